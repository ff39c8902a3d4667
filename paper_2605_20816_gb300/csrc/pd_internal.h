// pd_internal.h -- host-side interfaces between the parts of libpd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pd.h"
#include "pd_common.cuh"

namespace pd {

// One objective/gradient (v == nullptr) or Hessian-vector (v != nullptr)
// evaluation.  All pointers are device pointers.
struct EvalCall {
  Geom g;
  int dim, d, N, prec;
  double eps;
  const int32_t* labels;
  const double* theta;
  const double* v;  // HVP direction, or nullptr for objective/gradient
  double* obj;      // objective scalar, or nullptr
  double* grad;     // gradient, or nullptr
  double* hv;       // HVP output when v != nullptr
};

// Stream-ordered scratch: every get() draws from the device's default
// memory pool on stream `st`; everything is handed back on the same stream
// when the object goes out of scope, so later work on that stream may reuse
// it and work on other streams never sees it.
class Scratch {
 public:
  explicit Scratch(cudaStream_t st) : st_(st) {}
  ~Scratch() {
    for (void* p : ptrs_) cudaFreeAsync(p, st_);
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  template <typename T>
  T* get(size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    if (cudaMallocAsync(&p, n * sizeof(T), st_) != cudaSuccess) {
      cudaGetLastError();
      failed_ = true;
      return nullptr;
    }
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  bool ok() const { return !failed_; }

 private:
  cudaStream_t st_;
  std::vector<void*> ptrs_;
  bool failed_ = false;
};

int device_sm_count();

// Records a pair of CUDA events around the launches made during its
// lifetime when tracing is on (pd_prof_enable); a no-op otherwise.
class ProfScope {
 public:
  ProfScope(cudaStream_t st, const char* name);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  int idx_;
};
#define PD_TIMED(st, name, ...) \
  do {                          \
    ::pd::ProfScope pd_ps_(st, name); \
    __VA_ARGS__;                \
  } while (0)

// pd_simt.cu
int eval_simt(const EvalCall& c, cudaStream_t st);
int assign_simt(const Geom& g, int dim, int d, int N, const double* theta, int32_t* out, double* gap,
                const int32_t* ref, int64_t* mismatch, cudaStream_t st);
int features_simt(const Geom& g, int dim, int d, int prec, void* out, cudaStream_t st);
int moments_simt(const Geom& g, int dim, int dm, const int32_t* labels, int N, double* mom_out,
                 int64_t* counts_out, cudaStream_t st);
int check_labels_simt(const int32_t* labels, int64_t P, int N, int* bad_dev, cudaStream_t st);

// pd_tc.cu (tensor-core evaluation); PD_ENOTSUP where a shape is not covered
int eval_tc(const EvalCall& c, cudaStream_t st);
int eval_tc_hvp(const EvalCall& c, cudaStream_t st);  // pd_tc_hvp.cu
int selftest_wait_timeout(double seconds, int* status_out, cudaStream_t st);

// pd_noalloc.cu
void noalloc_forget_device();

// pd_capi.cu
int validate_grid(const pd_grid* grid, Geom* g);
int theta_from_apd_host(int dim, int d, int N, const double* y, const double* w, const double* A,
                        double* theta_out);

}  // namespace pd
