// pd_internal.h -- host-side interfaces between the parts of libpd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pd.h"
#include "pd_common.cuh"

namespace pd {

struct PlanState;

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
  // plan evaluations (pd_plan.cu): scratch from the plan's arena, or a
  // sizing pass; nullptr for the stream-ordered pool
  PlanState* plan = nullptr;
};

// The scratch arena of a plan for one kind of evaluation (pd_plan.cu):
// `base` (device memory, 256-byte aligned) of `cap` bytes, or base ==
// nullptr for a sizing pass, which records the bytes an evaluation needs in
// `need` and returns before any launch.  In plan mode an evaluation makes
// the same allocations on every call (buffers of optional outputs
// included), so data left in the arena by an earlier call stays where the
// next call looks for it: `features` says that the arena holds the centre
// features of every tile (grid only), `order` the grain order of the labels
// (labels only).
struct PlanState {
  char* base = nullptr;
  size_t cap = 0, need = 0;
  bool features = false, order = false;
};

// Scratch memory of one evaluation, in one of three modes:
//  * stream-ordered (the default): every get() draws from the device's
//    default memory pool on stream `st`, and everything is handed back on the
//    same stream when the object goes out of scope, so later work on that
//    stream may reuse it and work on other streams never sees it;
//  * arena: get() bumps through a caller-owned buffer [base, base + cap)
//    (256-byte aligned), nothing is freed; the same sequence of get() calls
//    returns the same addresses every time, so data left by an earlier
//    evaluation (a plan's label-dependent buffers) can be reused;
//  * sizing: get() only adds up the bytes an arena would need and returns a
//    placeholder; an evaluation returns right after its allocations.
class Scratch {
 public:
  explicit Scratch(cudaStream_t st) : st_(st) {}
  Scratch(cudaStream_t st, char* base, size_t cap) : st_(st), arena_(true), sizing_(base == nullptr), base_(base),
                                                      cap_(cap) {}
  // the plan's arena when ps != nullptr, else the stream-ordered pool
  Scratch(cudaStream_t st, const PlanState* ps)
      : st_(st), arena_(ps != nullptr), sizing_(ps && !ps->base), base_(ps ? ps->base : nullptr),
        cap_(ps ? ps->cap : 0) {}
  ~Scratch() {
    if (!arena_)
      for (void* p : ptrs_) cudaFreeAsync(p, st_);
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  template <typename T>
  T* get(size_t n) {
    if (n == 0) n = 1;
    if (arena_) {
      const size_t off = (used_ + 255) & ~(size_t)255;
      used_ = off + n * sizeof(T);
      if (sizing_) return reinterpret_cast<T*>(base_ + 256);  // placeholder, never dereferenced
      if (used_ > cap_) {
        failed_ = true;
        return nullptr;
      }
      return reinterpret_cast<T*>(base_ + off);
    }
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
  bool sizing() const { return sizing_; }
  size_t used() const { return used_; }

 private:
  cudaStream_t st_;
  bool arena_ = false, sizing_ = false;
  char* base_ = nullptr;
  size_t cap_ = 0, used_ = 0;
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
bool prof_enabled();  // pd_prof_enable is on
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

// A plan of evaluations on one pixel set and label map (pd_plan.cu): one
// device allocation holding the arena of the objective/gradient and, when
// asked for, the arena of the Hessian-vector product.
// The evaluation of one kind recorded as a CUDA graph, with the arguments
// it was recorded for.
struct PlanGraph {
  cudaGraphExec_t exec = nullptr;
  const double *theta = nullptr, *v = nullptr;
  double *obj = nullptr, *grad = nullptr, *hv = nullptr;
  double eps = 0.0;
  bool seen = false;  // the arguments were used by the last direct call
};
struct PlanCore {
  Geom g{};
  int dim = 0, d = 0, N = 0, prec = 0;
  const int32_t* labels = nullptr;
  PlanState eval, hvp;
  PlanGraph geval, ghvp;
  cudaStream_t cap = nullptr;  // capture stream (created on first use)
  bool graphs = true;          // false once a capture failed
  bool with_hvp = false;
  char* mem = nullptr;
  size_t bytes = 0;
};
int plan_init(PlanCore* p, const Geom& g, int dim, const int32_t* labels, int N, int d, int prec, bool with_hvp);
int plan_eval(PlanCore* p, const double* theta, double eps, double* obj, double* grad, cudaStream_t st);
int plan_hvp(PlanCore* p, const double* theta, const double* v, double eps, double* hv, cudaStream_t st);
void plan_free(PlanCore* p);

// pd_capi.cu
int validate_grid(const pd_grid* grid, Geom* g);
bool degree_ok(int dim, int d);  // 1 <= d <= the dimension's maximum degree
int theta_from_apd_host(int dim, int d, int N, const double* y, const double* w, const double* A,
                        double* theta_out);

}  // namespace pd
