// pd_peaks.cu -- throughput microbenchmarks of the execution units that
// bound the evaluation kernels (FP32 FMA, MUFU ex2, FP64 FMA), used to give
// the roofline its measured denominators (pd_microbench).
#include <cuda_runtime.h>

#include "pd.h"
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kChains = 8;

__global__ void k_bench_ffma(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = 1e-3f * (threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fmaf(a[q], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == 1234.5f) out[threadIdx.x] = s;  // keeps the chains alive
}

__global__ void k_bench_ex2(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = 1e-3f * (threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = Arith<float>::ex(-a[q]);  // converges near 0.64
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void k_bench_dfma(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = 1e-3 * (threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == 1234.5) out[threadIdx.x] = s;
}

}  // namespace
}  // namespace pd

extern "C" int pd_microbench(int kind, double* ops_per_s, void* stream) {
  using namespace pd;
  if (!ops_per_s || kind < 0 || kind > 2) return PD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = device_sm_count();
  const int threads = 256, blocks = sms * 8;
  const int iters = kind == 2 ? 256 : 4096;
  Scratch sc(st);
  double* buf = sc.get<double>(threads);
  if (!sc.ok()) return PD_ENOMEM;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return PD_ECUDA;
  auto launch = [&]() {
    if (kind == 0) k_bench_ffma<<<blocks, threads, 0, st>>>((float*)buf, iters, 0.999f, 1e-4f);
    else if (kind == 1) k_bench_ex2<<<blocks, threads, 0, st>>>((float*)buf, iters);
    else k_bench_dfma<<<blocks, threads, 0, st>>>(buf, iters, 0.999, 1e-4);
  };
  launch();  // warm-up
  cudaEventRecord(a, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(b, st);
  int rc = PD_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) rc = PD_ECUDA;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  const double ops = (double)reps * blocks * threads * (double)iters * kChains;
  *ops_per_s = ops / (ms * 1e-3);
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
}
