// pd_mlp.cu -- learned warm start: per-grain moment features, a three-layer
// perceptron (two ReLU hidden layers) with bf16 weights and fp32
// accumulation, its forward and backward kernels, Adam training, and the
// warm-start entry point that turns the network's prediction into starting
// parameters for the ascent scheme.  (Not from the paper.)
//
// Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with x the features
// of one grain and y its gauge-fixed (zero mean over grains), scale-
// normalised (unit root-mean-square norm over grains) parameter vector.
// The forward pass reads bf16 weights (rounded from the fp32 master copy
// after every update) and accumulates in fp32; the backward pass uses the
// same bf16 weights; weight gradients are summed over the batch in fixed
// order (split over the batch, then a fixed-order sum of the splits).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pd.h"
#include "pd_internal.h"
#include "pd_tc_common.cuh"

struct pd_mlp {
  int n_in = 0, n_h1 = 0, n_h2 = 0, n_out = 0;
  size_t n_params = 0;
  float* w = nullptr;        // fp32 master parameters: W1 b1 W2 b2 W3 b3
  __nv_bfloat16* wb = nullptr;  // bf16 copy used by the kernels
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  int64_t step = 0;
  size_t o_w1 = 0, o_b1 = 0, o_w2 = 0, o_b2 = 0, o_w3 = 0, o_b3 = 0;
};

namespace pd {
namespace {

// ---------------------------------------------------------------------------
// The network's GEMMs on the tensor cores (tcgen05.mma kind::f16, fp32
// accumulation in TMEM).
//
// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]) with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn]; EPI 0: plain, 1: ReLU, 2: multiply by
// (mask[m*ldm + n] > 0) (ReLU derivative).  Split-K over blockIdx.z writes
// slice z of C (C + z*M*ldc), k in [z*kchunk, (z+1)*kchunk).
//
// A CTA (4 warps) owns a 128 x kMmaN tile of C in TMEM.  The K range runs
// in chunks of 32, staged by all threads into shared memory (two stages) in
// the canonical K-major layout without swizzle: rows of A are the MMA's M
// rows, rows of B its N rows.  A bf16 operand (the weights) is one term; an
// fp32 operand (activations, gradients) is split into three bf16 terms
// hi + mid + lo (each the bf16 rounding of what the previous ones leave),
// which hold it to about 2^-24 relative, and the products are those of
// the terms whose weight reaches 2^-16 of the leading one (hh, hm, mh, hl,
// mm, lh: six for fp32 x fp32; three for fp32 x bf16), smallest first: the
// products of the network's bf16 weights with fp32 data, accumulated in
// fp32, as the CUDA cores would form them.  One thread issues the MMAs;
// every wait on the MMAs is bounded (a wait that gives up makes the tile
// NaN).
// ---------------------------------------------------------------------------
constexpr int kMmaN = 64;        // N of the MMA (columns of the C tile)
constexpr int kMmaKC = 32;       // K per staged chunk
constexpr int kGemmThreads = 128;
constexpr uint32_t kStageA = 128 * kMmaKC * 2;    // bytes of one A term per stage
constexpr uint32_t kStageB = kMmaN * kMmaKC * 2;  // bytes of one B term per stage

template <typename T>
__host__ __device__ constexpr int gemm_terms() { return std::is_same<T, float>::value ? 3 : 1; }
template <typename TA, typename TB>
__host__ __device__ constexpr uint32_t gemm_stage_bytes() {
  return gemm_terms<TA>() * kStageA + gemm_terms<TB>() * kStageB;
}

// bf16 terms of a value: three for fp32, the value itself for bf16.
__device__ __forceinline__ void bf16_terms(float a, __nv_bfloat16* t) {
  t[0] = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(t[0]);
  t[1] = __float2bfloat16_rn(r1);
  t[2] = __float2bfloat16_rn(r1 - __bfloat162float(t[1]));
}
__device__ __forceinline__ void bf16_terms(__nv_bfloat16 a, __nv_bfloat16* t) { t[0] = a; }

// Stages rows x kMmaKC values of an operand: value (r, kk) = X[(row0 + r) *
// sr + (k0 + kk) * sk] (zero outside rows < nrows, k < ke), term t at
// dst + t * term_bytes, K-major (row width kMmaKC).
template <typename T>
__device__ __forceinline__ void stage_operand(const T* __restrict__ X, int64_t sr, int64_t sk, int row0, int nrows,
                                              int k0, int ke, int rows, uint8_t* dst, uint32_t term_bytes) {
  constexpr int NT = gemm_terms<T>();
  const int n = rows * kMmaKC;
  // consecutive threads along the unit-stride index: coalesced loads
  const bool k_fast = sk == 1;
  for (int e = threadIdx.x; e < n; e += kGemmThreads) {
    const int r = k_fast ? e / kMmaKC : e % rows;
    const int kk = k_fast ? e % kMmaKC : e / rows;
    const int row = row0 + r, k = k0 + kk;
    __nv_bfloat16 t[3];
    if (row < nrows && k < ke) {
      bf16_terms(X[(int64_t)row * sr + (int64_t)k * sk], t);
    } else {
#pragma unroll
      for (int q = 0; q < NT; ++q) t[q] = __float2bfloat16_rn(0.f);
    }
    const uint32_t o = kmaj(r, kk, kMmaKC);
#pragma unroll
    for (int q = 0; q < NT; ++q) *reinterpret_cast<__nv_bfloat16*>(dst + q * term_bytes + o) = t[q];
  }
}

template <typename TA, typename TB, int EPI>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm(int M, int N, int K, const TA* __restrict__ A, int64_t sam, int64_t sak, const TB* __restrict__ B,
       int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc, const __nv_bfloat16* __restrict__ bias,
       const float* __restrict__ mask, int64_t ldm, int kchunk) {
  constexpr int NTA = gemm_terms<TA>(), NTB = gemm_terms<TB>();
  constexpr uint32_t kStage = gemm_stage_bytes<TA, TB>();
  extern __shared__ __align__(128) uint8_t gsm[];
  __shared__ uint64_t bar_mma[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * kMmaN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int n_chunks = ke > kb ? (ke - kb + kMmaKC - 1) / kMmaKC : 0;
  if (threadIdx.x == 0) {
    mbar_init(&bar_mma[0], 1);
    mbar_init(&bar_mma[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kMmaN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  constexpr uint32_t idesc = idesc_bf16(128, kMmaN);
  bool ok = true;
  int issued = 0;  // chunks whose MMAs were issued and committed
  for (int c = 0; c < n_chunks; ++c) {
    const int s = c & 1;
    // the stage is free once the MMAs of chunk c - 2 have read it
    if (c >= 2) ok = mbar_wait(&bar_mma[s], (uint32_t)(((c - 2) >> 1) & 1), &abort_flag, nullptr) && ok;
    ok = __syncthreads_and(ok);
    if (!ok) break;
    uint8_t* sa = gsm + s * kStage;
    uint8_t* sb = sa + NTA * kStageA;
    const int k0 = kb + c * kMmaKC;
    stage_operand<TA>(A, sam, sak, m0, M, k0, ke, 128, sa, kStageA);
    stage_operand<TB>(B, sbn, sbk, n0, N, k0, ke, kMmaN, sb, kStageB);
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_addr(sa), b0 = smem_addr(sb);
      uint32_t acc = c > 0 ? 1u : 0u;  // the tile's first product initialises the accumulator
#pragma unroll
      for (int kk = 0; kk < kMmaKC; kk += 16) {
        // products hh, hm, mh, hl, mm, lh (the available ones), smallest first
#pragma unroll
        for (int p = 5; p >= 0; --p) {
          const int ta = p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0);
          const int tb = p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0);
          if (ta >= NTA || tb >= NTB) continue;
          const uint64_t da = smem_desc(a0 + ta * kStageA + (uint32_t)kk * 16u, 128u, kMmaKC * 16u);
          const uint64_t db = smem_desc(b0 + tb * kStageB + (uint32_t)kk * 16u, 128u, kMmaKC * 16u);
          mma_bf16(tmem, da, db, idesc, acc);
          acc = 1u;
        }
      }
      mma_commit(&bar_mma[s]);
    }
    issued = c + 1;
  }
  // all MMAs of the tile complete (the last commit covers them all)
  if (issued > 0) {
    const int c = issued - 1;
    if (ok) ok = mbar_wait(&bar_mma[c & 1], (uint32_t)((c >> 1) & 1), &abort_flag, nullptr);
    else if (threadIdx.x == 0) mbar_wait_drain(&bar_mma[c & 1], (uint32_t)((c >> 1) & 1));
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();
  // epilogue: warp w holds rows m0 + 32 w + lane
  float* Cz = C + (int64_t)blockIdx.z * M * ldc;
  const int m = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < kMmaN; c0 += 32) {
    uint32_t r[32];
    if (n_chunks > 0 && ok) {
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      tmem_wait_ld();
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(ok ? 0.f : __int_as_float(0x7fc00000));
    }
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int n = n0 + c0 + j;
      if (n >= N) continue;
      float v = __uint_as_float(r[j]);
      if (bias) v += __bfloat162float(bias[n]);
      if (EPI == 1) v = fmaxf(v, 0.f);
      if (EPI == 2) v = mask[(int64_t)m * ldm + n] > 0.f ? v : 0.f;
      Cz[(int64_t)m * ldc + n] = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kMmaN);
  }
}

// out[q] = sum over s of part[s][q] (fixed order)
__global__ void k_sum_slices(const float* __restrict__ part, int S, int64_t n, float* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += part[(int64_t)z * n + q];
  out[q] = s;
}

// column sums of a [rows][cols] matrix (bias gradients), fixed order
__global__ void k_colsum(const float* __restrict__ X, int rows, int cols, float* __restrict__ out) {
  __shared__ float s[256];
  const int c = blockIdx.x;
  float a = 0.f;
  for (int r = threadIdx.x; r < rows; r += 256) a += X[(int64_t)r * cols + c];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = s[0];
}

// dY = 2 (Y - T) / (B n_out); per-block loss partials (fixed order)
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t n, float inv,
                      float* __restrict__ dY, float* __restrict__ part) {
  __shared__ float s[256];
  float a = 0.f;
  for (int64_t q = (int64_t)blockIdx.x * 256 + threadIdx.x; q < n; q += (int64_t)gridDim.x * 256) {
    const float e = Y[q] - T[q];
    a = fmaf(e, e, a);
    dY[q] = 2.f * e * inv;
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_mse_final(const float* __restrict__ part, int n, float inv, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int q = 0; q < n; ++q) s += part[q];
    *loss = s * inv;
  }
}

__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ g, int64_t n, float lr, float b1, float b2,
                       float c1, float c2, float epsa) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = b1 * m[q] + (1.f - b1) * gq;
  const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float wq = w[q] - lr * (mq * c1) / (sqrtf(vq * c2) + epsa);
  w[q] = wq;
  wb[q] = __float2bfloat16_rn(wq);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) wb[q] = __float2bfloat16_rn(w[q]);
}

// Counter-based uniform draw in [-1, 1) (splitmix64 of seed and index).
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
}

// He-uniform weights (limit sqrt(6 / fan_in)), zero biases.
__global__ void k_init(float* __restrict__ w, int64_t n, int64_t o_start, int fan_in, int is_bias, uint64_t seed) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  w[q] = is_bias ? 0.f : hash_uniform(seed, (uint64_t)(o_start + q)) * sqrtf(6.f / (float)fan_in);
}

// ---------------------------------------------------------------------------
// Features: normalised degree-4 moments of a grain and of its 8 nearest
// grains by centroid (nearest first, ties to the smaller index; padded with
// the grain's own vector).
// ---------------------------------------------------------------------------
constexpr int kNb = 8;

__global__ void k_norm_moments(const double* __restrict__ mom, const int64_t* __restrict__ cnt, int N, int Kd,
                               double* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)N * Kd) return;
  const int i = (int)(q / Kd);
  out[q] = cnt[i] ? mom[q] / (double)cnt[i] : 0.0;
}

__global__ void k_knn_features(const double* __restrict__ nm, int N, int Kd, int dim, float* __restrict__ feat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double dist[kNb];
  int nb[kNb];
  int have = 0;
  for (int j = 0; j < N; ++j) {
    if (j == i) continue;
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
      const double dx = nm[(int64_t)j * Kd + 1 + a] - nm[(int64_t)i * Kd + 1 + a];
      s += dx * dx;
    }
    int pos = have;
    while (pos > 0 && dist[pos - 1] > s) --pos;
    if (pos >= kNb) continue;
    const int last = have < kNb ? have : kNb - 1;
    for (int q = last; q > pos; --q) {
      dist[q] = dist[q - 1];
      nb[q] = nb[q - 1];
    }
    dist[pos] = s;
    nb[pos] = j;
    if (have < kNb) ++have;
  }
  const int F = (1 + kNb) * Kd;
  for (int k = 0; k < Kd; ++k) feat[(int64_t)i * F + k] = (float)nm[(int64_t)i * Kd + k];
  for (int q = 0; q < kNb; ++q) {
    const int j = q < have ? nb[q] : i;
    for (int k = 0; k < Kd; ++k) feat[(int64_t)i * F + (1 + q) * Kd + k] = (float)nm[(int64_t)j * Kd + k];
  }
}

template <typename TA, typename TB, int EPI>
int gemm(cudaStream_t st, int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk,
         int64_t sbn, float* C, int64_t ldc, const __nv_bfloat16* bias, const float* mask, int64_t ldm,
         int splits = 1) {
  const int kchunk = ((K + splits - 1) / splits + kMmaKC - 1) / kMmaKC * kMmaKC;
  const int sz = std::max(1, (K + kchunk - 1) / kchunk);
  dim3 grid((N + kMmaN - 1) / kMmaN, (M + 127) / 128, sz);
  constexpr int smem = 2 * (int)gemm_stage_bytes<TA, TB>();
  auto k = k_gemm<TA, TB, EPI>;
  // (a failure here is left in the runtime's last error, which the callers check)
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 1;
  PD_TIMED(st, "mlp_gemm_tc",
           (k<<<grid, kGemmThreads, smem, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, mask, ldm, kchunk)));
  return sz;
}

struct Acts {
  float *h1, *h2, *y;
};

int forward(const pd_mlp* net, const float* X, int B, Acts a, cudaStream_t st) {
  const __nv_bfloat16* W1 = net->wb + net->o_w1;
  const __nv_bfloat16* W2 = net->wb + net->o_w2;
  const __nv_bfloat16* W3 = net->wb + net->o_w3;
  gemm<float, __nv_bfloat16, 1>(st, B, net->n_h1, net->n_in, X, net->n_in, 1, W1, 1, net->n_in, a.h1, net->n_h1,
                                net->wb + net->o_b1, nullptr, 0);
  gemm<float, __nv_bfloat16, 1>(st, B, net->n_h2, net->n_h1, a.h1, net->n_h1, 1, W2, 1, net->n_h1, a.h2, net->n_h2,
                                net->wb + net->o_b2, nullptr, 0);
  gemm<float, __nv_bfloat16, 0>(st, B, net->n_out, net->n_h2, a.h2, net->n_h2, 1, W3, 1, net->n_h2, a.y, net->n_out,
                                net->wb + net->o_b3, nullptr, 0);
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
}

// Loss and gradients (into g, laid out like the parameters).
int loss_grad(const pd_mlp* net, const float* X, const float* T, int B, float* loss, float* g, cudaStream_t st) {
  Scratch sc(st);
  const int H1 = net->n_h1, H2 = net->n_h2, O = net->n_out, I = net->n_in;
  Acts a{sc.get<float>((size_t)B * H1), sc.get<float>((size_t)B * H2), sc.get<float>((size_t)B * O)};
  float* dy = sc.get<float>((size_t)B * O);
  float* d2 = sc.get<float>((size_t)B * H2);
  float* d1 = sc.get<float>((size_t)B * H1);
  const int splits = std::max(1, std::min(64, B / 512));
  const size_t slice = (size_t)std::max(H1 * I, std::max(H2 * H1, O * H2));
  float* part = sc.get<float>(slice * splits);
  const int mse_blocks = 256;
  float* lpart = sc.get<float>(mse_blocks);
  if (!sc.ok()) return PD_ENOMEM;
  int rc = forward(net, X, B, a, st);
  if (rc) return rc;
  const int64_t nY = (int64_t)B * O;
  k_mse<<<mse_blocks, 256, 0, st>>>(a.y, T, nY, 1.f / (float)nY, dy, lpart);
  k_mse_final<<<1, 32, 0, st>>>(lpart, mse_blocks, 1.f / (float)nY, loss);
  const __nv_bfloat16* W2 = net->wb + net->o_w2;
  const __nv_bfloat16* W3 = net->wb + net->o_w3;
  // layer 3: gW3 = dy^T h2, gb3 = colsum dy, d2 = (dy W3) * relu'(h2)
  int s = gemm<float, float, 0>(st, O, H2, B, dy, 1, O, a.h2, H2, 1, part, H2, nullptr, nullptr, 0, splits);
  k_sum_slices<<<(O * H2 + 255) / 256, 256, 0, st>>>(part, s, (int64_t)O * H2, g + net->o_w3);
  k_colsum<<<O, 256, 0, st>>>(dy, B, O, g + net->o_b3);
  gemm<float, __nv_bfloat16, 2>(st, B, H2, O, dy, O, 1, W3, H2, 1, d2, H2, nullptr, a.h2, H2);
  // layer 2
  s = gemm<float, float, 0>(st, H2, H1, B, d2, 1, H2, a.h1, H1, 1, part, H1, nullptr, nullptr, 0, splits);
  k_sum_slices<<<(H2 * H1 + 255) / 256, 256, 0, st>>>(part, s, (int64_t)H2 * H1, g + net->o_w2);
  k_colsum<<<H2, 256, 0, st>>>(d2, B, H2, g + net->o_b2);
  gemm<float, __nv_bfloat16, 2>(st, B, H1, H2, d2, H2, 1, W2, H1, 1, d1, H1, nullptr, a.h1, H1);
  // layer 1
  s = gemm<float, float, 0>(st, H1, I, B, d1, 1, H1, X, I, 1, part, I, nullptr, nullptr, 0, splits);
  k_sum_slices<<<(H1 * I + 255) / 256, 256, 0, st>>>(part, s, (int64_t)H1 * I, g + net->o_w1);
  k_colsum<<<H1, 256, 0, st>>>(d1, B, H1, g + net->o_b1);
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
}

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" int pd_mlp_create(int n_in, int n_h1, int n_h2, int n_out, uint64_t seed, pd_mlp** out) {
  if (!out || n_in < 1 || n_h1 < 1 || n_h2 < 1 || n_out < 1) return PD_EINVAL;
  pd_mlp* net = new pd_mlp();
  net->n_in = n_in;
  net->n_h1 = n_h1;
  net->n_h2 = n_h2;
  net->n_out = n_out;
  size_t o = 0;
  net->o_w1 = o; o += (size_t)n_h1 * n_in;
  net->o_b1 = o; o += n_h1;
  net->o_w2 = o; o += (size_t)n_h2 * n_h1;
  net->o_b2 = o; o += n_h2;
  net->o_w3 = o; o += (size_t)n_out * n_h2;
  net->o_b3 = o; o += n_out;
  net->n_params = o;
  if (cudaMalloc(&net->w, sizeof(float) * o) != cudaSuccess || cudaMalloc(&net->m, sizeof(float) * o) != cudaSuccess ||
      cudaMalloc(&net->v, sizeof(float) * o) != cudaSuccess ||
      cudaMalloc(&net->wb, sizeof(__nv_bfloat16) * o) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(net->w);
    cudaFree(net->m);
    cudaFree(net->v);
    delete net;
    return PD_ENOMEM;
  }
  cudaMemset(net->m, 0, sizeof(float) * o);
  cudaMemset(net->v, 0, sizeof(float) * o);
  struct L {
    size_t off, n;
    int fan, bias;
  } ls[] = {{net->o_w1, (size_t)n_h1 * n_in, n_in, 0}, {net->o_b1, (size_t)n_h1, n_in, 1},
            {net->o_w2, (size_t)n_h2 * n_h1, n_h1, 0}, {net->o_b2, (size_t)n_h2, n_h1, 1},
            {net->o_w3, (size_t)n_out * n_h2, n_h2, 0}, {net->o_b3, (size_t)n_out, n_h2, 1}};
  for (const L& l : ls)
    k_init<<<(unsigned)((l.n + 255) / 256), 256>>>(net->w + l.off, (int64_t)l.n, (int64_t)l.off, l.fan, l.bias, seed);
  k_to_bf16<<<(unsigned)((o + 255) / 256), 256>>>(net->w, net->wb, (int64_t)o);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    delete net;
    return PD_ECUDA;
  }
  *out = net;
  return PD_OK;
}

extern "C" void pd_mlp_destroy(pd_mlp* net) {
  if (!net) return;
  cudaDeviceSynchronize();
  cudaFree(net->w);
  cudaFree(net->wb);
  cudaFree(net->m);
  cudaFree(net->v);
  delete net;
}

extern "C" int64_t pd_mlp_num_params(const pd_mlp* net) { return net ? (int64_t)net->n_params : -1; }

extern "C" int pd_mlp_get_params(const pd_mlp* net, float* host, int rounded) {
  if (!net || !host) return PD_EINVAL;
  if (!rounded) return cudaMemcpy(host, net->w, sizeof(float) * net->n_params, cudaMemcpyDeviceToHost) == cudaSuccess
                           ? PD_OK
                           : PD_ECUDA;
  std::vector<__nv_bfloat16> b(net->n_params);
  if (cudaMemcpy(b.data(), net->wb, sizeof(__nv_bfloat16) * net->n_params, cudaMemcpyDeviceToHost) != cudaSuccess)
    return PD_ECUDA;
  for (size_t q = 0; q < net->n_params; ++q) host[q] = __bfloat162float(b[q]);
  return PD_OK;
}

extern "C" int pd_mlp_set_params(pd_mlp* net, const float* host) {
  if (!net || !host) return PD_EINVAL;
  if (cudaMemcpy(net->w, host, sizeof(float) * net->n_params, cudaMemcpyHostToDevice) != cudaSuccess) return PD_ECUDA;
  k_to_bf16<<<(unsigned)((net->n_params + 255) / 256), 256>>>(net->w, net->wb, (int64_t)net->n_params);
  return cudaDeviceSynchronize() == cudaSuccess ? PD_OK : PD_ECUDA;
}

extern "C" int pd_mlp_forward(const pd_mlp* net, const float* X, int B, float* Y, void* stream) {
  if (!net || !X || !Y || B < 0) return PD_EINVAL;
  if (B == 0) return PD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  Acts a{sc.get<float>((size_t)B * net->n_h1), sc.get<float>((size_t)B * net->n_h2), Y};
  if (!sc.ok()) return PD_ENOMEM;
  return forward(net, X, B, a, st);
}

extern "C" int pd_mlp_loss_grad(const pd_mlp* net, const float* X, const float* T, int B, float* loss_out,
                                float* grad_out, void* stream) {
  if (!net || !X || !T || !loss_out || !grad_out || B < 1) return PD_EINVAL;
  return loss_grad(net, X, T, B, loss_out, grad_out, (cudaStream_t)stream);
}

extern "C" int pd_mlp_train_step(pd_mlp* net, const float* X, const float* T, int B, float lr, float* loss_out,
                                 void* stream) {
  if (!net || !X || !T || !loss_out || B < 1 || !(lr > 0.f)) return PD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  float* g = sc.get<float>(net->n_params);
  if (!sc.ok()) return PD_ENOMEM;
  int rc = loss_grad(net, X, T, B, loss_out, g, st);
  if (rc) return rc;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f / (1.f - powf(b1, (float)net->step)), c2 = 1.f / (1.f - powf(b2, (float)net->step));
  PD_TIMED(st, "mlp_adam",
           (k_adam<<<(unsigned)((net->n_params + 255) / 256), 256, 0, st>>>(
               net->w, net->wb, net->m, net->v, g, (int64_t)net->n_params, lr, b1, b2, c1, c2, 1e-8f)));
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
}

extern "C" int pd_mlp_features(const pd_grid* grid, const int32_t* labels, int N, float* feat_out, void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (!labels || !feat_out || N < 1 || g.P < 1) return PD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int Kd = basis_K(grid->dim, 4);
  Scratch sc(st);
  double* mom = sc.get<double>((size_t)N * Kd);
  double* nm = sc.get<double>((size_t)N * Kd);
  int64_t* cnt = sc.get<int64_t>(N);
  if (!sc.ok()) return PD_ENOMEM;
  rc = moments_simt(g, grid->dim, 4, labels, N, mom, cnt, st);
  if (rc) return rc;
  const int64_t n = (int64_t)N * Kd;
  k_norm_moments<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mom, cnt, N, Kd, nm);
  PD_TIMED(st, "mlp_features", (k_knn_features<<<(N + 127) / 128, 128, 0, st>>>(nm, N, Kd, grid->dim, feat_out)));
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
}

// Training targets of one map: t_i = (theta_i - mean_j theta_j) / s with
// s^2 = mean_i |theta_i - mean_j theta_j|^2 (one block, fixed order).
static __global__ void k_mlp_targets(const double* __restrict__ theta, int N, int K, float* __restrict__ out) {
  __shared__ double mean[64];
  __shared__ double red[256];
  for (int k = 0; k < K; ++k) {
    double a = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) a += theta[(int64_t)i * K + k];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) mean[k] = red[0] / N;
    __syncthreads();
  }
  double a = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    for (int k = 0; k < K; ++k) {
      const double c = theta[(int64_t)i * K + k] - mean[k];
      a += c * c;
    }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double sc = red[0] > 0.0 ? 1.0 / sqrt(red[0] / N) : 1.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    for (int k = 0; k < K; ++k) out[(int64_t)i * K + k] = (float)((theta[(int64_t)i * K + k] - mean[k]) * sc);
}

extern "C" int pd_mlp_targets(const double* theta, int N, int K, float* out, void* stream) {
  if (!theta || !out || N < 1 || K < 1 || K > 64) return PD_EINVAL;
  k_mlp_targets<<<1, 256, 0, (cudaStream_t)stream>>>(theta, N, K, out);
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
}

// Synchronous: predict, restore the gauge and pick the scale.
extern "C" int pd_warm_start(const pd_mlp* net, const pd_grid* grid, const int32_t* labels, int N, int d, double eps,
                             int prec, double* theta_out, double* scale_out, void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (!net || !labels || !theta_out || N < 2 || d < 1 || !(eps > 0.0)) return PD_EINVAL;
  const int K = basis_K(grid->dim, d);
  const int Kd = basis_K(grid->dim, 4);
  if (net->n_in != (1 + kNb) * Kd || net->n_out != K) return PD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  float* feat = sc.get<float>((size_t)N * net->n_in);
  float* y = sc.get<float>((size_t)N * K);
  double* th = sc.get<double>((size_t)N * K);
  double* obj = sc.get<double>(1);
  if (!sc.ok()) return PD_ENOMEM;
  rc = pd_mlp_features(grid, labels, N, feat, stream);
  if (rc) return rc;
  rc = pd_mlp_forward(net, feat, N, y, stream);
  if (rc) return rc;
  std::vector<float> hy((size_t)N * K);
  if (cudaMemcpyAsync(hy.data(), y, sizeof(float) * hy.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PD_ECUDA;
  // gauge: theta_{N-1} = 0 (differences between grains are what the
  // network predicts; the common shift is free, Lemma 4.2)
  std::vector<double> base((size_t)N * K);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < K; ++k) base[(size_t)i * K + k] = (double)hy[(size_t)i * K + k] - (double)hy[(size_t)(N - 1) * K + k];
  // scale: maximise Phi(s * base) over s = 2^(q/2), then keep the best
  std::vector<double> trial(base.size());
  double best_phi = -INFINITY, best_s = 1.0;
  pd_eval_opts o{d, eps, prec};
  for (int q = -16; q <= 40; ++q) {
    const double s = pow(2.0, 0.5 * q);
    for (size_t e = 0; e < base.size(); ++e) trial[e] = s * base[e];
    if (cudaMemcpyAsync(th, trial.data(), sizeof(double) * trial.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return PD_ECUDA;
    rc = pd_objective_grad(grid, labels, N, th, &o, obj, nullptr, stream);
    if (rc) return rc;
    double phi = 0.0;
    if (cudaMemcpyAsync(&phi, obj, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PD_ECUDA;
    if (isfinite(phi) && phi > best_phi) {
      best_phi = phi;
      best_s = s;
    }
  }
  for (size_t e = 0; e < base.size(); ++e) trial[e] = best_s * base[e];
  if (scale_out) *scale_out = best_s;
  if (cudaMemcpyAsync(theta_out, trial.data(), sizeof(double) * trial.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PD_ECUDA;
  return PD_OK;
}
