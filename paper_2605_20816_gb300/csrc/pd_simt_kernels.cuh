// pd_simt_kernels.cuh -- CUDA-core (FFMA / DFMA) kernels of libpd:
//   objective + gradient (eqs. Phi, grad), Hessian-vector products
//   (eq. hess), arg-min assignment (eq. Li_def), features, grain moments.
//
// Evaluation structure (two passes over the pixels, nothing of size P x N is
// ever stored):
//   pass 1, one thread per pixel: features eta(x) in registers, logits of
//           every grain against parameter tiles staged in shared memory,
//           online log-sum-exp; writes log S(x) (4 or 8 bytes per pixel)
//           and a per-block partial of sum_x log p_{G(x)}(x).
//   pass 2, one thread per grain: pixel tiles (features, log S, label)
//           staged in shared memory, the thread recomputes its logit, forms
//           p_i(x) and accumulates (delta_{iG(x)} - p_i(x)) eta(x); per-tile
//           sums are carried in double per pixel chunk.
//   reduce: fixed-order double sum over chunks (bitwise reproducible).
// PD_FP64 runs this structure over the pixel-linear order.  PD_FP32 runs it
// over 128-pixel tiles (pd_tiles.cuh) with every logit relative to the
// tile's reference C(t): the centre offset theta'_i . eta(c) - C(t) in
// float-float, rounded once, plus the remainder theta'_i . (eta(x) -
// eta(c)) in float from divided differences of the recurrence; pass 2
// accumulates (delta - p) (eta(x) - eta(c)) and adds the tile's sum of
// (delta - p) times eta(c) at the end of the tile, so that the float
// accumulation acts on small numbers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pd_common.cuh"
#include "pd_internal.h"
#include "pd_tiles.cuh"

namespace pd {
// Everything here has internal linkage: each translation unit that includes
// this header gets its own copies of the kernels it instantiates.
namespace {

constexpr int kLseThreads = 256;
constexpr int kGradThreads = 128;  // grains per block in pass 2
constexpr int kPixTile = 128;      // pixels per shared-memory tile in pass 2
constexpr int kChunk = 8;          // grains per online-LSE rescale

template <int K, typename T>
__device__ __forceinline__ T dot_k(const T* __restrict__ a, const T* __restrict__ b) {
  T acc = a[0] * b[0];
#pragma unroll
  for (int k = 1; k < K; ++k) acc = fma(a[k], b[k], acc);
  return acc;
}

static __device__ __forceinline__ double block_sum_fixed(double v, double* sbuf) {
  // fixed-order block reduction: warp tree, then warp sums in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sbuf[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sbuf[w];
  }
  return s;
}

// ---------------------------------------------------------------------------
// theta -> scaled working copy thS[i][k] = theta[i][k] * scale, padded rows.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scale_theta(const double* __restrict__ theta, int N, int K, int KP,
                              double scale, T* __restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)N * KP) return;
  int i = (int)(q / KP), k = (int)(q % KP);
  out[q] = k < K ? (T)(theta[(int64_t)i * K + k] * scale) : (T)0;
}

template <typename T>
__global__ void k_copy_pad(const double* __restrict__ v, int N, int K, int KP, T* __restrict__ out) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)N * KP) return;
  int i = (int)(q / KP), k = (int)(q % KP);
  out[q] = k < K ? (T)v[(int64_t)i * K + k] : (T)0;
}

// ---------------------------------------------------------------------------
// Pass 1: per-pixel log-sum-exp (and, for HVP, ubar(x) = sum_k p_k u_k).
// ---------------------------------------------------------------------------
// One block of pass 1 (pixels block*kLseThreads*PPT ...); obj_slot receives
// the block's objective partial.  Called by the single-map kernel with the
// block index and by the batched persistent kernel for each work item.
template <typename T, int DIM, int D, int PPT, bool HVP>
__device__ __forceinline__ void pass1_block(const Geom& g, const int32_t* __restrict__ labels, int N,
                                            const T* __restrict__ thS, const T* __restrict__ vS,
                                            T* __restrict__ lse_out, T* __restrict__ ubar_out,
                                            double* __restrict__ obj_slot, int64_t block) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<T>(K);
  constexpr int GT = HVP ? 64 : 128;  // grains per shared tile
  __shared__ __align__(16) T sth[GT * KP];
  __shared__ __align__(16) T sv[HVP ? GT * KP : 1];
  __shared__ double sred[kLseThreads / 32];

  const int64_t base = block * (kLseThreads * PPT);
  T eta[PPT][K];
  T m[PPT], s[PPT], t[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int64_t j = base + q * kLseThreads + threadIdx.x;
    T x[DIM];
    if (j < g.P) {
      pixel_coords<DIM>(g, j, x);
    } else {
#pragma unroll
      for (int a = 0; a < DIM; ++a) x[a] = (T)0;
    }
    legendre_features<DIM, D>(x, eta[q]);
    m[q] = -INFINITY;
    s[q] = (T)0;
    t[q] = (T)0;
  }

  for (int g0 = 0; g0 < N; g0 += GT) {
    const int gn = min(GT, N - g0);
    __syncthreads();
    {
      // rows g0..g0+gn-1 are contiguous: gn*KP elements, 16-byte vectors
      constexpr int VE = 16 / sizeof(T);
      const int nv = gn * KP / VE;
      const uint4* src = reinterpret_cast<const uint4*>(thS + (int64_t)g0 * KP);
      uint4* dst = reinterpret_cast<uint4*>(sth);
      for (int e = threadIdx.x; e < nv; e += kLseThreads) dst[e] = src[e];
      if (HVP) {
        const uint4* srcv = reinterpret_cast<const uint4*>(vS + (int64_t)g0 * KP);
        uint4* dstv = reinterpret_cast<uint4*>(sv);
        for (int e = threadIdx.x; e < nv; e += kLseThreads) dstv[e] = srcv[e];
      }
    }
    __syncthreads();
    int i = 0;
    for (; i + kChunk <= gn; i += kChunk) {
      T l[PPT][kChunk];
      T u[PPT][HVP ? kChunk : 1];
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          l[q][c] = dot_k<K>(sth + (i + c) * KP, eta[q]);
          if (HVP) u[q][c] = dot_k<K>(sv + (i + c) * KP, eta[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        T cm = l[q][0];
#pragma unroll
        for (int c = 1; c < kChunk; ++c) cm = fmax(cm, l[q][c]);
        const T mn = fmax(m[q], cm);
        const T r = Arith<T>::ex(m[q] - mn);
        T add = (T)0, addu = (T)0;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
          const T e = Arith<T>::ex(l[q][c] - mn);
          add += e;
          if (HVP) addu = fma(e, u[q][c], addu);
        }
        s[q] = fma(s[q], r, add);
        if (HVP) t[q] = fma(t[q], r, addu);
        m[q] = mn;
      }
    }
    for (; i < gn; ++i) {
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const T l = dot_k<K>(sth + i * KP, eta[q]);
        const T mn = fmax(m[q], l);
        const T r = Arith<T>::ex(m[q] - mn);
        const T e = Arith<T>::ex(l - mn);
        s[q] = fma(s[q], r, e);
        if (HVP) {
          const T u = dot_k<K>(sv + i * KP, eta[q]);
          t[q] = fma(t[q], r, e * u);
        }
        m[q] = mn;
      }
    }
  }

  double racc = 0.0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int64_t j = base + q * kLseThreads + threadIdx.x;
    if (j >= g.P) continue;
    const T lse = m[q] + Arith<T>::lg(s[q]);
    if (lse_out) lse_out[j] = lse;
    if (HVP) ubar_out[j] = t[q] / s[q];
    if (!HVP && obj_slot) {
      const int G = labels[j];
      if ((unsigned)G < (unsigned)N) {
        const T lG = dot_k<K>(thS + (int64_t)G * KP, eta[q]);
        racc += (double)(lG - lse) * Arith<T>::to_nat;
      } else {
        racc = NAN;  // a label outside 0..N-1 poisons the objective
      }
    }
  }
  if (!HVP && obj_slot) {
    const double bs = block_sum_fixed(racc, sred);
    if (threadIdx.x == 0) *obj_slot = bs;
  }
}

template <typename T, int DIM, int D, int PPT, bool HVP>
__global__ void __launch_bounds__(kLseThreads)
k_pass1(Geom g, const int32_t* __restrict__ labels, int N, const T* __restrict__ thS,
        const T* __restrict__ vS, T* __restrict__ lse_out, T* __restrict__ ubar_out,
        double* __restrict__ obj_part) {
  pass1_block<T, DIM, D, PPT, HVP>(g, labels, N, thS, vS, lse_out, ubar_out,
                                   obj_part ? obj_part + blockIdx.x : nullptr, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Pass 2: one thread per grain over pixel tiles.
//   GRAD: c = delta_{iG(x)} - p_i(x)
//   HVP : c = p_i(x) (u_i(x) - ubar(x))
// accumulates c * eta(x) per chunk of pixels into part[chunk][i][k].  Two
// pixels per step give two independent dependency chains.  When c is zero
// for every grain of a warp at both pixels (p underflows to zero and no
// label matches, the common case for small eps) the accumulation is skipped:
// adding c * eta with c = 0 changes nothing, so results are identical.
// ---------------------------------------------------------------------------
// One block of pass 2: pixel chunk `chunk` (ppc pixels) and grain tile
// `gtile`; writes part[chunk][i][k] for the tile's grains.
template <typename T, int DIM, int D, bool HVP>
__device__ __forceinline__ void pass2_block(const Geom& g, const int32_t* __restrict__ labels, int N,
                                            const T* __restrict__ thS, const T* __restrict__ vS,
                                            const T* __restrict__ lse, const T* __restrict__ ubar, int64_t ppc,
                                            double* __restrict__ part, int64_t chunk, int gtile) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<T>(K);
  __shared__ __align__(16) T seta[kPixTile * KP];
  __shared__ T slse[kPixTile];
  __shared__ T subar[HVP ? kPixTile : 1];
  __shared__ int slab[kPixTile];
  __shared__ double sacc[K * kGradThreads];  // per-thread double accumulators

  const int i = gtile * kGradThreads + threadIdx.x;
  const bool vi = i < N;
  T th[K], vv[HVP ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    th[k] = vi ? thS[(int64_t)i * KP + k] : (T)0;
    if (HVP) vv[k] = vi ? vS[(int64_t)i * KP + k] : (T)0;
    sacc[k * kGradThreads + threadIdx.x] = 0.0;
  }

  const int64_t p0 = chunk * ppc;
  const int64_t p1 = min(p0 + ppc, g.P);
  for (int64_t t0 = p0; t0 < p1; t0 += kPixTile) {
    const int tn = (int)min((int64_t)kPixTile, p1 - t0);
    __syncthreads();
    if (threadIdx.x < tn) {
      const int64_t j = t0 + threadIdx.x;
      T x[DIM], e[K];
      pixel_coords<DIM>(g, j, x);
      legendre_features<DIM, D>(x, e);
#pragma unroll
      for (int k = 0; k < K; ++k) seta[threadIdx.x * KP + k] = e[k];
      slse[threadIdx.x] = lse[j];
      if (HVP) subar[threadIdx.x] = ubar[j];
      else slab[threadIdx.x] = labels[j];
    }
    __syncthreads();
    T acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = (T)0;
    auto coef = [&](int q, T l) -> T {
      const T p = Arith<T>::ex(l - slse[q]);
      T c;
      if (HVP) {
        const T u = dot_k<K>(vv, seta + q * KP);
        c = p * (u - subar[q]);
      } else {
        c = (slab[q] == i ? (T)1 : (T)0) - p;
      }
      return vi ? c : (T)0;
    };
    int q = 0;
    for (; q + 2 <= tn; q += 2) {
      const T* e0 = seta + q * KP;
      const T* e1 = e0 + KP;
      const T l0 = dot_k<K>(th, e0);
      const T l1 = dot_k<K>(th, e1);
      const T c0 = coef(q, l0);
      const T c1 = coef(q + 1, l1);
      if (__any_sync(0xffffffffu, c0 != (T)0 || c1 != (T)0)) {
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = fma(c1, e1[k], fma(c0, e0[k], acc[k]));
      }
    }
    if (q < tn) {
      const T* e0 = seta + q * KP;
      const T c0 = coef(q, dot_k<K>(th, e0));
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fma(c0, e0[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) sacc[k * kGradThreads + threadIdx.x] += (double)acc[k];
  }
  if (vi) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[(chunk * N + i) * K + k] = sacc[k * kGradThreads + threadIdx.x];
  }
  __syncthreads();  // the shared tiles may be reused by the next work item
}

template <typename T, int DIM, int D, bool HVP>
__global__ void __launch_bounds__(kGradThreads)
k_pass2(Geom g, const int32_t* __restrict__ labels, int N, const T* __restrict__ thS,
        const T* __restrict__ vS, const T* __restrict__ lse, const T* __restrict__ ubar,
        int64_t ppc, double* __restrict__ part) {
  pass2_block<T, DIM, D, HVP>(g, labels, N, thS, vS, lse, ubar, ppc, part, blockIdx.x, blockIdx.y);
}

// Fixed-order sum over chunks: out[q] = scale * sum_c part[c][q].  A block
// covers 32 consecutive q (coalesced) with 8 chunk phases; phase y sums the
// chunks c = y (mod 8) in ascending order, then the 8 phase sums are added
// in phase order: the same order every run.
constexpr int kRedPhases = 8;
static __global__ void __launch_bounds__(32 * kRedPhases)
k_reduce_parts(const double* __restrict__ part, int nchunks, int64_t NK, double scale, double* __restrict__ out) {
  __shared__ double ssum[kRedPhases][32];
  const int64_t q = (int64_t)blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (q < NK)
    for (int c = threadIdx.y; c < nchunks; c += kRedPhases) s += part[(int64_t)c * NK + q];
  ssum[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && q < NK) {
    double t = 0.0;
#pragma unroll
    for (int y = 0; y < kRedPhases; ++y) t += ssum[y][threadIdx.x];
    out[q] = t * scale;
  }
}

// Fixed-order sum of the per-block objective partials: *out = scale * sum.
static __global__ void k_reduce_obj(const double* __restrict__ part, int n, double scale,
                             double* __restrict__ out) {
  __shared__ double sred[32];
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += part[q];
  const double bs = block_sum_fixed(s, sred);
  if (threadIdx.x == 0) *out = bs * scale;
}

// ---------------------------------------------------------------------------
// FP32 evaluation on tiles (pd_tiles.cuh).  The logits of a pixel are kept
// relative to its tile's reference logit: l_i(x) - C(t) = o_i(t) +
// theta'_i . (eta(x) - eta(c)), with o_i(t) = theta'_i . eta(c) - C(t)
// formed in float-float inside the kernels (once per grain and tile) and
// rounded once; log2 S(x) is kept relative to the same C(t).  Pass 2 forms
// c = delta_{iG(x)} - p_i(x) from the same offsets and log2 S.
//   pass 1: a block = kT1Tiles tiles (two pixels a thread), grains in
//           shared-memory chunks with their offsets on the block's tiles;
//   pass 2: a block = 128 grains over a run of tiles; per tile the pixels'
//           features, feature differences, log2 S and labels in shared
//           memory and each thread's offset on the tile.
// ---------------------------------------------------------------------------
constexpr int kT1Tiles = 4;  // tiles per pass-1 block: 512 pixels, two a thread
static_assert(kGradThreads == kTilePix, "pass 2: one producer thread per tile row");

// log2 of a float sum S >= 1 (the largest term of a log-sum-exp is 1): the
// accurate library logarithm, so that log2 S of pixels whose sum is 1 plus
// tiny terms carries no approximation bias.
__device__ __forceinline__ float lse_log2(float s) { return log2f(s); }

template <int DIM, int D, bool HVP>
__device__ __forceinline__ void pass1_tiles_block(const Geom& g, const TileMap& tm, const int32_t* __restrict__ labels,
                                                  int N, const float* __restrict__ thH, const float* __restrict__ thL,
                                                  const float* __restrict__ vS, const float2* __restrict__ ecg,
                                                  const float2* __restrict__ refg, float* __restrict__ lse_out,
                                                  float* __restrict__ q_out, float* __restrict__ ubar_out,
                                                  float* __restrict__ dm_out, int* __restrict__ mx_out,
                                                  double* __restrict__ obj_slot, int64_t blk) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<float>(K);
  constexpr int GT = HVP ? 64 : 128;  // grains per shared chunk
  __shared__ __align__(16) float sth[GT * KP];
  __shared__ __align__(16) float stl[GT * KP];
  __shared__ __align__(16) float sv[HVP ? GT * KP : 1];
  __shared__ float soff[kT1Tiles][GT];
  __shared__ float2 sec[kT1Tiles][K];
  __shared__ float2 sref[kT1Tiles];
  __shared__ double sred[kLseThreads / 32];

  const int64_t t0 = blk * kT1Tiles;
  const int r = threadIdx.x & (kTilePix - 1), hq = threadIdx.x / kTilePix;  // row; local tiles hq, hq + 2
  for (int e = threadIdx.x; e < kT1Tiles * K; e += kLseThreads) {
    const int64_t t = t0 + e / K;
    sec[e / K][e % K] = t < tm.n_tiles ? ecg[t * K + e % K] : make_float2(0.f, 0.f);
  }
  if (threadIdx.x < kT1Tiles) {
    const int64_t t = t0 + threadIdx.x;
    sref[threadIdx.x] = t < tm.n_tiles ? refg[t] : make_float2(0.f, 0.f);
  }
  float de[2][K], eta[HVP ? 2 : 1][K];
  int64_t jq[2];
  // m: running max; s: the sum of 2^(l - m) over the grains other than the
  // pixel's label G (gradient) -- the label's term is added at the end, so
  // that 1 - p_G = s / (s + 2^(lG - m)) and log p_G carry no cancellation
  // when p_G is close to 1 (a well-fitted pixel).  For the HVP the grain
  // kept apart is the arg-max M (index mx, u_M = uM): s and tu sum 2^(l - m)
  // and 2^(l - m) u over the others, so that u_M - ubar = (uM s - tu) /
  // (1 + s) keeps its relative accuracy when p_M is close to 1.
  float m[2], s[2], tu[2], uM[2];
  int Gq[2], mx[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t t = t0 + hq + 2 * q;
    float x[DIM], c[DIM], dx[DIM];
    if (t < tm.n_tiles) {
      jq[q] = tile_pixel_dx<DIM>(g, tm, t, r, x, c, dx);
    } else {
      jq[q] = -1;
#pragma unroll
      for (int a = 0; a < DIM; ++a) x[a] = c[a] = dx[a] = 0.f;
    }
    legendre_delta<DIM, D>(x, c, dx, de[q], HVP ? eta[q] : nullptr);
    m[q] = -INFINITY;
    s[q] = 0.f;
    tu[q] = 0.f;
    uM[q] = 0.f;
    mx[q] = -1;
    Gq[q] = !HVP && jq[q] >= 0 ? labels[jq[q]] : -1;
  }

  for (int g0 = 0; g0 < N; g0 += GT) {
    const int gn = min(GT, N - g0);
    __syncthreads();
    {
      const int nv = gn * KP / 4;
      const uint4* src = reinterpret_cast<const uint4*>(thH + (int64_t)g0 * KP);
      const uint4* srcl = reinterpret_cast<const uint4*>(thL + (int64_t)g0 * KP);
      uint4* dst = reinterpret_cast<uint4*>(sth);
      uint4* dstl = reinterpret_cast<uint4*>(stl);
      for (int e = threadIdx.x; e < nv; e += kLseThreads) {
        dst[e] = src[e];
        dstl[e] = srcl[e];
      }
      if (HVP) {
        const uint4* srcv = reinterpret_cast<const uint4*>(vS + (int64_t)g0 * KP);
        uint4* dstv = reinterpret_cast<uint4*>(sv);
        for (int e = threadIdx.x; e < nv; e += kLseThreads) dstv[e] = srcv[e];
      }
    }
    __syncthreads();
    // the chunk's offsets on the block's tiles, one (grain, tile) pair a thread
    for (int e = threadIdx.x; e < gn * kT1Tiles; e += kLseThreads) {
      const int gi = e % gn, q = e / gn;
      soff[q][gi] = centre_offset<K>(sth + gi * KP, stl + gi * KP, sec[q], sref[q]);
    }
    __syncthreads();
    int i = 0;
    for (; i + kChunk <= gn; i += kChunk) {
      float l[2][kChunk];
      float u[2][HVP ? kChunk : 1];
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          l[q][c] = soff[hq + 2 * q][i + c] + dot_k<K>(sth + (i + c) * KP, de[q]);
          if (HVP) u[q][c] = dot_k<K>(sv + (i + c) * KP, eta[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float cm = l[q][0];
#pragma unroll
        for (int c = 1; c < kChunk; ++c) cm = fmaxf(cm, l[q][c]);
        if (HVP) {
          if (cm > m[q]) {
            // the max moves into this chunk: the old max's term joins the
            // sums, the first grain attaining cm is kept apart
            const float rr = Arith<float>::ex(m[q] - cm);
            float add = rr, addu = uM[q] * rr;
            bool found = false;
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
              const float e = Arith<float>::ex(l[q][c] - cm);
              const bool hit = !found && l[q][c] == cm;
              found = found || hit;
              if (hit) {
                uM[q] = u[q][c];
                mx[q] = g0 + i + c;
              } else {
                add += e;
                addu = fmaf(e, u[q][c], addu);
              }
            }
            s[q] = fmaf(s[q], rr, add);
            tu[q] = fmaf(tu[q], rr, addu);
            m[q] = cm;
          } else {
            float add = 0.f, addu = 0.f;
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
              const float e = Arith<float>::ex(l[q][c] - m[q]);
              add += e;
              addu = fmaf(e, u[q][c], addu);
            }
            s[q] += add;
            tu[q] += addu;
          }
          continue;
        }
        const float mn = fmaxf(m[q], cm);
        const float rr = Arith<float>::ex(m[q] - mn);
        float add = 0.f;
        const int lc = Gq[q] - (g0 + i);
        if ((unsigned)lc < (unsigned)kChunk) {
          // the chunk of the label: its term kept apart
#pragma unroll
          for (int c = 0; c < kChunk; ++c) {
            const float e = Arith<float>::ex(l[q][c] - mn);
            add += c == lc ? 0.f : e;
          }
        } else {
#pragma unroll
          for (int c = 0; c < kChunk; ++c) add += Arith<float>::ex(l[q][c] - mn);
        }
        s[q] = fmaf(s[q], rr, add);
        m[q] = mn;
      }
    }
    for (; i < gn; ++i) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float l = soff[hq + 2 * q][i] + dot_k<K>(sth + i * KP, de[q]);
        if (HVP) {
          const float uu = dot_k<K>(sv + i * KP, eta[q]);
          if (l > m[q]) {  // a new max: the old one's term joins the sums
            const float rr = Arith<float>::ex(m[q] - l);
            s[q] = fmaf(s[q], rr, rr);
            tu[q] = fmaf(tu[q], rr, uM[q] * rr);
            uM[q] = uu;
            mx[q] = g0 + i;
            m[q] = l;
          } else {
            const float e = Arith<float>::ex(l - m[q]);
            s[q] += e;
            tu[q] = fmaf(e, uu, tu[q]);
          }
          continue;
        }
        const float mn = fmaxf(m[q], l);
        const float rr = Arith<float>::ex(m[q] - mn);
        const float e = g0 + i == Gq[q] ? 0.f : Arith<float>::ex(l - mn);
        s[q] = fmaf(s[q], rr, e);
        m[q] = mn;
      }
    }
  }

  double racc = 0.0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t j = jq[q];
    if (j < 0) continue;
    if (HVP) {
      // S = 1 + s (the max's own term is 1)
      const float S = 1.f + s[q];
      if (lse_out) lse_out[j] = m[q] + lse_log2(S);
      ubar_out[j] = (uM[q] + tu[q]) / S;
      dm_out[j] = fmaf(uM[q], s[q], -tu[q]) / S;  // u_M - ubar
      mx_out[j] = mx[q];
      continue;
    }
    const int G = Gq[q];
    const bool lab_ok = (unsigned)G < (unsigned)N;
    float lG = NAN;  // the label logit, formed as in the loop
    if (lab_ok) {
      float h[K], l[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        h[k] = thH[(int64_t)G * KP + k];
        l[k] = thL[(int64_t)G * KP + k];
      }
      const int lt = hq + 2 * q;
      lG = centre_offset<K>(h, l, sec[lt], sref[lt]) + dot_k<K>(h, de[q]);
    }
    const LabelLse rl = label_lse(m[q], s[q], lG);
    if (lse_out) lse_out[j] = rl.lse;
    if (q_out) q_out[j] = rl.q;
    if (obj_slot) racc = lab_ok ? racc + rl.logp : NAN;  // a label outside 0..N-1 poisons the objective
  }
  if (!HVP && obj_slot) {
    const double bs = block_sum_fixed(racc, sred);
    if (threadIdx.x == 0) *obj_slot = bs;
  }
}

template <int DIM, int D, bool HVP>
__global__ void __launch_bounds__(kLseThreads)
k_pass1_tiles(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, const float* __restrict__ thH,
              const float* __restrict__ thL, const float* __restrict__ vS, const float2* __restrict__ ecg,
              const float2* __restrict__ refg, float* __restrict__ lse_out, float* __restrict__ q_out,
              float* __restrict__ ubar_out, float* __restrict__ dm_out, int* __restrict__ mx_out,
              double* __restrict__ obj_part) {
  pass1_tiles_block<DIM, D, HVP>(g, tm, labels, N, thH, thL, vS, ecg, refg, lse_out, q_out, ubar_out, dm_out, mx_out,
                                 obj_part ? obj_part + blockIdx.x : nullptr, blockIdx.x);
}

// The same for the longest feature vectors (K > 28), held to two blocks
// per SM: left free, the compiler gives them one.
template <int DIM, int D, bool HVP>
__global__ void __launch_bounds__(kLseThreads, 2)
k_pass1_tiles_2(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, const float* __restrict__ thH,
                const float* __restrict__ thL, const float* __restrict__ vS, const float2* __restrict__ ecg,
                const float2* __restrict__ refg, float* __restrict__ lse_out, float* __restrict__ q_out,
                float* __restrict__ ubar_out, float* __restrict__ dm_out, int* __restrict__ mx_out,
                double* __restrict__ obj_part) {
  pass1_tiles_block<DIM, D, HVP>(g, tm, labels, N, thH, thL, vS, ecg, refg, lse_out, q_out, ubar_out, dm_out, mx_out,
                                 obj_part ? obj_part + blockIdx.x : nullptr, blockIdx.x);
}

// Pass 2 on tiles: grain tile `gtile` over the tiles [chunk * tpc, ...).
//   GRAD: c = delta_{iG(x)} - p_i(x);  HVP: c = p_i(x) (u_i(x) - ubar(x)).
// Only the feature differences eta(x) - eta(c) are staged: the sum
// sum_x c eta(x) of a tile is sum_x c (eta(x) - eta(c)) + (sum_x c) eta(c),
// which reuses the operand the logit was formed from (and u = v.eta(c) +
// v.(eta(x) - eta(c)) for the HVP).  Rows lie kP2Stride floats apart, an
// odd number of 16-byte units, so that the producers' 16-byte stores of a
// warp hit distinct banks.  The float sums of kP2Flush tiles go into one
// double per grain and feature.
template <int KP>
__host__ __device__ constexpr int p2_stride() { return (KP / 4) % 2 == 0 ? KP + 4 : KP; }
constexpr int kP2Flush = 8;

template <int DIM, int D, bool HVP>
__device__ __forceinline__ void pass2_tiles_block(const Geom& g, const TileMap& tm, const int32_t* __restrict__ labels,
                                                  int N, const float* __restrict__ thH, const float* __restrict__ thL,
                                                  const float* __restrict__ vS, const float2* __restrict__ ecg,
                                                  const float2* __restrict__ refg, const float* __restrict__ lse,
                                                  const float* __restrict__ qin, const float* __restrict__ ubar,
                                                  const float* __restrict__ dmin, const int* __restrict__ mxin,
                                                  int64_t tpc, double* __restrict__ part, int64_t chunk, int gtile) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<float>(K);
  constexpr int RS = p2_stride<KP>();
  __shared__ __align__(16) float sde[kTilePix * RS];
  // per pixel: for the HVP one 16-byte word (log2 S, u_M - ubar, the
  // arg-max grain M, ubar); for the gradient log2 S, 1 - p_G and the label
  __shared__ float4 spx[HVP ? kTilePix : 1];
  __shared__ float slse[HVP ? 1 : kTilePix], sqv[HVP ? 1 : kTilePix];
  __shared__ int slab[HVP ? 1 : kTilePix];
  __shared__ float2 sec[K];
  __shared__ float2 sref;
  __shared__ double sacc[K * kGradThreads];

  const int i = gtile * kGradThreads + threadIdx.x;
  const bool vi = i < N;
  float th[K], vv[HVP ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    th[k] = vi ? thH[(int64_t)i * KP + k] : 0.f;
    if (HVP) vv[k] = vi ? vS[(int64_t)i * KP + k] : 0.f;
    sacc[k * kGradThreads + threadIdx.x] = 0.0;
  }
  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;
  const int64_t tb = chunk * tpc;
  const int64_t te = min(tb + tpc, tm.n_tiles);
  for (int64_t t = tb; t < te; ++t) {
    __syncthreads();
    {
      // row threadIdx.x of the tile (rows outside the set: log2 S = +inf
      // and no label, so that c = 0)
      float x[DIM], c[DIM], dx[DIM], dd[KP];
      const int64_t j = tile_pixel_dx<DIM>(g, tm, t, threadIdx.x, x, c, dx);
      legendre_delta<DIM, D>(x, c, dx, dd, nullptr);
#pragma unroll
      for (int k = K; k < KP; ++k) dd[k] = 0.f;
#pragma unroll
      for (int k = 0; k < KP; k += 4)
        *reinterpret_cast<float4*>(sde + threadIdx.x * RS + k) = make_float4(dd[k], dd[k + 1], dd[k + 2], dd[k + 3]);
      if (HVP)
        spx[threadIdx.x] = j >= 0 ? make_float4(lse[j], dmin[j], __int_as_float(mxin[j]), ubar[j])
                                  : make_float4(INFINITY, 0.f, __int_as_float(-1), 0.f);
      else {
        slse[threadIdx.x] = j >= 0 ? lse[j] : INFINITY;
        sqv[threadIdx.x] = j >= 0 ? qin[j] : 0.f;
        slab[threadIdx.x] = j >= 0 ? labels[j] : -1;
      }
      if (threadIdx.x < K) sec[threadIdx.x] = ecg[t * K + threadIdx.x];
      if (threadIdx.x == 0) sref = refg[t];
    }
    __syncthreads();
    // (the lo parts from L1 once per tile: registers are better spent on
    // the pixel loop)
    const float off = vi ? centre_offset<K>(th, thL + (int64_t)i * KP, sec, sref) : 0.f;
    float uc = 0.f;  // v_i . eta(c)
    if (HVP) {
#pragma unroll
      for (int k = 0; k < K; ++k) uc = fmaf(vv[k], sec[k].x, uc);
    }
    float cs = 0.f;  // sum of c over the tile
    auto coef = [&](int q, float l, const float* de) -> float {
      float cc;
      if (HVP) {
        const float4 px = spx[q];
        const float p = Arith<float>::ex(l - px.x);
        const bool own = __float_as_int(px.z) == i;
        // the arg-max grain's u_M - ubar from pass 1 (no cancellation near p_M = 1)
        const float u = uc + dot_k<K>(vv, de);
        cc = p * (own ? px.y : u - px.w);
      } else {
        // the label's c = 1 - p_G from pass 1 (no cancellation near p_G = 1)
        const float p = Arith<float>::ex(l - slse[q]);
        cc = slab[q] == i ? sqv[q] : -p;
      }
      return vi ? cc : 0.f;
    };
    // PS pixels a step: two independent chains where registers allow
    constexpr int PS = K <= 20 ? 2 : 1;
    for (int q = 0; q < kTilePix; q += PS) {
      float dq[PS][KP], cq[PS];
#pragma unroll
      for (int u = 0; u < PS; ++u) {
#pragma unroll
        for (int k = 0; k < KP; k += 4) {
          const float4 a = *reinterpret_cast<const float4*>(sde + (q + u) * RS + k);
          dq[u][k] = a.x;
          dq[u][k + 1] = a.y;
          dq[u][k + 2] = a.z;
          dq[u][k + 3] = a.w;
        }
      }
      bool nz = false;
#pragma unroll
      for (int u = 0; u < PS; ++u) {
        cq[u] = coef(q + u, off + dot_k<K>(th, dq[u]), dq[u]);
        nz |= cq[u] != 0.f;
      }
      if (__any_sync(0xffffffffu, nz)) {
#pragma unroll
        for (int u = 0; u < PS; ++u) {
#pragma unroll
          for (int k = 0; k < K; ++k) acc[k] = fmaf(cq[u], dq[u][k], acc[k]);
          cs += cq[u];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fmaf(cs, sec[k].x, acc[k]);
    if ((t - tb) % kP2Flush == kP2Flush - 1 || t == te - 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        sacc[k * kGradThreads + threadIdx.x] += (double)acc[k];
        acc[k] = 0.f;
      }
    }
  }
  if (vi) {
#pragma unroll
    for (int k = 0; k < K; ++k) part[(chunk * N + i) * K + k] = sacc[k * kGradThreads + threadIdx.x];
  }
  __syncthreads();  // the shared tiles may be reused by the next work item
}

template <int DIM, int D, bool HVP>
__global__ void __launch_bounds__(kGradThreads)
k_pass2_tiles(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, const float* __restrict__ thH,
              const float* __restrict__ thL, const float* __restrict__ vS, const float2* __restrict__ ecg,
              const float2* __restrict__ refg, const float* __restrict__ lse, const float* __restrict__ qin,
              const float* __restrict__ ubar, const float* __restrict__ dmin, const int* __restrict__ mxin,
              int64_t tpc, double* __restrict__ part) {
  pass2_tiles_block<DIM, D, HVP>(g, tm, labels, N, thH, thL, vS, ecg, refg, lse, qin, ubar, dmin, mxin, tpc, part,
                                 blockIdx.x, blockIdx.y);
}

// The same held to four blocks per SM, for the longer feature vectors
// (K > 15), where the compiler left free picks a slower schedule.
template <int DIM, int D, bool HVP>
__global__ void __launch_bounds__(kGradThreads, 4)
k_pass2_tiles_4(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, const float* __restrict__ thH,
              const float* __restrict__ thL, const float* __restrict__ vS, const float2* __restrict__ ecg,
              const float2* __restrict__ refg, const float* __restrict__ lse, const float* __restrict__ qin,
              const float* __restrict__ ubar, const float* __restrict__ dmin, const int* __restrict__ mxin,
              int64_t tpc, double* __restrict__ part) {
  pass2_tiles_block<DIM, D, HVP>(g, tm, labels, N, thH, thL, vS, ecg, refg, lse, qin, ubar, dmin, mxin, tpc, part,
                                 blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Arg-min assignment in double, smallest index on ties (eq. Li_def).
// ---------------------------------------------------------------------------
constexpr int kAssignThreads = 256;
constexpr int kAssignGT = 128;

template <int DIM, int D>
__global__ void __launch_bounds__(kAssignThreads)
k_assign(Geom g, int N, const double* __restrict__ theta, int32_t* __restrict__ out,
         double* __restrict__ gap, const int32_t* __restrict__ ref,
         unsigned long long* __restrict__ mismatch) {
  constexpr int K = basis_K(DIM, D);
  __shared__ double sth[kAssignGT * K];
  __shared__ int swarp[kAssignThreads / 32];
  const int64_t j = (int64_t)blockIdx.x * kAssignThreads + threadIdx.x;
  double x[DIM], eta[K];
  if (j < g.P) {
    pixel_coords<DIM>(g, j, x);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = 0.0;
  }
  legendre_features<DIM, D>(x, eta);
  double best = INFINITY, second = INFINITY;
  int bi = 0;
  for (int g0 = 0; g0 < N; g0 += kAssignGT) {
    const int gn = min(kAssignGT, N - g0);
    __syncthreads();
    for (int e = threadIdx.x; e < gn * K; e += kAssignThreads) sth[e] = theta[(int64_t)g0 * K + e];
    __syncthreads();
    for (int i = 0; i < gn; ++i) {
      const double h = dot_k<K>(sth + i * K, eta);
      if (h < best) {
        second = best;
        best = h;
        bi = g0 + i;
      } else if (h < second) {
        second = h;
      }
    }
  }
  int miss = 0;
  if (j < g.P) {
    out[j] = bi;
    if (gap) gap[j] = second - best;
    if (ref) miss = (ref[j] != bi);
  }
  if (mismatch) {
    const int wsum = __popc(__ballot_sync(0xffffffffu, miss));
    if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < kAssignThreads / 32; ++w) tot += swarp[w];
      if (tot) atomicAdd(mismatch, (unsigned long long)tot);
    }
  }
}

// ---------------------------------------------------------------------------
// Fast arg-min assignment: an fp32 pass with a certified margin, double
// precision for the pixels where the margin is not met.
//
// |P_m| <= 1 on [-1, 1], so every feature satisfies |eta_k(x)| <= 1 and
// every h_i(x) = theta_i . eta(x) computed in fp32 (fp32 parameters, fp32
// features from the recurrence, an fma chain) lies within
//   E = C 2^-24 max_i sum_k |theta_ik|,  C = 2 (K + 8 D + 8),
// of its exact value (the dot product contributes about K units of
// rounding, the rounding of theta one, the recurrence and the tensor
// products at most about 8 (D + 1); C doubles that).  A pixel whose fp32
// best and second-best values are more than 2E apart has the same arg-min
// in exact arithmetic, hence in double: its fp32 label is final.  The others
// are listed and assigned by the double-precision arg-min (smallest index on
// ties), so every label equals that of the double-precision kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_assign_prep(const double* __restrict__ theta, int N, int K, int KP, float* __restrict__ th32,
              float* __restrict__ margin, int* __restrict__ count, float c_bound) {
  __shared__ double smax[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double l1 = 0.0;
    for (int k = 0; k < K; ++k) l1 += fabs(theta[(int64_t)i * K + k]);
    m = fmax(m, l1);
  }
  for (int64_t q = threadIdx.x; q < (int64_t)N * KP; q += blockDim.x) {
    const int i = (int)(q / KP), k = (int)(q % KP);
    th32[q] = k < K ? (float)theta[(int64_t)i * K + k] : 0.f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, smax[w]);
    // twice the bound E (the two values compared), rounded up; NaN parameters
    // make it NaN, and no pixel is certified
    *margin = (float)(2.0 * c_bound * ldexp(mx, -24) * (1.0 + 1e-6));
    *count = 0;
  }
}

template <int DIM, int D>
__global__ void __launch_bounds__(kAssignThreads)
k_assign32(Geom g, int N, const float* __restrict__ th32, const float* __restrict__ margin, int32_t* __restrict__ out,
           const int32_t* __restrict__ ref, unsigned long long* __restrict__ mismatch, int* __restrict__ list,
           int* __restrict__ count) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<float>(K);
  __shared__ __align__(16) float sth[kAssignGT * KP];
  __shared__ int swarp[kAssignThreads / 32];
  const int64_t j = (int64_t)blockIdx.x * kAssignThreads + threadIdx.x;
  float x[DIM], eta[K];
  if (j < g.P) {
    pixel_coords<DIM>(g, j, x);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = 0.f;
  }
  legendre_features<DIM, D>(x, eta);
  float best = INFINITY, second = INFINITY;
  int bi = 0;
  for (int g0 = 0; g0 < N; g0 += kAssignGT) {
    const int gn = min(kAssignGT, N - g0);
    __syncthreads();
    {
      const uint4* src = reinterpret_cast<const uint4*>(th32 + (int64_t)g0 * KP);
      uint4* dst = reinterpret_cast<uint4*>(sth);
      for (int e = threadIdx.x; e < gn * KP / 4; e += kAssignThreads) dst[e] = src[e];
    }
    __syncthreads();
    for (int i = 0; i < gn; ++i) {
      const float h = dot_k<K>(sth + i * KP, eta);
      if (h < best) {
        second = best;
        best = h;
        bi = g0 + i;
      } else if (h < second) {
        second = h;
      }
    }
  }
  int miss = 0;
  if (j < g.P) {
    if (second - best > *margin) {  // certified (false for NaN)
      out[j] = bi;
      if (ref) miss = ref[j] != bi;
    } else {
      list[atomicAdd(count, 1)] = (int)j;
    }
  }
  if (mismatch) {
    const int wsum = __popc(__ballot_sync(0xffffffffu, miss));
    if ((threadIdx.x & 31) == 0) swarp[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < kAssignThreads / 32; ++w) tot += swarp[w];
      if (tot) atomicAdd(mismatch, (unsigned long long)tot);
    }
  }
}

// The listed pixels by the double-precision arg-min (one thread a pixel,
// parameters from the caches; a grid-stride loop over the device count).
template <int DIM, int D>
__global__ void __launch_bounds__(256)
k_assign64_list(Geom g, int N, const double* __restrict__ theta, const int* __restrict__ list,
                const int* __restrict__ count, int32_t* __restrict__ out, const int32_t* __restrict__ ref,
                unsigned long long* __restrict__ mismatch) {
  constexpr int K = basis_K(DIM, D);
  const int n = *count;
  int miss = 0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int64_t j = list[q];
    double x[DIM], eta[K];
    pixel_coords<DIM>(g, j, x);
    legendre_features<DIM, D>(x, eta);
    double best = INFINITY;
    int bi = 0;
    for (int i = 0; i < N; ++i) {
      const double h = dot_k<K>(theta + (int64_t)i * K, eta);
      if (h < best) {
        best = h;
        bi = i;
      }
    }
    out[j] = bi;
    if (ref) miss += ref[j] != bi;
  }
  if (mismatch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) miss += __shfl_down_sync(0xffffffffu, miss, o);
    if ((threadIdx.x & 31) == 0 && miss) atomicAdd(mismatch, (unsigned long long)miss);
  }
}

// ---------------------------------------------------------------------------
// Features (testing aid): eta_out[j][k].
// ---------------------------------------------------------------------------
template <typename T, int DIM, int D>
__global__ void k_features(Geom g, T* __restrict__ out) {
  constexpr int K = basis_K(DIM, D);
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= g.P) return;
  T x[DIM], eta[K];
  pixel_coords<DIM>(g, j, x);
  legendre_features<DIM, D>(x, eta);
#pragma unroll
  for (int k = 0; k < K; ++k) out[j * K + k] = eta[k];
}

// ---------------------------------------------------------------------------
// Grain moments in 64-bit fixed point (exact, order independent).
// ---------------------------------------------------------------------------
template <int DIM, int DM>
__global__ void k_moments(Geom g, const int32_t* __restrict__ labels, int N, double fx_scale,
                          unsigned long long* __restrict__ mom, unsigned long long* __restrict__ cnt) {
  constexpr int K = basis_K(DIM, DM);
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = j < g.P;
  int G = valid ? labels[j] : -1;
  if (G < 0 || G >= N) G = -1;
  double x[DIM], eta[K];
  if (valid) {
    pixel_coords<DIM>(g, j, x);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = 0.0;
  }
  legendre_features<DIM, DM>(x, eta);
  long long fx[K];
#pragma unroll
  for (int k = 0; k < K; ++k) fx[k] = (G >= 0) ? __double2ll_rn(eta[k] * fx_scale) : 0ll;
  // warp aggregation when the whole warp shares one label (common: grains
  // are spatially coherent); integer sums keep the result order independent
  const int G0 = __shfl_sync(0xffffffffu, G, 0);
  const bool uniform = __all_sync(0xffffffffu, G == G0) && G0 >= 0;
  if (uniform) {
    unsigned long long c = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      long long v = fx[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) atomicAdd(&mom[(int64_t)G0 * K + k], (unsigned long long)v);
    }
    c = 32;
    if ((threadIdx.x & 31) == 0) atomicAdd(&cnt[G0], c);
  } else if (G >= 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) atomicAdd(&mom[(int64_t)G * K + k], (unsigned long long)fx[k]);
    atomicAdd(&cnt[G], 1ull);
  }
}

static __global__ void k_moments_final(const unsigned long long* __restrict__ mom, int64_t n, double inv_scale,
                                double* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = (double)(long long)mom[q] * inv_scale;
}

static __global__ void k_check_labels(const int32_t* __restrict__ labels, int64_t P, int N, int* __restrict__ bad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool b = j < P && (labels[j] < 0 || labels[j] >= N);
  if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// ===========================================================================
// Launch of one objective/gradient or HVP evaluation for a fixed
// (precision, dimension, degree).
// ===========================================================================
inline int chunks_for(int64_t P, int grain_tiles, int sms) {
  int64_t tiles = (P + kPixTile - 1) / kPixTile;
  int64_t want = ((int64_t)sms * 6 + grain_tiles - 1) / grain_tiles;
  if (want < 1) want = 1;
  if (want > tiles) want = tiles;
  return (int)want;
}

// Launches of one FP32 tile evaluation into caller-provided scratch:
// parameters thH/thL/vS [N][KP], centre features ec [tiles][K], reference
// logits ref [tiles], lse [P], qv [P] (1 - p_G of the label, or u_M -
// ubar of the arg-max grain for the HVP), ubar and mx (the arg-max grain)
// [P], objective partials objp [tiles / kT1Tiles], gradient partials part
// [chunks][N][K].  Shared by the allocating and the allocation-free entry
// points.
template <int DIM, int D>
int launch_simt_tiles(const EvalCall& c, const TileMap& tm, float* thH, float* thL, float* vS, float2* ec,
                      float2* ref, float* lse, float* qv, float* ubar, int* mx, double* objp, double* part,
                      int64_t tpc, cudaStream_t st) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<float>(K);
  const int N = c.N;
  const int64_t P = c.g.P;
  const bool hvp = c.v != nullptr;
  const bool want_grad = c.grad != nullptr;
  const int64_t n_tiles = tm.n_tiles;
  const int64_t blocks1 = (n_tiles + kT1Tiles - 1) / kT1Tiles;
  const int gtiles = (N + kGradThreads - 1) / kGradThreads;
  const int nch = (int)((n_tiles + tpc - 1) / tpc);
  const int64_t nth = (int64_t)N * KP;
  PD_TIMED(st, "theta_ff",
           k_theta_ff<<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(c.theta, N, K, KP,
                                                                      Arith<float>::theta_scale(c.eps), thH, thL));
  if (hvp)
    PD_TIMED(st, "scale_theta", k_copy_pad<float><<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(c.v, N, K, KP, vS));
  if (!(c.plan && c.plan->features))
    PD_TIMED(st, "centre_features",
             (k_centre_features<DIM, D><<<centre_feature_blocks(n_tiles), kFeatThreads, 0, st>>>(c.g, tm, ec)));
  PD_TIMED(st, "tile_refs",
           (k_tile_refs<K><<<tile_centre_blocks(n_tiles), kRefThreads, 0, st>>>(thH, N, n_tiles, ec, ref)));
  const dim3 grid2(nch, gtiles);
  if (hvp) {
    PD_TIMED(st, "simt_hvp_pass1",
             (k_pass1_tiles<DIM, D, true><<<(unsigned)blocks1, kLseThreads, 0, st>>>(
                 c.g, tm, c.labels, N, thH, thL, vS, ec, ref, lse, nullptr, ubar, qv, mx, nullptr)));
    PD_TIMED(st, "simt_hvp_pass2",
             (k_pass2_tiles<DIM, D, true><<<grid2, kGradThreads, 0, st>>>(c.g, tm, c.labels, N, thH, thL, vS, ec, ref,
                                                                         lse, nullptr, ubar, qv, mx, tpc, part)));
  } else {
    auto k1 = k_pass1_tiles<DIM, D, false>;
    if constexpr (K > 28) k1 = k_pass1_tiles_2<DIM, D, false>;
    PD_TIMED(st, "simt_lse_pass1",
             (k1<<<(unsigned)blocks1, kLseThreads, 0, st>>>(c.g, tm, c.labels, N, thH, thL, nullptr, ec, ref, lse,
                                                             want_grad ? qv : nullptr, nullptr, nullptr, nullptr,
                                                             objp)));
    if (want_grad) {
      auto k2 = k_pass2_tiles<DIM, D, false>;
      if constexpr (K > 15) k2 = k_pass2_tiles_4<DIM, D, false>;
      PD_TIMED(st, "simt_grad_pass2",
               (k2<<<grid2, kGradThreads, 0, st>>>(c.g, tm, c.labels, N, thH, thL, nullptr, ec, ref, lse, qv,
                                                    nullptr, nullptr, nullptr, tpc, part)));
    }
  }
  if (c.obj && !hvp)
    PD_TIMED(st, "reduce_obj", k_reduce_obj<<<1, 1024, 0, st>>>(objp, (int)blocks1, 1.0 / (double)P, c.obj));
  if (want_grad || hvp) {
    const int64_t NK = (int64_t)N * K;
    const double scale = hvp ? -1.0 / (c.eps * c.eps * (double)P) : -1.0 / (c.eps * (double)P);
    PD_TIMED(st, "reduce_parts",
             k_reduce_parts<<<(unsigned)((NK + 31) / 32), dim3(32, kRedPhases), 0, st>>>(part, nch, NK, scale,
                                                                                       hvp ? c.hv : c.grad));
  }
  if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
  if (c.plan) c.plan->features = true;
  return PD_OK;
}

// Tiles per pass-2 chunk: about 6 CTAs per SM over the grain tiles.
inline int64_t tiles_per_chunk(int64_t n_tiles, int grain_tiles, int sms, int factor = 6) {
  int64_t want = ((int64_t)sms * factor + grain_tiles - 1) / grain_tiles;
  want = std::max<int64_t>(1, std::min<int64_t>(want, n_tiles));
  return (n_tiles + want - 1) / want;
}

// The FP32 evaluation on tiles (objective/gradient or HVP).
template <int DIM, int D>
int eval_simt_tiles(const EvalCall& c, cudaStream_t st) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<float>(K);
  const int N = c.N;
  const int64_t P = c.g.P;
  const bool hvp = c.v != nullptr;
  const bool want_grad = c.grad != nullptr;
  const int sms = device_sm_count();
  const TileMap tm = make_tiles<DIM>(c.g);
  const int64_t n_tiles = tm.n_tiles;
  const int64_t blocks1 = (n_tiles + kT1Tiles - 1) / kT1Tiles;
  const int gtiles = (N + kGradThreads - 1) / kGradThreads;
  const int64_t tpc = tiles_per_chunk(n_tiles, gtiles, sms);
  const int nch = (int)((n_tiles + tpc - 1) / tpc);

  // (a plan makes every allocation on every call, so that its arena keeps
  // the centre features at the same place)
  const bool all = c.plan != nullptr;
  Scratch sc(st, c.plan);
  float* thH = sc.get<float>((size_t)N * KP);
  float* thL = sc.get<float>((size_t)N * KP);
  float* vS = hvp ? sc.get<float>((size_t)N * KP) : nullptr;
  float2* ec = sc.get<float2>((size_t)n_tiles * K);
  float2* ref = sc.get<float2>((size_t)n_tiles);
  float* lse = (want_grad || hvp || all) ? sc.get<float>((size_t)P) : nullptr;
  float* qv = (want_grad || hvp || all) ? sc.get<float>((size_t)P) : nullptr;  // 1 - p_G, or u_M - ubar
  float* ubar = hvp ? sc.get<float>((size_t)P) : nullptr;
  int* mx = hvp ? sc.get<int>((size_t)P) : nullptr;  // the arg-max grain of each pixel (HVP)
  double* objp = (!hvp && (c.obj || all)) ? sc.get<double>((size_t)blocks1) : nullptr;
  double* part = (want_grad || hvp || all) ? sc.get<double>((size_t)nch * N * K) : nullptr;
  if (!sc.ok()) return PD_ENOMEM;
  if (sc.sizing()) {
    c.plan->need = sc.used();
    return PD_OK;
  }
  if (!c.obj) objp = nullptr;
  return launch_simt_tiles<DIM, D>(c, tm, thH, thL, vS, ec, ref, lse, qv, ubar, mx, objp, part, tpc, st);
}

template <typename T, int DIM, int D>
int eval_simt_dd(const EvalCall& c, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) return eval_simt_tiles<DIM, D>(c, st);
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<T>(K);
  const int N = c.N;
  const int64_t P = c.g.P;
  const bool hvp = c.v != nullptr;
  const bool want_grad = c.grad != nullptr;
  const int sms = device_sm_count();

  constexpr int ppt = 2;
  const int blocks1 = (int)((P + kLseThreads * ppt - 1) / (kLseThreads * ppt));
  const int gtiles = (N + kGradThreads - 1) / kGradThreads;
  const int nch = chunks_for(P, gtiles, sms);
  const int64_t tiles = (P + kPixTile - 1) / kPixTile;
  const int64_t ppc = ((tiles + nch - 1) / nch) * kPixTile;
  const int nch_eff = (int)((P + ppc - 1) / ppc);

  const bool all = c.plan != nullptr;  // a plan makes every allocation on every call
  Scratch sc(st, c.plan);
  T* thS = sc.get<T>((size_t)N * KP);
  T* vS = hvp ? sc.get<T>((size_t)N * KP) : nullptr;
  T* lse = (want_grad || hvp || all) ? sc.get<T>((size_t)P) : nullptr;
  T* ubar = hvp ? sc.get<T>((size_t)P) : nullptr;
  double* objp = (!hvp && (c.obj || all)) ? sc.get<double>((size_t)blocks1) : nullptr;
  double* part = (want_grad || hvp || all) ? sc.get<double>((size_t)nch_eff * N * K) : nullptr;
  if (!sc.ok()) return PD_ENOMEM;
  if (sc.sizing()) {
    c.plan->need = sc.used();
    return PD_OK;
  }

  const double tscale = Arith<T>::theta_scale(c.eps);
  const int64_t nth = (int64_t)N * KP;
  PD_TIMED(st, "scale_theta", k_scale_theta<T><<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(c.theta, N, K, KP, tscale, thS));
  if (hvp) {
    PD_TIMED(st, "scale_theta", k_copy_pad<T><<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(c.v, N, K, KP, vS));
    PD_TIMED(st, "simt_hvp_pass1", k_pass1<T, DIM, D, ppt, true><<<blocks1, kLseThreads, 0, st>>>(c.g, c.labels, N, thS, vS, lse, ubar, nullptr));
    dim3 grid2(nch_eff, gtiles);
    PD_TIMED(st, "simt_hvp_pass2", k_pass2<T, DIM, D, true><<<grid2, kGradThreads, 0, st>>>(c.g, c.labels, N, thS, vS, lse, ubar, ppc, part));
  } else {
    PD_TIMED(st, "simt_lse_pass1", k_pass1<T, DIM, D, ppt, false><<<blocks1, kLseThreads, 0, st>>>(c.g, c.labels, N, thS, nullptr, lse, nullptr, objp));
    if (want_grad) {
      dim3 grid2(nch_eff, gtiles);
      PD_TIMED(st, "simt_grad_pass2", k_pass2<T, DIM, D, false><<<grid2, kGradThreads, 0, st>>>(c.g, c.labels, N, thS, nullptr, lse, nullptr, ppc, part));
    }
  }
  if (c.obj && !hvp) PD_TIMED(st, "reduce_obj", k_reduce_obj<<<1, 1024, 0, st>>>(objp, blocks1, 1.0 / (double)P, c.obj));
  if (want_grad || hvp) {
    const int64_t NK = (int64_t)N * K;
    const double scale = hvp ? -1.0 / (c.eps * c.eps * (double)P) : -1.0 / (c.eps * (double)P);
    PD_TIMED(st, "reduce_parts", k_reduce_parts<<<(unsigned)((NK + 31) / 32), dim3(32, kRedPhases), 0, st>>>(part, nch_eff, NK, scale, hvp ? c.hv : c.grad));
  }
  if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
  return PD_OK;
}

}  // namespace
}  // namespace pd
