// pd_tiles.cuh -- pixel tiles and tile-centred logits, shared by the CUDA-core
// (FP32) and tensor-core evaluations.
//
// A tile is 128 pixels that are close in space: a 16 x 8 block of a 2-D grid,
// an 8 x 4 x 4 block of a 3-D grid, or 128 consecutive points of a point
// list.  Every logit of a pixel x in tile t is formed relative to the tile's
// centre c and to one reference logit C(t) of the tile:
//
//   l_i(x) - C(t) = [theta'_i . eta(c) - C(t)] + theta'_i . (eta(x) - eta(c)),
//
// theta' = -theta log2(e) / eps.  Subtracting one constant from all logits
// of a pixel changes neither p_i(x) nor log p_{G(x)}(x) (the log-sum-exp of
// eq. log-res-2 moves with it), so every quantity the evaluation keeps in
// float -- logits, log S, their differences -- is small: the large parts
// theta'_i . eta(c) (|theta|/eps reaches 1e3 and more) are formed in
// float-float arithmetic once per (tile, grain) and enter only through their
// difference with C(t), rounded once.  C(t) is the centre logit of the grain
// whose fp32 centre logit is largest (the smallest index on ties).
//
// The remainder is formed from eta(x) - eta(c) computed by a recurrence for
// the differences D_m = P_m(x) - P_m(c) themselves,
//   (m+1) D_{m+1} = (2m+1) (x D_m + (x - c) P_m(c)) - m D_{m-1},
//   D_0 = 0, D_1 = x - c,
// which follows from the three-term recurrence of Sec. 3.3 and keeps the
// relative accuracy of the small differences (their float difference would
// lose it), and the tensor products
//   psi_a(x) - psi_a(c) = sum_axes (prod of P(c) before) D (prod of P(x) after).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "pd_common.cuh"

namespace pd {
namespace {

constexpr int kTilePix = 128;  // pixels per tile

struct TileMap {
  int ntx, nty, ntz;      // tiles per axis (structured grids)
  int64_t n_tiles;
  int n0, n1, n2;         // grid sides
  float f0, f1, f2;       // 1 / n_a rounded to float
};

template <int DIM>
struct TileShape {
  static constexpr int X = DIM == 2 ? 16 : 8;
  static constexpr int Y = DIM == 2 ? 8 : 4;
  static constexpr int Z = DIM == 2 ? 1 : 4;
};

template <int DIM>
TileMap make_tiles(const Geom& g) {
  TileMap tm{1, 1, 1, 0, 1, 1, 1, 1.f, 1.f, 1.f};
  if (g.coords) {
    tm.n_tiles = (g.P + kTilePix - 1) / kTilePix;
    return tm;
  }
  using TS = TileShape<DIM>;
  tm.ntx = (int)((g.n0 + TS::X - 1) / TS::X);
  tm.nty = (int)((g.n1 + TS::Y - 1) / TS::Y);
  tm.ntz = DIM == 3 ? (int)((g.n2 + TS::Z - 1) / TS::Z) : 1;
  tm.n_tiles = (int64_t)tm.ntx * tm.nty * tm.ntz;
  tm.n0 = (int)g.n0;
  tm.n1 = (int)g.n1;
  tm.n2 = (int)g.n2;
  tm.f0 = (float)(1.0 / (double)g.n0);
  tm.f1 = (float)(1.0 / (double)g.n1);
  tm.f2 = (float)(1.0 / (double)g.n2);
  return tm;
}

// Integer position of row r of tile t and of the tile's centre pixel
// (structured grids).  The centre pixel is the middle of the tile, moved
// back to the grid's last pixel along an axis where the middle lies outside
// the grid (a ragged tile only): the centre then stays in [-1, 1], where
// |P_m| <= 1.  Outside, P_m grows like x^m, and on a grid narrower than a
// tile (a single pixel: x = 0 against a middle at 16) the centre logits and
// the remainders would be large terms that cancel in float.  Full tiles,
// the only ones the tile bounds are taken for, keep their middle.
template <int DIM>
__device__ __forceinline__ void tile_ints(const TileMap& tm, int64_t t, int r, int* k, int* kc) {
  using TS = TileShape<DIM>;
  const unsigned tt = (unsigned)t;
  const unsigned tx = tt % (unsigned)tm.ntx;
  const unsigned rest = tt / (unsigned)tm.ntx;
  const int ty = (int)(rest % (unsigned)tm.nty);
  const int tz = (int)(rest / (unsigned)tm.nty);
  kc[0] = min((int)tx * TS::X + TS::X / 2, tm.n0 - 1);
  kc[1] = min(ty * TS::Y + TS::Y / 2, tm.n1 - 1);
  k[0] = (int)tx * TS::X + (r % TS::X);
  k[1] = ty * TS::Y + ((r / TS::X) % TS::Y);
  if (DIM == 3) {
    kc[2] = min(tz * TS::Z + TS::Z / 2, tm.n2 - 1);
    k[2] = tz * TS::Z + (r / (TS::X * TS::Y));
  }
}

// Pixel index of row r of tile t (or -1 outside the pixel set), its
// coordinates x and the coordinates of the tile centre c, in fp32.  A
// coordinate -1 + (2k+1)/n is formed as the exact integer 2k+1-n times the
// float 1/n (exact when n is a power of two, else within an ulp); every pass
// uses this same function, so the log-sum-exp of pass 1 belongs to the very
// points of pass 2.  Rows outside the set get x = c.
template <int DIM>
__device__ __forceinline__ int64_t tile_pixel(const Geom& g, const TileMap& tm, int64_t t, int r, float* x,
                                              float* c) {
  if (g.coords) {
    const int64_t j0 = t * kTilePix;
#pragma unroll
    for (int a = 0; a < DIM; ++a) c[a] = (float)g.coords[j0 * DIM + a];
    const int64_t j = j0 + r;
    if (j >= g.P) {
#pragma unroll
      for (int a = 0; a < DIM; ++a) x[a] = c[a];
      return -1;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = (float)g.coords[j * DIM + a];
    return j;
  }
  int k[3], kc[3];
  tile_ints<DIM>(tm, t, r, k, kc);
  const float f[3] = {tm.f0, tm.f1, tm.f2};
  const int n[3] = {tm.n0, tm.n1, tm.n2};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    c[a] = (float)(2 * kc[a] + 1 - n[a]) * f[a];
    x[a] = (float)(2 * k[a] + 1 - n[a]) * f[a];
  }
  if (k[0] >= tm.n0 || k[1] >= tm.n1 || (DIM == 3 && k[2] >= tm.n2)) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = c[a];
    return -1;
  }
  return DIM == 2 ? k[0] + (int64_t)tm.n0 * k[1] : k[0] + (int64_t)tm.n0 * (k[1] + (int64_t)tm.n1 * k[2]);
}

// As tile_pixel, plus dx = x - c: the exact integer 2 (k - k_c) times 1/n
// on grids, the double difference rounded once on point lists (so that dx
// keeps its relative accuracy when x and c are close).  Rows outside the
// set get x = c, dx = 0.
template <int DIM>
__device__ __forceinline__ int64_t tile_pixel_dx(const Geom& g, const TileMap& tm, int64_t t, int r, float* x,
                                                 float* c, float* dx) {
  if (g.coords) {
    const int64_t j0 = t * kTilePix;
    const int64_t j = j0 + r;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const double cd = g.coords[j0 * DIM + a];
      const double xd = j < g.P ? g.coords[j * DIM + a] : cd;
      c[a] = (float)cd;
      x[a] = (float)xd;
      dx[a] = (float)(xd - cd);
    }
    return j < g.P ? j : -1;
  }
  int k[3], kc[3];
  tile_ints<DIM>(tm, t, r, k, kc);
  const float f[3] = {tm.f0, tm.f1, tm.f2};
  const int n[3] = {tm.n0, tm.n1, tm.n2};
  const bool out = k[0] >= tm.n0 || k[1] >= tm.n1 || (DIM == 3 && k[2] >= tm.n2);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    c[a] = (float)(2 * kc[a] + 1 - n[a]) * f[a];
    x[a] = out ? c[a] : (float)(2 * k[a] + 1 - n[a]) * f[a];
    dx[a] = out ? 0.f : (float)(2 * (k[a] - kc[a])) * f[a];
  }
  if (out) return -1;
  return DIM == 2 ? k[0] + (int64_t)tm.n0 * k[1] : k[0] + (int64_t)tm.n0 * (k[1] + (int64_t)tm.n1 * k[2]);
}

// The tile centre in double: -1 + (2 k_c + 1) / n on grids, the tile's first
// point on point lists.
template <int DIM>
__device__ __forceinline__ void tile_centre(const Geom& g, const TileMap& tm, int64_t t, double* c) {
  if (g.coords) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) c[a] = g.coords[t * kTilePix * DIM + a];
    return;
  }
  int k[3], kc[3];
  tile_ints<DIM>(tm, t, 0, k, kc);
  const int64_t n[3] = {g.n0, g.n1, g.n2};
#pragma unroll
  for (int a = 0; a < DIM; ++a) c[a] = -1.0 + (2.0 * (double)kc[a] + 1.0) / (double)n[a];
}

// ---------------------------------------------------------------------------
// Feature differences eta(x) - eta(c) (see the file comment) and the
// features eta(x), in float.
// ---------------------------------------------------------------------------
template <int DIM, int D, int k>
__device__ __forceinline__ float delta_product(const float (&Px)[DIM][D + 1], const float (&Pc)[DIM][D + 1],
                                               const float (&Dm)[DIM][D + 1]) {
  constexpr int e0 = basis_exp(DIM, D, k, 0);
  constexpr int e1 = basis_exp(DIM, D, k, 1);
  constexpr int e2 = basis_exp(DIM, D, k, 2);
  if constexpr (DIM == 2) {
    return fmaf(Dm[0][e0], Px[1][e1], Pc[0][e0] * Dm[1][e1]);
  } else {
    const float t2 = Pc[0][e0] * Pc[1][e1] * Dm[2][e2];
    const float t1 = fmaf(Pc[0][e0] * Dm[1][e1], Px[2][e2], t2);
    return fmaf(Dm[0][e0] * Px[1][e1], Px[2][e2], t1);
  }
}

template <int DIM, int D, int... Ks>
__device__ __forceinline__ void delta_all(const float (&Px)[DIM][D + 1], const float (&Pc)[DIM][D + 1],
                                          const float (&Dm)[DIM][D + 1], float* de, float* eta,
                                          std::integer_sequence<int, Ks...>) {
  ((de[Ks] = delta_product<DIM, D, Ks>(Px, Pc, Dm)), ...);
  if (eta) ((eta[Ks] = basis_product<DIM, D, Ks>(Px)), ...);
}

// de[k] = psi_k(x) - psi_k(c) from x, c and dx = x - c; eta (if not null)
// receives psi_k(x).
template <int DIM, int D>
__device__ __forceinline__ void legendre_delta(const float* x, const float* c, const float* dx, float* de,
                                               float* eta) {
  float Px[DIM][D + 1], Pc[DIM][D + 1], Dm[DIM][D + 1];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    Px[a][0] = 1.f;
    Pc[a][0] = 1.f;
    Dm[a][0] = 0.f;
    if (D >= 1) {
      Px[a][1] = x[a];
      Pc[a][1] = c[a];
      Dm[a][1] = dx[a];
    }
#pragma unroll
    for (int m = 1; m < D; ++m) {
      const float inv = 1.f / (float)(m + 1);
      Px[a][m + 1] = ((float)(2 * m + 1) * x[a] * Px[a][m] - (float)m * Px[a][m - 1]) * inv;
      Pc[a][m + 1] = ((float)(2 * m + 1) * c[a] * Pc[a][m] - (float)m * Pc[a][m - 1]) * inv;
      Dm[a][m + 1] = ((float)(2 * m + 1) * fmaf(x[a], Dm[a][m], dx[a] * Pc[a][m]) - (float)m * Dm[a][m - 1]) * inv;
    }
  }
  delta_all<DIM, D>(Px, Pc, Dm, de, eta, std::make_integer_sequence<int, basis_K(DIM, D)>{});
}

// ---------------------------------------------------------------------------
// Float-float arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2).  Every
// operation is an explicitly rounded intrinsic, so that the compiler cannot
// contract the error-free transformations into fused multiply-adds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Compensated dot product sum_k (ah_k + al_k)(bh_k + bl_k) as hi + lo: the
// leading products exactly (product and fma residue), the cross terms in
// float, the running sum by two-sum.
template <int K>
__device__ __forceinline__ float2 ff_dot(const float* ah, const float* al, const float2* b) {
  float s = 0.f, e = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float p = __fmul_rn(ah[k], b[k].x);
    const float pe = __fmaf_rn(ah[k], b[k].x, -p);
    float t, te;
    ff_two_sum(s, p, t, te);
    s = t;
    const float cross = __fmaf_rn(al[k], b[k].x, __fmul_rn(ah[k], b[k].y));
    e = __fadd_rn(e, __fadd_rn(te, __fadd_rn(pe, cross)));
  }
  float hi, lo;
  ff_two_sum(s, e, hi, lo);
  return make_float2(hi, lo);
}

// (a - r) rounded to float, a and r float-float.
__device__ __forceinline__ float ff_diff(float2 a, float2 r) {
  float d, de;
  ff_two_sum(a.x, -r.x, d, de);
  return __fadd_rn(d, __fadd_rn(de, __fsub_rn(a.y, r.y)));
}

// Scaled parameters theta' = theta * scale as a float-float pair per entry,
// rows padded to KP: hi[i][k] = fl(theta'), lo[i][k] = fl(theta' - hi).
__global__ void k_theta_ff(const double* __restrict__ theta, int N, int K, int KP, double scale,
                           float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)N * KP) return;
  const int i = (int)(q / KP), k = (int)(q % KP);
  const double v = k < K ? theta[(int64_t)i * K + k] * scale : 0.0;
  const float h = (float)v;
  hi[q] = h;
  lo[q] = (float)(v - (double)h);
}

// ---------------------------------------------------------------------------
// Per tile: eta(c) as float-float pairs (from the double centre) and the
// reference logit C(t).  C(t) only has to be one constant shared by all
// grains of the tile: it is the largest fp32 centre logit hi . fl(eta(c))
// over all grains, an exact float (lo part zero), so that the offsets of
// the grains that matter on the tile are small.  A block takes kRefTiles
// tiles.  Warp maxima use redux.sync on order-preserving integer images of
// the floats, and the block maximum an atomicMax in shared memory: the
// result does not depend on the order of the atomics.
// ---------------------------------------------------------------------------
constexpr int kRefTiles = 8;
constexpr int kRefThreads = 256;

struct TileBound {
  float d[32];  // D_k: |eta_k(x) - eta_k(c)| <= D_k inside a tile (structured grids)
};

__device__ __forceinline__ uint32_t ord_f32(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// The centre features eta(c_t) of every tile as float-float pairs, ec
// [tiles][K]: one thread per tile runs the Legendre recurrence of each axis
// in double (FP64 is slow on this part: once per axis, not per feature)
// and forms the products.  They depend on the pixel set only.  Small blocks
// (kFeatThreads) spread the double-precision work over all SMs.
constexpr int kFeatThreads = 32;
template <int DIM, int D>
__global__ void __launch_bounds__(kFeatThreads) k_centre_features(Geom g, TileMap tm, float2* __restrict__ ec) {
  constexpr int K = basis_K(DIM, D);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tm.n_tiles) return;
  double c[DIM], P[DIM][D + 1];
  tile_centre<DIM>(g, tm, t, c);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    P[a][0] = 1.0;
    if (D >= 1) P[a][1] = c[a];
#pragma unroll
    for (int m = 1; m < D; ++m) P[a][m + 1] = ((2.0 * m + 1.0) * c[a] * P[a][m] - (double)m * P[a][m - 1]) * (1.0 / (m + 1.0));
  }
  double eta[K];
  basis_all<DIM, D>(P, eta, std::make_integer_sequence<int, K>{});
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float h = (float)eta[k];
    ec[t * K + k] = make_float2(h, (float)(eta[k] - (double)h));
  }
}

inline unsigned centre_feature_blocks(int64_t n_tiles) {
  return (unsigned)((n_tiles + kFeatThreads - 1) / kFeatThreads);
}

// The centre features of tiles t0 .. t0+nt-1 from ec into shared memory:
// float-float pairs sec[q][k] and hi parts sech[q][k] (rows padded to a
// multiple of 4 for vector loads).  Ends with a barrier.
template <int K>
__device__ __forceinline__ void load_centre_features(const float2* __restrict__ ec, int64_t t0, int nt,
                                                     float2 (*sec)[K], float (*sech)[padded_K<float>(K)]) {
  constexpr int KP = padded_K<float>(K);
  for (int e = threadIdx.x; e < nt * KP; e += blockDim.x) {
    const int q = e / KP, k = e % KP;
    const float2 f = k < K ? ec[(t0 + q) * K + k] : make_float2(0.f, 0.f);
    if (k < K) sec[q][k] = f;
    sech[q][k] = f.x;
  }
  __syncthreads();
}

// fp32 centre logit hi_i . fl(eta(c)): parameters in registers (padded
// row), features from a padded shared row (16-byte aligned, vector loads).
template <int K>
__device__ __forceinline__ float centre_dot32(const float (&h)[padded_K<float>(K)], const float* __restrict__ e) {
  constexpr int KP = padded_K<float>(K);
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < KP; k += 4) {
    const float4 b = *reinterpret_cast<const float4*>(e + k);
    acc = fmaf(h[k], b.x, acc);
    if (k + 1 < K) acc = fmaf(h[k + 1], b.y, acc);
    if (k + 2 < K) acc = fmaf(h[k + 2], b.z, acc);
    if (k + 3 < K) acc = fmaf(h[k + 3], b.w, acc);
  }
  return acc;
}

// Block maximum over all grains of their fp32 centre logit on each of the
// nt tiles, into smax[q] (order-preserving bits; 0 = nothing).  Ends with a
// barrier.  thH: [N][KP] parameters (rows 16-byte aligned).
template <int K>
__device__ __forceinline__ void centre_max_block(const float* __restrict__ thH, int N, int nt,
                                                 const float (*sech)[padded_K<float>(K)], uint32_t* smax) {
  constexpr int KP = padded_K<float>(K);
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < N; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    float h[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) h[k] = i < N ? thH[(int64_t)i * KP + k] : 0.f;
    for (int q = 0; q < nt; ++q) {
      const float f = centre_dot32<K>(h, sech[q]);
      const uint32_t m = __reduce_max_sync(0xffffffffu, i < N ? ord_f32(f) : 0u);
      if (lane == 0 && m) atomicMax(&smax[q], m);
    }
  }
  __syncthreads();
}

template <int K>
__device__ __forceinline__ void tile_centres_block(const float* __restrict__ thH, int N, int64_t n_tiles,
                                                   const float2* __restrict__ ec, float2* __restrict__ ref,
                                                   int64_t t0, float2 (*sec)[K], float (*sech)[padded_K<float>(K)],
                                                   uint32_t* smax) {
  const int nt = (int)min((int64_t)kRefTiles, n_tiles - t0);
  __syncthreads();  // the block's previous use of the shared slots is over
  if (threadIdx.x < kRefTiles) smax[threadIdx.x] = 0u;
  load_centre_features<K>(ec, t0, nt, sec, sech);
  centre_max_block<K>(thH, N, nt, sech, smax);
  if (threadIdx.x < nt) {
    const uint32_t m = smax[threadIdx.x];
    ref[t0 + threadIdx.x] = make_float2(m ? unord_f32(m) : 0.f, 0.f);
  }
}

// Reference logits C(t) of every tile (ec from k_centre_features).
template <int K>
__global__ void __launch_bounds__(kRefThreads)
k_tile_refs(const float* __restrict__ thH, int N, int64_t n_tiles, const float2* __restrict__ ec,
            float2* __restrict__ ref) {
  __shared__ float2 sec[kRefTiles][K];
  __shared__ __align__(16) float sech[kRefTiles][padded_K<float>(K)];
  __shared__ uint32_t smax[kRefTiles];
  tile_centres_block<K>(thH, N, n_tiles, ec, ref, (int64_t)blockIdx.x * kRefTiles, sec, sech, smax);
}

inline unsigned tile_centre_blocks(int64_t n_tiles) { return (unsigned)((n_tiles + kRefTiles - 1) / kRefTiles); }

// The relative centre logit theta'_i . eta(c) - C(t) of grain i (float).
template <int K>
__device__ __forceinline__ float centre_offset(const float* h, const float* l, const float2* ec, float2 ref) {
  return ff_diff(ff_dot<K>(h, l, ec), ref);
}

}  // namespace
}  // namespace pd
