// pd_tc_hvp.cu -- tensor-core (tcgen05) Hessian-vector products, PD_BF16
// and PD_BF16X3:
//
//   (H v)_i = -(1/(eps^2 |Omega|)) sum_x p_i(x) (u_i(x) - ubar(x)) eta(x),
//   u_i(x) = v_i . eta(x),  ubar(x) = sum_k p_k(x) u_k(x)
//
// (eq. hess and the proof of Prop. 4.5).  The contraction u = V . eta is a
// second logit-shaped contraction: it runs on the tensor cores beside the
// logits, from an operand image of v built like the parameter image, and is
// split at the tile centre in the same way (centre part v_i . eta(c) in fp32
// on the CUDA cores, the remainder v_i . (eta(x) - eta(c)) on the tensor
// cores).
//
// pass 1  (persistent over 128-pixel tiles) per 128-grain tile: logits and
//   u into two TMEM accumulators; the epilogue keeps, per pixel, the online
//   log-sum-exp and the p-weighted sum of u (rescaled with the running max),
//   and writes log2 S(x) and ubar(x).
// pass 2  the gradient pass of pd_tc.cu with c = p_i (u_i - ubar) in place
//   of -p_i: logits and u of the tile into TMEM, c in fp16 into the gradient
//   operand, the contraction against fp16 eta (hi + lo for PD_BF16X3).
//
// v is scaled by a power of two s so that |v/s| <= 1: then |u| <= K and
// |c| <= 2K, inside fp16's range; the factor s returns at the reduction.
#include "pd_tc_common.cuh"

namespace pd {
namespace {

constexpr int kH1Tile = 128;  // pass-1 grains per MMA group
constexpr int kH1Bufs = 2;    // TMEM buffers: logits [256 b, +128), u [256 b + 128, +128)

// The power of two s >= max |v| (1 when v = 0): s and 1/s.
__global__ void k_tc_vscale(const double* __restrict__ v, int64_t n, double* __restrict__ out) {
  __shared__ double sm[32];
  double m = 0.0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) m = fmax(m, fabs(v[q]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, sm[w]);
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    out[0] = ldexp(1.0, e);
    out[1] = ldexp(1.0, -e);
  }
}

// ---------------------------------------------------------------------------
// Pass 1: log2 S(x) and ubar(x) per pixel.
// ---------------------------------------------------------------------------
template <int DIM, int D, int KS>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_hvp_pass1(Geom g, TileMap tm, int N, int Npad, int g0, int Ng, const uint8_t* __restrict__ img,
               const uint8_t* __restrict__ vimg, const float* __restrict__ offg, const float* __restrict__ uoffg,
               float* __restrict__ lse_out, float* __restrict__ ubar_out, float4* __restrict__ ms_out,
               const unsigned long long* __restrict__ masks, uint32_t* __restrict__ need_bits, int64_t n_words,
               int* __restrict__ status) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * n_terms(KS);
  constexpr uint32_t kRowBytes = KT * 2;
  constexpr uint32_t kTileBytes = kTcPixTile * kRowBytes;
  constexpr uint32_t IDESC = idesc_bf16(128, kH1Tile);

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;                                            // Ng x KT parameter image
  uint8_t* sV = sB + (size_t)Ng * kRowBytes;                     // Ng x KT image of v / s
  uint8_t* sA = sV + (size_t)Ng * kRowBytes;                     // 2 stages x 128 x KT pixel rows
  float* sOff = reinterpret_cast<float*>(sA + 2 * kTileBytes);   // 2 stages x Ng centre logits
  float* sUoff = sOff + 2 * Ng;                                  // 2 stages x Ng centre parts of u
  float4* sPart = reinterpret_cast<float4*>(sUoff + 2 * Ng);    // 2 stages x 128 (max, S, T) of half 1
  long long* sJ = reinterpret_cast<long long*>(sPart + 2 * 128);  // 2 stages x 128 pixel indices
  float* sBm = reinterpret_cast<float*>(sJ + 2 * 128);           // 2 stages x Ng/128 blocks x 2 halves x 128
  __shared__ __align__(8) uint64_t bar_img, bar_a_full[2], bar_a_empty[2], bar_off_free[2], bar_d_full[kH1Bufs],
      bar_d_empty[kH1Bufs], bar_part_full[2], bar_part_free[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ unsigned long long sMask[2];  // blocks visited on the stage's tile (bit q: image block q)

  const int tid = threadIdx.x, warp = tid >> 5;
  const int n_gt = Ng / kH1Tile;
  // the blocks of this launch visited on the tile of stage s: all, less
  // those whose exponentials the centre-logit bounds show to underflow
  const uint64_t all_q = n_gt >= 64 ? ~0ull : ((1ull << n_gt) - 1ull);
  auto tile_mask = [&](int s) -> uint64_t { return masks ? (sMask[s] >> (g0 / 128)) & all_q : all_q; };
  const int64_t n_tiles = tm.n_tiles;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar_img, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar_a_full[s], kTcProducers);
      mbar_init(&bar_a_empty[s], 1);
      mbar_init(&bar_off_free[s], kTcConsumers);
      mbar_init(&bar_part_full[s], 128);
      mbar_init(&bar_part_free[s], 128);
    }
    for (int b = 0; b < kH1Bufs; ++b) {
      mbar_init(&bar_d_full[b], 1);
      mbar_init(&bar_d_empty[b], kTcConsumers);
    }
    mbar_init(&bar_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTcMmaWarp) tmem_alloc(&tmem_slot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kTcMmaWarp) {
    if (tid == kTcMmaWarp * 32) {
      const uint32_t total = (uint32_t)Ng * kRowBytes;
      mbar_arrive_expect_tx(&bar_img, 2 * total);
      for (uint32_t off = 0; off < total; off += 32768u) {
        const uint32_t n = total - off < 32768u ? total - off : 32768u;
        bulk_g2s(sB + off, img + (size_t)g0 * kRowBytes + off, n, &bar_img);
        bulk_g2s(sV + off, vimg + (size_t)g0 * kRowBytes + off, n, &bar_img);
      }
      bool ok = mbar_wait(&bar_img, 0, &abort_flag, status);
      int64_t c = 0;
      int it = 0;
      for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
        const int s = it & 1;
        ok = mbar_wait(&bar_a_full[s], (it >> 1) & 1, &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        for (uint64_t msk = tile_mask(s); msk; msk &= msk - 1, ++c) {
          const int gt = __ffsll((long long)msk) - 1;
          const int b = (int)(c % kH1Bufs);
          if (c >= kH1Bufs) {
            ok = mbar_wait(&bar_d_empty[b], (uint32_t)(((c / kH1Bufs) - 1) & 1), &abort_flag, status);
            if (!ok) break;
            tc_fence_after();
          }
          const uint32_t aaddr = smem_addr(sA + s * kTileBytes);
          const size_t rows = (size_t)gt * kH1Tile * kRowBytes;
          mma_terms<KS, KW>(tmem + b * 256, aaddr, KT * 16, false, smem_addr(sB + rows), KT * 16, IDESC);
          mma_terms<KS, KW>(tmem + b * 256 + 128, aaddr, KT * 16, false, smem_addr(sV + rows), KT * 16, IDESC);
          mma_commit(&bar_d_full[b]);
        }
        if (!ok) break;
        mma_commit(&bar_a_empty[s]);
      }
      mma_commit(&bar_drain);
      mbar_wait_drain(&bar_drain, 0);
    }
    __syncwarp();
  } else if (is_producer(warp)) {
    // pixel rows p0 and p0 + 64 of every tile; the tile's centre parts of
    // the logits and of u by bulk copies on the stage's barrier
    const int p0 = tid - kTcConsumers;
    int it = 0;
    bool ok = true;
    // the tile's block mask, fetched a tile ahead (thread p0 == 0)
    unsigned long long maskn = masks && p0 == 0 && blockIdx.x < n_tiles ? masks[blockIdx.x] : 0ull;
    for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
      const int s = it & 1, use = it >> 1;
      const unsigned long long maskc = maskn;
      if (masks && p0 == 0 && t + gridDim.x < n_tiles) maskn = masks[t + gridDim.x];
      if (use >= 1 && (!mbar_wait_warp(&bar_a_empty[s], (uint32_t)((use - 1) & 1), &abort_flag, status) ||
                       !mbar_wait_warp(&bar_off_free[s], (uint32_t)((use - 1) & 1), &abort_flag, status)))
        break;
      if (p0 == 0) {
        sMask[s] = maskc;
        fence_proxy_async();
        mbar_expect_tx(&bar_a_full[s], (uint32_t)Ng * 8);
        bulk_g2s(sOff + s * Ng, offg + t * Npad + g0, (uint32_t)Ng * 4, &bar_a_full[s]);
        bulk_g2s(sUoff + s * Ng, uoffg + t * Npad + g0, (uint32_t)Ng * 4, &bar_a_full[s]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int p = p0 + 64 * u;
        float x[DIM], cc[DIM], dx[DIM], de[K];
        const int64_t j = tile_pixel_dx<DIM>(g, tm, t, p, x, cc, dx);
        legendre_delta<DIM, D>(x, cc, dx, de, nullptr);
        store_eta_row<K, KW, KS>(sA + s * kTileBytes, p, de);
        sJ[s * 128 + p] = (long long)j;
      }
      fence_proxy_async();
      mbar_arrive(&bar_a_full[s]);
    }
  } else {
    const int quad = warp & 3, half = warp >> 2, lane = tid & 31;
    const int row = quad * 32 + lane;  // pixel row of the tile == TMEM lane
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    // one 32-grain chunk: logits r + off, u = w + uoff; the online
    // log-sum-exp (m, S) and T = sum 2^(l - m) u share the rescaling
    auto chunk = [&](const uint32_t(&r)[32], const uint32_t(&w)[32], const float* off, const float* uoff, int nv,
                     float& m, float& S, float& T) -> float {
      if (nv <= 0) return -INFINITY;
      float v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = q < nv ? __uint_as_float(r[q]) + off[q] : -INFINITY;
      const float cm = tree_max32(v);
      if (__all_sync(0xffffffffu, cm < m - 127.f)) return cm;
      const float mn = fmaxf(m, cm);
      const float sc = Arith<float>::ex(m - mn);
      float es = 0.f, eu = 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float e = Arith<float>::ex(v[q] - mn);
        es += e;
        eu = fmaf(e, q < nv ? __uint_as_float(w[q]) + uoff[q] : 0.f, eu);
      }
      S = fmaf(S, sc, es);
      T = fmaf(T, sc, eu);
      m = mn;
      return cm;
    };
    uint32_t R[32], U[32];
    int it = 0;
    int64_t c = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
      const int s = it & 1;
      ok = mbar_wait_warp(&bar_a_full[s], (uint32_t)((it >> 1) & 1), &abort_flag, status);
      if (!ok) break;
      float m = -INFINITY, S = 0.f, T = 0.f;
      const uint64_t msk0 = tile_mask(s);
      for (uint64_t msk = msk0; msk; msk &= msk - 1, ++c) {
        const int gt = __ffsll((long long)msk) - 1;
        const int b = (int)(c % kH1Bufs);
        ok = mbar_wait_warp(&bar_d_full[b], (uint32_t)((c / kH1Bufs) & 1), &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        const int cbase = gt * kH1Tile + half * 64;
        const int nrem = N - g0 - cbase;
        float bm = -INFINITY;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const uint32_t col = (uint32_t)(b * 256 + half * 64 + 32 * h2);
          tmem_ld32(tmem + lane_base + col, R);
          tmem_ld32(tmem + lane_base + col + 128, U);
          tmem_wait_ld();
          if (h2 == 1) {
            tc_fence_before();
            mbar_arrive(&bar_d_empty[b]);  // both halves of the buffer are in registers
          }
          bm = fmaxf(bm, chunk(R, U, sOff + s * Ng + cbase + 32 * h2, sUoff + s * Ng + cbase + 32 * h2,
                               nrem - 32 * h2, m, S, T));
        }
        // the largest logit of this pixel in the thread's half of the block
        sBm[((s * n_gt + gt) * 2 + half) * 128 + row] = bm;
      }
      if (!ok) break;
      // combine the two column halves of each pixel
      if (half == 1) {
        if (it >= 2 && !mbar_wait_warp(&bar_part_free[s], (uint32_t)(((it >> 1) - 1) & 1), &abort_flag, status)) {
          ok = false;
          break;
        }
        sPart[s * 128 + row] = make_float4(m, S, T, 0.f);
        mbar_arrive(&bar_part_full[s]);
      } else {
        if (!mbar_wait_warp(&bar_part_full[s], (uint32_t)((it >> 1) & 1), &abort_flag, status)) {
          ok = false;
          break;
        }
        const float4 o = sPart[s * 128 + row];
        mbar_arrive(&bar_part_free[s]);
        const int64_t j = sJ[s * 128 + row];
        float lse = NAN;
        if (j >= 0) {
          const float mm = fmaxf(m, o.x);
          const float a = Arith<float>::ex(m - mm), bb = Arith<float>::ex(o.x - mm);
          const float Sm = S * a + o.y * bb, Tm = T * a + o.z * bb;
          // log2 S of the pixel, or of this group's part (a lower bound)
          lse = mm + log2f(Sm);
          if (ms_out) {
            ms_out[j] = make_float4(mm, Sm, Tm, 0.f);
          } else {
            lse_out[j] = lse;
            ubar_out[j] = Tm / Sm;
          }
        }
        if (need_bits) {
          // a 128-grain block is needed by the HVP pass 2 on this tile
          // unless every probability in it is below 2^-32: with |u - ubar|
          // <= 2K <= 64, every c = p (u - ubar) of it is below 2^-26 and
          // rounds to zero in fp16
          for (int q = 0; q < n_gt; ++q) {
            const float bmq = fmaxf(sBm[((s * n_gt + q) * 2) * 128 + row], sBm[((s * n_gt + q) * 2 + 1) * 128 + row]);
            const bool nd = ((msk0 >> q) & 1) && j >= 0 && !(bmq < lse - 32.f);
            const uint32_t bal = __ballot_sync(0xffffffffu, nd);
            if (lane == 0 && bal)
              atomicOr(&need_bits[(int64_t)(g0 / 128 + q) * n_words + (t >> 5)], 1u << (int)(t & 31));
          }
        }
      }
      mbar_arrive(&bar_off_free[s]);
    }
    tmem_wait_ld();
  }
  tc_fence_before();
  __syncthreads();
  if (abort_flag && tid == 0) atomicCAS(status, 0, PD_ETIMEOUT);
  if (warp == kTcMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

// Merge of a grain-split pass 1: (max, S, T) of every group per pixel.
__global__ void __launch_bounds__(256)
k_tc_hvp_merge(const float4* __restrict__ ms, int n_grp, int64_t P, float* __restrict__ lse_out,
               float* __restrict__ ubar_out) {
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (j >= P) return;
  float m = -INFINITY;
  for (int q = 0; q < n_grp; ++q) m = fmaxf(m, ms[(int64_t)q * P + j].x);
  float S = 0.f, T = 0.f;
  for (int q = 0; q < n_grp; ++q) {
    const float4 v = ms[(int64_t)q * P + j];
    if (v.y > 0.f) {
      const float e = Arith<float>::ex(v.x - m);
      S = fmaf(v.y, e, S);
      T = fmaf(v.z, e, T);
    }
  }
  lse_out[j] = m + log2f(S);
  ubar_out[j] = T / S;
}

// ---------------------------------------------------------------------------
// Pass 2: Hessian-vector partials of one grain block over a run of tiles.
// TMEM: logits [0, 128), u [128, 256) (one tile at a time), D2 two buffers
// of N2 columns from 256.
// ---------------------------------------------------------------------------
template <int DIM, int D, int KS>
struct HvpLayout {
  using L = Pass2Layout<DIM, D, KS>;
  static constexpr uint32_t kPerB = L::kPerB + 2 * kTcPixTile * 4;  // + ubar of the pixels, centre parts of u
  static constexpr size_t bytes(int nb, int na) {
    return 2 * (size_t)L::kABytes + (size_t)nb * kPerB + (size_t)na * L::kA2Bytes;
  }
};

template <int DIM, int D, int KS, int NB, int NA>
__global__ void __launch_bounds__(kP2Threads, 1)
k_tc_hvp_pass2(Geom g, TileMap tm, int N, int Npad, const uint8_t* __restrict__ img, const uint8_t* __restrict__ vimg,
               const float* __restrict__ offg, const float* __restrict__ uoffg, const float* __restrict__ lse,
               const float* __restrict__ ubar, const int* __restrict__ kept, const int* __restrict__ n_kept_gb,
               const int* __restrict__ perm, double* __restrict__ part, int* __restrict__ status) {
  using L = Pass2Layout<DIM, D, KS>;
  constexpr int K = L::K, KW = L::KW, KT = L::KT, ET = L::ET, N2 = L::N2, CT = L::CT;
  constexpr uint32_t IDESC1 = idesc_bf16(128, kTcPixTile);
  constexpr uint32_t IDESC2 = idesc_f16(128, N2);
  constexpr int D2COL = 2 * kTcPixTile;  // D2 buffer db at D2COL + db*CT*N2
  static_assert(D2COL + 2 * CT * N2 <= kTcCols, "TMEM columns");
  constexpr float kLoScale = 4096.f;      // c_lo = fl16((c - c_hi) * 2^12)

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                          // parameter block image
  uint8_t* sAv = sA + L::kABytes;              // v block image
  uint8_t* sB = sAv + L::kABytes;              // NB stages of eta - eta(c) rows
  uint8_t* sB2 = sB + NB * L::kBBytes;         // NB stages of eta^T (fp16)
  uint8_t* sA2 = sB2 + NB * L::kB2Bytes;       // NA stages of c (fp16, CT terms)
  float* sLse = reinterpret_cast<float*>(sA2 + NA * L::kA2Bytes);  // [NB][128]
  float* sOffP = sLse + NB * kTcPixTile;                           // [NB][128] centre logits of the block
  float* sUbar = sOffP + NB * 128;                                  // [NB][128]
  float* sUoffP = sUbar + NB * kTcPixTile;                          // [NB][128] centre parts of u
  __shared__ __align__(8) uint64_t bar_img, bar_b_full[NB], bar_b_empty[NB], bar_d1_full, bar_d1_empty,
      bar_a2_full[NA], bar_a2_empty[NA], bar_d2_full[2], bar_d2_free[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int gb = blockIdx.y;
  // this CTA's share of the tiles on which the grain block has a
  // non-negligible probability (all tiles without the lists), in order
  const int64_t n_list = kept ? (int64_t)n_kept_gb[gb] : tm.n_tiles;
  const int64_t k_lo = n_list * blockIdx.x / gridDim.x;
  const int n_pt = (int)(n_list * (blockIdx.x + 1) / gridDim.x - k_lo);
  const int* klist = kept ? kept + (int64_t)gb * tm.n_tiles + k_lo : nullptr;
  auto tile_of = [&](int t) -> int64_t { return klist ? (int64_t)klist[t] : k_lo + t; };
  const int n_items = (n_pt + kH2ChunkTiles - 1) / kH2ChunkTiles;  // chunks
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar_img, 1);
    for (int s = 0; s < NB; ++s) {
      mbar_init(&bar_b_full[s], kTcProducers);
      mbar_init(&bar_b_empty[s], 2);
    }
    mbar_init(&bar_d1_full, 1);
    mbar_init(&bar_d1_empty, kTcConsumers);
    for (int a = 0; a < NA; ++a) {
      mbar_init(&bar_a2_full[a], kTcConsumers);
      mbar_init(&bar_a2_empty[a], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_d2_full[b], 1);
      mbar_init(&bar_d2_free[b], 128);
    }
    mbar_init(&bar_drain, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTcMmaWarp) tmem_alloc(&tmem_slot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kTcMmaWarp) {
    // logits and u of tile t (one tile in TMEM at a time)
    if (tid == kTcMmaWarp * 32) {
      mbar_arrive_expect_tx(&bar_img, 2 * L::kABytes);
      bulk_g2s(sA, img + (size_t)gb * L::kABytes, L::kABytes, &bar_img);
      bulk_g2s(sAv, vimg + (size_t)gb * L::kABytes, L::kABytes, &bar_img);
      bool ok = mbar_wait(&bar_img, 0, &abort_flag, status);
      for (int t = 0; ok && t < n_pt; ++t) {
        const int s = t % NB;
        ok = mbar_wait(&bar_b_full[s], (uint32_t)((t / NB) & 1), &abort_flag, status);
        if (ok && t >= 1) ok = mbar_wait(&bar_d1_empty, (uint32_t)((t - 1) & 1), &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t baddr = smem_addr(sB + s * L::kBBytes);
        mma_terms<KS, KW>(tmem, smem_addr(sA), KT * 16, true, baddr, L::kSboB, IDESC1);
        mma_terms<KS, KW>(tmem + kTcPixTile, smem_addr(sAv), KT * 16, true, baddr, L::kSboB, IDESC1);
        mma_commit(&bar_d1_full);
        mma_commit(&bar_b_empty[s]);
      }
      mma_commit(&bar_drain);
      mbar_wait_drain(&bar_drain, 0);
    }
    __syncwarp();
  } else if (warp == kP2GradWarp) {
    // D2 += C . [eta_h | eta_l] (fp16), one accumulation per chunk
    if (tid == kP2GradWarp * 32) {
      bool ok = true;
      for (int t = 0; ok && t < n_pt; ++t) {
        const int s = t % NB, a = t % NA;
        const int u = t / kH2ChunkTiles, db = u & 1;
        const bool first = t % kH2ChunkTiles == 0, last = t % kH2ChunkTiles == kH2ChunkTiles - 1 || t == n_pt - 1;
        if (first && u >= 2) ok = mbar_wait(&bar_d2_free[db], (uint32_t)(((u >> 1) - 1) & 1), &abort_flag, status);
        if (ok) ok = mbar_wait(&bar_a2_full[a], (uint32_t)((t / NA) & 1), &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t a2 = smem_addr(sA2 + a * L::kA2Bytes), b2 = smem_addr(sB2 + s * L::kB2Bytes);
#pragma unroll 2
        for (int q = 0; q < kTcPixTile / 16; ++q) {
          const uint64_t bd = smem_desc(b2 + q * 2 * L::kLbo2, L::kLbo2, L::kSbo2);
#pragma unroll
          for (int ct = 0; ct < CT; ++ct) {
            const uint64_t ad = smem_desc(a2 + ct * L::kA2Term + q * 256, 128, kTcPixTile * 16);
            mma_bf16(tmem + D2COL + (db * CT + ct) * N2, ad, bd, IDESC2, (!first || q > 0) ? 1u : 0u);
          }
        }
        mma_commit(&bar_a2_empty[a]);
        mma_commit(&bar_b_empty[s]);
        if (last) mma_commit(&bar_d2_full[db]);
      }
      mma_commit(&bar_drain);
      mbar_wait_drain(&bar_drain, 0);
    }
    __syncwarp();
  } else if (is_producer(warp)) {
    const int q2 = 2 * (tid - kTcConsumers);
    float xn[2][DIM], cn[DIM], dxn[2][DIM], lsn[2], ubn[2];
    auto fetch = [&](int t) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t j = tile_pixel_dx<DIM>(g, tm, tile_of(t), q2 + u, xn[u], cn, dxn[u]);
        lsn[u] = j >= 0 ? lse[j] : INFINITY;
        ubn[u] = j >= 0 ? ubar[j] : 0.f;
      }
    };
    if (n_pt > 0) fetch(0);
    for (int t = 0; t < n_pt; ++t) {
      const int s = t % NB;
      float xc[2][DIM], cc[DIM], dxc[2][DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        xc[0][a] = xn[0][a];
        xc[1][a] = xn[1][a];
        dxc[0][a] = dxn[0][a];
        dxc[1][a] = dxn[1][a];
        cc[a] = cn[a];
      }
      const float2 lsc = make_float2(lsn[0], lsn[1]), ubc = make_float2(ubn[0], ubn[1]);
      if (t + 1 < n_pt) fetch(t + 1);
      if (t >= NB && !mbar_wait_warp(&bar_b_empty[s], (uint32_t)(((t / NB) - 1) & 1), &abort_flag, status)) break;
      if (q2 == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bar_b_full[s], 2 * 128 * 4);
        const int64_t tc = tile_of(t);
        bulk_g2s(sOffP + s * 128, offg + tc * Npad + gb * 128, 128 * 4, &bar_b_full[s]);
        bulk_g2s(sUoffP + s * 128, uoffg + tc * Npad + gb * 128, 128 * 4, &bar_b_full[s]);
      }
      float e0[K], e1[K];
      uint8_t* bs = sB + s * L::kBBytes;
      {
        float de[K];
        legendre_delta<DIM, D>(xc[0], cc, dxc[0], de, e0);
        store_eta_row<K, KW, KS, L::kSboB>(bs, q2, de);
        legendre_delta<DIM, D>(xc[1], cc, dxc[1], de, e1);
        store_eta_row<K, KW, KS, L::kSboB>(bs, q2 + 1, de);
      }
      uint8_t* b2 = sB2 + s * L::kB2Bytes;
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const float a0 = k < K ? e0[k] : 0.f, a1 = k < K ? e1[k] : 0.f;
        const __half2 h = __floats2half2_rn(a0, a1);
        const uint32_t o = kmaj_s(k, q2, L::kLbo2, L::kSbo2);
        *reinterpret_cast<uint32_t*>(b2 + o) = *reinterpret_cast<const uint32_t*>(&h);
        if (ET == 2) {
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn(a0 - hf.x, a1 - hf.y);
          *reinterpret_cast<uint32_t*>(b2 + L::kB2Term + o) = *reinterpret_cast<const uint32_t*>(&l);
        }
      }
      *reinterpret_cast<float2*>(sLse + s * kTcPixTile + q2) = lsc;
      *reinterpret_cast<float2*>(sUbar + s * kTcPixTile + q2) = ubc;
      fence_proxy_async();
      mbar_arrive(&bar_b_full[s]);
    }
  } else {
    const int quad = warp & 3, half = warp >> 2, lane = tid & 31;
    const int gr = quad * 32 + lane;
    const int i = gb * 128 + gr;  // row of the parameter image
    const int gi = perm ? perm[i] : (i < N ? i : -1);  // its grain (-1: padding)
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    int n_done = 0;
    // the CTA's partial of this grain (a row of part): the chunks added in
    // order, in double
    double* prow = gi >= 0 ? part + ((int64_t)blockIdx.x * N + gi) * K : nullptr;
    auto read_chunk = [&](int u) -> bool {
      const int db = u & 1;
      if (!mbar_wait_warp(&bar_d2_full[db], (uint32_t)((u >> 1) & 1), &abort_flag, status)) return false;
      tc_fence_after();
      const uint32_t base = tmem + lane_base + (uint32_t)(D2COL + db * CT * N2);
      // 16 features at a time: the eta_h and eta_l columns of each term of
      // c, added in fp32 (the accumulators' own precision), c_lo scaled back
#pragma unroll
      for (int kb = 0; kb < KW; kb += 16) {
        float f[16];
#pragma unroll
        for (int ct = 0; ct < CT; ++ct) {
          uint32_t r[ET][16];
#pragma unroll
          for (int et = 0; et < ET; ++et) tmem_ld16(base + (uint32_t)(ct * N2 + et * KW + kb), r[et]);
          tmem_wait_ld();
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            const float v = ET == 2 ? __uint_as_float(r[0][kk]) + __uint_as_float(r[ET - 1][kk]) : __uint_as_float(r[0][kk]);
            f[kk] = ct == 0 ? v : fmaf(v, 1.f / kLoScale, f[kk]);
          }
        }
        if (prow) {
#pragma unroll
          for (int kk = 0; kk < 16; ++kk) {
            const int k = kb + kk;
            if (k < K) prow[k] = u == 0 ? (double)f[kk] : prow[k] + (double)f[kk];
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&bar_d2_free[db]);
      n_done = u + 1;
      return true;
    };
    uint32_t R[32], U[32];
    bool ok = true;
    for (int t = 0; t < n_pt; ++t) {
      const int s = t % NB, a = t % NA;
      if (!mbar_wait_warp(&bar_b_full[s], (uint32_t)((t / NB) & 1), &abort_flag, status) ||
          !mbar_wait_warp(&bar_d1_full, (uint32_t)(t & 1), &abort_flag, status)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const float off = sOffP[s * 128 + gr], uoff = sUoffP[s * 128 + gr];
      if (t >= NA && !mbar_wait_warp(&bar_a2_empty[a], (uint32_t)(((t / NA) - 1) & 1), &abort_flag, status)) {
        ok = false;
        break;
      }
      uint8_t* a2 = sA2 + a * L::kA2Bytes;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const uint32_t col = (uint32_t)(half * 64 + 32 * h2);
        tmem_ld32(tmem + lane_base + col, R);
        tmem_ld32(tmem + lane_base + kTcPixTile + col, U);
        tmem_wait_ld();
        if (h2 == 1) {
          tc_fence_before();
          mbar_arrive(&bar_d1_empty);  // the tile's logits and u are in registers
        }
        const float* ls = sLse + s * kTcPixTile + col;
        const float* ub = sUbar + s * kTcPixTile + col;
#pragma unroll
        for (int q8 = 0; q8 < 32; q8 += 8) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            // c = p (u - ubar), p = 2^(l - log2 S), u = w + uoff
            const float p0 = Arith<float>::ex(__uint_as_float(R[q8 + u]) + (off - ls[q8 + u]));
            const float p1 = Arith<float>::ex(__uint_as_float(R[q8 + u + 1]) + (off - ls[q8 + u + 1]));
            const float c0 = p0 * ((__uint_as_float(U[q8 + u]) + uoff) - ub[q8 + u]);
            const float c1 = p1 * ((__uint_as_float(U[q8 + u + 1]) + uoff) - ub[q8 + u + 1]);
            const __half2 h = __floats2half2_rn(c0, c1);
            hw[u >> 1] = *reinterpret_cast<const uint32_t*>(&h);
            if (CT == 2) {
              const float2 hf = __half22float2(h);
              const __half2 l2 = __floats2half2_rn((c0 - hf.x) * kLoScale, (c1 - hf.y) * kLoScale);
              lw[u >> 1] = *reinterpret_cast<const uint32_t*>(&l2);
            }
          }
          const uint32_t o = kmaj(gr, (int)col + q8, kTcPixTile);
          *reinterpret_cast<uint4*>(a2 + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          if (CT == 2) *reinterpret_cast<uint4*>(a2 + L::kA2Term + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      }
      fence_proxy_async();
      mbar_arrive(&bar_a2_full[a]);
      if (half == 0 && t > kH2ChunkTiles && t % kH2ChunkTiles == 1 && !read_chunk(t / kH2ChunkTiles - 1)) {
        ok = false;
        break;
      }
    }
    tmem_wait_ld();
    if (half == 0) {
      for (int u = n_done; ok && u < n_items; ++u) ok = read_chunk(u);
      if (prow && (!ok || n_items == 0)) {
        for (int k = 0; k < K; ++k) prow[k] = ok ? 0.0 : NAN;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kTcMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int DIM, int D, int KS>
int eval_tc_hvp_dd(const EvalCall& c, cudaStream_t st) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * n_terms(KS);
  const int N = c.N;
  const int64_t P = c.g.P;
  const int Npad = (N + kH1Tile - 1) / kH1Tile * kH1Tile;
  const size_t row_bytes = (size_t)KT * 2;
  constexpr size_t kCap = 220 * 1024;
  // pass 1 keeps both images of ng grains resident; more grains run in
  // groups whose (max, S, T) are merged
  auto p1_bytes = [&](size_t ng) {
    return 2 * ng * row_bytes + 2 * kTcPixTile * row_bytes + 4 * ng * 4 + 2 * kTcPixTile * 16 + 2 * kTcPixTile * 8 +
           4 * ng * 4;
  };
  int n_grp = 1, Ng = Npad;
  while (p1_bytes((size_t)Ng) > kCap && Ng > kH1Tile) {
    ++n_grp;
    Ng = ((Npad + n_grp - 1) / n_grp + kH1Tile - 1) / kH1Tile * kH1Tile;
  }
  n_grp = (Npad + Ng - 1) / Ng;
  const size_t smem1 = p1_bytes((size_t)Ng);
  using H2 = HvpLayout<DIM, D, KS>;
  constexpr int NB = H2::bytes(3, 2) <= kCap ? 3 : (H2::bytes(2, 2) <= kCap ? 2 : (H2::bytes(2, 1) <= kCap ? 2 : 1));
  constexpr int NA = H2::bytes(NB, 2) <= kCap ? 2 : 1;
  const size_t smem2 = H2::bytes(NB, NA);
  if (smem1 > kCap || smem2 > kCap) return PD_ENOTSUP;
  if (!c.g.coords && std::max(c.g.n0, std::max(c.g.n1, c.g.n2)) > (int64_t(1) << 23)) return PD_ENOTSUP;
  const size_t smem1_req = std::max<size_t>(smem1, 120 * 1024);
  const size_t smem2_req = std::max<size_t>(smem2, 120 * 1024);

  const TileMap tm = make_tiles<DIM>(c.g);
  const int sms = device_sm_count();
  const int64_t n_tiles = tm.n_tiles;
  const int grid1 = (int)std::min<int64_t>(n_tiles, sms);
  const int gblocks = (N + 127) / 128;
  const int cpg = (int)std::min<int64_t>((n_tiles + kH2ChunkTiles - 1) / kH2ChunkTiles, std::max(1, sms / gblocks));
  // as for the gradient: pass 2 visits the (tile, block) pairs whose c can
  // survive in fp16, with the grains in the Morton order of their label
  // centroids (PD_TC_NO_SKIP=1: every pair, index order)
  const char* no_skip = getenv("PD_TC_NO_SKIP");
  const bool skip = !(no_skip && no_skip[0] && no_skip[0] != '0');
  // (labels may be NULL for the Hessian: then no grain order by label
  // centroids and no label reference for the block masks)
  const bool order = skip && Npad <= kOrderMax && c.labels != nullptr;
  // pass 1 leaves out the blocks that the centre-logit bounds place far
  // below the tile's reference logit (structured grids)
  const bool bounds = skip && !c.g.coords && Npad / 128 <= 64;
  const int64_t n_words = (n_tiles + 31) / 32;

  constexpr int KP = padded_K<float>(K);
  // (a plan makes every allocation on every call, so that its arena keeps
  // the centre features and the grain order at the same place)
  const bool all = c.plan != nullptr;
  Scratch sc(st, c.plan);
  double* vsc = sc.get<double>(2);
  float* thH = sc.get<float>((size_t)N * KP);  // float-float parameters for the centre logits
  float* thL = sc.get<float>((size_t)N * KP);
  uint8_t* img = sc.get<uint8_t>((size_t)Npad * row_bytes);
  uint8_t* vimg = sc.get<uint8_t>((size_t)Npad * row_bytes);
  float* th32t = sc.get<float>((size_t)K * Npad);
  float* v32t = sc.get<float>((size_t)K * Npad);
  float2* ecg = sc.get<float2>((size_t)n_tiles * K);  // centre features per tile
  float* offg = sc.get<float>((size_t)n_tiles * Npad);
  float* uoffg = sc.get<float>((size_t)n_tiles * Npad);
  float* lse = sc.get<float>((size_t)P);
  float* ubar = sc.get<float>((size_t)P);
  float4* ms = n_grp > 1 ? sc.get<float4>((size_t)n_grp * P) : nullptr;
  double* part = sc.get<double>((size_t)cpg * N * K);  // one partial per pass-2 CTA and grain
  uint32_t* need = (skip || all) ? sc.get<uint32_t>((size_t)gblocks * n_words) : nullptr;
  int* kept = (skip || all) ? sc.get<int>((size_t)gblocks * n_tiles) : nullptr;
  int* nkept = (skip || all) ? sc.get<int>((size_t)gblocks) : nullptr;
  constexpr int K1 = DIM + 1;  // label moments of degree <= 1: counts and centroids for the grain order
  unsigned long long* lmom = (order || all) ? sc.get<unsigned long long>((size_t)N * K1) : nullptr;
  int* perm = (order || all) ? sc.get<int>((size_t)Npad) : nullptr;
  int* rank = (order || all) ? sc.get<int>((size_t)N) : nullptr;
  unsigned long long* masks = (bounds || all) ? sc.get<unsigned long long>((size_t)n_tiles) : nullptr;
  int* status = sc.get<int>(1);
  if (!sc.ok()) return PD_ENOMEM;
  if (sc.sizing()) {
    c.plan->need = sc.used();
    return PD_OK;
  }
  if (!skip) need = nullptr, kept = nullptr, nkept = nullptr;
  if (!order) perm = nullptr, rank = nullptr;
  if (!bounds) masks = nullptr;
  const TileBound tb = bounds ? tile_bound<DIM, D>(c.g) : TileBound{};
  const bool have_features = c.plan && c.plan->features;
  const bool have_order = c.plan && c.plan->order;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return PD_ECUDA;
  if (need && cudaMemsetAsync(need, 0, sizeof(uint32_t) * (size_t)gblocks * n_words, st) != cudaSuccess)
    return PD_ECUDA;
  if (order && !have_order) {
    int bits = 0;
    while (bits < 62 && ((int64_t)1 << bits) <= P) ++bits;
    const float fx = ldexpf(1.f, 62 - bits);
    if (cudaMemsetAsync(lmom, 0, sizeof(unsigned long long) * N * K1, st) != cudaSuccess) return PD_ECUDA;
    const int64_t nthr = n_tiles * kTcPixTile;
    PD_TIMED(st, "tc_label_moments",
             (k_tc_label_moments<DIM, 1><<<(unsigned)((nthr + 255) / 256), 256, 0, st>>>(c.g, tm, c.labels, N, fx,
                                                                                       lmom)));
    PD_TIMED(st, "tc_grain_order",
             k_tc_grain_order<DIM><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(lmom, N, K1, Npad, perm, rank));
  }

  PD_TIMED(st, "tc_hvp_vscale", k_tc_vscale<<<1, 1024, 0, st>>>(c.v, (int64_t)N * K, vsc));
  {
    const int64_t n = (int64_t)Npad * KW;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    PD_TIMED(st, "tc_theta_image",
             k_tc_theta_image<KS><<<blocks, 256, 0, st>>>(c.theta, N, Npad, K, KW, Arith<float>::theta_scale(c.eps),
                                                          nullptr, perm, img, th32t, thH, thL, KP));
    PD_TIMED(st, "tc_v_image",
             k_tc_theta_image<KS><<<blocks, 256, 0, st>>>(c.v, N, Npad, K, KW, 1.0, vsc + 1, perm, vimg, v32t,
                                                          nullptr, nullptr, 0));
  }
  const dim3 gridc((unsigned)((Npad + 255) / 256),
                   (unsigned)std::min<int64_t>((n_tiles + kCentreTiles - 1) / kCentreTiles, 4096));
  // logits relative to the tiles' reference logits; u (not shift-invariant,
  // and of modest size) from plain fp32 centre parts
  if (!have_features)
    PD_TIMED(st, "centre_features",
             (k_centre_features<DIM, D><<<centre_feature_blocks(n_tiles), kFeatThreads, 0, st>>>(c.g, tm, ecg)));
  PD_TIMED(st, "tc_tile_setup",
           (k_tc_tile_setup<DIM, D><<<tile_centre_blocks(n_tiles), kRefThreads, 0, st>>>(
               c.g, tm, thH, thL, N, Npad, perm, ecg, offg, tb, bounds ? 1 : 0, masks)));
  PD_TIMED(st, "tc_centre_u", (k_tc_centre_logits<DIM, D><<<gridc, 256, 0, st>>>(c.g, tm, v32t, perm, N, Npad, uoffg, TileBound{}, nullptr, nullptr)));

  auto k1 = k_tc_hvp_pass1<DIM, D, KS>;
  if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1_req) != cudaSuccess)
    return PD_ECUDA;
  for (int q = 0; q < n_grp; ++q) {
    const int g0 = q * Ng, ng = std::min(Ng, Npad - g0);
    PD_TIMED(st, KS == 1 ? "tc_bf16_hvp_pass1" : "tc_bf16x3_hvp_pass1",
             k1<<<grid1, kTcThreads, smem1_req, st>>>(c.g, tm, N, Npad, g0, ng, img, vimg, offg, uoffg, lse, ubar,
                                                      ms ? ms + (size_t)q * P : nullptr, masks, need, n_words, status));
  }
  if (n_grp > 1)
    PD_TIMED(st, "tc_hvp_merge", k_tc_hvp_merge<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(ms, n_grp, P, lse, ubar));
  if (skip)
    PD_TIMED(st, "tc_kept_lists",
             k_tc_kept_lists<<<(unsigned)gblocks, 1024, 0, st>>>(need, n_words, n_tiles, kept, nkept));
  auto k2 = k_tc_hvp_pass2<DIM, D, KS, NB, NA>;
  if (cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2_req) != cudaSuccess)
    return PD_ECUDA;
  PD_TIMED(st, KS == 1 ? "tc_bf16_hvp_pass2" : "tc_bf16x3_hvp_pass2",
           (k2<<<dim3(cpg, gblocks), kP2Threads, smem2_req, st>>>(c.g, tm, N, Npad, img, vimg, offg, uoffg, lse, ubar,
                                                                 kept, nkept, perm, part, status)));
  const int64_t NK = (int64_t)N * K;
  PD_TIMED(st, "reduce_parts",
           k_tc_reduce_grad<<<(unsigned)((NK + 31) / 32), dim3(32, kRedPhases), 0, st>>>(
               part, cpg, NK, nullptr, 0.0, -1.0 / (c.eps * c.eps * (double)P), vsc, c.hv));
  if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
  if (c.plan) {
    c.plan->features = true;
    c.plan->order = c.plan->order || order;
  }
  return PD_OK;
}

template <int KS>
int eval_tc_hvp_ks(const EvalCall& c, cudaStream_t st) {
  if (c.dim == 2) {
    switch (c.d) {
      case 1: return eval_tc_hvp_dd<2, 1, KS>(c, st);
      case 2: return eval_tc_hvp_dd<2, 2, KS>(c, st);
      case 3: return eval_tc_hvp_dd<2, 3, KS>(c, st);
      case 4: return eval_tc_hvp_dd<2, 4, KS>(c, st);
      case 5: return eval_tc_hvp_dd<2, 5, KS>(c, st);
      case 6: return eval_tc_hvp_dd<2, 6, KS>(c, st);
      default: return PD_ENOTSUP;
    }
  }
  if (c.dim == 3) {
    switch (c.d) {
      case 1: return eval_tc_hvp_dd<3, 1, KS>(c, st);
      case 2: return eval_tc_hvp_dd<3, 2, KS>(c, st);
      case 3: return eval_tc_hvp_dd<3, 3, KS>(c, st);
      default: return PD_ENOTSUP;
    }
  }
  return PD_ENOTSUP;
}

}  // namespace

int eval_tc_hvp(const EvalCall& c, cudaStream_t st) {
  if (c.prec == PD_BF16) return eval_tc_hvp_ks<1>(c, st);
  if (c.prec == PD_BF16X3) return eval_tc_hvp_ks<6>(c, st);
  return PD_ENOTSUP;
}

}  // namespace pd
