// pd_tc.cu -- tensor-core (tcgen05) evaluation of the objective and
// gradient, PD_BF16 and PD_BF16X3.
//
// Both K-long contractions of eqs. (Phi) and (grad) run on the 5th-generation
// tensor cores with bf16/fp16 operands in shared memory and fp32
// accumulators in tensor memory (TMEM); the CUDA cores keep the
// soft-assignment arithmetic (one ex2 per pixel-grain pair and pass) and the
// per-pixel features.
//
// Pixels are processed in tiles of 128 neighbouring pixels (pd_tiles.cuh).
// Every logit is taken relative to a per-tile reference C(t):
//   l_i(x) - C(t) = [theta'_i . eta(c) - C(t)] + theta'_i . (eta(x) - eta(c)),
// c the tile's centre pixel, theta' = -theta log2(e) / eps.  The bracket
// (the centre offset, one float per tile and grain) is formed once per
// evaluation by k_tc_tile_setup from float-float parameters and features
// and rounded once; the tensor cores contract only the small remainder,
// whose features eta(x) - eta(c) come from divided differences of the
// Legendre recurrence (no cancellation).  The log-sum-exp is invariant
// under the per-pixel shift, so log2 S(x) is kept relative to C(t) as well.
//
// pass 1  (one CTA per SM, persistent over 128-pixel tiles)
//   A = eta(x) - eta(c) of 128 pixels (rows) x K, written by 128 producer
//       threads from the in-register recurrences;
//   B = all grains' scaled parameters (rows) x K, copied once per CTA from a
//       prepared global image by a bulk (TMA) copy;
//   D = A B^T, 128 pixels x 128 grains per MMA group, for the blocks of
//       grains that the tile's mask keeps; an epilogue warpgroup owns a
//       tile, adds the centre offsets, reads the label logit and keeps an
//       online log-sum-exp; out: log2 S(x) per pixel, per-CTA objective
//       partials, and one bit per (tile, 128-grain block): whether the
//       block holds a probability that can survive in the gradient pass's
//       fp16 operand, or the label of a pixel of the tile.
// pass 2  (CTA = 128 grains x a share of the tiles whose bit is set)
//   D1 = theta_block (128 grains x K) . (eta(x) - eta(c))^T (128 pixels):
//       the logits transposed, so that a thread owns one grain's row;
//   the thread forms c = delta_{i G(x)} - p_i(x) for its grain, written as
//       an fp16 A operand (grains x pixels, K-major) in two terms for
//       PD_BF16X3 (c_hi = fl16(c), c_lo = fl16((c - c_hi) 2^12)), one for
//       PD_BF16;
//   D2 += C (128 grains x 128 pixels) . eta(tile) (128 pixels x K, fp16 hi
//       and lo columns), one TMEM accumulator per term of c, read out every
//       kP2ChunkTiles tiles and summed in double to one partial per grain
//       and CTA.  Since c = delta - p is small wherever the fit is good, the
//       fp32 accumulation acts on small numbers.
//   A (tile, block) pair whose bit is clear would only add zeros: every
//   c = -p of it is below 2^-26 and rounds to zero in fp16, and no pixel of
//   the tile has a label in the block.  To make such pairs common, the
//   parameter image lists the grains in the Morton order of their label
//   centroids (k_tc_grain_order), so that a block of 128 grains is a
//   compact region and most tiles lie far from most blocks; the gradient
//   partials go back to the caller's grain order.
//
// PD_BF16X3 splits every logit operand into three bf16 terms (hi + mid +
// lo, about 24 significant bits) and forms the six products whose size is
// at least 2^-16 of the leading one (hh, hm, mh, hl, mm, lh), smallest
// first, which gives float-level logit remainders.  PD_BF16 uses one term.
// An operand row stores each term once, as KW-column slices side by side; a
// product is a run of MMAs whose two descriptors start at the slices of its
// terms.
#include "pd_tc_common.cuh"

namespace pd {
namespace {

// ---------------------------------------------------------------------------
// Pass 1: log2 S(x) per pixel and objective partials.
// ---------------------------------------------------------------------------
// Pass 1 takes the grains of a tile in blocks of 128 (one MMA of N = 128
// per block and product); the two epilogue warpgroups take alternate
// tiles, each all blocks of its tile (so that a pixel's log-sum-exp needs
// no exchange), through its own two 128-column TMEM buffers.  A block
// whose logits lie, everywhere in the tile, so far below the tile's
// largest logit that their exponentials underflow to zero (a bound from the
// centre offsets, see k_tc_tile_setup) is not visited.
constexpr int kP1Bufs = 4;
constexpr int kP1Stages = 3;  // pixel-operand stages at most (two tiles in the epilogue, one being written)

template <int DIM, int D, int KS>
__global__ void __launch_bounds__(kP1Threads, 1)
k_tc_pass1(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, int Npad, int g0, int Ng, int n_stages,
           const uint8_t* __restrict__ img, const float* __restrict__ th32t, int th_resident,
           const float* __restrict__ offg, const int* __restrict__ rank, float* __restrict__ lse_out,
           float* __restrict__ q_out, double* __restrict__ obj_part,
           float2* __restrict__ ms_out, float* __restrict__ lg_out, const unsigned long long* __restrict__ masks,
           uint32_t* __restrict__ need_bits, int64_t n_words, int* __restrict__ status) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * n_terms(KS);
  constexpr uint32_t kRowBytes = KT * 2;
  constexpr uint32_t kTileBytes = kTcPixTile * kRowBytes;
  constexpr uint32_t IDESC = idesc_bf16(128, 128);

  const int S = n_stages;  // 2 or 3
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;                                            // Ng x KT (this launch's grains)
  uint8_t* sA = smem + (size_t)Ng * kRowBytes;                   // S stages x 128 x KT
  float* sOff = reinterpret_cast<float*>(sA + S * kTileBytes);   // S stages x Ng centre logits (bulk copied)
  float* sLG = sOff + S * Ng;                                    // S stages x 128 starting max
  float* sLGv = sLG + S * 128;                                   // S stages x 128 label logits
  long long* sJ = reinterpret_cast<long long*>(sLGv + S * 128);  // S stages x 128 pixel indices
  int* sLRow = reinterpret_cast<int*>(sJ + S * 128);             // S stages x 128 image rows of the labels
  float* sBm = reinterpret_cast<float*>(sLRow + S * 128);        // S stages x Ng/128 x 128 block maxima
  float* sTh = sBm + S * Ng;                                     // K x Ng scaled parameters (when resident)
  __shared__ __align__(8) uint64_t bar_theta, bar_a_full[kP1Stages], bar_a_empty[kP1Stages], bar_off_free[kP1Stages],
      bar_d_full[kP1Bufs], bar_d_empty[kP1Bufs], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ double sred[kP1Threads / 32];
  __shared__ unsigned long long sMask[kP1Stages];  // blocks visited on the stage's tile (bit q: image block q)

  const int tid = threadIdx.x, warp = tid >> 5;
  const int nq = Ng / 128;  // grain blocks of this launch
  const int64_t n_tiles = tm.n_tiles;
  // the blocks of this launch visited on the tile of stage s
  const uint64_t all_q = nq >= 64 ? ~0ull : ((1ull << nq) - 1ull);
  auto tile_mask = [&](int s) -> uint64_t { return masks ? (sMask[s] >> (g0 / 128)) & all_q : all_q; };
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar_theta, 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(&bar_a_full[s], kP1Producers);
      mbar_init(&bar_a_empty[s], 1);
      mbar_init(&bar_off_free[s], 128);  // the warpgroup of the stage's tile
    }
    for (int b = 0; b < kP1Bufs; ++b) {
      mbar_init(&bar_d_full[b], 1);
      mbar_init(&bar_d_empty[b], 128);  // one warpgroup reads a buffer
    }
    mbar_init(&bar_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kP1MmaWarp) tmem_alloc(&tmem_slot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  double racc = 0.0;
  if (warp == kP1MmaWarp) {
    if (tid == kP1MmaWarp * 32) {
      // parameter image (and the float parameters when they fit): one bulk
      // copy per 32 KiB
      const uint32_t total = (uint32_t)Ng * kRowBytes;
      const uint32_t row_t = (uint32_t)Ng * 4;  // one feature row of the float parameters
      mbar_arrive_expect_tx(&bar_theta, total + (th_resident ? (uint32_t)K * row_t : 0u));
      const uint8_t* src = img + (size_t)g0 * kRowBytes;
      for (uint32_t off = 0; off < total; off += 32768u) {
        const uint32_t n = total - off < 32768u ? total - off : 32768u;
        bulk_g2s(sB + off, src + off, n, &bar_theta);
      }
      for (int k = 0; th_resident && k < K; ++k) {
        const uint8_t* rsrc = reinterpret_cast<const uint8_t*>(th32t + (size_t)k * Npad + g0);
        uint8_t* rdst = reinterpret_cast<uint8_t*>(sTh + (size_t)k * Ng);
        for (uint32_t off = 0; off < row_t; off += 32768u)
          bulk_g2s(rdst + off, rsrc + off, row_t - off < 32768u ? row_t - off : 32768u, &bar_theta);
      }
      bool ok = mbar_wait(&bar_theta, 0, &abort_flag, status);
      // Two cursors, one per epilogue warpgroup: cursor h holds a tile of
      // position parity h and issues its blocks into the warpgroup's two
      // TMEM buffers (h * 2, h * 2 + 1).  Tiles are taken in order, each
      // once its operands are in; the cursors alternate as their buffers
      // free, so that neither warpgroup waits behind the other's tile.
      // Every wait below is a non-blocking test inside one bounded loop.
      int it_next = 0;            // position of the next tile to take
      int it_of[2] = {0, 0};      // position of each cursor's tile
      uint64_t rem[2] = {0, 0};   // its blocks not yet issued
      bool act[2] = {false, false};
      int64_t cw[2] = {0, 0};     // blocks issued into each warpgroup's ring
      const int n_mine = (int)((n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);  // tiles of this CTA
      uint64_t t_last = global_ns();
      while (ok) {
        bool done = true, prog = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!act[h]) {
            if (it_next < n_mine && (it_next & 1) == h) {
              done = false;
              const int s = it_next % S;
              if (mbar_peek(&bar_a_full[s], (uint32_t)((it_next / S) & 1))) {
                tc_fence_after();
                it_of[h] = it_next++;
                rem[h] = tile_mask(s);
                act[h] = true;
                prog = true;
              }
            }
            continue;
          }
          done = false;
          const int s = it_of[h] % S;
          if (rem[h] == 0) {
            mma_commit(&bar_a_empty[s]);  // the tile's operands are no longer read
            act[h] = false;
            prog = true;
            continue;
          }
          const int b = h * 2 + (int)(cw[h] & 1);
          if (cw[h] >= 2 && !mbar_peek(&bar_d_empty[b], (uint32_t)(((cw[h] >> 1) - 1) & 1))) continue;
          tc_fence_after();
          const int q = __ffsll((long long)rem[h]) - 1;
          rem[h] &= rem[h] - 1;
          const uint32_t aaddr = smem_addr(sA + s * kTileBytes);
          const uint32_t baddr = smem_addr(sB + (size_t)q * 128 * kRowBytes);
          mma_terms<KS, KW>(tmem + b * 128, aaddr, KT * 16, false, baddr, KT * 16, IDESC);
          mma_commit(&bar_d_full[b]);
          ++cw[h];
          prog = true;
        }
        if (done) break;
        if (prog) {
          t_last = global_ns();
        } else if (abort_flag) {
          ok = false;
        } else if (global_ns() - t_last > kWaitLimitNs) {
          abort_flag = 1;
          atomicCAS(status, 0, PD_ETIMEOUT);
          ok = false;
        }
      }
      // every MMA issued above has completed before TMEM is released
      mma_commit(&bar_drain);
      mbar_wait_drain(&bar_drain, 0);
    }
    __syncwarp();
  } else if (warp >= kTcConsumers / 32 && warp < kP1MmaWarp) {
    // pixel row p0 of every tile (a producer warp on each SM sub-partition);
    // the next tile's pixel index, coordinates and label are fetched while
    // this one is written
    const int p0 = tid - kTcConsumers;
    // feature-major parameters: lanes that read consecutive grains hit
    // consecutive banks; grain i of this launch (global g0 + i)
    const float* thp = th_resident ? sTh : th32t + g0;
    const int ldt = th_resident ? Ng : Npad;
    auto dot_t = [&](int i, const float* e) {
      float acc = thp[i] * e[0];
#pragma unroll
      for (int k = 1; k < K; ++k) acc = fmaf(thp[(int64_t)k * ldt + i], e[k], acc);
      return acc;
    };
    // any grain (the label may lie outside this launch's grains)
    auto dot_g = [&](int G, const float* e) {
      if (G >= g0 && G < g0 + Ng) return dot_t(G - g0, e);
      float acc = th32t[G] * e[0];
#pragma unroll
      for (int k = 1; k < K; ++k) acc = fmaf(th32t[(int64_t)k * Npad + G], e[k], acc);
      return acc;
    };
    bool ok = !th_resident || mbar_wait_warp(&bar_theta, 0, &abort_flag, status);
    int64_t jn[kP1PixPerThread];
    float xn[kP1PixPerThread][DIM], cn[DIM], dxn[kP1PixPerThread][DIM];
    int Gn[kP1PixPerThread];
    unsigned long long maskn = 0;
    auto fetch = [&](int64_t t) {
#pragma unroll
      for (int u = 0; u < kP1PixPerThread; ++u) {
        jn[u] = tile_pixel_dx<DIM>(g, tm, t, p0 + kP1Producers * u, xn[u], cn, dxn[u]);
        Gn[u] = jn[u] >= 0 ? labels[jn[u]] : -1;
      }
      if (masks && p0 == 0) maskn = masks[t];
    };
    if (ok && blockIdx.x < n_tiles) fetch(blockIdx.x);
    int it = 0;
    for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
      const int s = it % S, use = it / S;
      int64_t jc[kP1PixPerThread];
      float xc[kP1PixPerThread][DIM], cc[DIM], dxc[kP1PixPerThread][DIM];
      int Gc[kP1PixPerThread];
#pragma unroll
      for (int u = 0; u < kP1PixPerThread; ++u) {
        jc[u] = jn[u];
        Gc[u] = Gn[u];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          xc[u][a] = xn[u][a];
          dxc[u][a] = dxn[u][a];
        }
      }
#pragma unroll
      for (int a = 0; a < DIM; ++a) cc[a] = cn[a];
      const unsigned long long maskc = maskn;
      if (t + gridDim.x < n_tiles) fetch(t + gridDim.x);
      if (use >= 1 && (!mbar_wait_warp(&bar_a_empty[s], (uint32_t)((use - 1) & 1), &abort_flag, status) ||
                       !mbar_wait_warp(&bar_off_free[s], (uint32_t)((use - 1) & 1), &abort_flag, status)))
        break;
      if (p0 == 0) {
        // the tile's centre offsets of this launch's grains, by one bulk
        // copy that the stage's barrier also waits for, and the blocks to
        // visit (one copy per visited block instead moves fewer bytes but
        // made the pass slower: the copies are issued one after another)
        sMask[s] = maskc;
        fence_proxy_async();
        mbar_expect_tx(&bar_a_full[s], (uint32_t)Ng * 4);
        bulk_g2s(sOff + s * Ng, offg + t * Npad + g0, (uint32_t)Ng * 4, &bar_a_full[s]);
      }
#pragma unroll
      for (int u = 0; u < kP1PixPerThread; ++u) {
        const int p = p0 + kP1Producers * u;
        float de[K];
        legendre_delta<DIM, D>(xc[u], cc, dxc[u], de, nullptr);
        store_eta_row<K, KW, KS>(sA + s * kTileBytes, p, de);
        float start = -INFINITY, lg = 0.f;
        int lrow = -1;
        if (jc[u] >= 0) {
          const int G = Gc[u];
          if ((unsigned)G < (unsigned)N) {
            // the label logit relative to the tile's reference logit: its
            // centre offset plus the remainder
            lrow = rank ? rank[G] : G;
            lg = offg[t * Npad + lrow] + dot_g(G, de);
            start = lg;
          } else {
            lg = NAN;
          }
          // one of the launches owns the label logit of a grain-split pass
          if (lg_out && (G >= g0 && G < g0 + Ng || ((unsigned)G >= (unsigned)N && g0 == 0))) lg_out[jc[u]] = lg;
        }
        sLG[s * 128 + p] = start;
        sLGv[s * 128 + p] = lg;
        sJ[s * 128 + p] = (long long)jc[u];
        sLRow[s * 128 + p] = lrow;
      }
      fence_proxy_async();
      mbar_arrive(&bar_a_full[s]);
    }
  } else {
    const int quad = warp & 3, half = warp >> 2, lane = tid & 31;
    const int row = quad * 32 + lane;  // pixel row of the tile == TMEM lane
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    // online log-sum-exp over 32 logits (grains cbase .. cbase+31, nv of
    // them valid); the running max starts at the label logit (a lower bound
    // of the max, usually the max itself), so most chunks of far-away grains
    // lie more than 127 below it: their exponentials underflow to exactly
    // zero in ex2.approx.ftz and the whole chunk is skipped.  The label's
    // own column (li, when in 0..31) is left out: ssum sums the other
    // grains only, and the label's term, from the producers' label logit,
    // joins at the end, so that 1 - p_G and log p_G carry no cancellation
    // when p_G is close to 1
    auto chunk = [&](const uint32_t(&r)[32], const float* off, int nv, int li, float& m, float& ssum) -> float {
      if (nv <= 0) return -INFINITY;
      float v[32];
      const float4* off4 = reinterpret_cast<const float4*>(off);  // 16-byte aligned: cbase is a multiple of 32
      if (nv >= 32) {  // (warp-uniform) a full chunk: packed adds, no masking
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          const float4 o = off4[q >> 2];
          const float2 a = __fadd2_rn(make_float2(__uint_as_float(r[q]), __uint_as_float(r[q + 1])), make_float2(o.x, o.y));
          const float2 b =
              __fadd2_rn(make_float2(__uint_as_float(r[q + 2]), __uint_as_float(r[q + 3])), make_float2(o.z, o.w));
          v[q] = a.x;
          v[q + 1] = a.y;
          v[q + 2] = b.x;
          v[q + 3] = b.y;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          const float4 o = off4[q >> 2];
          v[q] = q < nv ? __uint_as_float(r[q]) + o.x : -INFINITY;
          v[q + 1] = q + 1 < nv ? __uint_as_float(r[q + 1]) + o.y : -INFINITY;
          v[q + 2] = q + 2 < nv ? __uint_as_float(r[q + 2]) + o.z : -INFINITY;
          v[q + 3] = q + 3 < nv ? __uint_as_float(r[q + 3]) + o.w : -INFINITY;
        }
      }
      {
        const uint32_t lm = (unsigned)li < 32u ? 1u << li : 0u;
        if (__any_sync(0xffffffffu, lm != 0u)) {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = (lm >> q) & 1u ? -INFINITY : v[q];
        }
      }
      const float cm = tree_max32(v);
      if (__all_sync(0xffffffffu, cm < m - 127.f)) return cm;
      const float mn = fmaxf(m, cm);
      const float2 nmn = make_float2(-mn, -mn);
#pragma unroll
      for (int q = 0; q < 32; q += 2) {
        const float2 a = __fadd2_rn(make_float2(v[q], v[q + 1]), nmn);
        v[q] = Arith<float>::ex(a.x);
        v[q + 1] = Arith<float>::ex(a.y);
      }
      ssum = fmaf(ssum, Arith<float>::ex(m - mn), tree_sum32(v));
      m = mn;
      return cm;
    };
    // a block's 128 columns in four 32-column chunks, each loaded while the
    // one before is used; warpgroup `half` takes the tiles of even or odd
    // position and, in order, all their visited blocks
    uint32_t RA[32], RB[32];
    int it = 0;
    int64_t cw = 0;  // blocks this warpgroup has read
    bool ok = true;
    for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
      if ((it & 1) != half) continue;
      const int s = it % S;
      // the stage's operands and per-row values come from the producers
      ok = mbar_wait_warp(&bar_a_full[s], (uint32_t)((it / S) & 1), &abort_flag, status);
      if (!ok) break;
      float m = sLG[s * 128 + row], ssum = 0.f;
      const uint64_t msk0 = tile_mask(s);
      for (uint64_t msk = msk0; msk; msk &= msk - 1, ++cw) {
        const int q = __ffsll((long long)msk) - 1;
        const int b = half * 2 + (int)(cw & 1);  // this warpgroup's two buffers
        const uint32_t col = (uint32_t)(b * 128);
        ok = mbar_wait_warp(&bar_d_full[b], (uint32_t)((cw >> 1) & 1), &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        tmem_ld32(tmem + lane_base + col, RA);
        const int cbase = q * 128;
        const float* off = sOff + s * Ng + cbase;
        const int nrem = N - g0 - cbase;  // valid grains from this chunk on
        const int lb = sLRow[s * 128 + row] - g0 - cbase;  // the label's column in the block (when in 0..127)
        tmem_wait_ld();
        tmem_ld32(tmem + lane_base + col + 32, RB);
        float bm = chunk(RA, off, nrem, lb, m, ssum);
        tmem_wait_ld();
        tmem_ld32(tmem + lane_base + col + 64, RA);
        bm = fmaxf(bm, chunk(RB, off + 32, nrem - 32, lb - 32, m, ssum));
        tmem_wait_ld();
        tmem_ld32(tmem + lane_base + col + 96, RB);
        bm = fmaxf(bm, chunk(RA, off + 64, nrem - 64, lb - 64, m, ssum));
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&bar_d_empty[b]);  // the logits are in registers: release the TMEM buffer
        bm = fmaxf(bm, chunk(RB, off + 96, nrem - 96, lb - 96, m, ssum));
        // the largest logit of this pixel in the block
        sBm[s * Ng + q * 128 + row] = bm;
      }
      if (!ok) break;
      const int64_t j = sJ[s * 128 + row];
      float lse = NAN;
      if (j >= 0) {
        if (ms_out) {
          ms_out[j] = make_float2(m, ssum);  // this launch's grains only: merged later
          // a lower bound of the pixel's log2 S for the need bits: this
          // group's part, and the label logit (one term of the full sum)
          lse = fmaxf(m + Arith<float>::lg(ssum), sLG[s * 128 + row]);
        } else {
          // the label's term joins (a NaN label logit: a label outside 0..N-1)
          const LabelLse r = label_lse(m, ssum, sLGv[s * 128 + row]);
          lse = r.lse;
          lse_out[j] = r.lse;
          q_out[j] = r.q;
          racc += r.logp;
        }
      }
      if (need_bits) {
        // a 128-grain block is needed by the gradient pass on this tile
        // unless every probability in it is below 2^-26: the fp16
        // gradient operand would round all of them to zero
        for (int q = 0; q < nq; ++q) {
          const bool nd = ((msk0 >> q) & 1) && j >= 0 && !(sBm[s * Ng + q * 128 + row] < lse - 26.f);
          const uint32_t bal = __ballot_sync(0xffffffffu, nd);
          if (lane == 0 && bal)
            atomicOr(&need_bits[(int64_t)(g0 / 128 + q) * n_words + (t >> 5)], 1u << (int)(t & 31));
        }
        // the gradient pass forms c = delta - p, so the block of every
        // pixel's label is needed on its tile (set by the first launch)
        if (g0 == 0) {
          const int lrow = j >= 0 ? sLRow[s * 128 + row] : -1;
          const int lq = lrow >= 0 ? lrow / 128 : -1;
          const unsigned same = __match_any_sync(0xffffffffu, lq);
          if (lq >= 0 && lane == __ffs(same) - 1)
            atomicOr(&need_bits[(int64_t)lq * n_words + (t >> 5)], 1u << (int)(t & 31));
        }
      }
      mbar_arrive(&bar_off_free[s]);
    }
    tmem_wait_ld();  // no TMEM load may be outstanding when the columns are freed
    if (!ok) racc = NAN;
  }
  if (abort_flag) racc = NAN;
  // objective partial of this CTA (fixed order)
  {
    double v = racc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sred[warp] = v;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += sred[w];
    if (abort_flag) sum = NAN;
    obj_part[blockIdx.x] = sum;
  }
  if (warp == kP1MmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

// The gradient pass's CTAs per grain block, in proportion to the blocks'
// kept-tile counts: one to every block with kept tiles, the rest by the
// floor of the proportional share, the leftover one each to the first
// blocks with kept tiles.  p2_share gives CTA r its block, its index among
// the block's CTAs and their number; every caller computes the same split.
struct P2Share {
  int gb, idx, n;
};
// Walks the blocks in order with their first CTA and CTA count; stops when
// stop(b, first, count) returns true.  O(nb).
template <typename F>
__device__ __forceinline__ void p2_walk(const int* counts, int64_t n_tiles, int nb, int n_cta, F stop) {
  long long U = 0;
  int base = 0;
  for (int b = 0; b < nb; ++b) {
    const long long c = counts ? counts[b] : n_tiles;
    U += c;
    base += c > 0;
  }
  if (U == 0) return;
  const long long R = n_cta - base;
  long long floors = 0;
  for (int b = 0; b < nb; ++b) {
    const long long c = counts ? counts[b] : n_tiles;
    if (c > 0) floors += R * c / U;
  }
  long long left = R - floors;
  int pre = 0;
  for (int b = 0; b < nb; ++b) {
    const long long c = counts ? counts[b] : n_tiles;
    int a = 0;
    if (c > 0) {
      a = 1 + (int)(R * c / U);
      if (left > 0) {
        ++a;
        --left;
      }
    }
    if (stop(b, pre, a)) return;
    pre += a;
  }
}
__device__ __forceinline__ P2Share p2_share(const int* counts, int64_t n_tiles, int nb, int n_cta, int r) {
  P2Share sh{0, 0, 0};
  p2_walk(counts, n_tiles, nb, n_cta, [&](int b, int first, int a) {
    if (r < first + a) {
      sh = P2Share{b, r - first, a};
      return true;
    }
    return false;
  });
  return sh;
}

template <int DIM, int D, int KS, int NB, int NA>
__global__ void __launch_bounds__(kP2ThreadsG, 1)
k_tc_pass2(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, int Npad, const uint8_t* __restrict__ img,
           const float* __restrict__ offg, const float* __restrict__ lse, const float* __restrict__ qin,
           const int* __restrict__ kept, const int* __restrict__ n_kept_gb, int nb, const int* __restrict__ perm,
           double* __restrict__ part, int* __restrict__ status) {
  using L = Pass2Layout<DIM, D, KS>;
  constexpr int K = L::K, KW = L::KW, KT = L::KT, ET = L::ET, N2 = L::N2, CT = L::CT, LB = L::LB;
  constexpr uint32_t IDESC1 = idesc_bf16(128, kTcPixTile);
  constexpr uint32_t IDESC2 = idesc_f16(128, N2);
  constexpr int D2COL = LB * kTcPixTile;  // TMEM: D1 ring [0, LB*128); D2 buffer db at D2COL + db*CT*N2
  static_assert(D2COL + 2 * CT * N2 <= kTcCols, "TMEM columns");
  constexpr float kLoScale = 4096.f;       // c_lo = fl16((c - c_hi) * 2^12)

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                             // theta block image
  uint8_t* sB = sA + L::kABytes;                  // NB stages of eta - eta(c) rows
  uint8_t* sB2 = sB + NB * L::kBBytes;            // NB stages of eta^T
  uint8_t* sA2 = sB2 + NB * L::kB2Bytes;          // NA stages of c (CT terms)
  float* sLse = reinterpret_cast<float*>(sA2 + NA * L::kA2Bytes);  // [NB][128] log2 S of the pixels
  float* sOffP = sLse + NB * kTcPixTile;                           // [NB][128] centre logits of the block
  int* sLab = reinterpret_cast<int*>(sOffP + NB * 128);            // [NB][128] labels of the pixels
  float* sNq = reinterpret_cast<float*>(sLab + NB * kTcPixTile);  // [NB][128] -(1 - p_G) of the pixels
  __shared__ __align__(8) uint64_t bar_theta, bar_b_full[NB], bar_b_empty[NB], bar_d1_full[LB], bar_d1_empty[LB],
      bar_a2_full[NA], bar_a2_empty[NA], bar_d2_full[2], bar_d2_free[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5;
  // this CTA's grain block and share of the tiles on which the block has a
  // non-negligible probability or a label (all tiles without the lists), in
  // tile order; chunks of kP2ChunkTiles of them add up to one gradient partial
  const P2Share sh = p2_share(kept ? n_kept_gb : nullptr, tm.n_tiles, nb, gridDim.x, blockIdx.x);
  const int gb = sh.gb;  // grain block
  const int64_t n_list = sh.n > 0 ? (kept ? (int64_t)n_kept_gb[gb] : tm.n_tiles) : 0;
  const int64_t k_lo = sh.n > 0 ? n_list * sh.idx / sh.n : 0;
  const int n_kept = sh.n > 0 ? (int)(n_list * (sh.idx + 1) / sh.n - k_lo) : 0;
  const int* klist = kept ? kept + (int64_t)gb * tm.n_tiles + k_lo : nullptr;
  auto tile_of = [&](int t) -> int64_t { return klist ? (int64_t)klist[t] : k_lo + t; };
  const int n_used = (n_kept + kP2ChunkTiles - 1) / kP2ChunkTiles;  // chunks
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar_theta, 1);
    for (int s = 0; s < NB; ++s) {
      mbar_init(&bar_b_full[s], kP2Producers);
      mbar_init(&bar_b_empty[s], 2);  // both MMA issuers are done with the stage
    }
    for (int b = 0; b < LB; ++b) {
      mbar_init(&bar_d1_full[b], 1);
      mbar_init(&bar_d1_empty[b], kTcConsumers);
    }
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
  if (warp == kP2MmaWarp) tmem_alloc(&tmem_slot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kP2MmaWarp) {
    // logits D1(t) = theta_block . (eta - eta(c))^T, as far ahead of the
    // consumers as the TMEM ring and the operand stages allow
    if (tid == kP2MmaWarp * 32) {
      mbar_arrive_expect_tx(&bar_theta, L::kABytes);
      bulk_g2s(sA, img + (size_t)gb * L::kABytes, L::kABytes, &bar_theta);
      bool ok = mbar_wait(&bar_theta, 0, &abort_flag, status);
      for (int t = 0; ok && t < n_kept; ++t) {
        const int s = t % NB, b1 = t % LB;
        ok = mbar_wait(&bar_b_full[s], (uint32_t)((t / NB) & 1), &abort_flag, status);
        if (ok && t >= LB) ok = mbar_wait(&bar_d1_empty[b1], (uint32_t)(((t / LB) - 1) & 1), &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        mma_terms<KS, KW>(tmem + b1 * kTcPixTile, smem_addr(sA), KT * 16, true, smem_addr(sB + s * L::kBBytes),
                          L::kSboB, IDESC1);
        mma_commit(&bar_d1_full[b1]);
        mma_commit(&bar_b_empty[s]);
      }
      mma_commit(&bar_drain);
      mbar_wait_drain(&bar_drain, 0);
    }
    __syncwarp();
  } else if (warp == kP2GradWarpG) {
    // gradient D2 += C . [eta_h | eta_l] (fp16), one product per term of c
    // into its own columns; one D2 accumulation per chunk, alternating
    // between two TMEM buffers so that the consumers read one while the
    // next fills
    if (tid == kP2GradWarpG * 32) {
      bool ok = true;
      for (int t = 0; ok && t < n_kept; ++t) {
        const int s = t % NB, a = t % NA;
        const int u = t / kP2ChunkTiles, db = u & 1;
        const bool first = t % kP2ChunkTiles == 0, last = t % kP2ChunkTiles == kP2ChunkTiles - 1 || t == n_kept - 1;
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
  } else if (warp >= kP2ProdWarp0 && warp < kP2MmaWarp) {
    // pixel operands of every tile: the logit operand row (eta - eta(c)),
    // the transposed gradient operand (eta), log2 S and the label of the
    // pixel and (first thread) the block's centre logits.  A thread owns one
    // pixel row; the next tile's coordinates, log2 S and label are fetched
    // while the current tile is written.
    const int p = tid - kTcConsumers;
    float xn[DIM], cn[DIM], dxn[DIM], lsn = INFINITY, nqn = 0.f;
    int labn = -1;
    auto fetch = [&](int t) {
      const int64_t j = tile_pixel_dx<DIM>(g, tm, tile_of(t), p, xn, cn, dxn);
      lsn = j >= 0 ? lse[j] : INFINITY;
      labn = j >= 0 ? labels[j] : -1;
      nqn = j >= 0 ? -qin[j] : 0.f;
    };
    if (n_kept > 0) fetch(0);
    for (int t = 0; t < n_kept; ++t) {
      const int s = t % NB;
      float xc[DIM], cc[DIM], dxc[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        xc[a] = xn[a];
        cc[a] = cn[a];
        dxc[a] = dxn[a];
      }
      const float lsc = lsn, nqc = nqn;
      const int labc = labn;
      const int64_t tc = tile_of(t);
      if (t + 1 < n_kept) fetch(t + 1);
      if (t >= NB && !mbar_wait_warp(&bar_b_empty[s], (uint32_t)(((t / NB) - 1) & 1), &abort_flag, status)) break;
      if (p == 0) {
        // the block's centre logits for this tile, by one bulk copy that the
        // stage's barrier also waits for
        fence_proxy_async();
        mbar_expect_tx(&bar_b_full[s], 128 * 4);
        bulk_g2s(sOffP + s * 128, offg + tc * Npad + gb * 128, 128 * 4, &bar_b_full[s]);
      }
      float e0[K], de[K];
      legendre_delta<DIM, D>(xc, cc, dxc, de, e0);
      store_eta_row<K, KW, KS, L::kSboB>(sB + s * L::kBBytes, p, de);
      // eta^T in fp16 (hi, and lo for PD_BF16X3); neighbouring threads fill
      // the two halves of one 32-bit word (pixels outside the set have
      // c = 0, so their features need no masking)
      uint8_t* b2 = sB2 + s * L::kB2Bytes;
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const float a0 = k < K ? e0[k] : 0.f;
        const __half h = __float2half_rn(a0);
        const uint32_t o = kmaj_s(k, p, L::kLbo2, L::kSbo2);
        *reinterpret_cast<__half*>(b2 + o) = h;
        if (ET == 2) *reinterpret_cast<__half*>(b2 + L::kB2Term + o) = __float2half_rn(a0 - __half2float(h));
      }
      sLse[s * kTcPixTile + p] = lsc;
      sLab[s * kTcPixTile + p] = labc;
      sNq[s * kTcPixTile + p] = nqc;
      fence_proxy_async();
      mbar_arrive(&bar_b_full[s]);
    }
  } else {
    const int quad = warp & 3, half = warp >> 2, lane = tid & 31;
    const int gr = quad * 32 + lane;        // grain row of the block == TMEM lane
    const int i = gb * 128 + gr;            // this thread's row of the parameter image
    const int gi = perm ? perm[i] : (i < N ? i : -1);  // its grain (-1: padding)
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    int n_done = 0;  // chunks this thread has added up (first warpgroup)
    // the CTA's partial of this grain (a row of part): the D2 rows of its
    // chunks added in order, in double
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
    // c = p - delta for 32 pixels (columns q0 .. q0+31 of this thread's
    // half; the sign returns at the reduction), written as fp16 pairs, one
    // 16-byte core-matrix row per 8 pixels: c_hi = fl16(c) and, for
    // PD_BF16X3, c_lo = fl16((c - c_hi) 2^12).  The label's c = -(1 - p_G)
    // comes from pass 1 (no cancellation when p_G is close to 1).
    auto emit = [&](const uint32_t(&r)[32], const float* ls, const int* lab, const float* nq, float off,
                    uint8_t* a2, int q0) {
#pragma unroll
      for (int q8 = 0; q8 < 32; q8 += 8) {
        const float4 va = *reinterpret_cast<const float4*>(ls + q8);
        const float4 vb = *reinterpret_cast<const float4*>(ls + q8 + 4);
        const int4 la = *reinterpret_cast<const int4*>(lab + q8);
        const int4 lb = *reinterpret_cast<const int4*>(lab + q8 + 4);
        const float4 na = *reinterpret_cast<const float4*>(nq + q8);
        const float4 nb = *reinterpret_cast<const float4*>(nq + q8 + 4);
        const float lv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
        const int lg[8] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w};
        const float nv[8] = {na.x, na.y, na.z, na.w, nb.x, nb.y, nb.z, nb.w};
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          // l - log2 S = r + (off - lv); two pixels per packed fp32
          // operation throughout (each rounds as its scalar form would)
          const float2 t = __fadd2_rn(make_float2(off, off), make_float2(-lv[u], -lv[u + 1]));
          const float2 x = __fadd2_rn(make_float2(__uint_as_float(r[q8 + u]), __uint_as_float(r[q8 + u + 1])), t);
          // c = p - delta
          const float2 c = make_float2(lg[u] == gi ? nv[u] : Arith<float>::ex(x.x),
                                       lg[u + 1] == gi ? nv[u + 1] : Arith<float>::ex(x.y));
          const __half2 h = __floats2half2_rn(c.x, c.y);
          hw[u >> 1] = *reinterpret_cast<const uint32_t*>(&h);
          if (CT == 2) {
            // c - c_hi is exact in fp32, and the scaling by 2^12 too
            const float2 dlo = __ffma2_rn(__half22float2(h), make_float2(-1.f, -1.f), c);
            const float2 slo = __fmul2_rn(dlo, make_float2(kLoScale, kLoScale));
            const __half2 l2 = __floats2half2_rn(slo.x, slo.y);
            lw[u >> 1] = *reinterpret_cast<const uint32_t*>(&l2);
          }
        }
        const uint32_t o = kmaj(gr, q0 + q8, kTcPixTile);
        *reinterpret_cast<uint4*>(a2 + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        if (CT == 2) *reinterpret_cast<uint4*>(a2 + L::kA2Term + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    };
    // the two 32-column halves of the thread's logits: the second is loaded
    // while the first is used, and the first half of the next tile (when the
    // tensor cores have it ready) while the second is used
    uint32_t RA[32], RB[32];
    bool pre = false;
    bool ok = true;
    for (int t = 0; t < n_kept; ++t) {
      const int s = t % NB, b1 = t % LB, a = t % NA;
      const uint32_t col = (uint32_t)(b1 * kTcPixTile + half * 64);
      // sLse, sLab, sNq and sOffP of the stage were written by the producers
      if (!mbar_wait_warp(&bar_b_full[s], (uint32_t)((t / NB) & 1), &abort_flag, status)) { ok = false; break; }
      if (!pre) {
        if (!mbar_wait_warp(&bar_d1_full[b1], (uint32_t)((t / LB) & 1), &abort_flag, status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        tmem_ld32(tmem + lane_base + col, RA);
      }
      tmem_wait_ld();
      tmem_ld32(tmem + lane_base + col + 32, RB);
      // this grain's centre logit for the tile
      const float off = sOffP[s * 128 + gr];
      if (t >= NA && !mbar_wait_warp(&bar_a2_empty[a], (uint32_t)(((t / NA) - 1) & 1), &abort_flag, status)) {
        ok = false;
        break;
      }
      const float* ls = sLse + s * kTcPixTile + half * 64;
      const int* lb = sLab + s * kTcPixTile + half * 64;
      const float* nq = sNq + s * kTcPixTile + half * 64;
      uint8_t* a2 = sA2 + a * L::kA2Bytes;
      emit(RA, ls, lb, nq, off, a2, half * 64);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(&bar_d1_empty[b1]);  // the tile's logits are in registers: release its TMEM columns
      pre = false;
      if (t + 1 < n_kept) {
        const int bn = (t + 1) % LB;
        if (__all_sync(0xffffffffu, mbar_peek(&bar_d1_full[bn], (uint32_t)(((t + 1) / LB) & 1)))) {
          tc_fence_after();
          tmem_ld32(tmem + lane_base + (uint32_t)(bn * kTcPixTile + half * 64), RA);
          pre = true;
        }
      }
      emit(RB, ls + 32, lb + 32, nq + 32, off, a2, half * 64 + 32);
      fence_proxy_async();
      mbar_arrive(&bar_a2_full[a]);
      // the first warpgroup writes the previous chunk's partial one tile
      // into the next chunk, when its gradient MMAs are long done
      if (half == 0 && t > kP2ChunkTiles && t % kP2ChunkTiles == 1 && !read_chunk(t / kP2ChunkTiles - 1)) {
        ok = false;
        break;
      }
    }
    tmem_wait_ld();  // a prefetched load may be outstanding after an abort
    if (half == 0) {
      // the chunks not yet read: the last one (and, for a one-tile last
      // chunk, the one before); the CTA's partial is NaN after an abort
      for (int u = n_done; ok && u < n_used; ++u) ok = read_chunk(u);
      if (prow && (!ok || n_used == 0)) {
        for (int k = 0; k < K; ++k) prow[k] = ok ? 0.0 : NAN;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kP2MmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

// ---------------------------------------------------------------------------
// Log-sum-exp of a grain-split pass 1: the (max, sum) of every group of
// grains per pixel combine into log2 S(x); the objective terms l_G - log2 S
// are summed per block in a fixed order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_tc_merge_lse(const float2* __restrict__ ms, int n_grp, int64_t P, const float* __restrict__ lg,
               float* __restrict__ lse_out, float* __restrict__ q_out, double* __restrict__ obj_part,
               const int* __restrict__ status) {
  __shared__ double sred[8];
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double r = 0.0;
  if (j < P) {
    // every group's max starts at the label logit lG and its sum leaves the
    // label's own term out: the label joins here
    float m = -INFINITY;
    for (int q = 0; q < n_grp; ++q) m = fmaxf(m, ms[(int64_t)q * P + j].x);
    float sum = 0.f;
    for (int q = 0; q < n_grp; ++q) {
      const float2 v = ms[(int64_t)q * P + j];
      if (v.y > 0.f) sum = fmaf(v.y, Arith<float>::ex(v.x - m), sum);
    }
    const LabelLse t = label_lse(m, sum, lg[j]);
    lse_out[j] = t.lse;
    q_out[j] = t.q;
    r = t.logp;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sred[w];
    obj_part[blockIdx.x] = *status ? NAN : t;  // a pass-1 launch gave up
  }
}

// ---------------------------------------------------------------------------
// Gradient and objective of the evaluation: per grain the label part (64-bit
// fixed point) plus the pass-2 partials of its block's CTAs, in a fixed
// order; block 0 also sums the objective partials.  (The other CTAs' rows
// of the grain are never written.)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_tc_reduce_eval(const double* __restrict__ part, int n_cta, const int* __restrict__ n_kept_gb, int nb,
                 const int* __restrict__ rank, int64_t n_tiles, int K, int64_t NK,
                 const unsigned long long* __restrict__ base, double inv_fx, double scale, double* __restrict__ grad,
                 const double* __restrict__ objp, int n_obj, double obj_scale, double* __restrict__ obj) {
  __shared__ double ssum[8][32];
  if (obj && blockIdx.x == 0) {
    if (threadIdx.y == 0) {
      double v = 0.0;
      for (int q = threadIdx.x; q < n_obj; q += 32) v += objp[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (threadIdx.x == 0) *obj = v * obj_scale;
    }
  }
  if (!grad) return;
  const int64_t q = (int64_t)blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (q < NK) {
    // the CTAs of this grain's block, [r0, r0 + n), as the gradient pass
    // gave them out
    const int gi = (int)(q / K);
    const int gb = (rank ? rank[gi] : gi) / 128;
    int r0 = 0, n = 0;
    p2_walk(n_kept_gb, n_tiles, nb, n_cta, [&](int b, int first, int a) {
      if (b != gb) return false;
      r0 = first;
      n = a;
      return true;
    });
    for (int r = r0 + threadIdx.y; r < r0 + n; r += 8) s += part[(int64_t)r * NK + q];
  }
  ssum[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && q < NK) {
    double t = base ? (double)(long long)base[q] * inv_fx : 0.0;
#pragma unroll
    for (int y = 0; y < 8; ++y) t += ssum[y][threadIdx.x];
    grad[q] = t * scale;
  }
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits: one CTA waits on an mbarrier that nothing
// arrives at; the wait gives up after limit_ns and records PD_ETIMEOUT.
// ---------------------------------------------------------------------------
__global__ void k_selftest_timeout(uint64_t limit_ns, int* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint64_t t0 = global_ns();
  bool done = false;
  while (!(done = mbar_test(&bar, 0))) {
    if (abort_flag) break;
    if (global_ns() - t0 > limit_ns) {
      abort_flag = 1;
      break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !done) atomicCAS(status, 0, PD_ETIMEOUT);
}

template <int DIM, int D, int KS>
int eval_tc_dd(const EvalCall& c, cudaStream_t st) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * n_terms(KS);
  const int N = c.N;
  const int64_t P = c.g.P;
  const int Npad = (N + kTcGrainTile - 1) / kTcGrainTile * kTcGrainTile;  // parameter image rows
  const size_t row_bytes = (size_t)KT * 2;
  constexpr size_t kCap = 220 * 1024;
  // pass 1 keeps the image of ng grains resident: the image, and per
  // operand stage the pixel rows, centre logits, start and label logits,
  // pixel indices and block maxima; and the float parameters when they
  // fit too.  More grains than one SM holds are split into groups of ng,
  // one launch each, whose (max, sum) per pixel are merged afterwards.
  auto p1_bytes = [&](size_t ng, bool th_res, size_t S = 2) {
    return ng * row_bytes + S * (kTcPixTile * row_bytes + ng * 4 + 2 * kTcPixTile * 4 + kTcPixTile * 8 +
                                 kTcPixTile * 4 + ng * 4) +
           (th_res ? (size_t)K * ng * 4 : 0);
  };
  int n_grp = 1, Ng = Npad;
  while (p1_bytes((size_t)Ng, false) > kCap && Ng > kTcGrainTile) {
    ++n_grp;
    Ng = ((Npad + n_grp - 1) / n_grp + kTcGrainTile - 1) / kTcGrainTile * kTcGrainTile;
  }
  n_grp = (Npad + Ng - 1) / Ng;
  const int th_resident = p1_bytes((size_t)Ng, true) <= kCap ? 1 : 0;
  // a third operand stage where it fits beside the same grains
  const int p1_stages = p1_bytes((size_t)Ng, th_resident != 0, kP1Stages) <= kCap ? kP1Stages : 2;
  const size_t smem1 = p1_bytes((size_t)Ng, th_resident != 0, (size_t)p1_stages);
  // pass-2 stages: four pixel-operand and two gradient-operand stages when
  // they fit, else fewer
  using L2 = Pass2Layout<DIM, D, KS>;
  constexpr int NB = L2::bytes(4, 2) <= kCap ? 4 : (L2::bytes(3, 2) <= kCap ? 3 : (L2::bytes(2, 1) <= kCap ? 2 : 1));
  constexpr int NA = L2::bytes(NB, 2) <= kCap ? 2 : 1;
  const size_t smem2 = L2::bytes(NB, NA);
  if (smem1 > kCap || smem2 > kCap) return PD_ENOTSUP;
  // pixel-centre numerators 2k+1-n stay exact integers in fp32
  if (!c.g.coords && std::max(c.g.n0, std::max(c.g.n1, c.g.n2)) > (int64_t(1) << 23)) return PD_ENOTSUP;
  // at least 120 KiB of dynamic shared memory per CTA keeps one CTA per SM,
  // which owns all 512 TMEM columns
  const size_t smem1_req = std::max<size_t>(smem1, 120 * 1024);
  const size_t smem2_req = std::max<size_t>(smem2, 120 * 1024);

  const TileMap tm = make_tiles<DIM>(c.g);
  const int sms = device_sm_count();
  const int64_t n_tiles = tm.n_tiles;
  const int grid1 = (int)std::min<int64_t>(n_tiles, sms);
  const int gridm = (int)((P + 255) / 256);  // merge blocks of a grain-split pass 1
  const int gblocks = (N + 127) / 128;  // pass-2 grain blocks
  // pass 2: one wave of CTAs, at least one per grain block, the blocks
  // sharing the SMs in proportion to their kept tiles (p2_share); a CTA
  // takes a contiguous share of its block's tiles and writes one gradient
  // partial per grain of the block
  const int n_cta2 = std::max(sms, gblocks);
  // The gradient pass visits only the (tile, block) pairs with a
  // probability that survives in its fp16 operand (judged against a lower
  // bound of log2 S when pass 1 runs in grain groups), and the grains are
  // reordered so that blocks are compact regions.
  // (PD_TC_NO_SKIP=1 in the environment visits every pair in index order,
  // for tests that compare the two)
  const char* no_skip = getenv("PD_TC_NO_SKIP");
  const bool skip_on = !(no_skip && no_skip[0] && no_skip[0] != '0');
  const bool skip = c.grad && skip_on;
  // pass 1 leaves out the blocks that the centre-logit bounds show to be
  // far below the tile's reference logit (structured grids)
  const bool bounds = skip_on && !c.g.coords && Npad / 128 <= 64;
  const bool order = skip && Npad <= kOrderMax;

  constexpr int KP = padded_K<float>(K);
  constexpr int K1 = DIM + 1;  // label moments of degree <= 1: counts and centroids for the grain order
  // (a plan makes every allocation on every call, so that its arena keeps
  // the centre features and the grain order at the same place)
  const bool all = c.plan != nullptr;
  Scratch sc(st, c.plan);
  uint8_t* img = sc.get<uint8_t>((size_t)Npad * row_bytes);
  float* th32t = sc.get<float>((size_t)K * Npad);
  float* thH = sc.get<float>((size_t)N * KP);  // float-float parameters for the centre logits
  float* thL = sc.get<float>((size_t)N * KP);
  float2* ecg = sc.get<float2>((size_t)n_tiles * K);  // centre features per tile
  float* offg = sc.get<float>((size_t)n_tiles * Npad);  // relative centre logits [tile][image row]
  float* lse = sc.get<float>((size_t)P);
  float* qv = sc.get<float>((size_t)P);  // 1 - p_G per pixel
  double* objp = sc.get<double>((size_t)std::max(grid1, n_grp > 1 ? gridm : 1));
  float2* ms = n_grp > 1 ? sc.get<float2>((size_t)n_grp * P) : nullptr;
  float* lgb = n_grp > 1 ? sc.get<float>((size_t)P) : nullptr;
  double* part = (c.grad || all) ? sc.get<double>((size_t)n_cta2 * N * K) : nullptr;  // one partial per pass-2 CTA and grain
  // one bit per (128-grain block, tile): the block has a probability that
  // the gradient pass cannot neglect on the tile; then the tiles per block
  const int64_t n_words = (n_tiles + 31) / 32;
  uint32_t* need = (skip || all) ? sc.get<uint32_t>((size_t)(Npad / 128) * n_words) : nullptr;
  int* kept = (skip || all) ? sc.get<int>((size_t)(Npad / 128) * n_tiles) : nullptr;
  int* nkept = (skip || all) ? sc.get<int>((size_t)(Npad / 128)) : nullptr;
  int* perm = (order || all) ? sc.get<int>((size_t)Npad) : nullptr;
  int* rank = (order || all) ? sc.get<int>((size_t)N) : nullptr;
  unsigned long long* lmom = (order || all) ? sc.get<unsigned long long>((size_t)N * K1) : nullptr;
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
  if (need && cudaMemsetAsync(need, 0, sizeof(uint32_t) * (size_t)(Npad / 128) * n_words, st) != cudaSuccess)
    return PD_ECUDA;

  // |eta| <= 1, so a grain's label sum is bounded by P: the largest
  // power-of-two scale that keeps P * scale below 2^62
  int bits = 0;
  while (bits < 62 && ((int64_t)1 << bits) <= P) ++bits;
  const float fx = ldexpf(1.f, 62 - bits);
  if (order && !have_order) {
    // the grains' label centroids (sums of 1 and x per grain) for the order
    if (cudaMemsetAsync(lmom, 0, sizeof(unsigned long long) * N * K1, st) != cudaSuccess) return PD_ECUDA;
    const int64_t nthr = n_tiles * kTcPixTile;
    PD_TIMED(st, "tc_label_moments",
             (k_tc_label_moments<DIM, 1><<<(unsigned)((nthr + 255) / 256), 256, 0, st>>>(c.g, tm, c.labels, N, fx,
                                                                                       lmom)));
    PD_TIMED(st, "tc_grain_order",
             k_tc_grain_order<DIM><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(lmom, N, K1, Npad, perm, rank));
  }
  const double scale = Arith<float>::theta_scale(c.eps);
  {
    // the operand image, the transposed copy and the float-float parameters
    const int64_t n = (int64_t)Npad * KW;
    PD_TIMED(st, "tc_theta_image",
             k_tc_theta_image<KS><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.theta, N, Npad, K, KW, scale,
                                                                                nullptr, perm, img, th32t, thH, thL,
                                                                                KP));
  }
  if (!have_features)
    PD_TIMED(st, "centre_features",
             (k_centre_features<DIM, D><<<centre_feature_blocks(n_tiles), kFeatThreads, 0, st>>>(c.g, tm, ecg)));
  PD_TIMED(st, "tc_tile_setup",
           (k_tc_tile_setup<DIM, D><<<tile_centre_blocks(n_tiles), kRefThreads, 0, st>>>(
               c.g, tm, thH, thL, N, Npad, perm, ecg, offg, tb, bounds ? 1 : 0, masks)));
  auto k1 = k_tc_pass1<DIM, D, KS>;
  if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1_req) != cudaSuccess)
    return PD_ECUDA;
  for (int q = 0; q < n_grp; ++q) {
    const int g0 = q * Ng, ng = std::min(Ng, Npad - g0);
    PD_TIMED(st, KS == 1 ? "tc_bf16_lse_pass1" : "tc_bf16x3_lse_pass1",
             k1<<<grid1, kP1Threads, smem1_req, st>>>(c.g, tm, c.labels, N, Npad, g0, ng, p1_stages, img, th32t,
                                                      th_resident, offg, perm ? rank : nullptr,
                                                      lse, qv, objp, ms ? ms + (size_t)q * P : nullptr, lgb, masks, need,
                                                      n_words, status));
  }
  // a launch that fails (resources, configuration) is an error of this call
  if (cudaPeekAtLastError() != cudaSuccess) return PD_ECUDA;
  if (n_grp > 1)
    PD_TIMED(st, "tc_merge_lse", k_tc_merge_lse<<<gridm, 256, 0, st>>>(ms, n_grp, P, lgb, lse, qv, objp, status));
  if (c.grad) {
    if (skip)
      PD_TIMED(st, "tc_kept_lists",
               k_tc_kept_lists<<<(unsigned)(Npad / 128), 1024, 0, st>>>(need, n_words, n_tiles, kept, nkept));
    auto k2 = k_tc_pass2<DIM, D, KS, NB, NA>;
    if (cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2_req) != cudaSuccess)
      return PD_ECUDA;
    PD_TIMED(st, KS == 1 ? "tc_bf16_grad_pass2" : "tc_bf16x3_grad_pass2",
             k2<<<n_cta2, kP2ThreadsG, smem2_req, st>>>(c.g, tm, c.labels, N, Npad, img, offg, lse, qv, kept,
                                                        nkept, gblocks, perm, part, status));
    if (cudaPeekAtLastError() != cudaSuccess) return PD_ECUDA;
  }
  if (c.obj || c.grad) {
    const int64_t NK = (int64_t)N * K;
    const unsigned blocks = c.grad ? (unsigned)((NK + 31) / 32) : 1u;
    PD_TIMED(st, "reduce_eval",
             k_tc_reduce_eval<<<blocks, dim3(32, 8), 0, st>>>(
                 part, n_cta2, kept ? nkept : nullptr, gblocks, perm ? rank : nullptr, n_tiles, K, NK,
                 (const unsigned long long*)nullptr, 1.0 / (double)fx, 1.0 / (c.eps * (double)P), c.grad, objp, n_grp > 1 ? gridm : grid1, 1.0 / (double)P,
                 c.obj));
  }
  if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
  if (c.plan) {
    c.plan->features = true;
    c.plan->order = c.plan->order || order;
  }
  return PD_OK;
}

template <int KS>
int eval_tc_ks(const EvalCall& c, cudaStream_t st) {
  if (c.dim == 2) {
    switch (c.d) {
      case 1: return eval_tc_dd<2, 1, KS>(c, st);
      case 2: return eval_tc_dd<2, 2, KS>(c, st);
      case 3: return eval_tc_dd<2, 3, KS>(c, st);
      case 4: return eval_tc_dd<2, 4, KS>(c, st);
      case 5: return eval_tc_dd<2, 5, KS>(c, st);
      case 6: return eval_tc_dd<2, 6, KS>(c, st);
      default: return PD_ENOTSUP;
    }
  }
  if (c.dim == 3) {
    switch (c.d) {
      case 1: return eval_tc_dd<3, 1, KS>(c, st);
      case 2: return eval_tc_dd<3, 2, KS>(c, st);
      case 3: return eval_tc_dd<3, 3, KS>(c, st);
      default: return PD_ENOTSUP;
    }
  }
  return PD_ENOTSUP;
}

}  // namespace

int selftest_wait_timeout(double seconds, int* status_out, cudaStream_t st) {
  Scratch sc(st);
  int* dstat = sc.get<int>(1);
  if (!sc.ok()) return PD_ENOMEM;
  if (cudaMemsetAsync(dstat, 0, sizeof(int), st) != cudaSuccess) return PD_ECUDA;
  k_selftest_timeout<<<1, 32, 0, st>>>((uint64_t)(seconds * 1e9), dstat);
  if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
  if (cudaMemcpyAsync(status_out, dstat, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PD_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PD_OK : PD_ECUDA;
}

int eval_tc(const EvalCall& c, cudaStream_t st) {
  if (c.v) return eval_tc_hvp(c, st);
  if (c.prec == PD_BF16) return eval_tc_ks<1>(c, st);
  if (c.prec == PD_BF16X3) return eval_tc_ks<6>(c, st);
  return PD_ENOTSUP;
}

}  // namespace pd

extern "C" int pd_selftest_wait_timeout(double seconds, int* status_out, void* stream) {
  if (!status_out || !(seconds > 0.0) || seconds > 1.0) return PD_EINVAL;
  return pd::selftest_wait_timeout(seconds, status_out, (cudaStream_t)stream);
}
