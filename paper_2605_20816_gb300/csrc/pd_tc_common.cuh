// pd_tc_common.cuh -- building blocks of the tensor-core (tcgen05) passes:
// PTX wrappers for mbarriers, TMEM, MMAs and bulk copies, the operand layouts,
// the parameter images, the pixel tiles and the centre logits; included by
// the objective/gradient passes (pd_tc.cu) and the Hessian-vector passes
// (pd_tc_hvp.cu), each of which gets its own internal copy.
//
// Operands use the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, adjacent along K at 128 bytes (LBO) and along the
// rows at KT*16 bytes (SBO), KT = the operand's total K width.
//
// Every wait on an mbarrier is bounded by a 1 s timeout on the global timer:
// a wait that gives up sets PD_ETIMEOUT in a status word (the result then
// becomes NaN), raises a CTA-wide abort flag so that the other waits give up
// at once, and the CTA still frees its TMEM before it returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pd_simt_kernels.cuh"

namespace pd {
namespace {


constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
constexpr int kTcConsumers = 256;                 // warps 0..7: TMEM consumers
constexpr int kTcProducers = 64;                  // warps 8..9: pixel-operand producers, 2 pixels each
constexpr int kTcMmaWarp = 10;                    // TMEM allocation and MMA issue
constexpr int kTcThreads = 11 * 32;               // at most 3 warps per SM sub-partition
constexpr int kTcCols = 512;                      // TMEM columns per CTA (one CTA per SM)
constexpr int kTcGrainTile = 256;                 // pass-1 grains per MMA group (N of the MMA)
constexpr int kTcPixTile = kTilePix;              // pixels per tile (both passes)
// objective pass 1: 8 epilogue warps, 4 producer warps (one pixel per
// thread, one producer on each SM sub-partition), one MMA warp
constexpr int kP1Producers = 128;
constexpr int kP1PixPerThread = kTcPixTile / kP1Producers;
constexpr int kP1MmaWarp = (kTcConsumers + kP1Producers) / 32;
constexpr int kP1Threads = (kP1MmaWarp + 1) * 32;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  uint64_t state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(smem_addr(b)) : "memory");
  (void)state;
}
// Adds bytes to the transaction count of the current phase (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_addr(b)), "r"(bytes)
               : "memory");
  (void)state;
}
// Non-blocking probe of the phase (test_wait never suspends the thread).
__device__ __forceinline__ bool mbar_peek(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the completion of the phase with the given parity.  Returns false
// when the CTA aborted or the wait timed out (then the abort flag is raised
// and PD_ETIMEOUT recorded).
__device__ __noinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* status) {
  if (mbar_test(b, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_test(b, parity)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 > kWaitLimitNs) {
      *abort_flag = 1;
      if (status) atomicCAS(status, 0, PD_ETIMEOUT);
      return false;
    }
  }
}
// Warp-uniform variant for the epilogue warps: the tcgen05.ld that follow a
// wait are .sync.aligned, so the whole warp must agree on the outcome.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* status) {
  const bool ok = mbar_wait(b, parity, abort_flag, status);
  return __all_sync(0xffffffffu, ok);
}
// Bounded wait that ignores the abort flag: used once before TMEM is freed,
// so that no MMA still writes the columns being released.
__device__ __noinline__ void mbar_wait_drain(uint64_t* b, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_test(b, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) return;
  }
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D[tmem] (+)= A[smem] . B[smem]^T, both K-major, bf16 in, fp32 accumulate.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on the mbarrier when all previously issued MMAs of this
// thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(b))
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns: thread t of the warp reads
// lane (base lane + t), columns col .. col+31 of the address.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
}


// Shared-memory matrix descriptor, K-major, no swizzle (layout type 0),
// descriptor version 1; lbo/sbo in bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f16: fp32 D, bf16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same with fp16 A and B.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Byte offset of element (row r, column k) of a K-major no-swizzle operand
// whose core matrices lie lbo bytes apart along K and sbo bytes apart along
// the rows.
__host__ __device__ constexpr uint32_t kmaj_s(int r, int k, uint32_t lbo, uint32_t sbo) {
  return (uint32_t)((r >> 3) * sbo + (k >> 3) * lbo + (r & 7) * 16 + (k & 7) * 2);
}
// The dense case: rows KT elements wide.
__host__ __device__ constexpr uint32_t kmaj(int r, int k, int KT) { return kmaj_s(r, k, 128u, (uint32_t)KT * 16u); }


// Term split of the operands.  KS is the number of products per logit (1
// for PD_BF16, 6 for PD_BF16X3); n_terms(KS) the bf16 terms stored per
// value.  Product s pairs parameter term theta_term(s) with feature term
// eta_term(s): hh, hm, mh, hl, mm, lh.
__host__ __device__ constexpr int n_terms(int KS) { return KS == 1 ? 1 : 3; }
__host__ __device__ constexpr int theta_term(int s) { return s == 2 || s == 4 ? 1 : (s == 5 ? 2 : 0); }
__host__ __device__ constexpr int eta_term(int s) { return s == 1 || s == 4 ? 1 : (s == 3 ? 2 : 0); }

// The KS products of a logit chain: MMAs of K = 16 whose A and B
// descriptors start at the term slices of the two operands (rows of KT
// columns: slice t at column t*KW).  kind::f16, M = 128, N from idesc.
// The products are issued smallest first (lh, mm, hl, mh, hm, hh): the
// accumulator truncates, and its partial sums stay small until the last,
// leading product is added.
template <int KS, int KW>
__device__ __forceinline__ void mma_terms(uint32_t d, uint32_t aaddr, uint32_t a_sbo, bool a_theta, uint32_t baddr,
                                          uint32_t b_sbo, uint32_t idesc) {
#pragma unroll 1
  for (int si = 0; si < KS; ++si) {
    const int s = KS - 1 - si;
    const int ta = KS == 1 ? 0 : (a_theta ? theta_term(s) : eta_term(s));
    const int tb = KS == 1 ? 0 : (a_theta ? eta_term(s) : theta_term(s));
#pragma unroll
    for (int q = 0; q < KW / 16; ++q) {
      const uint64_t ad = smem_desc(aaddr + (uint32_t)(ta * KW * 16 + q * 256), 128, a_sbo);
      const uint64_t bd = smem_desc(baddr + (uint32_t)(tb * KW * 16 + q * 256), 128, b_sbo);
      mma_bf16(d, ad, bd, idesc, (si > 0 || q > 0) ? 1u : 0u);
    }
  }
}

// Writes the terms of a feature row (pixel r) into a K-major operand.
template <int K, int KW, int KS, uint32_t SBO = (uint32_t)KW * n_terms(KS) * 16>
__device__ __forceinline__ void store_eta_row(uint8_t* base, int r, const float* eta) {
  // hi, mid, lo bf16 terms (round to nearest, each of the remainder of the
  // previous ones), two adjacent columns per 32-bit word
  constexpr int NT = n_terms(KS);
  uint32_t w[NT][KW / 2];
#pragma unroll
  for (int k = 0; k < KW; k += 2) {
    float v0 = k < K ? eta[k] : 0.f, v1 = k + 1 < K ? eta[k + 1] : 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      w[t][k >> 1] = *reinterpret_cast<const uint32_t*>(&h);
      if (t + 1 < NT) {
        const float2 f = __bfloat1622float2(h);
        v0 -= f.x;
        v1 -= f.y;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
#pragma unroll
    for (int k8 = 0; k8 < KW; k8 += 8) {
      const uint4 v = make_uint4(w[t][k8 / 2], w[t][k8 / 2 + 1], w[t][k8 / 2 + 2], w[t][k8 / 2 + 3]);
      *reinterpret_cast<uint4*>(base + kmaj_s(r, t * KW + k8, 128u, SBO)) = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Parameter images: rows = grains (in the order perm gives, when given;
// padded to Npad with zero rows), K-major no-swizzle, one slice of KW
// columns per term; plus a transposed float copy (K x Npad, in the
// caller's grain order) used for the label logit of the objective, and
// (thH != nullptr) the float-float parameters [N][KP] in the caller's order
// (as k_theta_ff writes them) for the centre offsets.
// ---------------------------------------------------------------------------
template <int KS>
__global__ void k_tc_theta_image(const double* __restrict__ theta, int N, int Npad, int K, int KW, double scale,
                                 const double* __restrict__ dscale, const int* __restrict__ perm,
                                 uint8_t* __restrict__ img, float* __restrict__ th32t, float* __restrict__ thH,
                                 float* __restrict__ thL, int KP) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (row, k) pairs
  if (q >= (int64_t)Npad * KW) return;
  const int r = (int)(q / KW), k = (int)(q % KW);
  const int src = perm ? perm[r] : (r < N ? r : -1);  // row r holds grain src (-1: zero padding)
  const double t = (src >= 0 && k < K) ? theta[(int64_t)src * K + k] * (dscale ? scale * *dscale : scale) : 0.0;
  const uint16_t h = __bfloat16_as_ushort(__double2bfloat16(t));
  const double r1 = t - (double)__bfloat162float(__ushort_as_bfloat16(h));
  const uint16_t m = __bfloat16_as_ushort(__double2bfloat16(r1));
  const double r2 = r1 - (double)__bfloat162float(__ushort_as_bfloat16(m));
  const uint16_t l = __bfloat16_as_ushort(__double2bfloat16(r2));
  const uint16_t parts[3] = {h, m, l};
  const int KT = KW * n_terms(KS);
  for (int t = 0; t < n_terms(KS); ++t) *reinterpret_cast<uint16_t*>(img + kmaj(r, t * KW + k, KT)) = parts[t];
  // transposed float copy in the caller's grain order, zero rows beyond N
  if (k < K) th32t[(int64_t)k * Npad + (src >= 0 ? src : r)] = (float)t;
  if (thH && src >= 0 && k < KP) {
    const float h32 = (float)t;
    thH[(int64_t)src * KP + k] = h32;
    thL[(int64_t)src * KP + k] = (float)(t - (double)h32);
  }
}

// ---------------------------------------------------------------------------
// Pixel tiles (pd_tiles.cuh).  The logits of a tile's pixels are formed
// relative to the tile's reference logit C(t): the centre part
// theta'_i . eta(c) - C(t) per grain and tile from float-float arithmetic
// (k_tc_tile_setup), the small remainder theta'_i . (eta(x) - eta(c)) on
// the tensor cores, whose fp32 accumulation truncates (its biased error must
// act on small numbers).
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ float dot_f(const float* __restrict__ a, const float* __restrict__ b) {
  float acc = a[0] * b[0];
#pragma unroll
  for (int k = 1; k < K; ++k) acc = fmaf(a[k], b[k], acc);
  return acc;
}

// three-input maximum (a non-NaN operand wins over NaN, as in fmaxf)
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float tree_max32(const float* v) {
  float a[11];
#pragma unroll
  for (int q = 0; q < 10; ++q) a[q] = fmax3f(v[3 * q], v[3 * q + 1], v[3 * q + 2]);
  a[10] = fmaxf(v[30], v[31]);
  const float b0 = fmax3f(a[0], a[1], a[2]), b1 = fmax3f(a[3], a[4], a[5]), b2 = fmax3f(a[6], a[7], a[8]);
  return fmax3f(b0, b1, fmax3f(b2, a[9], a[10]));
}
// pairwise sums in packed fp32 adds (fixed order)
__device__ __forceinline__ float tree_sum32(const float* v) {
  float2 a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    a[q] = __fadd2_rn(make_float2(v[4 * q], v[4 * q + 1]), make_float2(v[4 * q + 2], v[4 * q + 3]));
#pragma unroll
  for (int w = 4; w >= 1; w >>= 1)
#pragma unroll
    for (int q = 0; q < w; ++q) a[q] = __fadd2_rn(a[q], a[q + w]);
  return a[0].x + a[0].y;
}

// ---------------------------------------------------------------------------
// Warp roles (both passes): warps 0..7 consume TMEM (warp w reads lanes
// 32 (w mod 4) .. +31, the access rule of tcgen05.ld, and the column half
// w / 4 of each 128-column tile); warps 8..9 produce the pixel-side
// operands of upcoming tiles (two pixels per thread); warp 10 allocates
// TMEM and one of its threads issues every MMA.  Eleven warps keep at most
// three on each SM sub-partition, which leaves 168 registers per thread.  Producers run ahead of the
// consumers by the number of operand stages, so their global loads and
// feature arithmetic overlap the consumers' work.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_consumer(int warp) { return warp < 8; }
__device__ __forceinline__ bool is_producer(int warp) { return warp >= 8 && warp < kTcMmaWarp; }

// ---------------------------------------------------------------------------
// Centre parts theta'_i . eta(c_t) of every tile t and grain i in plain
// fp32 (zero for padding grains): the Hessian passes take u = v . eta split
// at the tile centre with these (u is not shift-invariant and of modest
// size, so it needs no reference).  A block takes 256 grains (parameters in
// registers) and kCentreTiles tiles (centre features in shared memory); the
// same fma order as a per-grain fp32 dot product.
//
// With bounds (structured grids): the features of a tile's pixels differ
// from those at its centre pixel by |eta_k(x) - eta_k(c)| <= D_k, where
// D_k = sum_a alpha_a (alpha_a + 1) / 2 * h_a, since |P_m| <= 1 and
// |P_m'| <= m (m + 1) / 2 on [-1, 1] and |x_a - c_a| <= h_a in the tile.
// So every logit of grain i in tile t lies within A_i = sum_k |theta'_ik| D_k
// of the centre logit, and the kernel writes A_i and, per tile and
// 128-grain block, the largest off_i + A_i (+inf for a tile that crosses
// the grid edge, whose centre may lie outside [-1, 1]).
// ---------------------------------------------------------------------------
constexpr int kCentreTiles = 32;


template <int DIM, int D>
__global__ void __launch_bounds__(256)
k_tc_centre_logits(Geom g, TileMap tm, const float* __restrict__ th32t, const int* __restrict__ perm, int N,
                   int Npad, float* __restrict__ off, TileBound tb, float* __restrict__ amax, float* __restrict__ mb) {
  constexpr int K = basis_K(DIM, D);
  __shared__ float sec[kCentreTiles][K];
  __shared__ float smx[kCentreTiles][8];
  __shared__ int srag[kCentreTiles];
  const int i = blockIdx.x * 256 + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nblk = Npad / 128;
  const bool live = i < Npad;  // (every thread takes part in the barriers)
  // the grain of image row i (the float copy is in the caller's order)
  const int src = perm ? (live ? perm[i] : -1) : (i < N ? i : -1);
  float th[K];
#pragma unroll
  for (int k = 0; k < K; ++k) th[k] = src >= 0 ? th32t[(int64_t)k * Npad + src] : 0.f;
  float A = 0.f;
  if (mb) {
#pragma unroll
    for (int k = 0; k < K; ++k) A = fmaf(fabsf(th[k]), tb.d[k], A);
    if (blockIdx.y == 0 && live) amax[i] = A;
  }
  for (int64_t t0 = (int64_t)blockIdx.y * kCentreTiles; t0 < tm.n_tiles; t0 += (int64_t)gridDim.y * kCentreTiles) {
    const int nt = (int)min((int64_t)kCentreTiles, tm.n_tiles - t0);
    __syncthreads();  // the previous group's features and maxima are used up
    if (threadIdx.x < nt) {
      float x[DIM], c[DIM], ec[K];
      tile_pixel<DIM>(g, tm, t0 + threadIdx.x, 0, x, c);
      legendre_features<DIM, D>(c, ec);
#pragma unroll
      for (int k = 0; k < K; ++k) sec[threadIdx.x][k] = ec[k];
      // the tile's last pixel lies outside the grid: a ragged tile
      srag[threadIdx.x] = tile_pixel<DIM>(g, tm, t0 + threadIdx.x, kTcPixTile - 1, x, c) < 0;
    }
    __syncthreads();
    for (int q = 0; q < nt; ++q) {
      float acc = th[0] * sec[q][0];
#pragma unroll
      for (int k = 1; k < K; ++k) acc = fmaf(th[k], sec[q][k], acc);
      if (live) off[(t0 + q) * Npad + i] = acc;
      if (mb) {
        float v = src >= 0 ? acc + A : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) smx[q][wid] = v;
      }
    }
    if (mb) {
      __syncthreads();
      if (threadIdx.x < 2 * nt) {
        const int q = threadIdx.x >> 1, h = threadIdx.x & 1, blk = blockIdx.x * 2 + h;
        const float v = fmaxf(fmaxf(smx[q][4 * h], smx[q][4 * h + 1]), fmaxf(smx[q][4 * h + 2], smx[q][4 * h + 3]));
        if (blk < nblk) mb[(t0 + q) * nblk + blk] = srag[q] ? INFINITY : v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Pass 2: gradient partials of one grain block over a contiguous run of
// tiles (one wave of CTAs per grain block).  NB pixel-operand stages (up to
// 4) and NA gradient-operand stages (up to 2), as many as shared memory
// holds.  Two warps issue MMAs: one the logits, as far ahead as the three
// TMEM logit buffers and the operand stages allow, the other the gradient
// contractions, so neither waits behind the other.  The consumers pick the
// next tile's logits up early when they are already there.  The gradient
// accumulates in TMEM over chunks of kP2ChunkTiles tiles (two buffers,
// alternating), and the chunks add up in double to one partial per grain.
//
// Shared-memory operand layouts (all K-major, no swizzle):
//   sB   pixel rows x KT feature differences; the 8-row groups lie
//        KT*16 + 16 bytes apart, so that the producers' stores of even and
//        of odd rows spread over all banks;
//   sB2  features x 128 pixels (eta transposed); the 8-pixel core matrices
//        lie 144 bytes apart along K, so that 32 threads storing one 32-bit
//        word (two adjacent pixels) each hit 32 different banks;
//   sA2  grains x 128 pixels of c, dense.
// ---------------------------------------------------------------------------
template <int DIM, int D, int KS>
struct Pass2Layout {
  static constexpr int K = basis_K(DIM, D);
  static constexpr int KW = (K + 15) / 16 * 16;
  static constexpr int KT = KW * n_terms(KS);
  static constexpr int ET = KS == 1 ? 1 : 2;  // fp16 terms of eta in the gradient contraction
  static constexpr int N2 = ET * KW;           // its MMA N: eta_h (and eta_l) columns
  static constexpr int CT = KS == 1 ? 1 : 2;  // fp16 terms of c (hi, and lo scaled by 2^12)

  static constexpr uint32_t kABytes = 128u * KT * 2;             // theta block
  static constexpr uint32_t kSboB = (uint32_t)KT * 16 + 16;
  static constexpr uint32_t kBBytes = 16 * kSboB;                // 128 pixel rows
  static constexpr uint32_t kLbo2 = 144;
  static constexpr uint32_t kSbo2 = 16 * kLbo2;
  static constexpr uint32_t kB2Term = (KW / 8) * kSbo2;
  static constexpr uint32_t kB2Bytes = ET * kB2Term;           // rows: eta_h features, then eta_l
  static constexpr uint32_t kA2Term = 128u * kTcPixTile * 2;     // one term of c: 128 grains x 128 pixels, fp16
  static constexpr uint32_t kA2Bytes = CT * kA2Term;
  // + log2 S, centre logits of the block, labels of the pixels, -(1 - p_G)
  static constexpr uint32_t kPerB = kBBytes + kB2Bytes + kTcPixTile * 4 + 128 * 4 + kTcPixTile * 4 + kTcPixTile * 4;
  static constexpr size_t bytes(int nb, int na) { return kABytes + (size_t)nb * kPerB + (size_t)na * kA2Bytes; }
  // TMEM: the logit ring (128 columns a tile) and two gradient buffers of
  // CT x N2 columns; three logit buffers where they fit
  static constexpr int LB = 3 * kTcPixTile + 2 * CT * N2 <= kTcCols ? 3 : 2;
};

constexpr int kP2GradWarp = 11;       // pass 2: the gradient MMAs have their own issuing warp
constexpr int kP2Threads = 12 * 32;   // three warps on every SM sub-partition
// The gradient pass of pd_tc.cu: 8 epilogue warps, 4 producer warps (one
// pixel a thread, one warp on every SM sub-partition), one warp for the
// logit MMAs (and TMEM), one for the gradient MMAs.
constexpr int kP2ProdWarp0 = 8;
constexpr int kP2Producers = 128;
constexpr int kP2MmaWarp = 12;
constexpr int kP2GradWarpG = 13;
constexpr int kP2ThreadsG = 14 * 32;
constexpr int kP2ChunkTiles = 32;     // tiles per gradient partial (fp32 accumulation length)
// tiles per Hessian-vector partial: the accumulator truncates, and c = p (u -
// ubar) has no exact cancellation to keep its partial sums small, so it is
// read out more often
constexpr int kH2ChunkTiles = 8;

// out[q] = scale * mul * (base[q] / fx + sum_c part[c][q]), fixed order;
// base (fixed-point label moments) and mul (a device-side factor) optional
__global__ void __launch_bounds__(32 * kRedPhases)
k_tc_reduce_grad(const double* __restrict__ part, int nchunks, int64_t NK, const unsigned long long* __restrict__ base,
                 double inv_fx, double scale, const double* __restrict__ mul, double* __restrict__ out) {
  __shared__ double ssum[kRedPhases][32];
  const int64_t q = (int64_t)blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (q < NK)
    for (int c = threadIdx.y; c < nchunks; c += kRedPhases) s += part[(int64_t)c * NK + q];
  ssum[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && q < NK) {
    double t = base ? (double)(long long)base[q] * inv_fx : 0.0;
#pragma unroll
    for (int y = 0; y < kRedPhases; ++y) t += ssum[y][threadIdx.x];
    out[q] = t * (mul ? scale * *mul : scale);
  }
}

// ---------------------------------------------------------------------------
// Label part of eq. (grad): sum_{x in G_i} eta(x) per grain, at the points
// of the tile walk of the two passes.  A warp sums the features of each
// group of equal labels in fp32 (a fixed butterfly order), and lane k adds
// the group's feature-k sum to the grain's 64-bit fixed-point accumulator,
// so that the result does not depend on the order of the atomics.
// ---------------------------------------------------------------------------
template <int DIM, int D>
__global__ void __launch_bounds__(256)
k_tc_label_moments(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, float fx_scale,
                   unsigned long long* __restrict__ acc) {
  constexpr int K = basis_K(DIM, D);
  static_assert(K <= 32, "one lane per feature");
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = q / kTcPixTile;
  int G = -1;
  float x[DIM], c[DIM], eta[K];
#pragma unroll
  for (int a = 0; a < DIM; ++a) x[a] = 0.f;
  if (t < tm.n_tiles) {
    const int64_t j = tile_pixel<DIM>(g, tm, t, (int)(q % kTcPixTile), x, c);
    if (j >= 0) {
      G = labels[j];
      if ((unsigned)G >= (unsigned)N) G = -1;
    }
  }
  legendre_features<DIM, D>(x, eta);
  const int lane = threadIdx.x & 31;
  unsigned todo = __ballot_sync(0xffffffffu, G >= 0);
  while (todo) {
    const int L = __shfl_sync(0xffffffffu, G, __ffs(todo) - 1);
    const bool mine = G == L;
    float pick = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float v = mine ? eta[k] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == k) pick = v;
    }
    if (lane < K) atomicAdd(&acc[(int64_t)L * K + lane], (unsigned long long)__float2ll_rn(pick * fx_scale));
    todo &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// ---------------------------------------------------------------------------
// Grain order of the gradient pass.  Grains sorted by the Morton code of
// their label centroid (from the fixed-point label sums: feature 0 is 1,
// features 1..DIM are x_1..x_DIM) make a 128-grain block of the parameter
// image a compact region of the domain, so that most (tile, block) pairs
// carry only negligible probabilities.  Ties, and grains without pixels
// (last), go by index: the order is deterministic.  perm[r] is the grain
// of image row r (-1 beyond N), rank its inverse.  N <= kOrderMax; one
// thread per grain.
// ---------------------------------------------------------------------------
constexpr int kOrderMax = 2048;

__device__ __forceinline__ uint32_t spread_bits(uint32_t v, int dim) {
  // bit b of v moves to bit dim * b
  uint32_t r = 0;
  for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (dim * b);
  return r;
}

template <int DIM>
__global__ void __launch_bounds__(256)
k_tc_grain_order(const unsigned long long* __restrict__ lmom, int N, int K, int Npad, int* __restrict__ perm,
                 int* __restrict__ rank) {
  __shared__ unsigned long long key[kOrderMax];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const long long cnt = (long long)lmom[(int64_t)i * K];
    uint32_t code = 0xffffffffu;
    if (cnt > 0) {
      code = 0;
      // (a 10-bit cell per axis: float division is ample, and the
      // double-precision one cost most of this kernel)
      const float inv = 1.f / (float)cnt;
      for (int a = 0; a < DIM; ++a) {
        const float c = (float)(long long)lmom[(int64_t)i * K + 1 + a] * inv;  // in [-1, 1]
        int v = (int)((c + 1.f) * 512.f);
        v = v < 0 ? 0 : (v > 1023 ? 1023 : v);
        code |= spread_bits((uint32_t)v, DIM) << a;
      }
    }
    key[i] = ((unsigned long long)code << 32) | (uint32_t)i;
  }
  __syncthreads();
  // the keys are distinct (index in the low half): a grain's rank is the
  // number of smaller keys; every CTA holds all keys and ranks its 256
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    const unsigned long long ki = key[i];
    int r = 0;
    for (int j = 0; j < N; ++j) r += key[j] < ki;
    perm[r] = i;
    rank[i] = r;
  }
  if (blockIdx.x == 0)
    for (int r = N + threadIdx.x; r < Npad; r += blockDim.x) perm[r] = -1;
}

// ---------------------------------------------------------------------------
// Per 128-grain block, the tiles whose need bit pass 1 set, in increasing
// order (an ordered compaction, one CTA per block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_tc_kept_lists(const uint32_t* __restrict__ need, int64_t n_words, int64_t n_tiles, int* __restrict__ lists,
                int* __restrict__ counts) {
  __shared__ int wsum[32];
  __shared__ int base;
  const int gb = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t* row = need + (int64_t)gb * n_words;
  int* out = lists + (int64_t)gb * n_tiles;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int64_t w0 = 0; w0 < n_words; w0 += 1024) {
    const int64_t w = w0 + threadIdx.x;
    uint32_t bits = w < n_words ? row[w] : 0u;
    const int c = __popc(bits);
    int x = c;  // inclusive scan in the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int v = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;  // inclusive over warps
    }
    __syncthreads();
    int pos = base + (wid > 0 ? wsum[wid - 1] : 0) + x - c;
    while (bits) {
      const int b = __ffs((int)bits) - 1;
      out[pos++] = (int)(w * 32 + b);
      bits &= bits - 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[gb] = base;
}

// A block of grains is left out of a log-sum-exp pass when every logit of
// it lies more than kP1Far (log2 units) below the pixel's maximum: its
// exponentials underflow to zero in ex2.approx.ftz.
constexpr float kP1Far = 130.f;

// ---------------------------------------------------------------------------
// Per-tile set-up of the tensor-core passes, one block per kRefTiles tiles:
// the centre features (double, kept as float-float pairs), the reference
// logit C(t) of each tile (the largest fp32 centre logit, pd_tiles.cuh),
// the relative centre logits o_i(t) = theta'_i . eta(c_t) - C(t) of every
// image row (zero for padding rows), and on structured grids the 128-grain
// blocks pass 1 visits on each tile.
//
// Bounds: the features of a tile's pixels differ from those at its centre
// by |eta_k(x) - eta_k(c)| <= D_k = sum_a alpha_a (alpha_a + 1)/2 h_a,
// since |P_m| <= 1 and |P_m'| <= m (m + 1)/2 on [-1, 1] and |x_a - c_a|
// <= h_a in the tile, so every logit of grain i on tile t lies within
// A_i = sum_k |theta'_ik| D_k of o_i(t).  Hence every pixel's largest logit
// is at least L(t) = max_j (o_j - A_j) (taken over the fp32 offsets, less a
// margin of kSetupMargin for their rounding), and
//  * a grain with o_i + A_i < L(t) - 160 has every exponential exactly zero
//    in float however its offset is rounded: it keeps the fp32 offset and
//    the float-float dot product is formed for the others only;
//  * a 128-grain block with max (o_i + A_i) < L(t) - kP1Far only adds
//    exponentials that underflow to zero: pass 1 does not visit it.
// A tile that crosses the grid edge (its centre may lie outside [-1, 1])
// takes the compensated offsets and visits every block.
// ---------------------------------------------------------------------------
constexpr float kSetupMargin = 1.f;
constexpr int kSetupChunk = 512;  // image rows per chunk of passes B and C (a multiple of 128)

template <int DIM, int D>
__global__ void __launch_bounds__(kRefThreads)
k_tc_tile_setup(Geom g, TileMap tm, const float* __restrict__ thH, const float* __restrict__ thL, int N, int Npad,
                const int* __restrict__ perm, const float2* __restrict__ ec, float* __restrict__ off, TileBound tb,
                int bounds, unsigned long long* __restrict__ masks) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<float>(K);
  __shared__ float2 sec[kRefTiles][K];
  __shared__ __align__(16) float sech[kRefTiles][KP];
  __shared__ uint32_t smax[kRefTiles], slow[kRefTiles];
  __shared__ int srag[kRefTiles];
  __shared__ uint32_t smb[kRefTiles][64];        // per tile and block: max of o + A, order-preserving bits
  __shared__ float so[kRefTiles][kSetupChunk];   // offsets of the chunk's rows
  __shared__ float sA[kSetupChunk];              // A of the chunk's rows (-1: no grain)
  __shared__ uint32_t slist[kRefTiles * kSetupChunk];  // (tile, row) pairs that take the float-float offset
  __shared__ int scount;

  const int64_t t0 = (int64_t)blockIdx.x * kRefTiles;
  const int nt = (int)min((int64_t)kRefTiles, tm.n_tiles - t0);
  const int nblk = Npad / 128;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kRefTiles) {
    smax[threadIdx.x] = 0u;
    slow[threadIdx.x] = 0u;
  }
  for (int e = threadIdx.x; e < kRefTiles * 64; e += blockDim.x) smb[e / 64][e % 64] = 0u;
  if (threadIdx.x < nt) {
    float x[DIM], c[DIM];
    srag[threadIdx.x] = g.coords ? 1 : (tile_pixel<DIM>(g, tm, t0 + threadIdx.x, kTcPixTile - 1, x, c) < 0);
  }
  load_centre_features<K>(ec, t0, nt, sec, sech);  // (its barrier covers the set-up above)
  // pass A: C(t) = max_i f_i and max_i (f_i - A_i) over all grains (caller
  // order), as running maxima per thread (order-preserving bits, 0 =
  // nothing) reduced once per tile and warp
  uint32_t mo[kRefTiles], mlo[kRefTiles];
#pragma unroll
  for (int q = 0; q < kRefTiles; ++q) mo[q] = mlo[q] = 0u;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float h[KP];
#pragma unroll
    for (int k = 0; k < KP; k += 4) {
      const float4 v = *reinterpret_cast<const float4*>(thH + (int64_t)i * KP + k);
      h[k] = v.x, h[k + 1] = v.y, h[k + 2] = v.z, h[k + 3] = v.w;
    }
    float A = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) A = fmaf(fabsf(h[k]), tb.d[k], A);
#pragma unroll
    for (int q = 0; q < kRefTiles; ++q)
      if (q < nt) {
        const float f = centre_dot32<K>(h, sech[q]);
        mo[q] = max(mo[q], ord_f32(f));
        mlo[q] = max(mlo[q], ord_f32(f - A));
        asm volatile("" ::: "memory");  // one tile at a time: no feature rows of later tiles held early
      }
  }
#pragma unroll
  for (int q = 0; q < kRefTiles; ++q)
    if (q < nt) {
      const uint32_t m = __reduce_max_sync(0xffffffffu, mo[q]);
      const uint32_t lo = __reduce_max_sync(0xffffffffu, mlo[q]);
      if (lane == 0) {
        if (m) atomicMax(&smax[q], m);
        if (lo) atomicMax(&slow[q], lo);
      }
    }
  // passes B and C, per chunk of image rows
  for (int r0 = 0; r0 < Npad; r0 += kSetupChunk) {
    const int nr = min(kSetupChunk, Npad - r0);  // a multiple of 128: whole warps in every loop below
    __syncthreads();  // pass A's maxima are complete; the previous chunk is written out
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    // pass B: the fp32 offset of every (tile, row); the rows whose offset
    // can matter (not far below the tile's reference) are listed for the
    // float-float offset, so that only they pay for it
    float Cq[kRefTiles], Lq[kRefTiles];
#pragma unroll
    for (int q = 0; q < kRefTiles; ++q) {
      Cq[q] = unord_f32(smax[q]);
      Lq[q] = unord_f32(slow[q]) - Cq[q] - kSetupMargin;
    }
    for (int rr = threadIdx.x; rr < nr; rr += blockDim.x) {
      const int r = r0 + rr;
      const int src = perm ? perm[r] : (r < N ? r : -1);
      float h[KP];
#pragma unroll
      for (int k = 0; k < KP; k += 4) {
        const float4 v = src >= 0 ? *reinterpret_cast<const float4*>(thH + (int64_t)src * KP + k)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        h[k] = v.x, h[k + 1] = v.y, h[k + 2] = v.z, h[k + 3] = v.w;
      }
      float A = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) A = fmaf(fabsf(h[k]), tb.d[k], A);
      sA[rr] = src >= 0 ? A : -1.f;
#pragma unroll
      for (int q = 0; q < kRefTiles; ++q)
        if (q < nt) {
          const float o32 = centre_dot32<K>(h, sech[q]) - Cq[q];
          const bool far = bounds && !srag[q] && o32 + A < Lq[q] - 160.f;
          const bool near = src >= 0 && !far;
          const unsigned bal = __ballot_sync(0xffffffffu, near);
          if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&scount, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (near) slist[base + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)q << 16) | (uint32_t)rr;
          }
          so[q][rr] = src >= 0 ? o32 : 0.f;
          asm volatile("" ::: "memory");
        }
    }
    __syncthreads();
    const int cnt = scount;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int q = (int)(slist[e] >> 16), rr = (int)(slist[e] & 0xffffu);
      const int r = r0 + rr;
      const int src = perm ? perm[r] : r;
      const float C = unord_f32(smax[q]);
      so[q][rr] = ff_diff(ff_dot<K>(thH + (int64_t)src * KP, thL + (int64_t)src * KP, sec[q]), make_float2(C, 0.f));
    }
    __syncthreads();
    // pass C: write the chunk out, and the block maxima of o + A
    for (int rr = threadIdx.x; rr < nr; rr += blockDim.x) {
      const int r = r0 + rr;  // (a warp's 32 rows lie in one 128-row block)
      const float A = sA[rr];
#pragma unroll
      for (int q = 0; q < kRefTiles; ++q)
        if (q < nt) {
          const float o = so[q][rr];
          off[(t0 + q) * Npad + r] = o;
          if (bounds) {
            const uint32_t m = __reduce_max_sync(0xffffffffu, A >= 0.f ? ord_f32(o + A) : 0u);
            if (lane == 0 && m) atomicMax(&smb[q][r / 128], m);
          }
        }
    }
  }
  __syncthreads();
  if (bounds && threadIdx.x < nt) {
    const int q = threadIdx.x;
    unsigned long long msk = nblk >= 64 ? ~0ull : ((1ull << nblk) - 1ull);
    if (!srag[q] && smax[q]) {
      const float lim = unord_f32(slow[q]) - unord_f32(smax[q]) - kSetupMargin - kP1Far;
      for (int b = 0; b < nblk && b < 64; ++b)
        if (!smb[q][b] || unord_f32(smb[q][b]) < lim) msk &= ~(1ull << b);  // (no grain in the block: left out)
    }
    masks[t0 + q] = msk;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// D_k of the tile bounds for a structured grid: the largest offset of
// a tile's pixel from its centre pixel is TileShape_a / n_a along axis a.
template <int DIM, int D>
TileBound tile_bound(const Geom& g) {
  using TS = TileShape<DIM>;
  const double h[3] = {(double)TS::X / (double)g.n0, (double)TS::Y / (double)g.n1,
                       DIM == 3 ? (double)TS::Z / (double)g.n2 : 0.0};
  TileBound tb{};
  for (int k = 0; k < basis_K(DIM, D); ++k) {
    double dk = 0.0;
    for (int a = 0; a < DIM; ++a) {
      const int e = basis_exp(DIM, D, k, a);
      dk += 0.5 * e * (e + 1) * h[a];
    }
    tb.d[k] = (float)(dk * (1.0 + 1e-6));  // rounded up
  }
  return tb;
}

}  // namespace
}  // namespace pd
