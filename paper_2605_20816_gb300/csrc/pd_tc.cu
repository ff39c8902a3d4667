// pd_tc.cu -- tensor-core (tcgen05) evaluation of the objective and
// gradient, PD_BF16 and PD_BF16X3.
//
// Both K-long contractions of eqs. (Phi) and (grad) run on the 5th-generation
// tensor cores with bf16 operands in shared memory and fp32 accumulators in
// tensor memory (TMEM); the CUDA cores keep only the soft-assignment
// arithmetic (one ex2 per pixel-grain pair and pass) and the per-pixel
// features.
//
// Pixels are processed in tiles of 128 neighbouring pixels, and every logit
// is split at the tile centre (see TileMap below).
//
// pass 1  (one CTA per SM, persistent over 128-pixel tiles)
//   A = features of 128 pixels (rows) x K, written by the 128 epilogue
//       threads from the in-register Legendre recurrence;
//   B = all grains' scaled parameters -theta*log2(e)/eps (rows) x K, copied
//       once per CTA from a prepared global image by a bulk (TMA) copy;
//   D = A B^T, 128 pixels x 128 grains per MMA group, double-buffered in
//       TMEM; the epilogue warps read their pixel row of logits and keep an
//       online log-sum-exp; out: log2 S(x) per pixel and per-CTA objective
//       partials.
// pass 2  (CTA = 128 grains x a chunk of pixels)
//   D1 = theta_block (128 grains x K) . eta(tile)^T (128 pixels): the
//       logits transposed, so that a thread owns one grain's row;
//   the thread forms c = delta_{i G(x)} - ex2(l - log2 S(x)) for its grain
//       and writes it as the A operand (grains x pixels, K-major);
//   D2 += C (128 grains x 128 pixels) . eta(tile) (128 pixels x K): the
//       gradient contraction, accumulated in TMEM over the chunk, then
//       written as one double partial per grain and chunk.
//
// PD_BF16X3 splits every operand into three bf16 terms (hi + mid + lo,
// about 24 significant bits) and forms the six products whose size is at
// least 2^-16 of the leading one (hh, hm, mh, hl, mm, lh), which gives
// float-level logits; the gradient uses two-term splits (hh, lh, hl).
// PD_BF16 uses one term everywhere.
//
// Operands use the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, adjacent along K at 128 bytes (LBO) and along the
// rows at KT*16 bytes (SBO), KT = the operand's total K width.
//
// Every wait on an mbarrier is bounded by a 1 s timeout on the global timer:
// a wait that gives up sets PD_ETIMEOUT in a status word (the objective then
// becomes NaN), raises a CTA-wide abort flag so that the other waits give up
// at once, and the CTA still frees its TMEM before it returns.
#include <cuda_bf16.h>

#include "pd_simt_kernels.cuh"

namespace pd {
namespace {

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
constexpr int kTcConsumers = 256;                 // warps 0..7: TMEM consumers
constexpr int kTcProducers = 64;                  // warps 8..9: pixel-operand producers, 2 pixels each
constexpr int kTcMmaWarp = 10;                    // TMEM allocation and MMA issue
constexpr int kTcThreads = 11 * 32;               // at most 3 warps per SM sub-partition
constexpr int kTcCols = 512;                      // TMEM columns per CTA (one CTA per SM)
constexpr int kTcGrainTile = 128;                 // pass-1 grains per MMA group
constexpr int kTcPixTile = 128;                   // pixels per tile (both passes)

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
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  uint64_t state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
               : "=l"(state)
               : "r"(smem_addr(b)), "r"(bytes)
               : "memory");
  (void)state;
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
// Byte offset of element (row r, column k) of a K-major no-swizzle operand
// whose rows are KT elements wide.
__host__ __device__ constexpr uint32_t kmaj(int r, int k, int KT) {
  return (uint32_t)((r >> 3) * (KT * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float bf16_val(uint16_t b) {
  return __bfloat162float(__ushort_as_bfloat16(b));
}

// Term split of the operands.  Slice s of a BF16X3 operand holds, for the
// parameters (theta side), term kThetaTerm[s] and, for the features, term
// kEtaTerm[s]: products hh, hm, mh, hl, mm, lh.
__host__ __device__ constexpr int theta_term(int s) { return s == 2 || s == 4 ? 1 : (s == 5 ? 2 : 0); }
__host__ __device__ constexpr int eta_term(int s) { return s == 1 || s == 4 ? 1 : (s == 3 ? 2 : 0); }

// Writes the KS slices of a feature row (pixel r) into a K-major operand.
template <int K, int KW, int KS>
__device__ __forceinline__ void store_eta_row(uint8_t* base, int r, const float* eta) {
  constexpr int KT = KW * KS;
  uint16_t parts[3][KW];
#pragma unroll
  for (int k = 0; k < KW; ++k) {
    const float v = k < K ? eta[k] : 0.f;
    const uint16_t h = bf16_bits(v);
    const float r1 = v - bf16_val(h);
    const uint16_t m = bf16_bits(r1);
    const float r2 = r1 - bf16_val(m);
    parts[0][k] = h;
    parts[1][k] = m;
    parts[2][k] = bf16_bits(r2);
  }
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    const int t = KS == 1 ? 0 : eta_term(s);
#pragma unroll
    for (int k8 = 0; k8 < KW; k8 += 8) {
      uint4 v;
      v.x = (uint32_t)parts[t][k8 + 0] | ((uint32_t)parts[t][k8 + 1] << 16);
      v.y = (uint32_t)parts[t][k8 + 2] | ((uint32_t)parts[t][k8 + 3] << 16);
      v.z = (uint32_t)parts[t][k8 + 4] | ((uint32_t)parts[t][k8 + 5] << 16);
      v.w = (uint32_t)parts[t][k8 + 6] | ((uint32_t)parts[t][k8 + 7] << 16);
      *reinterpret_cast<uint4*>(base + kmaj(r, s * KW + k8, KT)) = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Parameter images: rows = grains (padded to Npad with zero rows), K-major
// no-swizzle, KS slices of KW columns; plus the float copy used for the
// label logit of the objective.
// ---------------------------------------------------------------------------
template <int KS>
__global__ void k_tc_theta_image(const double* __restrict__ theta, int N, int Npad, int K, int KW, double scale,
                                 uint8_t* __restrict__ img, float* __restrict__ th32, int KP32) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (row, k) pairs
  if (q >= (int64_t)Npad * KW) return;
  const int r = (int)(q / KW), k = (int)(q % KW);
  const double t = (r < N && k < K) ? theta[(int64_t)r * K + k] * scale : 0.0;
  const uint16_t h = __bfloat16_as_ushort(__double2bfloat16(t));
  const double r1 = t - (double)__bfloat162float(__ushort_as_bfloat16(h));
  const uint16_t m = __bfloat16_as_ushort(__double2bfloat16(r1));
  const double r2 = r1 - (double)__bfloat162float(__ushort_as_bfloat16(m));
  const uint16_t l = __bfloat16_as_ushort(__double2bfloat16(r2));
  const uint16_t parts[3] = {h, m, l};
  const int KT = KW * KS;
  for (int s = 0; s < KS; ++s) {
    const int term = KS == 1 ? 0 : theta_term(s);
    *reinterpret_cast<uint16_t*>(img + kmaj(r, s * KW + k, KT)) = parts[term];
  }
  if (r < N && k < KP32) th32[(int64_t)r * KP32 + k] = k < K ? (float)t : 0.f;
}

// ---------------------------------------------------------------------------
// Pixel tiles.  A tile is 128 pixels that are close in space: a 16 x 8 block
// of a 2-D grid or an 8 x 4 x 4 block of a 3-D grid (128 consecutive points
// of a point list).  Every logit is split at the tile centre c,
//   l_i(x) = theta'_i . eta(c) + theta'_i . (eta(x) - eta(c)),
// the first part (one per grain and tile) on the CUDA cores in fp32 and the
// second, small part on the tensor cores.  The tensor cores accumulate with
// truncation, whose error is biased; keeping their operand small (|x - c|
// is a few pixels) keeps that bias far below the float rounding of the
// logits, which is unbiased.
// ---------------------------------------------------------------------------
struct TileMap {
  int ntx, nty, ntz;      // tiles per axis (structured grids)
  int64_t n_tiles;
  double inv0, inv1, inv2;  // 1 / n_a
};

template <int DIM>
struct TileShape {
  static constexpr int X = DIM == 2 ? 16 : 8;
  static constexpr int Y = DIM == 2 ? 8 : 4;
  static constexpr int Z = DIM == 2 ? 1 : 4;
};

// Pixel index of row r of tile t (or -1 outside the pixel set), its
// coordinates x and the coordinates of the tile centre c.  Only 32-bit
// divisions by the (uniform) tile counts; pixel centres from reciprocals.
template <int DIM>
__device__ __forceinline__ int64_t tile_pixel(const Geom& g, const TileMap& tm, int64_t t, int r, float* x,
                                              float* c) {
  if (g.coords) {
    const int64_t j0 = t * kTcPixTile;
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
  using TS = TileShape<DIM>;
  const unsigned tt = (unsigned)t;
  const unsigned tx = tt % (unsigned)tm.ntx;
  const unsigned rest = tt / (unsigned)tm.ntx;
  const unsigned ty = rest % (unsigned)tm.nty;
  const unsigned tz = rest / (unsigned)tm.nty;
  const int64_t px = (int64_t)tx * TS::X + (r % TS::X);
  const int64_t py = (int64_t)ty * TS::Y + ((r / TS::X) % TS::Y);
  const int64_t pz = (int64_t)tz * TS::Z + (r / (TS::X * TS::Y));
  c[0] = (float)fma(2.0 * (double)(tx * TS::X + TS::X / 2) + 1.0, tm.inv0, -1.0);
  c[1] = (float)fma(2.0 * (double)(ty * TS::Y + TS::Y / 2) + 1.0, tm.inv1, -1.0);
  if (DIM == 3) c[2] = (float)fma(2.0 * (double)(tz * TS::Z + TS::Z / 2) + 1.0, tm.inv2, -1.0);
  x[0] = (float)fma(2.0 * (double)px + 1.0, tm.inv0, -1.0);
  x[1] = (float)fma(2.0 * (double)py + 1.0, tm.inv1, -1.0);
  if (DIM == 3) x[2] = (float)fma(2.0 * (double)pz + 1.0, tm.inv2, -1.0);
  if (px >= g.n0 || py >= g.n1 || (DIM == 3 && pz >= g.n2)) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = c[a];
    return -1;
  }
  return DIM == 2 ? px + g.n0 * py : px + g.n0 * (py + g.n1 * pz);
}

template <int K>
__device__ __forceinline__ float dot_f(const float* __restrict__ a, const float* __restrict__ b) {
  float acc = a[0] * b[0];
#pragma unroll
  for (int k = 1; k < K; ++k) acc = fmaf(a[k], b[k], acc);
  return acc;
}

__device__ __forceinline__ float tree_max32(const float* v) {
  float a[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = fmaxf(v[q], v[q + 16]);
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int q = 0; q < w; ++q) a[q] = fmaxf(a[q], a[q + w]);
  return a[0];
}
__device__ __forceinline__ float tree_sum32(const float* v) {
  float a[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = v[q] + v[q + 16];
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int q = 0; q < w; ++q) a[q] = a[q] + a[q + w];
  return a[0];
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
// Pass 1: log2 S(x) per pixel and objective partials.
// ---------------------------------------------------------------------------
constexpr int kP1Bufs = 4;  // logit tiles in flight in TMEM (4 x 128 columns)

template <int DIM, int D, int KS>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_pass1(Geom g, TileMap tm, const int32_t* __restrict__ labels, int N, int Npad, const uint8_t* __restrict__ img,
           const float* __restrict__ th32, float* __restrict__ lse_out, double* __restrict__ obj_part,
           int* __restrict__ status) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * KS;
  constexpr int KP32 = padded_K<float>(K);
  constexpr uint32_t kRowBytes = KT * 2;
  constexpr uint32_t kTileBytes = kTcPixTile * kRowBytes;
  constexpr uint32_t IDESC = idesc_bf16(128, kTcGrainTile);

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sB = smem;                                            // Npad x KT
  uint8_t* sA = smem + (size_t)Npad * kRowBytes;                 // 2 stages x 128 x KT
  float* sOff = reinterpret_cast<float*>(sA + 2 * kTileBytes);   // 2 stages x Npad centre logits
  float2* sPart = reinterpret_cast<float2*>(sOff + 2 * Npad);   // 2 stages x 128 (max, sum) of half 1
  float* sLG = reinterpret_cast<float*>(sPart + 2 * 128);        // 2 stages x 128 starting max
  float* sLGv = sLG + 2 * 128;                                   // 2 stages x 128 label logits
  long long* sJ = reinterpret_cast<long long*>(sLGv + 2 * 128);  // 2 stages x 128 pixel indices
  __shared__ __align__(8) uint64_t bar_theta, bar_a_full[2], bar_a_empty[2], bar_off_free[2], bar_d_full[kP1Bufs],
      bar_d_empty[kP1Bufs], bar_part_full[2], bar_part_free[2], bar_drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ double sred[kTcThreads / 32];

  const int tid = threadIdx.x, warp = tid >> 5;
  const int n_gt = Npad / kTcGrainTile;
  const int64_t n_tiles = tm.n_tiles;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar_theta, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar_a_full[s], kTcProducers);
      mbar_init(&bar_a_empty[s], 1);
      mbar_init(&bar_off_free[s], kTcConsumers);
      mbar_init(&bar_part_full[s], 128);
      mbar_init(&bar_part_free[s], 128);
    }
    for (int b = 0; b < kP1Bufs; ++b) {
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

  double racc = 0.0;
  if (warp == kTcMmaWarp) {
    if (tid == kTcMmaWarp * 32) {
      // parameter image: one bulk copy per 32 KiB
      const uint32_t total = (uint32_t)Npad * kRowBytes;
      mbar_arrive_expect_tx(&bar_theta, total);
      for (uint32_t off = 0; off < total; off += 32768u) {
        const uint32_t n = total - off < 32768u ? total - off : 32768u;
        bulk_g2s(sB + off, img + off, n, &bar_theta);
      }
      bool ok = mbar_wait(&bar_theta, 0, &abort_flag, status);
      int64_t c = 0;  // grain-tile counter over the whole loop
      int it = 0;
      for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
        const int s = it & 1;
        ok = mbar_wait(&bar_a_full[s], (it >> 1) & 1, &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        for (int gt = 0; gt < n_gt; ++gt, ++c) {
          const int b = (int)(c % kP1Bufs);
          if (c >= kP1Bufs) {
            ok = mbar_wait(&bar_d_empty[b], (uint32_t)(((c / kP1Bufs) - 1) & 1), &abort_flag, status);
            if (!ok) break;
            tc_fence_after();
          }
          const uint32_t aaddr = smem_addr(sA + s * kTileBytes);
          const uint32_t baddr = smem_addr(sB + (size_t)gt * kTcGrainTile * kRowBytes);
#pragma unroll
          for (int q = 0; q < KT / 16; ++q) {
            const uint64_t ad = smem_desc(aaddr + q * 256, 128, KT * 16);
            const uint64_t bd = smem_desc(baddr + q * 256, 128, KT * 16);
            mma_bf16(tmem + b * kTcGrainTile, ad, bd, IDESC, q > 0);
          }
          mma_commit(&bar_d_full[b]);
        }
        if (!ok) break;
        mma_commit(&bar_a_empty[s]);
      }
      // every MMA issued above has completed before TMEM is released
      mma_commit(&bar_drain);
      mbar_wait_drain(&bar_drain, 0);
    }
    __syncwarp();
  } else if (is_producer(warp)) {
    const int p0 = tid - kTcConsumers;  // pixel rows p0 and p0 + 64 of the tile
    int it = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++it) {
      const int s = it & 1, use = it >> 1;
      if (use >= 1 && (!mbar_wait_warp(&bar_a_empty[s], (uint32_t)((use - 1) & 1), &abort_flag, status) ||
                       !mbar_wait_warp(&bar_off_free[s], (uint32_t)((use - 1) & 1), &abort_flag, status)))
        break;
      float c[DIM], ec[K];
      for (int p = p0; p < kTcPixTile; p += kTcProducers) {
        float x[DIM], eta[K];
        const int64_t j = tile_pixel<DIM>(g, tm, t, p, x, c);
        legendre_features<DIM, D>(c, ec);
        legendre_features<DIM, D>(x, eta);
        float de[K];
#pragma unroll
        for (int k = 0; k < K; ++k) de[k] = eta[k] - ec[k];
        store_eta_row<K, KW, KS>(sA + s * kTileBytes, p, de);
        float start = -INFINITY, lg = 0.f;
        if (j >= 0) {
          const int G = labels[j];
          if ((unsigned)G < (unsigned)N) {
            const float* rowp = th32 + (int64_t)G * KP32;
            lg = dot_f<K>(rowp, ec) + dot_f<K>(rowp, de);
            start = lg;
          } else {
            lg = NAN;
          }
        }
        sLG[s * 128 + p] = start;
        sLGv[s * 128 + p] = lg;
        sJ[s * 128 + p] = (long long)j;
      }
      for (int i = p0; i < Npad; i += kTcProducers)
        sOff[s * Npad + i] = i < N ? dot_f<K>(th32 + (int64_t)i * KP32, ec) : 0.f;
      fence_proxy_async();
      mbar_arrive(&bar_a_full[s]);
    }
  } else {
    const int quad = warp & 3, half = warp >> 2, lane = tid & 31;
    const int row = quad * 32 + lane;  // pixel row of the tile == TMEM lane
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    int it = 0;
    int64_t c = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++it) {
      const int s = it & 1;
      // the stage's operands and per-row values come from the producers
      ok = mbar_wait_warp(&bar_a_full[s], (uint32_t)((it >> 1) & 1), &abort_flag, status);
      if (!ok) break;
      // the running max starts at the label logit (a lower bound of the max,
      // usually the max itself), so most chunks of far-away grains lie more
      // than 127 below it: their exponentials underflow to exactly zero in
      // ex2.approx.ftz and the whole chunk is skipped
      float m = sLG[s * 128 + row], ssum = 0.f;
      // logits of grain tile gt are loaded while tile gt-1 is processed
      uint32_t n0[32], n1[32];
      {
        const int b = (int)(c % kP1Bufs);
        ok = mbar_wait_warp(&bar_d_full[b], (uint32_t)((c / kP1Bufs) & 1), &abort_flag, status);
        if (!ok) break;
        tc_fence_after();
        const uint32_t col = (uint32_t)(b * kTcGrainTile + half * 64);
        tmem_ld32(tmem + lane_base + col, n0);
        tmem_ld32(tmem + lane_base + col + 32, n1);
      }
      for (int gt = 0; gt < n_gt; ++gt, ++c) {
        const int b = (int)(c % kP1Bufs);
        tmem_wait_ld();
        tc_fence_before();
        mbar_arrive(&bar_d_empty[b]);  // the logits are in registers: release the TMEM tile
        uint32_t r0[32], r1[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          r0[q] = n0[q];
          r1[q] = n1[q];
        }
        if (gt + 1 < n_gt) {
          const int bn = (int)((c + 1) % kP1Bufs);
          ok = mbar_wait_warp(&bar_d_full[bn], (uint32_t)(((c + 1) / kP1Bufs) & 1), &abort_flag, status);
          if (!ok) break;
          tc_fence_after();
          const uint32_t col = (uint32_t)(bn * kTcGrainTile + half * 64);
          tmem_ld32(tmem + lane_base + col, n0);
          tmem_ld32(tmem + lane_base + col + 32, n1);
        }
        const int cbase = gt * kTcGrainTile + half * 64;
        const float* off = sOff + s * Npad + cbase;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int nv = N - (cbase + 32 * h2);
          if (nv <= 0) break;
          const uint32_t* r = h2 ? r1 : r0;
          float v[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = q < nv ? __uint_as_float(r[q]) + off[32 * h2 + q] : -INFINITY;
          const float cm = tree_max32(v);
          if (__all_sync(0xffffffffu, cm < m - 127.f)) continue;
          const float mn = fmaxf(m, cm);
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = Arith<float>::ex(v[q] - mn);
          ssum = fmaf(ssum, Arith<float>::ex(m - mn), tree_sum32(v));
          m = mn;
        }
      }
      if (!ok) break;
      // combine the two column halves of each pixel (bounded mbarrier
      // hand-off between the warpgroups; slot s is reused every 2 tiles)
      if (half == 1) {
        if (it >= 2 && !mbar_wait_warp(&bar_part_free[s], (uint32_t)(((it >> 1) - 1) & 1), &abort_flag, status)) {
          ok = false;
          break;
        }
        sPart[s * 128 + row] = make_float2(m, ssum);
        mbar_arrive(&bar_part_full[s]);
      } else {
        if (!mbar_wait_warp(&bar_part_full[s], (uint32_t)((it >> 1) & 1), &abort_flag, status)) {
          ok = false;
          break;
        }
        const float2 o = sPart[s * 128 + row];
        mbar_arrive(&bar_part_free[s]);
        const int64_t j = sJ[s * 128 + row];
        if (j >= 0) {
          const float mm = fmaxf(m, o.x);
          const float sum = ssum * Arith<float>::ex(m - mm) + o.y * Arith<float>::ex(o.x - mm);
          const float lse = mm + Arith<float>::lg(sum);
          lse_out[j] = lse;
          racc += (double)(sLGv[s * 128 + row] - lse) * Arith<float>::to_nat;
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
  if (warp == kTcMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcCols);
  }
}

// ---------------------------------------------------------------------------
// Pass 2: gradient partials for one grain block and one chunk of tiles.
// NB pixel-operand stages and NA gradient-operand stages (2 when shared
// memory holds them, else 1); with NB = 2 the MMA warp issues the logits of
// tile t+1 before the gradient of tile t, so the tensor cores always have
// the next tile's logits ready when the consumers finish a tile.
// ---------------------------------------------------------------------------
template <int DIM, int D, int KS, int NB, int NA>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_pass2(Geom g, TileMap tm, int N, const uint8_t* __restrict__ img, const float* __restrict__ th32,
           const float* __restrict__ lse, int64_t tiles_per_chunk, double* __restrict__ part, int* __restrict__ status) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * KS;                     // logits operands
  constexpr int KP32 = padded_K<float>(K);
  constexpr int GT = KS == 1 ? 1 : 2;             // gradient terms of c and eta
  constexpr uint32_t kRowBytes = KT * 2;
  constexpr uint32_t kABytes = 128 * kRowBytes;   // theta block
  constexpr uint32_t kBBytes = kTcPixTile * kRowBytes;
  constexpr uint32_t kB2Term = KW * kTcPixTile * 2;        // eta^T term: rows KW, K = 128 pixels
  constexpr uint32_t kB2Bytes = GT * kB2Term;
  constexpr uint32_t kA2Term = 128 * kTcPixTile * 2;       // c term: rows 128 grains, K = 128 pixels
  constexpr uint32_t kA2Bytes = GT * kA2Term;
  constexpr uint32_t IDESC1 = idesc_bf16(128, kTcPixTile);
  constexpr uint32_t IDESC2 = idesc_bf16(128, KW);
  constexpr int D2COL = 2 * kTcPixTile;  // TMEM columns: D1 [0,256) double-buffered, D2 [256, 256+KW)

  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;                           // theta block image
  uint8_t* sB = sA + kABytes;                   // NB stages of eta rows
  uint8_t* sB2 = sB + NB * kBBytes;             // NB stages of eta^T
  uint8_t* sA2 = sB2 + NB * kB2Bytes;           // NA stages of c
  float* sLse = reinterpret_cast<float*>(sA2 + NA * kA2Bytes);     // [NB][128]
  float* sCen = sLse + NB * kTcPixTile;                             // [NB][4] tile centres
  __shared__ __align__(8) uint64_t bar_theta, bar_b_full[NB], bar_b_empty[NB], bar_d1_full[2], bar_d1_empty[2],
      bar_a2_full[NA], bar_a2_empty[NA], bar_d2_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5;
  const int gb = blockIdx.y;                 // grain block
  const int64_t t_begin = (int64_t)blockIdx.x * tiles_per_chunk;
  const int64_t t_end = min(t_begin + tiles_per_chunk, tm.n_tiles);
  const int n_pt = (int)(t_end - t_begin);
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bar_theta, 1);
    for (int s = 0; s < NB; ++s) {
      mbar_init(&bar_b_full[s], kTcProducers);
      mbar_init(&bar_b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_d1_full[b], 1);
      mbar_init(&bar_d1_empty[b], kTcConsumers);
    }
    for (int a = 0; a < NA; ++a) {
      mbar_init(&bar_a2_full[a], kTcConsumers);
      mbar_init(&bar_a2_empty[a], 1);
    }
    mbar_init(&bar_d2_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTcMmaWarp) tmem_alloc(&tmem_slot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kTcMmaWarp) {
    if (tid == kTcMmaWarp * 32) {
      mbar_arrive_expect_tx(&bar_theta, kABytes);
      bulk_g2s(sA, img + (size_t)gb * kABytes, kABytes, &bar_theta);
      bool ok = mbar_wait(&bar_theta, 0, &abort_flag, status);
      auto logits = [&](int t) -> bool {
        const int s = t % NB, b1 = t & 1;
        if (!mbar_wait(&bar_b_full[s], (uint32_t)((t / NB) & 1), &abort_flag, status)) return false;
        if (t >= 2 && !mbar_wait(&bar_d1_empty[b1], (uint32_t)(((t >> 1) - 1) & 1), &abort_flag, status))
          return false;
        tc_fence_after();
        const uint32_t aaddr = smem_addr(sA), baddr = smem_addr(sB + s * kBBytes);
#pragma unroll
        for (int q = 0; q < KT / 16; ++q)
          mma_bf16(tmem + b1 * kTcPixTile, smem_desc(aaddr + q * 256, 128, KT * 16),
                   smem_desc(baddr + q * 256, 128, KT * 16), IDESC1, q > 0);
        mma_commit(&bar_d1_full[b1]);
        return true;
      };
      auto grad = [&](int t) -> bool {
        const int s = t % NB, a = t % NA;
        if (!mbar_wait(&bar_a2_full[a], (uint32_t)((t / NA) & 1), &abort_flag, status)) return false;
        tc_fence_after();
        // D2 += C . eta: products (c_h, eta_h), then (c_l, eta_h), (c_h, eta_l)
        const uint32_t a2 = smem_addr(sA2 + a * kA2Bytes), b2 = smem_addr(sB2 + s * kB2Bytes);
        constexpr int NPROD = GT == 1 ? 1 : 3;
#pragma unroll
        for (int pr = 0; pr < NPROD; ++pr) {
          const int ct = pr == 1 ? 1 : 0, et = pr == 2 ? 1 : 0;
#pragma unroll
          for (int q = 0; q < kTcPixTile / 16; ++q) {
            const uint64_t ad = smem_desc(a2 + ct * kA2Term + q * 256, 128, kTcPixTile * 16);
            const uint64_t bd = smem_desc(b2 + et * kB2Term + q * 256, 128, kTcPixTile * 16);
            mma_bf16(tmem + D2COL, ad, bd, IDESC2, (t > 0 || pr > 0 || q > 0) ? 1u : 0u);
          }
        }
        mma_commit(&bar_a2_empty[a]);
        mma_commit(&bar_b_empty[s]);
        return true;
      };
      if (NB == 2) {
        if (ok && n_pt > 0) ok = logits(0);
        for (int t = 0; ok && t < n_pt; ++t) {
          if (t + 1 < n_pt) ok = logits(t + 1);
          if (ok) ok = grad(t);
        }
      } else {
        for (int t = 0; ok && t < n_pt; ++t) {
          ok = logits(t);
          if (ok) ok = grad(t);
        }
      }
      mma_commit(&bar_d2_done);
      mbar_wait_drain(&bar_d2_done, 0);
    }
    __syncwarp();
  } else if (is_producer(warp)) {
    // pixel operands of every tile: the logit operand rows, the transposed
    // gradient operand, log2 S of the pixels and the tile centre
    const int p0 = tid - kTcConsumers;
    for (int t = 0; t < n_pt; ++t) {
      const int s = t % NB;
      if (t >= NB && !mbar_wait_warp(&bar_b_empty[s], (uint32_t)(((t / NB) - 1) & 1), &abort_flag, status)) break;
      for (int p = p0; p < kTcPixTile; p += kTcProducers) {
      float x[DIM], c[DIM], eta[K], ec[K];
      const int64_t j = tile_pixel<DIM>(g, tm, t_begin + t, p, x, c);
      const bool vj = j >= 0;
      const float lsev = vj ? lse[j] : INFINITY;
      legendre_features<DIM, D>(c, ec);
      legendre_features<DIM, D>(x, eta);
      float de[K];
#pragma unroll
      for (int k = 0; k < K; ++k) de[k] = eta[k] - ec[k];
      store_eta_row<K, KW, KS>(sB + s * kBBytes, p, de);
      uint8_t* b2 = sB2 + s * kB2Bytes;
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const float v = (k < K && vj) ? eta[k] : 0.f;
        const uint16_t h = bf16_bits(v);
        *reinterpret_cast<uint16_t*>(b2 + kmaj(k, p, kTcPixTile)) = h;
        if (GT == 2) *reinterpret_cast<uint16_t*>(b2 + kB2Term + kmaj(k, p, kTcPixTile)) = bf16_bits(v - bf16_val(h));
      }
      sLse[s * kTcPixTile + p] = lsev;
      if (p == 0) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) sCen[s * 4 + a] = c[a];
      }
      }
      fence_proxy_async();
      mbar_arrive(&bar_b_full[s]);
    }
  } else {
    const int quad = warp & 3, half = warp >> 2, lane = tid & 31;
    const int gr = quad * 32 + lane;        // grain row of the block == TMEM lane
    const int i = gb * 128 + gr;            // this thread's grain
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    float th[K];
#pragma unroll
    for (int k = 0; k < K; ++k) th[k] = i < N ? th32[(int64_t)i * KP32 + k] : 0.f;
    // logits of tile t+1 are loaded from TMEM while tile t is processed
    // (NB == 2: the MMA warp issues them before the gradient of tile t)
    uint32_t n0[32], n1[32];
    bool loaded = false;
    auto load_logits = [&](int t) -> bool {
      const int b1 = t & 1;
      if (!mbar_wait_warp(&bar_d1_full[b1], (uint32_t)((t >> 1) & 1), &abort_flag, status)) return false;
      tc_fence_after();
      const uint32_t col = (uint32_t)(b1 * kTcPixTile + half * 64);
      tmem_ld32(tmem + lane_base + col, n0);
      tmem_ld32(tmem + lane_base + col + 32, n1);
      loaded = true;
      return true;
    };
    bool ok = true;
    for (int t = 0; ok && t < n_pt; ++t) {
      const int s = t % NB, b1 = t & 1, a = t % NA;
      // sLse and sCen of the stage were written by the producers
      if (!mbar_wait_warp(&bar_b_full[s], (uint32_t)((t / NB) & 1), &abort_flag, status)) { ok = false; break; }
      if (!loaded && !load_logits(t)) { ok = false; break; }
      tmem_wait_ld();
      loaded = false;
      tc_fence_before();
      mbar_arrive(&bar_d1_empty[b1]);  // the logits are in registers: release the TMEM tile
      uint32_t r0[32], r1[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        r0[q] = n0[q];
        r1[q] = n1[q];
      }
      if (NB == 2 && t + 1 < n_pt && !load_logits(t + 1)) { ok = false; break; }
      // this grain's centre logit for the tile
      float c[DIM], ec[K];
#pragma unroll
      for (int q = 0; q < DIM; ++q) c[q] = sCen[s * 4 + q];
      legendre_features<DIM, D>(c, ec);
      const float off = dot_f<K>(th, ec);
      if (t >= NA && !mbar_wait_warp(&bar_a2_empty[a], (uint32_t)(((t / NA) - 1) & 1), &abort_flag, status)) {
        ok = false;
        break;
      }
      const float* ls = sLse + s * kTcPixTile + half * 64;
      uint8_t* a2 = sA2 + a * kA2Bytes;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const uint32_t* r = h2 ? r1 : r0;
        uint32_t hi[16], lo[16];
        float lsv[32];
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          const float4 v4 = *reinterpret_cast<const float4*>(ls + 32 * h2 + q);
          lsv[q] = v4.x - off;
          lsv[q + 1] = v4.y - off;
          lsv[q + 2] = v4.z - off;
          lsv[q + 3] = v4.w - off;
        }
#pragma unroll
        for (int q = 0; q < 32; q += 2) {
          // c = -p; the label term delta_{i G(x)} enters through the grain
          // moments added at the final reduction
          const float c0 = -Arith<float>::ex(__uint_as_float(r[q]) - lsv[q]);
          const float c1 = -Arith<float>::ex(__uint_as_float(r[q + 1]) - lsv[q + 1]);
          const __nv_bfloat162 h = __floats2bfloat162_rn(c0, c1);
          hi[q >> 1] = *reinterpret_cast<const uint32_t*>(&h);
          if (GT == 2) {
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(c0 - hf.x, c1 - hf.y);
            lo[q >> 1] = *reinterpret_cast<const uint32_t*>(&l);
          }
        }
#pragma unroll
        for (int q8 = 0; q8 < 32; q8 += 8) {
          const uint32_t o = kmaj(gr, half * 64 + 32 * h2 + q8, kTcPixTile);
          *reinterpret_cast<uint4*>(a2 + o) = make_uint4(hi[q8 / 2], hi[q8 / 2 + 1], hi[q8 / 2 + 2], hi[q8 / 2 + 3]);
          if (GT == 2)
            *reinterpret_cast<uint4*>(a2 + kA2Term + o) =
                make_uint4(lo[q8 / 2], lo[q8 / 2 + 1], lo[q8 / 2 + 2], lo[q8 / 2 + 3]);
        }
      }
      fence_proxy_async();
      mbar_arrive(&bar_a2_full[a]);
    }
    tmem_wait_ld();  // a prefetched load may be outstanding after an abort
    // chunk result: D2 row of this grain (first warpgroup)
    if (ok && n_pt > 0) ok = mbar_wait_warp(&bar_d2_done, 0, &abort_flag, status);
    if (half == 0) {
      if (ok && n_pt > 0) {
        tc_fence_after();
        uint32_t r[32];
        if (KW == 16) {
          tmem_ld16(tmem + lane_base + (uint32_t)D2COL, r);
        } else {
          tmem_ld32(tmem + lane_base + (uint32_t)D2COL, r);
        }
        tmem_wait_ld();
        if (i < N) {
#pragma unroll
          for (int k = 0; k < K; ++k)
            part[((int64_t)blockIdx.x * N + i) * K + k] = abort_flag ? NAN : (double)__uint_as_float(r[k]);
        }
      } else if (i < N) {
        for (int k = 0; k < K; ++k) part[((int64_t)blockIdx.x * N + i) * K + k] = n_pt > 0 ? NAN : 0.0;
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
// Label term of eq. (grad): sum_{x in G_i} eta(x) per grain, fp32 features
// summed exactly in 64-bit fixed point (order independent).
// ---------------------------------------------------------------------------
template <int DIM, int D>
__global__ void k_tc_label_moments(Geom g, const int32_t* __restrict__ labels, int N, double fx_scale,
                                   unsigned long long* __restrict__ acc) {
  constexpr int K = basis_K(DIM, D);
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = j < g.P;
  int G = valid ? labels[j] : -1;
  if (G < 0 || G >= N) G = -1;
  float x[DIM], eta[K];
  if (valid) {
    pixel_coords<DIM>(g, j, x);
  } else {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = 0.f;
  }
  legendre_features<DIM, D>(x, eta);
  long long fx[K];
#pragma unroll
  for (int k = 0; k < K; ++k) fx[k] = G >= 0 ? __double2ll_rn((double)eta[k] * fx_scale) : 0ll;
  // one warp-wide sum (and one atomic per feature) for each distinct label
  // of the warp: spatially coherent labels make that one or two groups
  unsigned todo = __ballot_sync(0xffffffffu, G >= 0);
  const int lane = threadIdx.x & 31;
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int L = __shfl_sync(0xffffffffu, G, leader);
    const unsigned grp = __ballot_sync(0xffffffffu, G == L);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      long long v = (G == L) ? fx[k] : 0ll;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) atomicAdd(&acc[(int64_t)L * K + k], (unsigned long long)v);
    }
    todo &= ~grp;
  }
}

// out[q] = scale * (base[q] / fx + sum_c part[c][q]), fixed order
__global__ void __launch_bounds__(32 * kRedPhases)
k_tc_reduce_grad(const double* __restrict__ part, int nchunks, int64_t NK, const unsigned long long* __restrict__ base,
                 double inv_fx, double scale, double* __restrict__ out) {
  __shared__ double ssum[kRedPhases][32];
  const int64_t q = (int64_t)blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (q < NK)
    for (int c = threadIdx.y; c < nchunks; c += kRedPhases) s += part[(int64_t)c * NK + q];
  ssum[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && q < NK) {
    double t = (double)(long long)base[q] * inv_fx;
#pragma unroll
    for (int y = 0; y < kRedPhases; ++y) t += ssum[y][threadIdx.x];
    out[q] = t * scale;
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int DIM>
TileMap make_tiles(const Geom& g) {
  TileMap tm{1, 1, 1, 0, 1.0, 1.0, 1.0};
  if (g.coords) {
    tm.n_tiles = (g.P + kTcPixTile - 1) / kTcPixTile;
    return tm;
  }
  using TS = TileShape<DIM>;
  tm.ntx = (int)((g.n0 + TS::X - 1) / TS::X);
  tm.nty = (int)((g.n1 + TS::Y - 1) / TS::Y);
  tm.ntz = DIM == 3 ? (int)((g.n2 + TS::Z - 1) / TS::Z) : 1;
  tm.n_tiles = (int64_t)tm.ntx * tm.nty * tm.ntz;
  tm.inv0 = 1.0 / (double)g.n0;
  tm.inv1 = 1.0 / (double)g.n1;
  tm.inv2 = 1.0 / (double)g.n2;
  return tm;
}

template <int DIM, int D, int KS>
int eval_tc_dd(const EvalCall& c, cudaStream_t st) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KW = (K + 15) / 16 * 16;
  constexpr int KT = KW * KS;
  constexpr int KP32 = padded_K<float>(K);
  constexpr int GT = KS == 1 ? 1 : 2;
  const int N = c.N;
  const int64_t P = c.g.P;
  const int Npad = (N + 127) / 128 * 128;
  const size_t row_bytes = (size_t)KT * 2;
  // image, 2 operand stages, 2 x centre logits, 2 x (max, sum), 2 x start,
  // 2 x label logit, 2 x pixel index
  const size_t smem1 = (size_t)Npad * row_bytes + 2 * kTcPixTile * row_bytes + 2 * (size_t)Npad * 4 +
                       2 * kTcPixTile * 8 + 4 * kTcPixTile * 4 + 2 * kTcPixTile * 8;
  constexpr size_t kCap = 220 * 1024;
  // pass-2 stages: two of each when they fit, else one
  constexpr size_t kS2Fixed = (size_t)128 * KT * 2;
  constexpr size_t kS2PerB = (size_t)kTcPixTile * KT * 2 + (size_t)GT * KW * kTcPixTile * 2 + kTcPixTile * 4 + 16;
  constexpr size_t kS2PerA = (size_t)GT * 128 * kTcPixTile * 2;
  constexpr int NB = kS2Fixed + 2 * kS2PerB + 2 * kS2PerA <= kCap ? 2 : (kS2Fixed + 2 * kS2PerB + kS2PerA <= kCap ? 2 : 1);
  constexpr int NA = kS2Fixed + 2 * kS2PerB + 2 * kS2PerA <= kCap ? 2 : 1;
  const size_t smem2 = kS2Fixed + NB * kS2PerB + NA * kS2PerA;
  if (smem1 > kCap || smem2 > kCap) return PD_ENOTSUP;  // too many grains for a resident image
  // at least 120 KiB of dynamic shared memory per CTA keeps one CTA per SM,
  // which owns all 512 TMEM columns
  const size_t smem1_req = std::max<size_t>(smem1, 120 * 1024);
  const size_t smem2_req = std::max<size_t>(smem2, 120 * 1024);

  const TileMap tm = make_tiles<DIM>(c.g);
  const int sms = device_sm_count();
  const int64_t n_tiles = tm.n_tiles;
  const int grid1 = (int)std::min<int64_t>(n_tiles, sms);
  const int gblocks = Npad / 128;
  // tile chunks of pass 2: about 4 waves of CTAs, at most 32 tiles per chunk
  int64_t nch = std::max<int64_t>((int64_t)sms * 4 / gblocks, 1);
  nch = std::max<int64_t>(nch, (n_tiles + 31) / 32);
  nch = std::min<int64_t>(nch, n_tiles);
  const int64_t tpc = (n_tiles + nch - 1) / nch;
  const int nch_eff = (int)((n_tiles + tpc - 1) / tpc);

  Scratch sc(st);
  uint8_t* img = sc.get<uint8_t>((size_t)Npad * row_bytes);
  float* th32 = sc.get<float>((size_t)N * KP32);
  float* lse = sc.get<float>((size_t)P);
  double* objp = sc.get<double>((size_t)grid1);
  double* part = c.grad ? sc.get<double>((size_t)nch_eff * N * K) : nullptr;
  unsigned long long* lmom = c.grad ? sc.get<unsigned long long>((size_t)N * K) : nullptr;
  int* status = sc.get<int>(1);
  if (!sc.ok()) return PD_ENOMEM;
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return PD_ECUDA;

  const double scale = Arith<float>::theta_scale(c.eps);
  {
    const int64_t n = (int64_t)Npad * KW;
    PD_TIMED(st, "tc_theta_image",
             k_tc_theta_image<KS><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c.theta, N, Npad, K, KW, scale, img,
                                                                                th32, KP32));
  }
  auto k1 = k_tc_pass1<DIM, D, KS>;
  if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1_req) != cudaSuccess)
    return PD_ECUDA;
  PD_TIMED(st, KS == 1 ? "tc_bf16_lse_pass1" : "tc_bf16x3_lse_pass1",
           k1<<<grid1, kTcThreads, smem1_req, st>>>(c.g, tm, c.labels, N, Npad, img, th32, lse, objp, status));
  // |eta| <= 1, so a grain's label sum is bounded by P: the largest
  // power-of-two scale that keeps P * scale below 2^62
  int bits = 0;
  while (bits < 62 && ((int64_t)1 << bits) <= P) ++bits;
  const double fx = ldexp(1.0, 62 - bits);
  if (c.grad) {
    if (cudaMemsetAsync(lmom, 0, sizeof(unsigned long long) * N * K, st) != cudaSuccess) return PD_ECUDA;
    PD_TIMED(st, "tc_label_moments",
             (k_tc_label_moments<DIM, D><<<(unsigned)((P + 255) / 256), 256, 0, st>>>(c.g, c.labels, N, fx, lmom)));
    auto k2 = k_tc_pass2<DIM, D, KS, NB, NA>;
    if (cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2_req) != cudaSuccess)
      return PD_ECUDA;
    dim3 grid2(nch_eff, gblocks);
    PD_TIMED(st, KS == 1 ? "tc_bf16_grad_pass2" : "tc_bf16x3_grad_pass2",
             k2<<<grid2, kTcThreads, smem2_req, st>>>(c.g, tm, N, img, th32, lse, tpc, part, status));
  }
  if (c.obj) PD_TIMED(st, "reduce_obj", k_reduce_obj<<<1, 1024, 0, st>>>(objp, grid1, 1.0 / (double)P, c.obj));
  if (c.grad) {
    const int64_t NK = (int64_t)N * K;
    PD_TIMED(st, "reduce_parts",
             k_tc_reduce_grad<<<(unsigned)((NK + 31) / 32), dim3(32, kRedPhases), 0, st>>>(
                 part, nch_eff, NK, lmom, 1.0 / fx, -1.0 / (c.eps * (double)P), c.grad));
  }
  return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
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
  if (c.v) return PD_ENOTSUP;
  if (c.prec == PD_BF16) return eval_tc_ks<1>(c, st);
  if (c.prec == PD_BF16X3) return eval_tc_ks<6>(c, st);
  return PD_ENOTSUP;
}

}  // namespace pd

extern "C" int pd_selftest_wait_timeout(double seconds, int* status_out, void* stream) {
  if (!status_out || !(seconds > 0.0) || seconds > 1.0) return PD_EINVAL;
  return pd::selftest_wait_timeout(seconds, status_out, (cudaStream_t)stream);
}
