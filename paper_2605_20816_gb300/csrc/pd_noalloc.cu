// pd_noalloc.cu -- pd_objective_grad_noalloc: the CUDA-core objective and
// gradient evaluation with every scratch buffer carved from one fixed
// device array compiled into the library, for callers that cannot allocate
// device memory.  The kernels are the same as those of pd_objective_grad;
// only where their scratch lives differs.
#include <mutex>

#include "pd_simt_kernels.cuh"

namespace pd {
namespace {

// The fixed scratch.  Every device that loads the library holds it until
// the process exits.  In host code `g_noalloc_scratch` is only a host-side
// stand-in for the symbol, never a device address: the address is obtained
// once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call made with that device current).
int scratch_base(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PD_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return PD_ENOTSUP;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PD_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<char*>(g_addr[dev]);
  return PD_OK;
}

struct FixedArena {
  char* base;
  size_t cap, used;
  static size_t round_up(size_t v) { return (v + 255) & ~(size_t)255; }
  template <typename T>
  T* take(size_t n) {
    const size_t off = round_up(used);
    const size_t bytes = (n ? n : 1) * sizeof(T);
    if (off > cap || bytes > cap - off) return nullptr;
    used = off + bytes;
    return reinterpret_cast<T*>(base + off);
  }
};

template <typename T, int DIM, int D>
int noalloc_eval_dd(const EvalCall& c, cudaStream_t st, char* base) {
  constexpr int K = basis_K(DIM, D);
  constexpr int KP = padded_K<T>(K);
  const int N = c.N;
  const int64_t P = c.g.P;
  const bool want_grad = c.grad != nullptr;
  const int gtiles = (N + kGradThreads - 1) / kGradThreads;
  FixedArena fx{base, (size_t)PD_NOALLOC_SCRATCH_BYTES, 0};
  // every scratch word is written before it is read (parameters, centre
  // features and reference logits, log S, one objective partial per block,
  // one gradient partial per chunk and grain), so nothing left by an
  // earlier call needs clearing
  if constexpr (std::is_same<T, float>::value) {
    // the tile evaluation of pd_objective_grad in FP32
    const TileMap tm = make_tiles<DIM>(c.g);
    const int64_t n_tiles = tm.n_tiles;
    const int64_t blocks1 = (n_tiles + kT1Tiles - 1) / kT1Tiles;
    const size_t fixed = 2 * FixedArena::round_up(sizeof(float) * (size_t)N * KP) +
                         FixedArena::round_up(sizeof(float2) * (size_t)n_tiles * K) +
                         FixedArena::round_up(sizeof(float2) * (size_t)n_tiles) +
                         (want_grad ? 2 : 1) * FixedArena::round_up(sizeof(float) * (size_t)P) +
                         FixedArena::round_up(sizeof(double) * (size_t)blocks1) + 256;
    if (fixed > (size_t)PD_NOALLOC_SCRATCH_BYTES) return PD_ESCRATCH;
    int64_t tpc = tiles_per_chunk(n_tiles, gtiles, device_sm_count());
    if (want_grad) {
      // fewer, longer chunks when their partials do not fit
      const size_t per_chunk = sizeof(double) * (size_t)N * K;
      const size_t room = (size_t)PD_NOALLOC_SCRATCH_BYTES - fixed;
      if (room / per_chunk < 1) return PD_ESCRATCH;
      const int64_t max_ch = (int64_t)(room / per_chunk);
      if ((n_tiles + tpc - 1) / tpc > max_ch) tpc = (n_tiles + max_ch - 1) / max_ch;
    }
    const int nch = (int)((n_tiles + tpc - 1) / tpc);
    float* thH = fx.take<float>((size_t)N * KP);
    float* thL = fx.take<float>((size_t)N * KP);
    float2* ec = fx.take<float2>((size_t)n_tiles * K);
    float2* ref = fx.take<float2>((size_t)n_tiles);
    float* lse = fx.take<float>((size_t)P);
    float* qv = want_grad ? fx.take<float>((size_t)P) : nullptr;
    double* objp = fx.take<double>((size_t)blocks1);
    double* part = want_grad ? fx.take<double>((size_t)nch * N * K) : nullptr;
    if (!thH || !thL || !ec || !ref || !lse || !objp || (want_grad && (!part || !qv))) return PD_ESCRATCH;
    return launch_simt_tiles<DIM, D>(c, tm, thH, thL, nullptr, ec, ref, lse, qv, nullptr, nullptr, objp, part, tpc,
                                     st);
  } else {
    constexpr int ppt = 2;
    const int blocks1 = (int)((P + kLseThreads * ppt - 1) / (kLseThreads * ppt));
    const int64_t tiles = (P + kPixTile - 1) / kPixTile;
    // fixed part of the footprint, then as many pixel chunks as still fit
    const size_t fixed = FixedArena::round_up(sizeof(T) * (size_t)N * KP) +
                         FixedArena::round_up(sizeof(T) * (size_t)P) +
                         FixedArena::round_up(sizeof(double) * (size_t)blocks1) + 256;
    if (fixed > (size_t)PD_NOALLOC_SCRATCH_BYTES) return PD_ESCRATCH;
    int nch = chunks_for(P, gtiles, device_sm_count());
    if (want_grad) {
      const size_t per_chunk = sizeof(double) * (size_t)N * K;
      const size_t room = (size_t)PD_NOALLOC_SCRATCH_BYTES - fixed;
      if (room / per_chunk < 1) return PD_ESCRATCH;
      if ((size_t)nch > room / per_chunk) nch = (int)(room / per_chunk);
    }
    const int64_t ppc = ((tiles + nch - 1) / nch) * kPixTile;
    const int nch_eff = (int)((P + ppc - 1) / ppc);
    T* thS = fx.take<T>((size_t)N * KP);
    T* lse = fx.take<T>((size_t)P);
    double* objp = fx.take<double>((size_t)blocks1);
    double* part = want_grad ? fx.take<double>((size_t)nch_eff * N * K) : nullptr;
    if (!thS || !lse || !objp || (want_grad && !part)) return PD_ESCRATCH;

    const double tscale = Arith<T>::theta_scale(c.eps);
    const int64_t nth = (int64_t)N * KP;
    k_scale_theta<T><<<(unsigned)((nth + 255) / 256), 256, 0, st>>>(c.theta, N, K, KP, tscale, thS);
    k_pass1<T, DIM, D, ppt, false><<<blocks1, kLseThreads, 0, st>>>(c.g, c.labels, N, thS, nullptr, lse, nullptr,
                                                                     objp);
    if (want_grad) {
      dim3 grid2(nch_eff, gtiles);
      k_pass2<T, DIM, D, false><<<grid2, kGradThreads, 0, st>>>(c.g, c.labels, N, thS, nullptr, lse, nullptr, ppc,
                                                                part);
    }
    if (c.obj) k_reduce_obj<<<1, 1024, 0, st>>>(objp, blocks1, 1.0 / (double)P, c.obj);
    if (want_grad) {
      const int64_t NK = (int64_t)N * K;
      k_reduce_parts<<<(unsigned)((NK + 31) / 32), dim3(32, kRedPhases), 0, st>>>(part, nch_eff, NK,
                                                                                  -1.0 / (c.eps * (double)P), c.grad);
    }
    return cudaGetLastError() == cudaSuccess ? PD_OK : PD_ECUDA;
  }
}

template <typename T>
int noalloc_eval_2d(const EvalCall& c, cudaStream_t st, char* base) {
  switch (c.d) {
    case 1: return noalloc_eval_dd<T, 2, 1>(c, st, base);
    case 2: return noalloc_eval_dd<T, 2, 2>(c, st, base);
    case 3: return noalloc_eval_dd<T, 2, 3>(c, st, base);
    case 4: return noalloc_eval_dd<T, 2, 4>(c, st, base);
    case 5: return noalloc_eval_dd<T, 2, 5>(c, st, base);
    case 6: return noalloc_eval_dd<T, 2, 6>(c, st, base);
    case 7: return noalloc_eval_dd<T, 2, 7>(c, st, base);
    default: return PD_ENOTSUP;
  }
}

}  // namespace

// Forgets the cached address of the current device's array (pd_release):
// after a device reset the module is loaded again and the array may move.
void noalloc_forget_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  g_addr[dev] = nullptr;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_objective_grad_noalloc(const pd_grid* grid, const int32_t* labels, int N, const double* theta,
                                         const pd_eval_opts* opts, double* obj_out, double* grad_out,
                                         void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (!opts || !theta || !labels || N < 2 || g.P < 1 || (!obj_out && !grad_out)) return PD_EINVAL;
  if (!(opts->eps > 0.0) || !isfinite(opts->eps) || opts->d < 1) return PD_EINVAL;
  if (opts->prec < PD_FP64 || opts->prec > PD_BF16X3) return PD_EINVAL;  // as pd_objective_grad
  if (grid->dim != 2 || opts->d > PD_MAX_DEGREE_2D) return PD_ENOTSUP;
  if (opts->prec != PD_FP64 && opts->prec != PD_FP32) return PD_ENOTSUP;
  char* base = nullptr;
  rc = scratch_base(&base);
  if (rc) return rc;
  EvalCall c{g, grid->dim, opts->d, N, opts->prec, opts->eps, labels, theta, nullptr, obj_out, grad_out, nullptr};
  cudaStream_t st = (cudaStream_t)stream;
  return opts->prec == PD_FP64 ? noalloc_eval_2d<double>(c, st, base) : noalloc_eval_2d<float>(c, st, base);
}
