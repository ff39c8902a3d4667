// pd_batch.cu -- batched evaluation of many grain maps of uneven sizes and
// grain counts in one persistent launch per pass, replayed as a CUDA graph,
// with launch shapes chosen by a small autotuner; and the lockstep batched
// ascent scheme built on it (pd_fit_batched).
//
// On the tensor cores (PD_BF16, PD_BF16X3) every map has a plan of the
// single-map evaluation (pd_plan.cu: scratch, centre features and grain
// order made once), and the evaluations of all maps are captured as one
// graph in which the maps run on a few parallel chains, heaviest first,
// each map on the chain with the least work so far; the autotuner picks the
// number of chains.  A map's results are those of a single-map call.
//
// Work items: pass 1 = (map, 512-pixel block), pass 2 = (map, pixel chunk,
// 128-grain tile); in FP32 the pixels are the tiles of the single-map FP32
// evaluation (pd_tiles.cuh): pass 1 = (map, block of four tiles), pass 2 =
// (map, run of tiles, 128-grain tile), with each map's centre features and
// reference logits formed first.  A CTA takes items from a global counter until none are
// left, heaviest maps first (items are listed in decreasing N), and runs
// for each item exactly the per-block code of the single-map kernels, so a
// map's partial sums are those of a single-map call with the same chunking
// and its results are reproducible run to run.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "pd_fit_core.h"
#include "pd_simt_kernels.cuh"

namespace pd {
namespace {

struct BatchMapDev {
  Geom g;
  TileMap tm;        // FP32: the map's tiles
  const int32_t* labels;
  const double* theta;
  void* thS;         // scaled parameters (FP32: the hi parts)
  float* thL;        // FP32: the lo parts
  float2* ec;        // FP32: centre features [tiles][K]
  float2* ref;       // FP32: reference logits [tiles]
  void* lse;
  float* q;          // FP32: 1 - p_G per pixel
  double* objp;
  double* part;
  double* obj_out;
  double* grad_out;
  int64_t ppc;       // pixels (FP64) or tiles (FP32) per pass-2 chunk
  int N, nch, blocks1, pad;
};

template <typename T>
__global__ void k_batch_scale(const BatchMapDev* __restrict__ maps, int K, int KP, double scale,
                              const int* __restrict__ active) {
  const int m = blockIdx.y;
  if (!active[m]) return;
  const BatchMapDev mp = maps[m];
  T* out = static_cast<T*>(mp.thS);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)mp.N * KP;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / KP), k = (int)(q % KP);
    const double v = k < K ? mp.theta[(int64_t)i * K + k] * scale : 0.0;
    out[q] = (T)v;
    if (mp.thL) mp.thL[q] = (float)(v - (double)(T)v);
  }
}

// FP32: centre features of every map's tiles (they depend on the pixel set
// only: formed once when the plan is built).
template <int D>
__global__ void __launch_bounds__(256) k_batch_features(const BatchMapDev* __restrict__ maps) {
  const BatchMapDev& mp = maps[blockIdx.y];
  constexpr int K = basis_K(2, D);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < mp.tm.n_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    double c[2], P[2][D + 1];
    tile_centre<2>(mp.g, mp.tm, t, c);
    for (int a = 0; a < 2; ++a) {
      P[a][0] = 1.0;
      P[a][1] = c[a];
      for (int m = 1; m < D; ++m) P[a][m + 1] = ((2.0 * m + 1.0) * c[a] * P[a][m] - (double)m * P[a][m - 1]) * (1.0 / (m + 1.0));
    }
    double eta[K];
    basis_all<2, D>(P, eta, std::make_integer_sequence<int, K>{});
    for (int k = 0; k < K; ++k) {
      const float h = (float)eta[k];
      mp.ec[t * K + k] = make_float2(h, (float)(eta[k] - (double)h));
    }
  }
}

// FP32: reference logits of every map's tiles (blockIdx.y = map; blocks walk
// the map's groups of kRefTiles tiles).
template <int D>
__global__ void __launch_bounds__(kRefThreads)
k_batch_refs(const BatchMapDev* __restrict__ maps, const int* __restrict__ active) {
  constexpr int K = basis_K(2, D);
  __shared__ float2 sec[kRefTiles][K];
  __shared__ __align__(16) float sech[kRefTiles][padded_K<float>(K)];
  __shared__ uint32_t smax[kRefTiles];
  const int m = blockIdx.y;
  if (!active[m]) return;
  const BatchMapDev& mp = maps[m];
  for (int64_t t0 = (int64_t)blockIdx.x * kRefTiles; t0 < mp.tm.n_tiles; t0 += (int64_t)gridDim.x * kRefTiles)
    tile_centres_block<K>(static_cast<const float*>(mp.thS), mp.N, mp.tm.n_tiles, mp.ec, mp.ref, t0, sec, sech, smax);
}

__device__ __forceinline__ int next_item(int* counter) {
  __shared__ int s_item;
  __syncthreads();
  if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  __syncthreads();
  return s_item;
}

template <typename T, int D>
__global__ void __launch_bounds__(kLseThreads)
k_batch_pass1(const BatchMapDev* __restrict__ maps, const int2* __restrict__ items, int n_items,
              int* __restrict__ counter, const int* __restrict__ active) {
  for (;;) {
    const int it = next_item(counter);
    if (it >= n_items) break;
    const int2 w = items[it];
    if (!active[w.x]) continue;
    const BatchMapDev& mp = maps[w.x];
    if constexpr (std::is_same<T, float>::value)
      pass1_tiles_block<2, D, false>(mp.g, mp.tm, mp.labels, mp.N, static_cast<const float*>(mp.thS), mp.thL,
                                     nullptr, mp.ec, mp.ref, static_cast<float*>(mp.lse), mp.q, nullptr, nullptr,
                                     nullptr, mp.objp + w.y, w.y);
    else
      pass1_block<T, 2, D, 2, false>(mp.g, mp.labels, mp.N, static_cast<const T*>(mp.thS), nullptr,
                                     static_cast<T*>(mp.lse), nullptr, mp.objp + w.y, w.y);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kGradThreads)
k_batch_pass2(const BatchMapDev* __restrict__ maps, const int2* __restrict__ items, int n_items,
              int* __restrict__ counter, const int* __restrict__ active) {
  for (;;) {
    const int it = next_item(counter);
    if (it >= n_items) break;
    const int2 w = items[it];
    if (!active[w.x]) continue;
    const BatchMapDev& mp = maps[w.x];
    if (!mp.grad_out) continue;
    const int gtiles = (mp.N + kGradThreads - 1) / kGradThreads;
    if constexpr (std::is_same<T, float>::value)
      pass2_tiles_block<2, D, false>(mp.g, mp.tm, mp.labels, mp.N, static_cast<const float*>(mp.thS), mp.thL,
                                     nullptr, mp.ec, mp.ref, static_cast<const float*>(mp.lse), mp.q, nullptr,
                                     nullptr, nullptr, mp.ppc, mp.part, w.y / gtiles, w.y % gtiles);
    else
      pass2_block<T, 2, D, false>(mp.g, mp.labels, mp.N, static_cast<const T*>(mp.thS), nullptr,
                                  static_cast<const T*>(mp.lse), nullptr, mp.ppc, mp.part, w.y / gtiles,
                                  w.y % gtiles);
  }
}

__global__ void k_batch_reduce_obj(const BatchMapDev* __restrict__ maps, const int* __restrict__ active) {
  __shared__ double sred[32];
  const int m = blockIdx.x;
  if (!active[m]) return;
  const BatchMapDev& mp = maps[m];
  double s = 0.0;
  for (int q = threadIdx.x; q < mp.blocks1; q += blockDim.x) s += mp.objp[q];
  const double bs = block_sum_fixed(s, sred);
  if (threadIdx.x == 0) *mp.obj_out = bs / (double)mp.g.P;
}

__global__ void __launch_bounds__(32 * kRedPhases)
k_batch_reduce_parts(const BatchMapDev* __restrict__ maps, int K, double eps, const int* __restrict__ active) {
  __shared__ double ssum[kRedPhases][32];
  const int m = blockIdx.y;
  if (!active[m]) return;
  const BatchMapDev& mp = maps[m];
  if (!mp.grad_out) return;
  const int64_t NK = (int64_t)mp.N * K;
  if ((int64_t)blockIdx.x * 32 >= NK) return;
  const int64_t q = (int64_t)blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (q < NK)
    for (int c = threadIdx.y; c < mp.nch; c += kRedPhases) s += mp.part[(int64_t)c * NK + q];
  ssum[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && q < NK) {
    double t = 0.0;
#pragma unroll
    for (int y = 0; y < kRedPhases; ++y) t += ssum[y][threadIdx.x];
    mp.grad_out[q] = t * (-1.0 / (eps * (double)mp.g.P));
  }
}

// ---------------------------------------------------------------------------
// The plan: device tables, scratch, the captured graph.
// ---------------------------------------------------------------------------
struct Tune {
  int chunk_factor;  // pass-2 CTAs per SM the chunking aims at (single-map default: 6);
                     // tensor cores: the number of parallel chains
  int occ_div;       // persistent grid = SMs x occupancy / occ_div (tensor cores: unused, 0)
};
constexpr int kMaxChains = 8;

struct BatchKey {
  int d, prec, nmap_bucket, work_bucket;
  bool operator<(const BatchKey& o) const {
    return std::tie(d, prec, nmap_bucket, work_bucket) < std::tie(o.d, o.prec, o.nmap_bucket, o.work_bucket);
  }
};
std::mutex g_tune_mu;
std::map<BatchKey, std::pair<Tune, double>> g_tune_cache;

}  // namespace
}  // namespace pd

struct pd_batch {
  int n_maps = 0, d = 0, prec = 0, K = 0, KP = 0;
  double eps = 0.0;
  std::vector<pd_map> maps;
  std::vector<pd::BatchMapDev> hmaps;
  pd::BatchMapDev* d_maps = nullptr;
  int2* d_items1 = nullptr;
  int2* d_items2 = nullptr;
  int* d_counters = nullptr;
  int* d_active = nullptr;
  void* d_scratch = nullptr;
  int n_items1 = 0, n_items2 = 0, grid1 = 0, grid2 = 0;
  pd::Tune tune{6, 1};
  double tuned_ms = 0.0;
  bool tuned = false;
  cudaGraphExec_t exec = nullptr;
  int occ1 = 1, occ2 = 1;
  // tensor-core precisions
  std::vector<pd::PlanCore> plans;  // one per map
  std::vector<int> order;           // maps by decreasing pixels x grains
  std::vector<int> chain;           // map -> chain
  std::vector<int32_t> h_active;    // host copy of the active flags
  bool all_active = true;
  int n_chains = 1;
  cudaStream_t cst[pd::kMaxChains] = {};
  cudaEvent_t fork = nullptr, join[pd::kMaxChains] = {};
  double* tc_zero = nullptr;        // theta = 0 for the tuning replays (largest N x K)
  double* tc_out = nullptr;         // outputs of the tuning replays (Phi per map, then gradients)
  std::vector<size_t> tc_off;       // gradient offset of each map in tc_out
};

namespace pd {
namespace {

template <typename T, int D>
void launch_batch(pd_batch* b, cudaStream_t st) {
  const double scale = Arith<T>::theta_scale(b->eps);
  int maxNK = 0, maxNKP = 0;
  for (const auto& m : b->hmaps) {
    maxNK = std::max(maxNK, m.N * b->K);
    maxNKP = std::max(maxNKP, m.N * b->KP);
  }
  cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(int), st);
  k_batch_scale<T><<<dim3((maxNKP + 255) / 256, b->n_maps), 256, 0, st>>>(b->d_maps, b->K, b->KP, scale,
                                                                          b->d_active);
  if (std::is_same<T, float>::value) {
    int64_t max_tiles = 1;
    for (const auto& m : b->hmaps) max_tiles = std::max<int64_t>(max_tiles, m.tm.n_tiles);
    const unsigned gx = std::min<unsigned>(tile_centre_blocks(max_tiles), 1024u);
    k_batch_refs<D><<<dim3(gx, b->n_maps), kRefThreads, 0, st>>>(b->d_maps, b->d_active);
  }
  k_batch_pass1<T, D><<<b->grid1, kLseThreads, 0, st>>>(b->d_maps, b->d_items1, b->n_items1, b->d_counters,
                                                         b->d_active);
  k_batch_pass2<T, D><<<b->grid2, kGradThreads, 0, st>>>(b->d_maps, b->d_items2, b->n_items2, b->d_counters + 1,
                                                          b->d_active);
  k_batch_reduce_obj<<<b->n_maps, 1024, 0, st>>>(b->d_maps, b->d_active);
  k_batch_reduce_parts<<<dim3((maxNK + 31) / 32, b->n_maps), dim3(32, kRedPhases), 0, st>>>(b->d_maps, b->K,
                                                                                             b->eps, b->d_active);
}

template <typename T>
void launch_batch_d(pd_batch* b, cudaStream_t st) {
  switch (b->d) {
    case 1: launch_batch<T, 1>(b, st); break;
    case 2: launch_batch<T, 2>(b, st); break;
    case 3: launch_batch<T, 3>(b, st); break;
    case 4: launch_batch<T, 4>(b, st); break;
    case 5: launch_batch<T, 5>(b, st); break;
    case 6: launch_batch<T, 6>(b, st); break;
    case 7: launch_batch<T, 7>(b, st); break;
    default: break;
  }
}

template <typename T>
void occupancy(pd_batch* b) {
  int o1 = 1, o2 = 1;
  auto occ = [&](auto k1, auto k2) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k1, kLseThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k2, kGradThreads, 0);
  };
  switch (b->d) {
    case 1: occ(k_batch_pass1<T, 1>, k_batch_pass2<T, 1>); break;
    case 2: occ(k_batch_pass1<T, 2>, k_batch_pass2<T, 2>); break;
    case 3: occ(k_batch_pass1<T, 3>, k_batch_pass2<T, 3>); break;
    case 4: occ(k_batch_pass1<T, 4>, k_batch_pass2<T, 4>); break;
    case 5: occ(k_batch_pass1<T, 5>, k_batch_pass2<T, 5>); break;
    case 6: occ(k_batch_pass1<T, 6>, k_batch_pass2<T, 6>); break;
    case 7: occ(k_batch_pass1<T, 7>, k_batch_pass2<T, 7>); break;
    default: break;
  }
  b->occ1 = std::max(o1, 1);
  b->occ2 = std::max(o2, 1);
}

void free_plan_device(pd_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  cudaFree(b->d_maps);
  cudaFree(b->d_items1);
  cudaFree(b->d_items2);
  cudaFree(b->d_scratch);
  b->d_maps = nullptr;
  b->d_items1 = b->d_items2 = nullptr;
  b->d_scratch = nullptr;
}

// (Re)lays out scratch, work items and the graph for a tuning choice.
int build_plan(pd_batch* b, const Tune& tu) {
  free_plan_device(b);
  const int sms = device_sm_count();
  const size_t esz = b->prec == PD_FP64 ? 8 : 4;
  std::vector<int> order(b->n_maps);
  for (int m = 0; m < b->n_maps; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->maps[a].N > b->maps[c].N; });
  // scratch layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  std::vector<size_t> o_th(b->n_maps), o_lse(b->n_maps), o_objp(b->n_maps), o_part(b->n_maps);
  std::vector<size_t> o_thl(b->n_maps, 0), o_ec(b->n_maps, 0), o_ref(b->n_maps, 0), o_q(b->n_maps, 0);
  b->hmaps.assign(b->n_maps, BatchMapDev{});
  std::vector<int2> items1, items2;
  for (int m = 0; m < b->n_maps; ++m) {
    const pd_map& mp = b->maps[m];
    BatchMapDev& h = b->hmaps[m];
    validate_grid(&mp.grid, &h.g);
    h.labels = mp.labels;
    h.theta = mp.theta;
    h.obj_out = mp.obj_out;
    h.grad_out = mp.grad_out;
    h.N = mp.N;
    const int64_t P = h.g.P;
    const int gtiles = (mp.N + kGradThreads - 1) / kGradThreads;
    const bool f32 = b->prec == PD_FP32;
    if (f32) {
      h.tm = make_tiles<2>(h.g);
      h.blocks1 = (int)((h.tm.n_tiles + kT1Tiles - 1) / kT1Tiles);
      h.ppc = tiles_per_chunk(h.tm.n_tiles, gtiles, sms, tu.chunk_factor);
      h.nch = (int)((h.tm.n_tiles + h.ppc - 1) / h.ppc);
      o_thl[m] = take(4 * (size_t)mp.N * b->KP);
      o_ec[m] = take(sizeof(float2) * (size_t)h.tm.n_tiles * b->K);
      o_ref[m] = take(sizeof(float2) * (size_t)h.tm.n_tiles);
      o_q[m] = take(4 * (size_t)P);
    } else {
      h.blocks1 = (int)((P + kLseThreads * 2 - 1) / (kLseThreads * 2));
      const int64_t tiles = (P + kPixTile - 1) / kPixTile;
      int64_t want = ((int64_t)sms * tu.chunk_factor + gtiles - 1) / gtiles;
      want = std::max<int64_t>(1, std::min<int64_t>(want, tiles));
      h.ppc = ((tiles + want - 1) / want) * kPixTile;
      h.nch = (int)((P + h.ppc - 1) / h.ppc);
    }
    o_th[m] = take(esz * (size_t)mp.N * b->KP);
    o_lse[m] = take(esz * (size_t)P);
    o_objp[m] = take(8 * (size_t)h.blocks1);
    o_part[m] = mp.grad_out ? take(8 * (size_t)h.nch * mp.N * b->K) : 0;
  }
  for (int m : order) {
    const BatchMapDev& h = b->hmaps[m];
    for (int q = 0; q < h.blocks1; ++q) items1.push_back(make_int2(m, q));
    if (b->maps[m].grad_out) {
      const int gtiles = (h.N + kGradThreads - 1) / kGradThreads;
      for (int q = 0; q < h.nch * gtiles; ++q) items2.push_back(make_int2(m, q));
    }
  }
  if (cudaMalloc(&b->d_scratch, std::max<size_t>(off, 256)) != cudaSuccess) {
    cudaGetLastError();
    return PD_ENOMEM;
  }
  char* base = static_cast<char*>(b->d_scratch);
  for (int m = 0; m < b->n_maps; ++m) {
    BatchMapDev& h = b->hmaps[m];
    h.thS = base + o_th[m];
    h.lse = base + o_lse[m];
    if (b->prec == PD_FP32) {
      h.thL = reinterpret_cast<float*>(base + o_thl[m]);
      h.ec = reinterpret_cast<float2*>(base + o_ec[m]);
      h.ref = reinterpret_cast<float2*>(base + o_ref[m]);
      h.q = reinterpret_cast<float*>(base + o_q[m]);
    }
    h.objp = reinterpret_cast<double*>(base + o_objp[m]);
    h.part = b->maps[m].grad_out ? reinterpret_cast<double*>(base + o_part[m]) : nullptr;
  }
  b->n_items1 = (int)items1.size();
  b->n_items2 = (int)items2.size();
  if (cudaMalloc(&b->d_maps, sizeof(BatchMapDev) * b->n_maps) != cudaSuccess ||
      cudaMalloc(&b->d_items1, sizeof(int2) * std::max<size_t>(items1.size(), 1)) != cudaSuccess ||
      cudaMalloc(&b->d_items2, sizeof(int2) * std::max<size_t>(items2.size(), 1)) != cudaSuccess) {
    cudaGetLastError();
    return PD_ENOMEM;
  }
  if (cudaMemcpy(b->d_maps, b->hmaps.data(), sizeof(BatchMapDev) * b->n_maps, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (!items1.empty() &&
       cudaMemcpy(b->d_items1, items1.data(), sizeof(int2) * items1.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      (!items2.empty() &&
       cudaMemcpy(b->d_items2, items2.data(), sizeof(int2) * items2.size(), cudaMemcpyHostToDevice) != cudaSuccess))
    return PD_ECUDA;
  if (b->prec == PD_FP32) {
    // the maps' centre features, once per plan
    int64_t max_tiles = 1;
    for (const auto& m : b->hmaps) max_tiles = std::max<int64_t>(max_tiles, m.tm.n_tiles);
    const unsigned gx = (unsigned)std::min<int64_t>((max_tiles + 255) / 256, 1024);
    switch (b->d) {
      case 1: k_batch_features<1><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      case 2: k_batch_features<2><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      case 3: k_batch_features<3><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      case 4: k_batch_features<4><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      case 5: k_batch_features<5><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      case 6: k_batch_features<6><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      case 7: k_batch_features<7><<<dim3(gx, b->n_maps), 256>>>(b->d_maps); break;
      default: break;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return PD_ECUDA;
  }
  b->grid1 = std::max(1, std::min(b->n_items1, sms * std::max(1, b->occ1 / tu.occ_div)));
  b->grid2 = std::max(1, std::min(std::max(b->n_items2, 1), sms * std::max(1, b->occ2 / tu.occ_div)));
  b->tune = tu;
  // capture the whole evaluation as one graph
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PD_ECUDA;
  cudaGraph_t graph = nullptr;
  int rc = PD_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PD_ECUDA;
  if (rc == PD_OK) {
    if (b->prec == PD_FP64) launch_batch_d<double>(b, cs);
    else launch_batch_d<float>(b, cs);
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) rc = PD_ECUDA;
  }
  if (rc == PD_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = PD_ECUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (rc) cudaGetLastError();
  return rc;
}

bool is_tc(int prec) { return prec == PD_BF16 || prec == PD_BF16X3; }

// Chains for the tensor-core maps: heaviest map first, each on the chain
// with the least work so far.
void assign_chains(pd_batch* b, int n_chains) {
  b->n_chains = n_chains;
  b->chain.assign(b->n_maps, 0);
  std::vector<double> load(n_chains, 0.0);
  for (int m : b->order) {
    const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->chain[m] = c;
    load[c] += (double)b->maps[m].grid.P * (double)b->maps[m].N;
  }
}

// Enqueues the evaluations of the maps (all, or the active ones) on the
// chains, forked from and joined back to st; `tuning` evaluates theta = 0
// into the plan's own outputs instead of the maps' buffers.
int tc_enqueue(pd_batch* b, cudaStream_t st, bool tuning, bool only_active) {
  if (cudaEventRecord(b->fork, st) != cudaSuccess) return PD_ECUDA;
  for (int c = 0; c < b->n_chains; ++c)
    if (cudaStreamWaitEvent(b->cst[c], b->fork, 0) != cudaSuccess) return PD_ECUDA;
  int rc = PD_OK;
  for (int m : b->order) {
    if (only_active && !b->h_active[m]) continue;
    const pd_map& mp = b->maps[m];
    const double* th = tuning ? b->tc_zero : mp.theta;
    double* obj = tuning ? b->tc_out + m : mp.obj_out;
    double* grad = tuning ? b->tc_out + b->tc_off[m] : mp.grad_out;
    rc = plan_eval(&b->plans[m], th, b->eps, obj, grad, b->cst[b->chain[m]]);
    if (rc) break;
  }
  // (the chains join back even after an error, so that a capture can end)
  for (int c = 0; c < b->n_chains; ++c)
    if (cudaEventRecord(b->join[c], b->cst[c]) != cudaSuccess || cudaStreamWaitEvent(st, b->join[c], 0) != cudaSuccess)
      rc = rc ? rc : PD_ECUDA;
  return rc;
}

// Captures the tensor-core evaluation of all maps as the plan's graph.
int tc_capture(pd_batch* b, bool tuning) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PD_ECUDA;
  cudaGraph_t graph = nullptr;
  int rc = PD_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PD_ECUDA;
  if (rc == PD_OK) {
    rc = tc_enqueue(b, cs, tuning, false);
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && rc == PD_OK) rc = PD_ECUDA;
  }
  if (rc == PD_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) rc = PD_ECUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (rc) cudaGetLastError();
  return rc;
}

void tc_free(pd_batch* b) {
  for (auto& p : b->plans) plan_free(&p);
  b->plans.clear();
  for (int c = 0; c < kMaxChains; ++c) {
    if (b->cst[c]) cudaStreamDestroy(b->cst[c]);
    if (b->join[c]) cudaEventDestroy(b->join[c]);
    b->cst[c] = nullptr;
    b->join[c] = nullptr;
  }
  if (b->fork) cudaEventDestroy(b->fork);
  b->fork = nullptr;
  cudaFree(b->tc_zero);
  cudaFree(b->tc_out);
  b->tc_zero = b->tc_out = nullptr;
}

double time_plan(pd_batch* b, int reps);

// The tensor-core batch: plans, chains, tuning, the graph.
int tc_build(pd_batch* b, int autotune) {
  b->plans.assign(b->n_maps, PlanCore{});
  size_t max_nk = 1, tot = (size_t)b->n_maps;
  b->tc_off.assign(b->n_maps, 0);
  for (int m = 0; m < b->n_maps; ++m) {
    Geom g;
    validate_grid(&b->maps[m].grid, &g);
    const int rc = plan_init(&b->plans[m], g, 2, b->maps[m].labels, b->maps[m].N, b->d, b->prec, false);
    if (rc) return rc;
    const size_t nk = (size_t)b->maps[m].N * b->K;
    max_nk = std::max(max_nk, nk);
    b->tc_off[m] = tot;
    tot += nk;
  }
  if (cudaMalloc(&b->tc_zero, sizeof(double) * max_nk) != cudaSuccess ||
      cudaMalloc(&b->tc_out, sizeof(double) * tot) != cudaSuccess) {
    cudaGetLastError();
    return PD_ENOMEM;
  }
  if (cudaMemset(b->tc_zero, 0, sizeof(double) * max_nk) != cudaSuccess) return PD_ECUDA;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return PD_ECUDA;
  for (int c = 0; c < kMaxChains; ++c)
    if (cudaStreamCreateWithFlags(&b->cst[c], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming) != cudaSuccess)
      return PD_ECUDA;
  // one direct evaluation of every map leaves its centre features and grain
  // order in its plan, so that the graph holds only the per-call work
  assign_chains(b, 1);
  int rc = tc_enqueue(b, 0, true, false);
  if (rc) return rc;
  if (cudaDeviceSynchronize() != cudaSuccess) return PD_ECUDA;
  int best = 4;
  if (autotune) {
    double best_ms = 1e30;
    for (int nc : {1, 2, 4, 8}) {
      assign_chains(b, nc);
      rc = tc_capture(b, true);
      if (rc) return rc;
      const double ms = time_plan(b, 3);
      if (ms < best_ms) {
        best_ms = ms;
        best = nc;
      }
    }
    b->tuned_ms = best_ms;
  }
  assign_chains(b, best);
  b->tune = Tune{best, 0};
  return tc_capture(b, false);
}

double time_plan(pd_batch* b, int reps) {
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaGraphLaunch(b->exec, st);  // warm-up
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r) cudaGraphLaunch(b->exec, st);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  return ms / reps;
}

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" int pd_batch_create(int n_maps, const pd_map* maps, const pd_eval_opts* opts, int autotune,
                               pd_batch** out) {
  if (!out || n_maps < 1 || !maps || !opts) return PD_EINVAL;
  *out = nullptr;
  if (!(opts->eps > 0.0) || !isfinite(opts->eps) || opts->d < 1) return PD_EINVAL;
  if (opts->prec < PD_FP64 || opts->prec > PD_BF16X3) return PD_EINVAL;
  if (opts->d > PD_MAX_DEGREE_2D) return PD_ENOTSUP;
  for (int m = 0; m < n_maps; ++m) {
    Geom g;
    int rc = validate_grid(&maps[m].grid, &g);
    if (rc) return rc;
    if (maps[m].grid.dim != 2) return PD_ENOTSUP;
    if (g.P < 1 || maps[m].N < 2 || !maps[m].labels || !maps[m].theta || !maps[m].obj_out) return PD_EINVAL;
  }
  pd_batch* b = new pd_batch();
  b->n_maps = n_maps;
  b->d = opts->d;
  b->prec = opts->prec;
  b->eps = opts->eps;
  b->K = basis_K(2, opts->d);
  b->KP = opts->prec == PD_FP64 ? padded_K<double>(b->K) : padded_K<float>(b->K);
  b->maps.assign(maps, maps + n_maps);
  if (cudaMalloc(&b->d_counters, 2 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_active, sizeof(int) * n_maps) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return PD_ENOMEM;
  }
  std::vector<int> ones(n_maps, 1);
  cudaMemcpy(b->d_active, ones.data(), sizeof(int) * n_maps, cudaMemcpyHostToDevice);
  b->h_active.assign(n_maps, 1);
  b->order.resize(n_maps);
  for (int m = 0; m < n_maps; ++m) b->order[m] = m;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
    return (double)maps[a].grid.P * maps[a].N > (double)maps[c].grid.P * maps[c].N;
  });
  if (is_tc(b->prec)) {
    const int rc = tc_build(b, autotune);
    b->tuned = autotune != 0;
    if (rc) {
      pd_batch_destroy(b);
      return rc;
    }
    *out = b;
    return PD_OK;
  }
  if (b->prec == PD_FP64) occupancy<double>(b);
  else occupancy<float>(b);
  // autotune: the pass-2 chunking and the persistent grid size, cached per
  // (degree, precision, batch size, total work) bucket
  int64_t work = 0;
  for (int m = 0; m < n_maps; ++m) work += maps[m].grid.P * (int64_t)maps[m].N;
  BatchKey key{opts->d, opts->prec, (int)std::log2((double)n_maps + 1.0), (int)std::log2((double)work + 1.0)};
  Tune best{6, 1};
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto itc = g_tune_cache.find(key);
    if (itc != g_tune_cache.end()) {
      best = itc->second.first;
      b->tuned_ms = itc->second.second;
      cached = true;
    }
  }
  int rc = PD_OK;
  if (autotune && !cached) {
    double best_ms = 1e30;
    const Tune cands[] = {{3, 1}, {6, 1}, {12, 1}, {6, 2}, {12, 2}};
    for (const Tune& tu : cands) {
      rc = build_plan(b, tu);
      if (rc) break;
      const double ms = time_plan(b, 3);
      if (ms < best_ms) {
        best_ms = ms;
        best = tu;
      }
    }
    if (rc == PD_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = {best, best_ms};
      b->tuned_ms = best_ms;
    }
  }
  if (rc == PD_OK) rc = build_plan(b, best);
  b->tuned = autotune != 0;
  if (rc) {
    free_plan_device(b);
    cudaFree(b->d_counters);
    cudaFree(b->d_active);
    delete b;
    return rc;
  }
  *out = b;
  return PD_OK;
}

extern "C" int pd_batch_eval(pd_batch* b, void* stream) {
  if (!b || !b->exec) return PD_EINVAL;
  // tensor cores with some maps inactive: the active maps' evaluations are
  // launched directly (the graph runs all maps)
  if (is_tc(b->prec) && !b->all_active) return tc_enqueue(b, (cudaStream_t)stream, false, true);
  return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? PD_OK : PD_ECUDA;
}

extern "C" int pd_batch_set_active(pd_batch* b, const int32_t* active, void* stream) {
  if (!b || !active) return PD_EINVAL;
  if (is_tc(b->prec)) {
    b->all_active = true;
    for (int m = 0; m < b->n_maps; ++m) {
      b->h_active[m] = active[m] != 0;
      b->all_active = b->all_active && b->h_active[m];
    }
    return PD_OK;
  }
  return cudaMemcpyAsync(b->d_active, active, sizeof(int) * b->n_maps, cudaMemcpyHostToDevice,
                         (cudaStream_t)stream) == cudaSuccess
             ? PD_OK
             : PD_ECUDA;
}

extern "C" int pd_batch_info(const pd_batch* b, int* chunk_factor, int* occ_div, double* tuned_ms) {
  if (!b) return PD_EINVAL;
  if (chunk_factor) *chunk_factor = b->tune.chunk_factor;
  if (occ_div) *occ_div = b->tune.occ_div;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return PD_OK;
}

extern "C" void pd_batch_destroy(pd_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  tc_free(b);
  free_plan_device(b);
  cudaFree(b->d_counters);
  cudaFree(b->d_active);
  delete b;
}

// ---------------------------------------------------------------------------
// Lockstep batched ascent: one host thread per map runs the same optimiser
// as pd_fit; every objective/gradient request goes to a coordinator that,
// once all running maps have asked, evaluates all of them with one replay
// of the batch graph (maps that are not asking are masked off).  A batch
// plan is built when a round first needs its precision (the FP64 plan only
// once some map refines), autotuned only for batches of at least
// kTuneMaps maps (the timing costs more than it saves on a few maps), and
// the trial parameters and results pass through pinned host buffers.
// ---------------------------------------------------------------------------
namespace pd {
namespace {

constexpr int kTuneMaps = 16;

class Coordinator {
 public:
  // maps: the batch with theta/obj/grad pointing into d_theta/d_obj/d_grad
  Coordinator(const std::vector<pd_map>& maps, int K, int d, double eps, double* d_theta, double* d_obj,
              double* d_grad, cudaStream_t st)
      : n_((int)maps.size()), K_(K), d_(d), eps_(eps), maps_(maps), d_theta_(d_theta), d_obj_(d_obj),
        d_grad_(d_grad), st_(st), running_((int)maps.size()) {
    off_.resize(n_ + 1, 0);
    for (int m = 0; m < n_; ++m) off_[m + 1] = off_[m] + (size_t)maps_[m].N * K_;
    if (cudaMallocHost((void**)&h_theta_, sizeof(double) * std::max<size_t>(off_[n_], 1)) != cudaSuccess ||
        cudaMallocHost((void**)&h_grad_, sizeof(double) * std::max<size_t>(off_[n_], 1)) != cudaSuccess ||
        cudaMallocHost((void**)&h_obj_, sizeof(double) * n_) != cudaSuccess) {
      cudaGetLastError();
      ok_ = false;
    }
    want_.assign(n_, -1);
    want_eps_.assign(n_, 0.0);
  }
  ~Coordinator() {
    for (auto& kv : plans_) pd_batch_destroy(kv.second);
    if (h_theta_) cudaFreeHost(h_theta_);
    if (h_grad_) cudaFreeHost(h_grad_);
    if (h_obj_) cudaFreeHost(h_obj_);
  }
  bool ok() const { return ok_; }
  int64_t rounds = 0;

  // called from map m's thread; theta/grad are full [N][K] blocks
  int eval(int m, int prec, double eps, const double* theta, double* phi, double* grad) {
    std::unique_lock<std::mutex> lk(mu_);
    memcpy(&h_theta_[off_[m]], theta, sizeof(double) * maps_[m].N * K_);
    want_[m] = prec;
    want_eps_[m] = eps;
    ++waiting_;
    const int64_t my_round = round_;
    if (waiting_ == running_) {
      run_round();
    } else {
      cv_.wait(lk, [&] { return round_ != my_round; });
    }
    if (rc_) return rc_;
    *phi = h_obj_[m];
    memcpy(grad, &h_grad_[off_[m]], sizeof(double) * maps_[m].N * K_);
    return PD_OK;
  }
  void finish() {
    std::unique_lock<std::mutex> lk(mu_);
    --running_;
    if (running_ > 0 && waiting_ == running_) run_round();
  }

 private:
  // the batch plan of a precision and eps, built on first use
  int plan(int prec, double eps, pd_batch** out) {
    pd_batch*& b = plans_[std::make_pair(prec, eps)];
    if (!b) {
      pd_eval_opts eo{d_, eps, prec};
      const int rc = pd_batch_create(n_, maps_.data(), &eo, n_ >= kTuneMaps ? 1 : 0, &b);
      if (rc) return rc;
    }
    *out = b;
    return PD_OK;
  }

  void run_round() {  // with mu_ held
    std::vector<int32_t> act(n_);
    int rc = PD_OK;
    if (cudaMemcpyAsync(d_theta_, h_theta_, sizeof(double) * off_[n_], cudaMemcpyHostToDevice, st_) != cudaSuccess)
      rc = PD_ECUDA;
    // one replay per (precision, eps) that some waiting map asked for (maps
    // in different annealing stages ask for different eps)
    std::vector<std::pair<int, double>> kinds;
    for (int m = 0; m < n_; ++m)
      if (want_[m] >= 0 && std::find(kinds.begin(), kinds.end(), std::make_pair(want_[m], want_eps_[m])) == kinds.end())
        kinds.push_back(std::make_pair(want_[m], want_eps_[m]));
    for (const auto& kd : kinds) {
      if (rc != PD_OK) break;
      for (int m = 0; m < n_; ++m) act[m] = want_[m] == kd.first && want_eps_[m] == kd.second;
      pd_batch* b = nullptr;
      rc = plan(kd.first, kd.second, &b);
      if (rc == PD_OK) rc = pd_batch_set_active(b, act.data(), st_);
      if (rc == PD_OK) rc = pd_batch_eval(b, st_);
    }
    if (rc == PD_OK &&
        (cudaMemcpyAsync(h_obj_, d_obj_, sizeof(double) * n_, cudaMemcpyDeviceToHost, st_) != cudaSuccess ||
         cudaMemcpyAsync(h_grad_, d_grad_, sizeof(double) * off_[n_], cudaMemcpyDeviceToHost, st_) != cudaSuccess))
      rc = PD_ECUDA;
    if (rc == PD_OK && cudaStreamSynchronize(st_) != cudaSuccess) rc = PD_ECUDA;
    rc_ = rc;
    for (int m = 0; m < n_; ++m) want_[m] = -1;
    waiting_ = 0;
    ++round_;
    ++rounds;
    cv_.notify_all();
  }

  int n_, K_, d_;
  double eps_;
  std::vector<pd_map> maps_;
  std::map<std::pair<int, double>, pd_batch*> plans_;
  std::vector<double> want_eps_;
  double *d_theta_, *d_obj_, *d_grad_;
  cudaStream_t st_;
  std::vector<size_t> off_;
  double *h_theta_ = nullptr, *h_grad_ = nullptr, *h_obj_ = nullptr;  // pinned
  bool ok_ = true;
  std::vector<int> want_;
  std::mutex mu_;
  std::condition_variable cv_;
  int running_, waiting_ = 0;
  int64_t round_ = 0;
  int rc_ = PD_OK;
};

// Evaluator of one map that goes through the coordinator.
class BatchedMap : public Evaluator {
 public:
  BatchedMap(Coordinator* co, int m, int N, int K, double eps)
      : co_(co), m_(m), N_(N), K_(K), eps_(eps), th_((size_t)N * K), gr_((size_t)N * K) {}
  int n_free() const override { return (N_ - 1) * K_; }
  void set_eps(double e) { eps_ = e; }
  int eval(const Vec& x, int prec, double* f, Vec* gf) override {
    for (int q = 0; q < n_free(); ++q) th_[q] = x[q];
    for (int k = 0; k < K_; ++k) th_[(size_t)(N_ - 1) * K_ + k] = 0.0;
    double phi = 0.0;
    const int rc = co_->eval(m_, prec, eps_, th_.data(), &phi, gr_.data());
    if (rc) return rc;
    ++evals;
    *f = -phi;
    if (gf) {
      gf->resize(n_free());
      for (int q = 0; q < n_free(); ++q) (*gf)[q] = -gr_[q];
    }
    return PD_OK;
  }
  int hvp(const Vec&, const Vec&, int, Vec*) override { return PD_ENOTSUP; }

 private:
  Coordinator* co_;
  int m_, N_, K_;
  double eps_;
  std::vector<double> th_, gr_;
};

}  // namespace
}  // namespace pd

extern "C" int pd_fit_batched(int n_maps, const pd_map* maps, double* const* theta_io, const pd_fit_opts* opts,
                              pd_fit_report* reports, void* stream) {
  using namespace pd;
  const auto t0 = std::chrono::steady_clock::now();
  if (n_maps < 1 || !maps || !theta_io || !opts || !reports) return PD_EINVAL;
  if (opts->method != PD_METHOD_LBFGS || opts->lbfgs_m < 1) return PD_ENOTSUP;
  if (opts->prec < PD_FP64 || opts->prec > PD_BF16X3) return PD_EINVAL;
  if (opts->init != PD_INIT_ZERO && opts->init != PD_INIT_GIVEN) return PD_ENOTSUP;
  const bool anneal = opts->anneal_eps0 > opts->eps;
  if (anneal && (!isfinite(opts->anneal_eps0) || !(opts->anneal_factor > 0.0 && opts->anneal_factor < 1.0) ||
                 opts->anneal_iter < 1))
    return PD_EINVAL;
  if (opts->err_stop) return PD_ENOTSUP;  // Err-aligned stopping: pd_fit only
  cudaStream_t st = (cudaStream_t)stream;
  const int K = basis_K(2, opts->d);
  for (int m = 0; m < n_maps; ++m) {
    if (maps[m].grid.dim != 2 || maps[m].N < 2 || !theta_io[m]) return PD_EINVAL;
    int rc = pd_check_labels(&maps[m].grid, maps[m].labels, maps[m].N, stream);
    if (rc) return rc;
  }
  // concatenated device buffers for the trial parameters and results
  std::vector<size_t> off(n_maps + 1, 0);
  for (int m = 0; m < n_maps; ++m) off[m + 1] = off[m] + (size_t)maps[m].N * K;
  double *d_theta = nullptr, *d_grad = nullptr, *d_obj = nullptr;
  if (cudaMalloc(&d_theta, sizeof(double) * off[n_maps]) != cudaSuccess ||
      cudaMalloc(&d_grad, sizeof(double) * off[n_maps]) != cudaSuccess ||
      cudaMalloc(&d_obj, sizeof(double) * n_maps) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_theta);
    cudaFree(d_grad);
    return PD_ENOMEM;
  }
  std::vector<pd_map> bm(maps, maps + n_maps);
  for (int m = 0; m < n_maps; ++m) {
    bm[m].theta = d_theta + off[m];
    bm[m].obj_out = d_obj + m;
    bm[m].grad_out = d_grad + off[m];
  }
  int rc = PD_OK;
  std::vector<std::vector<double>> th0(n_maps);
  for (int m = 0; rc == PD_OK && m < n_maps; ++m) {
    th0[m].assign((size_t)maps[m].N * K, 0.0);
    if (opts->init == PD_INIT_GIVEN &&
        cudaMemcpy(th0[m].data(), theta_io[m], sizeof(double) * th0[m].size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = PD_ECUDA;
  }
  auto release = [&]() {
    cudaFree(d_theta);
    cudaFree(d_grad);
    cudaFree(d_obj);
  };
  if (rc) {
    release();
    return rc;
  }
  std::vector<int> rcs(n_maps, PD_OK);
  {
    Coordinator co(bm, K, opts->d, opts->eps, d_theta, d_obj, d_grad, st);
    if (!co.ok()) {
      release();
      return PD_ENOMEM;
    }
    std::vector<std::thread> threads;
    threads.reserve(n_maps);
    for (int m = 0; m < n_maps; ++m) {
      threads.emplace_back([&, m]() {
        const int N = maps[m].N;
        BatchedMap ev(&co, m, N, K, opts->eps);
        FitState fs;
        pd_fit_opts om = *opts;
        if (!isnan(maps[m].target_phi)) om.target_phi = maps[m].target_phi;
        // the stages of eps-annealing, as in pd_fit: each warm-started from
        // the last, the last at eps with the full schedule
        std::vector<double> ths = th0[m];
        double eps_k = anneal ? opts->anneal_eps0 : opts->eps;
        int r = PD_OK, stages = 0, iters = 0, iters1 = 0;
        for (;;) {
          const bool last = eps_k <= opts->eps;
          if (last) eps_k = opts->eps;
          ev.set_eps(eps_k);
          pd_fit_opts so = om;
          so.eps = eps_k;
          if (!last) {
            so.max_iter = opts->anneal_iter;
            so.refine_iter = 0;
            so.target_phi = -INFINITY;
            so.switch_rtol = 0.0;
          }
          r = fit_run(ev, ths, N, K, so, &fs);
          if (r) break;
          ++stages;
          iters += fs.iters;
          iters1 += last ? fs.iters_phase1 : fs.iters;
          for (size_t q = 0; q < fs.cur.x.size(); ++q) ths[q] = fs.cur.x[q];
          for (int k = 0; k < K; ++k) ths[(size_t)(N - 1) * K + k] = 0.0;
          if (last) break;
          eps_k *= opts->anneal_factor;
        }
        fs.iters = iters;
        fs.iters_phase1 = iters1;
        // final double-precision evaluation for the report
        if (r == PD_OK && fs.final_prec != PD_FP64) {
          std::vector<double> gf;
          r = ev.eval(fs.cur.x, PD_FP64, &fs.cur.f, &gf);
          if (r == PD_OK) fs.cur.g = gf;
        }
        co.finish();
        pd_fit_report& rep = reports[m];
        memset(&rep, 0, sizeof(rep));
        rep.phi = -fs.cur.f;
        rep.gnorm = sqrt(dot(fs.cur.g, fs.cur.g));
        rep.iters = fs.iters;
        rep.iters_phase1 = fs.iters_phase1;
        rep.evals = ev.evals;
        rep.status = fs.status;
        rep.eps_final = eps_k;
        rep.stages = stages;
        rcs[m] = r;
        // gauge-fixed result
        std::vector<double> th((size_t)N * K, 0.0);
        for (int q = 0; q < (N - 1) * K; ++q) th[q] = fs.cur.x[q];
        if (r == PD_OK && cudaMemcpy(theta_io[m], th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice) !=
                              cudaSuccess)
          rcs[m] = PD_ECUDA;
      });
    }
    for (auto& t : threads) t.join();
  }  // (the coordinator's batch plans are freed here)
  // Err per map (double-precision assignment on the caller's stream)
  int64_t* d_mis = nullptr;
  int32_t* d_lab = nullptr;
  int64_t Pmax = 1;
  for (int m = 0; m < n_maps; ++m) Pmax = std::max<int64_t>(Pmax, maps[m].grid.P);
  if (cudaMalloc(&d_mis, sizeof(int64_t)) == cudaSuccess && cudaMalloc(&d_lab, sizeof(int32_t) * Pmax) == cudaSuccess) {
    for (int m = 0; m < n_maps; ++m) {
      int64_t miss = 0;
      if (pd_assign(&maps[m].grid, maps[m].N, opts->d, theta_io[m], d_lab, nullptr, maps[m].labels, d_mis, stream) ==
              PD_OK &&
          cudaMemcpyAsync(&miss, d_mis, sizeof(int64_t), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
          cudaStreamSynchronize(st) == cudaSuccess)
        reports[m].err = (double)miss / (double)maps[m].grid.P;
    }
  } else {
    cudaGetLastError();
  }
  cudaFree(d_mis);
  cudaFree(d_lab);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int m = 0; m < n_maps; ++m) reports[m].seconds = secs;
  release();
  for (int m = 0; m < n_maps; ++m)
    if (rcs[m]) return rcs[m];
  return PD_OK;
}
