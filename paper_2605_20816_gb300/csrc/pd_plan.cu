// pd_plan.cu -- plans: the scratch of repeated evaluations on one pixel set
// and one label map, sized once and allocated once, with the parts of an
// evaluation that depend on the pixel set or the labels alone (centre
// features of the tiles, grain order) computed by the first call and kept.
//
// An evaluation in plan mode allocates the same buffers, in the same order
// and of the same sizes, on every call (optional outputs included), so a
// bump allocator over one buffer hands out the same addresses each time.
// A sizing pass runs the evaluation's allocation sequence without a buffer
// and records the bytes it needs; it returns before any launch, so its
// pointer arguments are never read.
//
// Repeated calls with the same arguments (the same parameter, direction and
// output pointers and the same eps, as in every evaluation of a fit) replay
// a CUDA graph of the evaluation: the first call with new arguments runs
// directly (and leaves the cached data), the second records the launches
// on a private stream as a graph, and it and every later call launch that
// graph on the caller's stream (one launch instead of about ten).  Tracing
// (pd_prof_enable) runs every call directly.
#include <cuda_runtime.h>
#include <math.h>
#include <new>

#include "pd.h"
#include "pd_internal.h"

namespace pd {
namespace {

// stands in for the device pointers of a sizing pass (never dereferenced)
const double kSizingArg = 0.0;

int run(PlanCore* p, PlanState* ps, const double* theta, const double* v, double eps, double* obj, double* grad,
        double* hv, cudaStream_t st) {
  EvalCall c{p->g, p->dim, p->d, p->N, p->prec, eps, p->labels, theta, v, obj, grad, hv};
  c.plan = ps;
  const bool tc = p->prec == PD_BF16 || p->prec == PD_BF16X3;
  return tc ? eval_tc(c, st) : eval_simt(c, st);
}

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

int plan_init(PlanCore* p, const Geom& g, int dim, const int32_t* labels, int N, int d, int prec, bool with_hvp) {
  *p = PlanCore{};
  p->g = g;
  p->dim = dim;
  p->d = d;
  p->N = N;
  p->prec = prec;
  p->labels = labels;
  p->with_hvp = with_hvp;
  device_sm_count();
  double* out = const_cast<double*>(&kSizingArg);
  int rc = run(p, &p->eval, &kSizingArg, nullptr, 1.0, out, out, nullptr, nullptr);
  if (rc) return rc;
  if (with_hvp) {
    rc = run(p, &p->hvp, &kSizingArg, &kSizingArg, 1.0, nullptr, nullptr, out, nullptr);
    if (rc) return rc;
  }
  const size_t e = round256(p->eval.need), h = with_hvp ? round256(p->hvp.need) : 0;
  p->bytes = e + h;
  if (cudaMalloc((void**)&p->mem, p->bytes) != cudaSuccess) {
    cudaGetLastError();
    p->mem = nullptr;
    return PD_ENOMEM;
  }
  p->eval.base = p->mem;
  p->eval.cap = e;
  if (with_hvp) {
    p->hvp.base = p->mem + e;
    p->hvp.cap = h;
  }
  return PD_OK;
}

namespace {

bool same_args(const PlanGraph& g, const double* theta, const double* v, double eps, double* obj, double* grad,
               double* hv) {
  return g.theta == theta && g.v == v && g.eps == eps && g.obj == obj && g.grad == grad && g.hv == hv;
}

// One evaluation of kind ps (graph gr): directly, or through the graph.
int run_cached(PlanCore* p, PlanState* ps, PlanGraph* gr, const double* theta, const double* v, double eps,
               double* obj, double* grad, double* hv, cudaStream_t st) {
  // (a call recorded into the caller's own graph, as the tensor-core batch
  // does, runs its launches directly into that graph)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;
  }
  if (cs != cudaStreamCaptureStatusNone) return run(p, ps, theta, v, eps, obj, grad, hv, st);
  const bool same = same_args(*gr, theta, v, eps, obj, grad, hv);
  if (!p->graphs || prof_enabled() || !same || (!gr->exec && !gr->seen)) {
    if (!same) {
      gr->theta = theta, gr->v = v, gr->eps = eps, gr->obj = obj, gr->grad = grad, gr->hv = hv;
      if (gr->exec) cudaGraphExecDestroy(gr->exec);
      gr->exec = nullptr;
    }
    gr->seen = true;
    return run(p, ps, theta, v, eps, obj, grad, hv, st);
  }
  if (!gr->exec) {
    // record the launches of this call (no work runs on the capture stream)
    if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      p->graphs = false;
      return run(p, ps, theta, v, eps, obj, grad, hv, st);
    }
    cudaGraph_t graph = nullptr;
    int rc = PD_OK;
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PD_ECUDA;
    if (rc == PD_OK) {
      rc = run(p, ps, theta, v, eps, obj, grad, hv, p->cap);
      if (cudaStreamEndCapture(p->cap, &graph) != cudaSuccess && rc == PD_OK) rc = PD_ECUDA;
    }
    if (rc == PD_OK && cudaGraphInstantiate(&gr->exec, graph, 0) != cudaSuccess) {
      gr->exec = nullptr;
      rc = PD_ECUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc != PD_OK) {
      // a capture that failed leaves nothing behind: run directly from now on
      cudaGetLastError();
      p->graphs = false;
      return run(p, ps, theta, v, eps, obj, grad, hv, st);
    }
  }
  return cudaGraphLaunch(gr->exec, st) == cudaSuccess ? PD_OK : PD_ECUDA;
}

}  // namespace

int plan_eval(PlanCore* p, const double* theta, double eps, double* obj, double* grad, cudaStream_t st) {
  return run_cached(p, &p->eval, &p->geval, theta, nullptr, eps, obj, grad, nullptr, st);
}

int plan_hvp(PlanCore* p, const double* theta, const double* v, double eps, double* hv, cudaStream_t st) {
  if (!p->with_hvp) return PD_EINVAL;
  return run_cached(p, &p->hvp, &p->ghvp, theta, v, eps, nullptr, nullptr, hv, st);
}

void plan_free(PlanCore* p) {
  if (p->geval.exec) cudaGraphExecDestroy(p->geval.exec);
  if (p->ghvp.exec) cudaGraphExecDestroy(p->ghvp.exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->mem) cudaFree(p->mem);
  *p = PlanCore{};
}

}  // namespace pd

struct pd_plan {
  pd::PlanCore core;
};

extern "C" {

int pd_plan_create(const pd_grid* grid, const int32_t* labels, int N, int d, int prec, int flags,
                   pd_plan** plan_out) {
  if (!plan_out) return PD_EINVAL;
  *plan_out = nullptr;
  pd::Geom g;
  int rc = pd::validate_grid(grid, &g);
  if (rc) return rc;
  if (!labels || N < 2 || g.P < 1 || d < 1 || (flags & ~PD_PLAN_HVP)) return PD_EINVAL;
  if (!pd::degree_ok(grid->dim, d)) return PD_ENOTSUP;
  if (prec < PD_FP64 || prec > PD_BF16X3) return PD_EINVAL;
  pd_plan* p = new (std::nothrow) pd_plan;
  if (!p) return PD_ENOMEM;
  rc = pd::plan_init(&p->core, g, grid->dim, labels, N, d, prec, (flags & PD_PLAN_HVP) != 0);
  if (rc) {
    pd::plan_free(&p->core);
    delete p;
    return rc;
  }
  *plan_out = p;
  return PD_OK;
}

int pd_plan_objective_grad(pd_plan* plan, const double* theta, double eps, double* obj_out, double* grad_out,
                           void* stream) {
  if (!plan || !theta || (!obj_out && !grad_out) || !(eps > 0.0) || !isfinite(eps)) return PD_EINVAL;
  return pd::plan_eval(&plan->core, theta, eps, obj_out, grad_out, (cudaStream_t)stream);
}

int pd_plan_hvp(pd_plan* plan, const double* theta, const double* v, double eps, double* hv_out, void* stream) {
  if (!plan || !theta || !v || !hv_out || !(eps > 0.0) || !isfinite(eps)) return PD_EINVAL;
  return pd::plan_hvp(&plan->core, theta, v, eps, hv_out, (cudaStream_t)stream);
}

int pd_plan_scratch_bytes(const pd_plan* plan, size_t* bytes_out) {
  if (!plan || !bytes_out) return PD_EINVAL;
  *bytes_out = plan->core.bytes;
  return PD_OK;
}

void pd_plan_destroy(pd_plan* plan) {
  if (!plan) return;
  pd::plan_free(&plan->core);
  delete plan;
}

}  // extern "C"
