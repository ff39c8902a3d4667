// pd_fit.cu -- the ascent scheme (Sec. 5.2): maximise Phi over the
// gauge-fixed parameters (theta_{N-1} = 0, Remark 4.3) by L-BFGS with a
// strong-Wolfe line search, or by truncated Newton with Hessian-vector
// products (eq. hess).  The host runs the optimiser in double; every
// objective/gradient or Hessian-vector evaluation is one device evaluation
// of this library.
//
// Constants (the paper fixes none of them): L-BFGS memory m (10); strong
// Wolfe c1 = 1e-4, c2 = 0.9, at most 25 evaluations per line search;
// bracketing doubles the step; zooming uses a cubic interpolant kept at
// least 10% of the bracket away from its ends, else bisection; the first
// iteration tries the step 1/||g||_2, later ones the unit step; the initial
// inverse Hessian is gamma I with gamma = s.y / y.y of the newest pair; a
// pair is stored only if s.y > 1e-300; a non-descent direction restarts the
// memory.  Newton-CG: conjugate gradients on (-H) s = grad Phi to relative
// residual min(0.5, sqrt(||g||)), at most max_cg steps, stopping at
// non-positive curvature (steepest ascent when that happens at once).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "pd.h"
#include "pd_fit_core.h"
#include "pd_internal.h"

namespace pd {

// Eight interleaved partial sums, combined in a fixed order: the same
// result on every call, and eight independent add chains instead of one
// (a single running sum over tens of thousands of terms is bound by the
// add latency and dominated the host side of an L-BFGS iteration).
double dot(const Vec& a, const Vec& b) {
  const size_t n = a.size();
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  size_t q = 0;
  for (; q + 8 <= n; q += 8)
    for (int u = 0; u < 8; ++u) s[u] += a[q + u] * b[q + u];
  for (int u = 0; q < n; ++q, ++u) s[u] += a[q] * b[q];
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

namespace {

class Problem : public Evaluator {
 public:
  // hvp: the fit takes Hessian-vector products (Newton-CG)
  Problem(const pd_grid* grid, const Geom& g, const int32_t* labels, int N, int d, double eps, bool hvp,
          cudaStream_t st)
      : grid_(grid), g_(g), labels_(labels), N_(N), d_(d), K_(basis_K(grid->dim, d)), eps_(eps), hvp_(hvp), st_(st),
        sc_(st) {
    d_theta_ = sc_.get<double>((size_t)N * K_);
    d_grad_ = sc_.get<double>((size_t)N * K_);
    d_v_ = sc_.get<double>((size_t)N * K_);
    d_obj_ = sc_.get<double>(1);
    d_mis_ = sc_.get<int64_t>(1);
    d_lab_ = sc_.get<int32_t>((size_t)(g.P > 0 ? g.P : 1));
    // pinned staging: the uploads run asynchronously, and the one
    // synchronisation per evaluation (after the read-back) also orders
    // them before the next overwrite of these buffers
    const size_t nk = (size_t)N * K_;
    if (cudaMallocHost((void**)&h_theta_, sizeof(double) * nk) != cudaSuccess) h_theta_ = nullptr;
    if (cudaMallocHost((void**)&h_v_, sizeof(double) * nk) != cudaSuccess) h_v_ = nullptr;
    if (cudaMallocHost((void**)&h_grad_, sizeof(double) * (nk + 1)) != cudaSuccess) h_grad_ = nullptr;
  }
  ~Problem() override {
    for (PlanCore& p : plans_) plan_free(&p);
    if (h_theta_) cudaFreeHost(h_theta_);
    if (h_v_) cudaFreeHost(h_v_);
    if (h_grad_) cudaFreeHost(h_grad_);
  }
  bool ok() const { return sc_.ok() && h_theta_ && h_v_ && h_grad_; }
  void set_eps(double e) { eps_ = e; }
  int n_free() const override { return (N_ - 1) * K_; }
  int K() const { return K_; }

  // f = -Phi, gf = -grad Phi on the free blocks
  int eval(const Vec& x, int prec, double* f, Vec* gf) override {
    int rc = upload(x, d_theta_, h_theta_);
    if (rc) return rc;
    PlanCore* pl = nullptr;
    rc = plan(prec, &pl);
    if (rc) return rc;
    rc = plan_eval(pl, d_theta_, eps_, d_obj_, gf ? d_grad_ : nullptr, st_);
    if (rc) return rc;
    const size_t nk = (size_t)N_ * K_;
    double* h_phi = h_grad_ + nk;
    if (cudaMemcpyAsync(h_phi, d_obj_, sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess) return PD_ECUDA;
    if (gf && cudaMemcpyAsync(h_grad_, d_grad_, sizeof(double) * nk, cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return PD_ECUDA;
    if (cudaStreamSynchronize(st_) != cudaSuccess) return PD_ECUDA;
    ++evals;
    const double phi = *h_phi;
    *f = -phi;
    if (gf) {
      gf->resize(n_free());
      for (int q = 0; q < n_free(); ++q) (*gf)[q] = -h_grad_[q];
    }
    return PD_OK;
  }

  // out = (Hessian of -Phi) v on the free blocks
  int hvp(const Vec& x, const Vec& v, int prec, Vec* out) override {
    int rc = upload(x, d_theta_, h_theta_);
    if (rc) return rc;
    rc = upload(v, d_v_, h_v_);
    if (rc) return rc;
    PlanCore* pl = nullptr;
    rc = plan(prec, &pl);
    if (rc) return rc;
    rc = plan_hvp(pl, d_theta_, d_v_, eps_, d_grad_, st_);
    if (rc) return rc;
    if (cudaMemcpyAsync(h_grad_, d_grad_, sizeof(double) * (size_t)N_ * K_, cudaMemcpyDeviceToHost, st_) !=
        cudaSuccess)
      return PD_ECUDA;
    if (cudaStreamSynchronize(st_) != cudaSuccess) return PD_ECUDA;
    ++hvps;
    out->resize(n_free());
    for (int q = 0; q < n_free(); ++q) (*out)[q] = -h_grad_[q];
    return PD_OK;
  }

  int mismatch(const Vec& x, int64_t* miss) {
    int rc = upload(x, d_theta_, h_theta_);
    if (rc) return rc;
    rc = assign_simt(g_, grid_->dim, d_, N_, d_theta_, d_lab_, nullptr, labels_, d_mis_, st_);
    if (rc) return rc;
    if (cudaMemcpyAsync(miss, d_mis_, sizeof(int64_t), cudaMemcpyDeviceToHost, st_) != cudaSuccess) return PD_ECUDA;
    return cudaStreamSynchronize(st_) == cudaSuccess ? PD_OK : PD_ECUDA;
  }

  int write_theta(const Vec& x, double* dst) {
    int rc = upload(x, d_theta_, h_theta_);
    if (rc) return rc;
    if (cudaMemcpyAsync(dst, d_theta_, sizeof(double) * (size_t)N_ * K_, cudaMemcpyDeviceToDevice, st_) !=
        cudaSuccess)
      return PD_ECUDA;
    return cudaStreamSynchronize(st_) == cudaSuccess ? PD_OK : PD_ECUDA;
  }

 private:
  // the plan of precision prec, made on first use: the scratch of every
  // evaluation in that precision, and the centre features and grain order
  // computed once for the whole fit
  int plan(int prec, PlanCore** out) {
    if (prec < PD_FP64 || prec > PD_BF16X3) return PD_EINVAL;
    PlanCore& p = plans_[prec];
    if (!p.mem) {
      const int rc = plan_init(&p, g_, grid_->dim, labels_, N_, d_, prec, hvp_);
      if (rc) {
        plan_free(&p);
        return rc;
      }
    }
    *out = &p;
    return PD_OK;
  }

  // free blocks x -> full [N][K] with the last block zero, through the
  // pinned staging buffer h (asynchronous: every caller synchronises the
  // stream before it returns, so h is not rewritten while in flight)
  int upload(const Vec& x, double* dst, double* h) {
    for (int q = 0; q < n_free(); ++q) h[q] = x[q];
    for (int k = 0; k < K_; ++k) h[(size_t)(N_ - 1) * K_ + k] = 0.0;
    return cudaMemcpyAsync(dst, h, sizeof(double) * (size_t)N_ * K_, cudaMemcpyHostToDevice, st_) == cudaSuccess
               ? PD_OK
               : PD_ECUDA;
  }

  const pd_grid* grid_;
  Geom g_;
  const int32_t* labels_;
  int N_, d_, K_;
  double eps_;
  bool hvp_;
  cudaStream_t st_;
  PlanCore plans_[PD_BF16X3 + 1];
  Scratch sc_;
  double *d_theta_, *d_grad_, *d_v_, *d_obj_;
  int64_t* d_mis_;
  int32_t* d_lab_;
  double* h_theta_ = nullptr;  // pinned [N][K]
  double* h_v_ = nullptr;      // pinned [N][K]
  double* h_grad_ = nullptr;   // pinned [N][K] + 1 (objective)
};

// Safeguarded cubic step between (a, fa, ga) and (b, fb, gb).
double cubic_step(double a, double fa, double ga, double b, double fb, double gb) {
  const double lo = fmin(a, b), hi = fmax(a, b);
  const double t1 = ga + gb - 3.0 * (fa - fb) / (a - b);
  const double rad = t1 * t1 - ga * gb;
  if (rad >= 0.0) {
    double t2 = sqrt(rad);
    if (b < a) t2 = -t2;
    const double z = b - (b - a) * ((gb + t2 - t1) / (gb - ga + 2.0 * t2));
    if (isfinite(z) && z >= lo && z <= hi) return z;
  }
  return 0.5 * (a + b);
}

// Strong-Wolfe search along dir from cur; returns the step (0 on failure,
// with *out = cur re-evaluated).
int wolfe(Evaluator& pb, int prec, const Point& cur, const Vec& dir, double a0, Point* out, double* step) {
  const double c1 = 1e-4, c2 = 0.9;
  const int budget = 25;
  const int n = (int)cur.x.size();
  const double d0 = dot(cur.g, dir);
  int used = 0;
  auto try_at = [&](double a, Point* p) {
    p->x.resize(n);
    for (int q = 0; q < n; ++q) p->x[q] = cur.x[q] + a * dir[q];
    ++used;
    return pb.eval(p->x, prec, &p->f, &p->g);
  };
  double ap = 0.0, fp = cur.f, dp = d0;
  double a = a0;
  double lo = 0, flo = 0, glo = 0, hi = 0, fhi = 0, ghi = 0;
  bool have_bracket = false;
  Point p;
  while (used < budget) {
    int rc = try_at(a, &p);
    if (rc) return rc;
    const double da = dot(p.g, dir);
    if (!isfinite(p.f) || p.f > cur.f + c1 * a * d0 || (used > 1 && p.f >= fp)) {
      lo = ap; flo = fp; glo = dp;
      hi = a; fhi = p.f; ghi = da;
      have_bracket = true;
      break;
    }
    if (fabs(da) <= -c2 * d0) {
      *out = p;
      *step = a;
      return PD_OK;
    }
    if (da >= 0.0) {
      lo = a; flo = p.f; glo = da;
      hi = ap; fhi = fp; ghi = dp;
      have_bracket = true;
      break;
    }
    ap = a; fp = p.f; dp = da;
    a *= 2.0;
  }
  if (have_bracket) {
    const double xnorm = sqrt(dot(cur.x, cur.x)), dnorm = sqrt(dot(dir, dir));
    while (used < budget) {
      const double w = fabs(hi - lo);
      double t = isfinite(fhi) ? cubic_step(lo, flo, glo, hi, fhi, ghi) : 0.5 * (lo + hi);
      if (t < fmin(lo, hi) + 0.1 * w || t > fmax(lo, hi) - 0.1 * w) t = 0.5 * (lo + hi);
      int rc = try_at(t, &p);
      if (rc) return rc;
      const double dt = dot(p.g, dir);
      if (!isfinite(p.f) || p.f > cur.f + c1 * t * d0 || p.f >= flo) {
        hi = t; fhi = p.f; ghi = dt;
      } else {
        if (fabs(dt) <= -c2 * d0) {
          *out = p;
          *step = t;
          return PD_OK;
        }
        if (dt * (hi - lo) >= 0.0) { hi = lo; fhi = flo; ghi = glo; }
        lo = t; flo = p.f; glo = dt;
      }
      if (fabs(hi - lo) * dnorm < 1e-16 * (1.0 + xnorm)) break;
    }
    if (lo > 0.0) {
      int rc = try_at(lo, &p);
      if (rc) return rc;
      *out = p;
      *step = lo;
      return PD_OK;
    }
  }
  // failure: stay at the current point (re-evaluated, as a search would)
  Point back;
  back.x = cur.x;
  int rc = pb.eval(back.x, prec, &back.f, &back.g);
  if (rc) return rc;
  *out = back;
  *step = 0.0;
  return PD_OK;
}

struct PhaseResult {
  int iters = 0;
  int status = 0;  // 0 budget, 1 gtol, 2 stalled, 3 target, 4 switch
};

int lbfgs_phase(Evaluator& pb, int prec, Point& cur, int max_iter, int m, double gtol, double target_phi,
                double switch_rtol, bool first_scaled, PhaseResult* res) {
  const int n = (int)cur.x.size();
  std::vector<Vec> S, Y;
  std::vector<double> rho;
  Vec dir(n), alpha(m);
  int it = 0;
  for (; it < max_iter; ++it) {
    const double gn = sqrt(dot(cur.g, cur.g));
    if (gn <= gtol) { res->status = 1; break; }
    if (isfinite(target_phi) && -cur.f >= target_phi) { res->status = 3; break; }
    for (int q = 0; q < n; ++q) dir[q] = -cur.g[q];
    const int h = (int)S.size();  // newest pair last
    for (int j = h - 1; j >= 0; --j) {
      alpha[j] = rho[j] * dot(S[j], dir);
      for (int q = 0; q < n; ++q) dir[q] -= alpha[j] * Y[j][q];
    }
    if (h > 0) {
      const double gamma = dot(S[h - 1], Y[h - 1]) / dot(Y[h - 1], Y[h - 1]);
      for (int q = 0; q < n; ++q) dir[q] *= gamma;
    }
    for (int j = 0; j < h; ++j) {
      const double beta = rho[j] * dot(Y[j], dir);
      for (int q = 0; q < n; ++q) dir[q] += (alpha[j] - beta) * S[j][q];
    }
    if (dot(dir, cur.g) >= 0.0) {
      S.clear(); Y.clear(); rho.clear();
      for (int q = 0; q < n; ++q) dir[q] = -cur.g[q];
    }
    const double a0 = (it == 0 && first_scaled) ? 1.0 / gn : 1.0;
    Point nxt;
    double step = 0.0;
    int rc = wolfe(pb, prec, cur, dir, a0, &nxt, &step);
    if (rc) return rc;
    if (step == 0.0) { res->status = 2; break; }
    Vec s(n), y(n);
    for (int q = 0; q < n; ++q) { s[q] = nxt.x[q] - cur.x[q]; y[q] = nxt.g[q] - cur.g[q]; }
    const double sy = dot(s, y);
    if (sy > 1e-300) {
      if ((int)S.size() == m) { S.erase(S.begin()); Y.erase(Y.begin()); rho.erase(rho.begin()); }
      S.push_back(std::move(s)); Y.push_back(std::move(y)); rho.push_back(1.0 / sy);
    }
    const double gain = cur.f - nxt.f;
    cur = std::move(nxt);
    if (switch_rtol > 0.0 && gain <= switch_rtol * fabs(cur.f)) { ++it; res->status = 4; break; }
  }
  res->iters = it;
  return PD_OK;
}

int newton_phase(Evaluator& pb, int prec, Point& cur, int max_iter, int max_cg, double gtol, double target_phi,
                 PhaseResult* res) {
  const int n = (int)cur.x.size();
  Vec s(n), r(n), p(n), hp;
  int it = 0;
  for (; it < max_iter; ++it) {
    const double gn = sqrt(dot(cur.g, cur.g));
    if (gn <= gtol) { res->status = 1; break; }
    if (isfinite(target_phi) && -cur.f >= target_phi) { res->status = 3; break; }
    const double tol = (gn < 0.25 ? sqrt(gn) : 0.5) * gn;
    for (int q = 0; q < n; ++q) { s[q] = 0.0; r[q] = -cur.g[q]; p[q] = r[q]; }
    double rr = dot(r, r);
    for (int j = 0; j < max_cg; ++j) {
      int rc = pb.hvp(cur.x, p, prec, &hp);
      if (rc) return rc;
      const double curv = dot(p, hp);
      if (curv <= 0.0) {
        if (j == 0)
          for (int q = 0; q < n; ++q) s[q] = -cur.g[q];
        break;
      }
      const double a = rr / curv;
      for (int q = 0; q < n; ++q) { s[q] += a * p[q]; r[q] -= a * hp[q]; }
      const double rr2 = dot(r, r);
      if (sqrt(rr2) <= tol) break;
      const double b = rr2 / rr;
      for (int q = 0; q < n; ++q) p[q] = r[q] + b * p[q];
      rr = rr2;
    }
    if (dot(s, cur.g) >= 0.0)
      for (int q = 0; q < n; ++q) s[q] = -cur.g[q];
    Point nxt;
    double step = 0.0;
    int rc = wolfe(pb, prec, cur, s, 1.0, &nxt, &step);
    if (rc) return rc;
    if (step == 0.0) { res->status = 2; break; }
    cur = std::move(nxt);
  }
  res->iters = it;
  return PD_OK;
}

}  // namespace

int fit_run(Evaluator& ev, const Vec& th, int N, int K, const pd_fit_opts& o, FitState* out) {
  const int n = (N - 1) * K;
  Point& cur = out->cur;
  cur.x.resize(n);
  for (int i = 0; i < N - 1; ++i)
    for (int k = 0; k < K; ++k) cur.x[(size_t)i * K + k] = th[(size_t)i * K + k] - th[(size_t)(N - 1) * K + k];
  for (double v : cur.x)
    if (!isfinite(v)) return PD_ENAN;
  const double target = isnan(o.target_phi) ? -INFINITY : o.target_phi;
  int prec = o.prec;
  int rc = ev.eval(cur.x, prec, &cur.f, &cur.g);
  if (rc) return rc;
  PhaseResult r1, r2;
  if (o.method == PD_METHOD_LBFGS)
    rc = lbfgs_phase(ev, prec, cur, o.max_iter, o.lbfgs_m, o.gtol, target, o.switch_rtol, true, &r1);
  else
    rc = newton_phase(ev, prec, cur, o.max_iter, o.max_cg, o.gtol, target, &r1);
  if (rc) return rc;
  int status = r1.status;
  // a target reached in reduced precision counts only once the FP64
  // objective confirms it (the objective alone: no gradient pass); otherwise
  // the FP64 refinement continues from a full FP64 evaluation
  if (o.refine_iter > 0 && status == 3 && prec != PD_FP64) {
    double f64 = 0.0;
    rc = ev.eval(cur.x, PD_FP64, &f64, nullptr);
    if (rc) return rc;
    prec = PD_FP64;
    if (-f64 >= target) {
      cur.f = f64;  // the gradient stays that of the reduced-precision phase
    } else {
      status = 0;
      rc = ev.eval(cur.x, prec, &cur.f, &cur.g);
      if (rc) return rc;
    }
  }
  if (o.refine_iter > 0 && status != 3) {
    if (prec != PD_FP64) {
      prec = PD_FP64;
      rc = ev.eval(cur.x, prec, &cur.f, &cur.g);
      if (rc) return rc;
    }
    if (o.method == PD_METHOD_LBFGS)
      rc = lbfgs_phase(ev, prec, cur, o.refine_iter, o.lbfgs_m, o.gtol, target, 0.0, false, &r2);
    else
      rc = newton_phase(ev, prec, cur, o.refine_iter, o.max_cg, o.gtol, target, &r2);
    if (rc) return rc;
    status = r2.status;
  }
  out->iters = r1.iters + r2.iters;
  out->iters_phase1 = r1.iters;
  out->status = status == 4 ? 0 : status;
  out->final_prec = prec;
  return PD_OK;
}

}  // namespace pd

using namespace pd;

extern "C" int pd_fit(const pd_grid* grid, const int32_t* labels, int N, const pd_fit_opts* opts, double* theta_io,
                      pd_fit_report* report, void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (!opts || !labels || !theta_io || !report || N < 2 || g.P < 1) return PD_EINVAL;
  if (!(opts->eps > 0.0) || !isfinite(opts->eps) || opts->d < 1 || opts->max_iter < 0 || opts->refine_iter < 0)
    return PD_EINVAL;
  if (opts->prec < PD_FP64 || opts->prec > PD_BF16X3) return PD_EINVAL;
  if (opts->method != PD_METHOD_LBFGS && opts->method != PD_METHOD_NEWTON_CG) return PD_EINVAL;
  if (opts->method == PD_METHOD_LBFGS && opts->lbfgs_m < 1) return PD_EINVAL;
  if (pd_K(grid->dim, opts->d) < 0) return PD_EINVAL;
  const bool anneal = opts->anneal_eps0 > opts->eps;
  if (anneal && (!isfinite(opts->anneal_eps0) || !(opts->anneal_factor > 0.0 && opts->anneal_factor < 1.0) ||
                 opts->anneal_iter < 1))
    return PD_EINVAL;
  if ((grid->dim == 2 && opts->d > PD_MAX_DEGREE_2D) || (grid->dim == 3 && opts->d > PD_MAX_DEGREE_3D))
    return PD_ENOTSUP;
  memset(report, 0, sizeof(*report));
  cudaStream_t st = (cudaStream_t)stream;
  device_sm_count();
  rc = pd_check_labels(grid, labels, N, stream);
  if (rc) return rc;

  Problem pb(grid, g, labels, N, opts->d, opts->eps, opts->method == PD_METHOD_NEWTON_CG, st);
  if (!pb.ok()) return PD_ENOMEM;
  const int K = pb.K();

  // initial parameters
  std::vector<double> th((size_t)N * K, 0.0);
  if (opts->init == PD_INIT_HEURISTIC) {
    rc = pd_heuristic_init(grid, labels, N, opts->d, theta_io, stream);
    if (rc) return rc;
  } else if (opts->init != PD_INIT_GIVEN && opts->init != PD_INIT_ZERO) {
    return PD_EINVAL;
  }
  if (opts->init != PD_INIT_ZERO) {
    if (cudaMemcpyAsync(th.data(), theta_io, sizeof(double) * th.size(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return PD_ECUDA;
  }
  // the ascent scheme, in stages of decreasing eps when annealing
  FitState fs;
  int stages = 0, iters = 0, iters_phase1 = 0, status = 0;
  double eps_k = anneal ? opts->anneal_eps0 : opts->eps;
  for (;;) {
    const bool last = eps_k <= opts->eps;
    if (last) eps_k = opts->eps;
    pb.set_eps(eps_k);
    pd_fit_opts so = *opts;
    so.eps = eps_k;
    if (!last) {
      so.max_iter = opts->anneal_iter;
      so.refine_iter = 0;
      so.target_phi = -INFINITY;
      so.switch_rtol = 0.0;
    }
    rc = fit_run(pb, th, N, K, so, &fs);
    if (rc) return rc;
    ++stages;
    iters += fs.iters;
    iters_phase1 += last ? fs.iters_phase1 : fs.iters;
    status = fs.status;
    // the stage's parameters (gauge-fixed) start the next stage
    for (size_t q = 0; q < fs.cur.x.size(); ++q) th[q] = fs.cur.x[q];
    for (int k = 0; k < K; ++k) th[(size_t)(N - 1) * K + k] = 0.0;
    if (last) break;
    if (opts->err_stop) {
      // Err^G = 0: certified by Phi > -log 2 / |Omega| (Cor. 4.10, Phi in
      // FP64), else counted by the double-precision assignment
      double f64 = fs.cur.f;
      if (fs.final_prec != PD_FP64) {
        rc = pb.eval(fs.cur.x, PD_FP64, &f64, nullptr);
        if (rc) return rc;
      }
      bool done = -f64 > -log(2.0) / (double)g.P;
      if (!done) {
        int64_t miss = 0;
        rc = pb.mismatch(fs.cur.x, &miss);
        if (rc) return rc;
        done = miss == 0;
      }
      if (done) {
        status = 5;
        break;
      }
    }
    eps_k *= opts->anneal_factor;
  }
  Point& cur = fs.cur;
  const int prec = fs.final_prec;
  // final report in double precision
  double f_final = cur.f;
  std::vector<double> gfin = cur.g;
  if (prec != PD_FP64) {
    rc = pb.eval(cur.x, PD_FP64, &f_final, &gfin);
    if (rc) return rc;
  }
  int64_t miss = 0;
  rc = pb.mismatch(cur.x, &miss);
  if (rc) return rc;
  rc = pb.write_theta(cur.x, theta_io);
  if (rc) return rc;
  report->phi = -f_final;
  report->gnorm = sqrt(dot(gfin, gfin));
  report->err = (double)miss / (double)g.P;
  report->iters = iters;
  report->iters_phase1 = iters_phase1;
  report->evals = pb.evals;
  report->hvps = pb.hvps;
  report->status = status;
  report->eps_final = eps_k;
  report->stages = stages;
  report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return isfinite(report->phi) ? PD_OK : PD_ENAN;
}
