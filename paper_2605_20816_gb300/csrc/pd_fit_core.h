// pd_fit_core.h -- the optimiser of the ascent scheme (Sec. 5.2), shared by
// the single-map fit (pd_fit.cu) and the batched fit (pd_batch.cu).  It
// works on the free parameters x = theta_0..theta_{N-2} (theta_{N-1} = 0)
// and minimises f = -Phi through an Evaluator.
#pragma once

#include <stdint.h>

#include <vector>

#include "pd.h"

namespace pd {

using Vec = std::vector<double>;

double dot(const Vec& a, const Vec& b);

// f(x) = -Phi and its gradient (and Hessian products) at free parameters x.
class Evaluator {
 public:
  virtual ~Evaluator() = default;
  virtual int n_free() const = 0;
  virtual int eval(const Vec& x, int prec, double* f, Vec* gf) = 0;
  virtual int hvp(const Vec& x, const Vec& v, int prec, Vec* out) = 0;
  int64_t evals = 0, hvps = 0;
};

struct Point {
  Vec x, g;
  double f = 0.0;
};

struct FitState {
  Point cur;
  int iters = 0, iters_phase1 = 0;
  int status = 0;  // 0 budget, 1 gtol, 2 line search stalled, 3 target
  int final_prec = PD_FP64;
};

// Runs the phases requested by opts from theta0 (full [N][K], gauge-fixed
// here by subtracting its last block); the result is in out->cur.
int fit_run(Evaluator& ev, const Vec& theta0, int N, int K, const pd_fit_opts& opts, FitState* out);

}  // namespace pd
