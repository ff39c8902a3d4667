/*
 * pd_oracle.c -- slow, plain FP64 CPU oracle for polynomial-diagram fitting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library; the two are independent restatements of the paper
 * "Polynomial diagrams for microstructure modelling" (Bourne, Buze,
 * Gallouet, Merigot).
 *
 * Every routine is written for clarity: one pixel at a time, one grain at a
 * time, in the order the paper's formulas are written, in double precision.
 * Sums over pixels use Neumaier-compensated accumulation (same left-to-right
 * order, no blocking) so that the oracle's own rounding error stays far
 * below the 1e-10 parity bar even at 1.7e7 pixels.
 *
 * Conventions (readings of places where the paper is silent):
 *  - pixel centres (Sec. 2.1): x_a = -1 + (2 k_a + 1) / n_a for the 0-based
 *    index k_a along axis a; the linear pixel index is
 *    j = k_1 + n_1 (k_2 + n_2 k_3) (axis 1 fastest).  An explicit point list
 *    (the paper's "any finite set of sample points") replaces the grid when
 *    coords != NULL.
 *  - multi-index order of A_d (Sec. 3.1 only asks for "a fixed ordering"):
 *    ascending total degree; within one degree descending alpha_1, then
 *    descending alpha_2 (3-D).  2-D, d = 2: (0,0),(1,0),(0,1),(2,0),(1,1),(0,2).
 *  - grains are 0-based: labels in 0..N-1.
 *  - gauge fixing (Remark 4.3): the last grain's parameter block is 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXDIM 3
#define OR_MAXDEG 16

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) accumulator.                                      */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } or_acc;

static void acc_add(or_acc* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double acc_val(const or_acc* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Multi-index set A_d and K_d (Sec. 3.1; 3-D by the same tensor product).  */
/* ------------------------------------------------------------------------ */
int or_K(int dim, int d) {
  if (d < 0) return -1;
  if (dim == 2) return (d + 1) * (d + 2) / 2;
  if (dim == 3) return (d + 1) * (d + 2) * (d + 3) / 6;
  return -1;
}

/* alpha: [K][dim] exponents in the fixed order described above. */
int or_alpha(int dim, int d, int* alpha) {
  int k = 0;
  for (int g = 0; g <= d; ++g) {
    if (dim == 2) {
      for (int a1 = g; a1 >= 0; --a1) {
        alpha[2 * k + 0] = a1;
        alpha[2 * k + 1] = g - a1;
        ++k;
      }
    } else {
      for (int a1 = g; a1 >= 0; --a1)
        for (int a2 = g - a1; a2 >= 0; --a2) {
          alpha[3 * k + 0] = a1;
          alpha[3 * k + 1] = a2;
          alpha[3 * k + 2] = g - a1 - a2;
          ++k;
        }
    }
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Legendre polynomials by the three-term recurrence (Sec. 3.3):            */
/* (m+1) P_{m+1}(t) = (2m+1) t P_m(t) - m P_{m-1}(t),  P_0 = 1, P_1 = t.     */
/* ------------------------------------------------------------------------ */
double or_legendre(int m, double t) {
  if (m == 0) return 1.0;
  double p_prev = 1.0, p = t;
  for (int j = 1; j < m; ++j) {
    double p_next = ((2.0 * j + 1.0) * t * p - (double)j * p_prev) / (j + 1.0);
    p_prev = p;
    p = p_next;
  }
  return p;
}

/* ------------------------------------------------------------------------ */
/* Pixel centres (Sec. 2.1) or an explicit point list.                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int dim;
  int64_t n[3];          /* grid extents (ignored when coords != NULL)       */
  const double* coords;  /* NULL, or [P][dim] explicit points in [-1,1]^dim  */
  int64_t P;             /* number of pixels                                 */
} or_grid;

void or_point(const or_grid* g, int64_t j, double* x) {
  if (g->coords) {
    for (int a = 0; a < g->dim; ++a) x[a] = g->coords[j * g->dim + a];
    return;
  }
  int64_t r = j;
  for (int a = 0; a < g->dim; ++a) {
    int64_t k = r % g->n[a];
    r /= g->n[a];
    x[a] = -1.0 + (2.0 * (double)k + 1.0) / (double)g->n[a];
  }
}

/* Tensor-product Legendre design function eta_L^(d)(x) (Sec. 3.3):
 * psi_alpha(x) = prod_a P_{alpha_a}(x_a). */
static void legendre_features(int dim, int d, const int* alpha, int K,
                              const double* x, double* eta) {
  for (int k = 0; k < K; ++k) {
    double v = 1.0;
    for (int a = 0; a < dim; ++a) v *= or_legendre(alpha[k * dim + a], x[a]);
    eta[k] = v;
  }
  (void)d;
}

/* Monomial design function eta^(d)(x) = (x^alpha) (Sec. 3.2). */
static void monomial_features(int dim, const int* alpha, int K,
                              const double* x, double* eta) {
  for (int k = 0; k < K; ++k) {
    double v = 1.0;
    for (int a = 0; a < dim; ++a)
      for (int e = 0; e < alpha[k * dim + a]; ++e) v *= x[a];
    eta[k] = v;
  }
}

static int* make_alpha(int dim, int d, int* K_out) {
  int K = or_K(dim, d);
  if (K <= 0) return NULL;
  int* alpha = (int*)malloc(sizeof(int) * (size_t)K * (size_t)dim);
  or_alpha(dim, d, alpha);
  *K_out = K;
  return alpha;
}

/* Design matrix eta(Omega) written pixel-major: eta_out[j][k].
 * basis: 0 = Legendre, 1 = monomial. */
int or_features(const or_grid* g, int d, int basis, double* eta_out) {
  int K;
  int* alpha = make_alpha(g->dim, d, &K);
  if (!alpha) return -1;
  double x[OR_MAXDIM];
  for (int64_t j = 0; j < g->P; ++j) {
    or_point(g, j, x);
    if (basis == 0) legendre_features(g->dim, d, alpha, K, x, eta_out + j * K);
    else monomial_features(g->dim, alpha, K, x, eta_out + j * K);
  }
  free(alpha);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel soft assignment (eq. p-e) with the usual max shift.            */
/* h[i] = theta_i . eta(x); l[i] = -h[i]/eps; returns log S - (-max) etc.   */
/* Fills p[i] = exp(l_i - m) / sum_j exp(l_j - m) and returns              */
/* LSE = m + log(sum_j exp(l_j - m)) = log S_theta^eps(x).                  */
/* ------------------------------------------------------------------------ */
static void logits_at(int N, int K, const double* theta, const double* eta,
                      double eps, double* l) {
  for (int i = 0; i < N; ++i) {
    double h = 0.0;
    for (int k = 0; k < K; ++k) h += theta[i * K + k] * eta[k];
    l[i] = -h / eps;
  }
}

static double softmax_at(int N, const double* l, double* p) {
  double m = l[0];
  for (int i = 1; i < N; ++i)
    if (l[i] > m) m = l[i];
  double S = 0.0;
  for (int i = 0; i < N; ++i) S += exp(l[i] - m);
  if (p)
    for (int i = 0; i < N; ++i) p[i] = exp(l[i] - m) / S;
  return m + log(S);
}

/* ------------------------------------------------------------------------ */
/* Objective (eqs. log-res-2 / Phi) and gradient (eq. grad).                */
/*   Phi = (1/|Omega|) sum_x [ l_{G(x)}(x) - log S(x) ]                     */
/*   grad_i = -(1/(eps |Omega|)) sum_x (delta_{i G(x)} - p_i(x)) eta(x)     */
/* basis: 0 = Legendre, 1 = monomial.  grad may be NULL.                    */
/* Returns 0 on success, -1 on invalid arguments or labels.                 */
/* ------------------------------------------------------------------------ */
int or_objective_grad(const or_grid* g, const int32_t* labels, int N, int d,
                      int basis, double eps, const double* theta,
                      double* phi_out, double* grad) {
  int K;
  int* alpha = make_alpha(g->dim, d, &K);
  if (!alpha || N < 2 || !(eps > 0.0)) { free(alpha); return -1; }
  double* eta = (double*)malloc(sizeof(double) * K);
  double* l = (double*)malloc(sizeof(double) * N);
  double* p = (double*)malloc(sizeof(double) * N);
  or_acc* gacc = NULL;
  if (grad) gacc = (or_acc*)calloc((size_t)N * K, sizeof(or_acc));
  or_acc phi = {0.0, 0.0};
  double x[OR_MAXDIM];
  int bad = 0;
  for (int64_t j = 0; j < g->P; ++j) {
    int G = labels[j];
    if (G < 0 || G >= N) { bad = 1; break; }
    or_point(g, j, x);
    if (basis == 0) legendre_features(g->dim, d, alpha, K, x, eta);
    else monomial_features(g->dim, alpha, K, x, eta);
    logits_at(N, K, theta, eta, eps, l);
    double lse = softmax_at(N, l, grad ? p : NULL);
    acc_add(&phi, l[G] - lse);
    if (grad) {
      for (int i = 0; i < N; ++i) {
        double c = (i == G ? 1.0 : 0.0) - p[i];
        for (int k = 0; k < K; ++k) acc_add(&gacc[(size_t)i * K + k], c * eta[k]);
      }
    }
  }
  if (!bad) {
    *phi_out = acc_val(&phi) / (double)g->P;
    if (grad) {
      double scale = -1.0 / (eps * (double)g->P);
      for (size_t q = 0; q < (size_t)N * K; ++q) grad[q] = scale * acc_val(&gacc[q]);
    }
  }
  free(alpha); free(eta); free(l); free(p); free(gacc);
  return bad ? -1 : 0;
}

/* Per-pixel log-probability r_x = l_{G(x)} - log S(x) and log S(x), for
 * checking single pixels of very large problems. */
int or_pixel_terms(const or_grid* g, const int32_t* labels, int N, int d,
                   double eps, const double* theta, int64_t n_idx,
                   const int64_t* idx, double* r_out, double* lse_out) {
  int K;
  int* alpha = make_alpha(g->dim, d, &K);
  if (!alpha || N < 2 || !(eps > 0.0)) { free(alpha); return -1; }
  double* eta = (double*)malloc(sizeof(double) * K);
  double* l = (double*)malloc(sizeof(double) * N);
  double x[OR_MAXDIM];
  for (int64_t q = 0; q < n_idx; ++q) {
    int64_t j = idx[q];
    or_point(g, j, x);
    legendre_features(g->dim, d, alpha, K, x, eta);
    logits_at(N, K, theta, eta, eps, l);
    double lse = softmax_at(N, l, NULL);
    if (lse_out) lse_out[q] = lse;
    if (r_out) r_out[q] = l[labels[j]] - lse;
  }
  free(alpha); free(eta); free(l);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Hessian-vector product from eq. (hess):                                  */
/*  (Hv)_i = -(1/(eps^2 |Omega|)) sum_x p_i (u_i - sum_k p_k u_k) eta(x),   */
/*  u_i = v_i . eta(x).                                                     */
/* ------------------------------------------------------------------------ */
int or_hvp(const or_grid* g, const int32_t* labels, int N, int d, double eps,
           const double* theta, const double* v, double* hv) {
  int K;
  int* alpha = make_alpha(g->dim, d, &K);
  if (!alpha || N < 2 || !(eps > 0.0)) { free(alpha); return -1; }
  double* eta = (double*)malloc(sizeof(double) * K);
  double* l = (double*)malloc(sizeof(double) * N);
  double* p = (double*)malloc(sizeof(double) * N);
  double* u = (double*)malloc(sizeof(double) * N);
  or_acc* acc = (or_acc*)calloc((size_t)N * K, sizeof(or_acc));
  double x[OR_MAXDIM];
  for (int64_t j = 0; j < g->P; ++j) {
    or_point(g, j, x);
    legendre_features(g->dim, d, alpha, K, x, eta);
    logits_at(N, K, theta, eta, eps, l);
    softmax_at(N, l, p);
    double ubar = 0.0;
    for (int i = 0; i < N; ++i) {
      double ui = 0.0;
      for (int k = 0; k < K; ++k) ui += v[i * K + k] * eta[k];
      u[i] = ui;
      ubar += p[i] * ui;
    }
    for (int i = 0; i < N; ++i) {
      double c = p[i] * (u[i] - ubar);
      for (int k = 0; k < K; ++k) acc_add(&acc[(size_t)i * K + k], c * eta[k]);
    }
  }
  double scale = -1.0 / (eps * eps * (double)g->P);
  for (size_t q = 0; q < (size_t)N * K; ++q) hv[q] = scale * acc_val(&acc[q]);
  (void)labels;
  free(alpha); free(eta); free(l); free(p); free(u); free(acc);
  return 0;
}

/* Dense Hessian, eq. (hess), for tiny problems: H[(i,a)][(k,b)]. */
int or_hessian(const or_grid* g, int N, int d, double eps, const double* theta,
               double* H) {
  int K;
  int* alpha = make_alpha(g->dim, d, &K);
  if (!alpha || N < 2 || !(eps > 0.0)) { free(alpha); return -1; }
  int n = N * K;
  double* eta = (double*)malloc(sizeof(double) * K);
  double* l = (double*)malloc(sizeof(double) * N);
  double* p = (double*)malloc(sizeof(double) * N);
  or_acc* acc = (or_acc*)calloc((size_t)n * n, sizeof(or_acc));
  double x[OR_MAXDIM];
  for (int64_t j = 0; j < g->P; ++j) {
    or_point(g, j, x);
    legendre_features(g->dim, d, alpha, K, x, eta);
    logits_at(N, K, theta, eta, eps, l);
    softmax_at(N, l, p);
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < N; ++k) {
        double w = p[i] * ((i == k ? 1.0 : 0.0) - p[k]);
        for (int a = 0; a < K; ++a)
          for (int b = 0; b < K; ++b)
            acc_add(&acc[(size_t)(i * K + a) * n + (k * K + b)], w * eta[a] * eta[b]);
      }
  }
  double scale = -1.0 / (eps * eps * (double)g->P);
  for (size_t q = 0; q < (size_t)n * n; ++q) H[q] = scale * acc_val(&acc[q]);
  free(alpha); free(eta); free(l); free(p); free(acc);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Arg-min assignment F_theta (Sec. 2.1, eq. Li_def): the smallest index    */
/* attaining the minimum of h_i(x) = theta_i . eta(x).  gap_out (optional)  */
/* receives the second-smallest minus the smallest h over all grains.       */
/* ------------------------------------------------------------------------ */
int or_assign(const or_grid* g, int N, int d, int basis, const double* theta,
              int32_t* labels_out, double* gap_out) {
  int K;
  int* alpha = make_alpha(g->dim, d, &K);
  if (!alpha || N < 1) { free(alpha); return -1; }
  double* eta = (double*)malloc(sizeof(double) * K);
  double* h = (double*)malloc(sizeof(double) * N);
  double x[OR_MAXDIM];
  for (int64_t j = 0; j < g->P; ++j) {
    or_point(g, j, x);
    if (basis == 0) legendre_features(g->dim, d, alpha, K, x, eta);
    else monomial_features(g->dim, alpha, K, x, eta);
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += theta[i * K + k] * eta[k];
      h[i] = s;
    }
    int best = 0;
    for (int i = 1; i < N; ++i)
      if (h[i] < h[best]) best = i;
    labels_out[j] = best;
    if (gap_out) {
      double second = INFINITY;
      for (int i = 0; i < N; ++i)
        if (i != best && h[i] < second) second = h[i];
      gap_out[j] = second - h[best];
    }
  }
  free(alpha); free(eta); free(h);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Grain moments: counts |G_i| and sum_{x in G_i} psi_alpha(x) (Legendre,   */
/* degree dm), used by the moment heuristic (Sec. 5.5.2) and as learned-    */
/* warm-start inputs.                                                       */
/* ------------------------------------------------------------------------ */
int or_grain_moments(const or_grid* g, const int32_t* labels, int N, int dm,
                     double* mom, int64_t* counts) {
  int K;
  int* alpha = make_alpha(g->dim, dm, &K);
  if (!alpha || N < 1) { free(alpha); return -1; }
  double* eta = (double*)malloc(sizeof(double) * K);
  or_acc* acc = (or_acc*)calloc((size_t)N * K, sizeof(or_acc));
  for (int i = 0; i < N; ++i) counts[i] = 0;
  double x[OR_MAXDIM];
  int bad = 0;
  for (int64_t j = 0; j < g->P; ++j) {
    int G = labels[j];
    if (G < 0 || G >= N) { bad = 1; break; }
    or_point(g, j, x);
    legendre_features(g->dim, dm, alpha, K, x, eta);
    counts[G] += 1;
    for (int k = 0; k < K; ++k) acc_add(&acc[(size_t)G * K + k], eta[k]);
  }
  for (size_t q = 0; q < (size_t)N * K; ++q) mom[q] = acc_val(&acc[q]);
  free(alpha); free(eta); free(acc);
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Basis change (Remark 3.1): monomial -> Legendre.                         */
/* 1-D: t^a = sum_m c[a][m] P_m(t), built from t P_m = ((m+1) P_{m+1} +     */
/* m P_{m-1}) / (2m+1), which is the Legendre recurrence solved for t P_m.  */
/* Tensorised: x^alpha = prod_a sum_m c[alpha_a][m] P_m(x_a), so            */
/* theta_L[beta] = sum_alpha theta_mono[alpha] prod_a c[alpha_a][beta_a].   */
/* T is written [K][K] with theta_L = T theta_mono (row beta, col alpha).   */
/* ------------------------------------------------------------------------ */
static void power_to_legendre_1d(int d, double c[OR_MAXDEG + 1][OR_MAXDEG + 2]) {
  for (int a = 0; a <= d; ++a)
    for (int m = 0; m <= d + 1; ++m) c[a][m] = 0.0;
  c[0][0] = 1.0;
  for (int a = 0; a < d; ++a) {
    /* t^{a+1} = t * sum_m c[a][m] P_m */
    for (int m = 0; m <= a; ++m) {
      double cm = c[a][m];
      if (cm == 0.0) continue;
      c[a + 1][m + 1] += cm * (m + 1.0) / (2.0 * m + 1.0);
      if (m >= 1) c[a + 1][m - 1] += cm * (double)m / (2.0 * m + 1.0);
    }
  }
}

int or_mono_to_legendre(int dim, int d, double* T) {
  if (d > OR_MAXDEG) return -1;
  int K;
  int* alpha = make_alpha(dim, d, &K);
  if (!alpha) return -1;
  double c[OR_MAXDEG + 1][OR_MAXDEG + 2];
  power_to_legendre_1d(d, c);
  for (int b = 0; b < K; ++b)
    for (int a = 0; a < K; ++a) {
      double v = 1.0;
      for (int ax = 0; ax < dim; ++ax) {
        int ea = alpha[a * dim + ax], eb = alpha[b * dim + ax];
        v *= (eb <= ea) ? c[ea][eb] : 0.0;
      }
      T[b * K + a] = v;
    }
  free(alpha);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Physical parameters -> linear parameters (Sec. 2.3).                     */
/* An (anisotropic) power diagram cost |x - y_i|^2_{A_i} - w_i expands to   */
/*   x.A x - 2 (A y).x + (y.A y - w):                                       */
/* monomial coefficients x_a^2 -> A_aa, x_a x_b (a<b) -> 2 A_ab,            */
/* x_a -> -2 (A y)_a, 1 -> y.A y - w.  With A = NULL (power diagram) the    */
/* quadratic part |x|^2 is the same for every grain and is dropped: a       */
/* function added to every h_i changes neither F nor p nor Phi.             */
/* Output: Legendre coefficients theta[N][K_d] (higher degrees zero).       */
/* ------------------------------------------------------------------------ */
static int alpha_index(int dim, int d, const int* e) {
  int K = or_K(dim, d);
  int* alpha = (int*)malloc(sizeof(int) * K * dim);
  or_alpha(dim, d, alpha);
  int found = -1;
  for (int k = 0; k < K && found < 0; ++k) {
    int ok = 1;
    for (int a = 0; a < dim; ++a) ok &= (alpha[k * dim + a] == e[a]);
    if (ok) found = k;
  }
  free(alpha);
  return found;
}

int or_theta_from_apd(int dim, int d, int N, const double* y, const double* w,
                      const double* A, double* theta) {
  if ((A && d < 2) || d < 1 || (dim != 2 && dim != 3)) return -1;
  int K = or_K(dim, d);
  double* mono = (double*)calloc((size_t)K, sizeof(double));
  double* T = (double*)malloc(sizeof(double) * K * K);
  or_mono_to_legendre(dim, d, T);
  for (int i = 0; i < N; ++i) {
    const double* yi = y + i * dim;
    double Ai[9];
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b)
        Ai[a * dim + b] = A ? A[(size_t)i * dim * dim + a * dim + b] : (a == b ? 1.0 : 0.0);
    for (int k = 0; k < K; ++k) mono[k] = 0.0;
    int e[3];
    /* quadratic part (only with an explicit A) */
    if (A) {
      for (int a = 0; a < dim; ++a)
        for (int b = a; b < dim; ++b) {
          for (int q = 0; q < dim; ++q) e[q] = 0;
          e[a] += 1; e[b] += 1;
          mono[alpha_index(dim, d, e)] = (a == b) ? Ai[a * dim + a] : 2.0 * Ai[a * dim + b];
        }
    }
    /* linear part: -2 (A y) */
    double yAy = 0.0;
    for (int a = 0; a < dim; ++a) {
      double Ay = 0.0;
      for (int b = 0; b < dim; ++b) Ay += Ai[a * dim + b] * yi[b];
      for (int q = 0; q < dim; ++q) e[q] = 0;
      e[a] = 1;
      mono[alpha_index(dim, d, e)] = -2.0 * Ay;
      yAy += yi[a] * Ay;
    }
    for (int q = 0; q < dim; ++q) e[q] = 0;
    mono[alpha_index(dim, d, e)] = yAy - w[i];
    for (int b = 0; b < K; ++b) {
      double s = 0.0;
      for (int a = 0; a < K; ++a) s += T[b * K + a] * mono[a];
      theta[(size_t)i * K + b] = s;
    }
  }
  free(mono); free(T);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Moment heuristic initialisation (Sec. 5.5.2, eqs. centroid-guess ..      */
/* w-guess):                                                                */
/*   y'_i = mean of the pixels of G_i;                                      */
/*   B'_i = (1/|G_i|) sum (x - y'_i)(x - y'_i)^T;                           */
/*   A'_i = B'_i^{-1} if invertible (else the identity);                    */
/*   w'_i = sqrt(det A'_i) |G_i| / (|Omega| pi)      (2-D, as printed)      */
/*        = sqrt(det A'_i) |G_i| / (|Omega| 4 pi/3)  (3-D ellipsoid reading)*/
/* power diagrams (anisotropic = 0) use A'_i = Id.  The result is converted */
/* to Legendre coefficients of degree d, higher-degree terms zero.          */
/* Empty grains get y' = 0, w' = 0, A' = Id.                                */
/* ------------------------------------------------------------------------ */
static double det_sym(int dim, const double* B) {
  if (dim == 2) return B[0] * B[3] - B[1] * B[2];
  return B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
         B[2] * (B[3] * B[7] - B[4] * B[6]);
}
static void inv_sym(int dim, const double* B, double det, double* Ainv) {
  if (dim == 2) {
    Ainv[0] = B[3] / det; Ainv[1] = -B[1] / det;
    Ainv[2] = -B[2] / det; Ainv[3] = B[0] / det;
    return;
  }
  Ainv[0] = (B[4] * B[8] - B[5] * B[7]) / det;
  Ainv[1] = (B[2] * B[7] - B[1] * B[8]) / det;
  Ainv[2] = (B[1] * B[5] - B[2] * B[4]) / det;
  Ainv[3] = (B[5] * B[6] - B[3] * B[8]) / det;
  Ainv[4] = (B[0] * B[8] - B[2] * B[6]) / det;
  Ainv[5] = (B[2] * B[3] - B[0] * B[5]) / det;
  Ainv[6] = (B[3] * B[7] - B[4] * B[6]) / det;
  Ainv[7] = (B[1] * B[6] - B[0] * B[7]) / det;
  Ainv[8] = (B[0] * B[4] - B[1] * B[3]) / det;
}

int or_heuristic_params(const or_grid* g, const int32_t* labels, int N,
                        int anisotropic, double* y, double* w, double* A) {
  int dim = g->dim;
  int64_t* cnt = (int64_t*)calloc((size_t)N, sizeof(int64_t));
  or_acc* sx = (or_acc*)calloc((size_t)N * dim, sizeof(or_acc));
  or_acc* sxx = (or_acc*)calloc((size_t)N * dim * dim, sizeof(or_acc));
  double x[OR_MAXDIM];
  for (int64_t j = 0; j < g->P; ++j) {
    int G = labels[j];
    if (G < 0 || G >= N) { free(cnt); free(sx); free(sxx); return -1; }
    or_point(g, j, x);
    cnt[G] += 1;
    for (int a = 0; a < dim; ++a) acc_add(&sx[G * dim + a], x[a]);
  }
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < dim; ++a)
      y[i * dim + a] = cnt[i] ? acc_val(&sx[i * dim + a]) / (double)cnt[i] : 0.0;
  for (int64_t j = 0; j < g->P; ++j) {
    int G = labels[j];
    or_point(g, j, x);
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b)
        acc_add(&sxx[(size_t)G * dim * dim + a * dim + b],
                (x[a] - y[G * dim + a]) * (x[b] - y[G * dim + b]));
  }
  const double vol = (dim == 2) ? M_PI : 4.0 * M_PI / 3.0;
  for (int i = 0; i < N; ++i) {
    double B[9], Ai[9];
    for (int q = 0; q < dim * dim; ++q)
      B[q] = cnt[i] ? acc_val(&sxx[(size_t)i * dim * dim + q]) / (double)cnt[i] : 0.0;
    double det = det_sym(dim, B);
    int use_id = !anisotropic || cnt[i] == 0 || !(det > 0.0) || !isfinite(det);
    if (use_id) {
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) Ai[a * dim + b] = (a == b) ? 1.0 : 0.0;
    } else {
      inv_sym(dim, B, det, Ai);
    }
    double detA = det_sym(dim, Ai);
    w[i] = sqrt(detA) * (double)cnt[i] / ((double)g->P * vol);
    if (A)
      for (int q = 0; q < dim * dim; ++q) A[(size_t)i * dim * dim + q] = Ai[q];
  }
  free(cnt); free(sx); free(sxx);
  return 0;
}

int or_heuristic_theta(const or_grid* g, const int32_t* labels, int N, int d,
                       double* theta) {
  int dim = g->dim;
  int anis = d >= 2;
  double* y = (double*)malloc(sizeof(double) * N * dim);
  double* w = (double*)malloc(sizeof(double) * N);
  double* A = (double*)malloc(sizeof(double) * N * dim * dim);
  int rc = or_heuristic_params(g, labels, N, anis, y, w, A);
  if (rc == 0) rc = or_theta_from_apd(dim, d, N, y, w, anis ? A : NULL, theta);
  free(y); free(w); free(A);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* The ascent scheme (Sec. 5.2): maximise Phi over the gauge-fixed          */
/* variables theta_0..theta_{N-2} (theta_{N-1} = 0, Remark 4.3) by L-BFGS   */
/* [Liu & Nocedal 1989] on f = -Phi.  The paper fixes neither the memory,   */
/* the line search nor the tolerances; this oracle uses: memory m; a        */
/* strong-Wolfe line search (c1 = 1e-4, c2 = 0.9) by bracketing and         */
/* zooming with safeguarded cubic interpolation (Nocedal & Wright, Alg.     */
/* 3.5/3.6); initial trial step 1, except 1/||g||_2 on the first iteration; */
/* the standard initial inverse-Hessian scaling gamma = s.y / y.y.          */
/* ------------------------------------------------------------------------ */
typedef struct {
  const or_grid* g;
  const int32_t* labels;
  int N, d, K;
  double eps;
  double* theta;  /* [N][K], last block kept 0 */
  double* gfull;  /* [N][K] */
  int64_t evals;
} or_fitctx;

/* f(x) = -Phi(theta(x)), grad f = -grad Phi restricted to the free blocks. */
static int fit_eval(or_fitctx* c, const double* xv, double* f, double* gf) {
  int n = (c->N - 1) * c->K;
  memcpy(c->theta, xv, sizeof(double) * n);
  for (int k = 0; k < c->K; ++k) c->theta[n + k] = 0.0;
  double phi;
  int rc = or_objective_grad(c->g, c->labels, c->N, c->d, 0, c->eps, c->theta, &phi, c->gfull);
  if (rc) return rc;
  *f = -phi;
  for (int q = 0; q < n; ++q) gf[q] = -c->gfull[q];
  c->evals += 1;
  return 0;
}

static double dotv(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int q = 0; q < n; ++q) s += a[q] * b[q];
  return s;
}

/* Safeguarded cubic interpolation minimiser of a 1-D function given two
 * points with values and derivatives; falls back to bisection. */
static double cubic_min(double a, double fa, double da, double b, double fb,
                        double db) {
  double d1 = da + db - 3.0 * (fa - fb) / (a - b);
  double disc = d1 * d1 - da * db;
  double lo = a < b ? a : b, hi = a < b ? b : a;
  if (disc >= 0.0) {
    double d2 = sqrt(disc);
    if (b < a) d2 = -d2;
    double t = b - (b - a) * ((db + d2 - d1) / (db - da + 2.0 * d2));
    if (isfinite(t) && t >= lo && t <= hi) return t;
  }
  return 0.5 * (a + b);
}

typedef struct {
  double c1, c2;
  int max_ls;
} or_lsopts;

/* Strong-Wolfe line search along direction dv from xv (value f0, grad g0).
 * On return xn, fn, gn hold the accepted point; returns the step or 0 on
 * failure (then xn/fn/gn hold the best point with sufficient decrease or x). */
static double wolfe_search(or_fitctx* c, int n, const double* xv, double f0,
                           const double* g0, const double* dv, double a_init,
                           const or_lsopts* o, double* xn, double* fn,
                           double* gn) {
  double dphi0 = dotv(n, g0, dv);
  double a_prev = 0.0, f_prev = f0, dp_prev = dphi0;
  double a = a_init;
  double lo = 0, flo = 0, dlo = 0, hi = 0, fhi = 0, dhi = 0;
  int zoom = 0;
  int evals = 0;
  for (;;) {
    if (evals >= o->max_ls) goto fail;
    for (int q = 0; q < n; ++q) xn[q] = xv[q] + a * dv[q];
    if (fit_eval(c, xn, fn, gn)) goto fail;
    ++evals;
    double dp = dotv(n, gn, dv);
    if (!isfinite(*fn) || *fn > f0 + o->c1 * a * dphi0 || (evals > 1 && *fn >= f_prev)) {
      lo = a_prev; flo = f_prev; dlo = dp_prev;
      hi = a; fhi = *fn; dhi = dp;
      zoom = 1;
      break;
    }
    if (fabs(dp) <= -o->c2 * dphi0) return a;
    if (dp >= 0.0) {
      lo = a; flo = *fn; dlo = dp;
      hi = a_prev; fhi = f_prev; dhi = dp_prev;
      zoom = 1;
      break;
    }
    a_prev = a; f_prev = *fn; dp_prev = dp;
    a = 2.0 * a;
  }
  if (zoom) {
    for (;;) {
      if (evals >= o->max_ls) break;
      double width = fabs(hi - lo);
      double t = isfinite(fhi) ? cubic_min(lo, flo, dlo, hi, fhi, dhi) : 0.5 * (lo + hi);
      double lb = (lo < hi ? lo : hi) + 0.1 * width, ub = (lo < hi ? hi : lo) - 0.1 * width;
      if (t < lb || t > ub) t = 0.5 * (lo + hi);
      for (int q = 0; q < n; ++q) xn[q] = xv[q] + t * dv[q];
      if (fit_eval(c, xn, fn, gn)) break;
      ++evals;
      double dp = dotv(n, gn, dv);
      if (!isfinite(*fn) || *fn > f0 + o->c1 * t * dphi0 || *fn >= flo) {
        hi = t; fhi = *fn; dhi = dp;
      } else {
        if (fabs(dp) <= -o->c2 * dphi0) return t;
        if (dp * (hi - lo) >= 0.0) { hi = lo; fhi = flo; dhi = dlo; }
        lo = t; flo = *fn; dlo = dp;
      }
      if (fabs(hi - lo) * sqrt(dotv(n, dv, dv)) < 1e-16 * (1.0 + sqrt(dotv(n, xv, xv)))) break;
    }
    /* accept the best point with sufficient decrease, if any */
    if (lo > 0.0) {
      for (int q = 0; q < n; ++q) xn[q] = xv[q] + lo * dv[q];
      if (fit_eval(c, xn, fn, gn) == 0) return lo;
    }
  }
fail:
  memcpy(xn, xv, sizeof(double) * n);
  fit_eval(c, xn, fn, gn);
  return 0.0;
}

typedef struct {
  int iters;        /* completed iterations */
  int64_t evals;    /* objective+gradient evaluations */
  double phi;       /* final Phi */
  double gnorm;     /* final ||grad Phi||_2 over the free blocks */
  int status;       /* 0 budget reached, 1 gradient tolerance, 2 line-search failure */
} or_fitreport;

/* theta_io: [N][K] initial parameters in, fitted parameters out (gauge-fixed:
 * the last block is subtracted from every block first).  phi_trace (may be
 * NULL) receives Phi after each iteration (max_iter entries). */
int or_lbfgs_fit(const or_grid* g, const int32_t* labels, int N, int d,
                 double eps, double* theta_io, int max_iter, int m, double gtol,
                 double* phi_trace, or_fitreport* rep) {
  int K = or_K(g->dim, d);
  if (K <= 0 || N < 2 || m < 1) return -1;
  int n = (N - 1) * K;
  or_fitctx c = {g, labels, N, d, K, eps, NULL, NULL, 0};
  c.theta = (double*)malloc(sizeof(double) * N * K);
  c.gfull = (double*)malloc(sizeof(double) * N * K);
  double* xv = (double*)malloc(sizeof(double) * n);
  double* gv = (double*)malloc(sizeof(double) * n);
  double* xn = (double*)malloc(sizeof(double) * n);
  double* gn = (double*)malloc(sizeof(double) * n);
  double* dv = (double*)malloc(sizeof(double) * n);
  double* S = (double*)malloc(sizeof(double) * (size_t)m * n);
  double* Y = (double*)malloc(sizeof(double) * (size_t)m * n);
  double* rho = (double*)malloc(sizeof(double) * m);
  double* al = (double*)malloc(sizeof(double) * m);
  for (int i = 0; i < N - 1; ++i)
    for (int k = 0; k < K; ++k) xv[i * K + k] = theta_io[i * K + k] - theta_io[(N - 1) * K + k];
  double f;
  int rc = fit_eval(&c, xv, &f, gv);
  if (rc) goto done;
  or_lsopts lso = {1e-4, 0.9, 25};
  int hist = 0, head = 0, it = 0, status = 0;
  for (it = 0; it < max_iter; ++it) {
    double gn2 = sqrt(dotv(n, gv, gv));
    if (gn2 <= gtol) { status = 1; break; }
    /* two-loop recursion: dv = -H g */
    for (int q = 0; q < n; ++q) dv[q] = -gv[q];
    for (int h = 0; h < hist; ++h) {
      int s = (head - 1 - h + m) % m;
      al[s] = rho[s] * dotv(n, S + (size_t)s * n, dv);
      for (int q = 0; q < n; ++q) dv[q] -= al[s] * Y[(size_t)s * n + q];
    }
    if (hist > 0) {
      int s = (head - 1 + m) % m;
      double gamma = dotv(n, S + (size_t)s * n, Y + (size_t)s * n) /
                     dotv(n, Y + (size_t)s * n, Y + (size_t)s * n);
      for (int q = 0; q < n; ++q) dv[q] *= gamma;
    }
    for (int h = hist - 1; h >= 0; --h) {
      int s = (head - 1 - h + m) % m;
      double be = rho[s] * dotv(n, Y + (size_t)s * n, dv);
      for (int q = 0; q < n; ++q) dv[q] += (al[s] - be) * S[(size_t)s * n + q];
    }
    if (dotv(n, dv, gv) >= 0.0) { /* not a descent direction: restart */
      hist = 0; head = 0;
      for (int q = 0; q < n; ++q) dv[q] = -gv[q];
    }
    double a0 = (it == 0) ? 1.0 / gn2 : 1.0;
    double fn;
    double step = wolfe_search(&c, n, xv, f, gv, dv, a0, &lso, xn, &fn, gn);
    if (step == 0.0) { status = 2; break; }
    /* curvature pair */
    double* sn = S + (size_t)head * n;
    double* yn = Y + (size_t)head * n;
    for (int q = 0; q < n; ++q) { sn[q] = xn[q] - xv[q]; yn[q] = gn[q] - gv[q]; }
    double sy = dotv(n, sn, yn);
    if (sy > 1e-300) {
      rho[head] = 1.0 / sy;
      head = (head + 1) % m;
      if (hist < m) ++hist;
    }
    memcpy(xv, xn, sizeof(double) * n);
    memcpy(gv, gn, sizeof(double) * n);
    f = fn;
    if (phi_trace) phi_trace[it] = -f;
  }
  for (int i = 0; i < N - 1; ++i)
    for (int k = 0; k < K; ++k) theta_io[i * K + k] = xv[i * K + k];
  for (int k = 0; k < K; ++k) theta_io[(N - 1) * K + k] = 0.0;
  if (rep) {
    rep->iters = it;
    rep->evals = c.evals;
    rep->phi = -f;
    rep->gnorm = sqrt(dotv(n, gv, gv));
    rep->status = status;
  }
done:
  free(c.theta); free(c.gfull); free(xv); free(gv); free(xn); free(gn); free(dv);
  free(S); free(Y); free(rho); free(al);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Truncated Newton (Newton-CG) ascent using Hessian-vector products        */
/* (eq. hess).  Not in the paper (which uses L-BFGS); a textbook scheme:    */
/* solve (-H) s = grad Phi on the gauge-fixed subspace by conjugate          */
/* gradients to relative residual min(0.5, sqrt(||g||)), at most max_cg     */
/* steps, stop at non-positive curvature; then the same strong-Wolfe line   */
/* search with trial step 1.                                                */
/* ------------------------------------------------------------------------ */
static int fit_hvp(or_fitctx* c, const double* xv, const double* vfree, double* out) {
  int n = (c->N - 1) * c->K;
  double* v = (double*)calloc((size_t)c->N * c->K, sizeof(double));
  double* hv = (double*)malloc(sizeof(double) * c->N * c->K);
  memcpy(c->theta, xv, sizeof(double) * n);
  for (int k = 0; k < c->K; ++k) c->theta[n + k] = 0.0;
  memcpy(v, vfree, sizeof(double) * n);
  int rc = or_hvp(c->g, c->labels, c->N, c->d, c->eps, c->theta, v, hv);
  for (int q = 0; q < n; ++q) out[q] = -hv[q]; /* Hessian of f = -Phi */
  free(v); free(hv);
  return rc;
}

int or_newton_cg_fit(const or_grid* g, const int32_t* labels, int N, int d,
                     double eps, double* theta_io, int max_iter, int max_cg,
                     double gtol, double* phi_trace, or_fitreport* rep) {
  int K = or_K(g->dim, d);
  if (K <= 0 || N < 2) return -1;
  int n = (N - 1) * K;
  or_fitctx c = {g, labels, N, d, K, eps, NULL, NULL, 0};
  c.theta = (double*)malloc(sizeof(double) * N * K);
  c.gfull = (double*)malloc(sizeof(double) * N * K);
  double* xv = (double*)malloc(sizeof(double) * n);
  double* gv = (double*)malloc(sizeof(double) * n);
  double* xn = (double*)malloc(sizeof(double) * n);
  double* gn = (double*)malloc(sizeof(double) * n);
  double* sv = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* pv = (double*)malloc(sizeof(double) * n);
  double* hp = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < N - 1; ++i)
    for (int k = 0; k < K; ++k) xv[i * K + k] = theta_io[i * K + k] - theta_io[(N - 1) * K + k];
  double f;
  int rc = fit_eval(&c, xv, &f, gv);
  int it = 0, status = 0;
  or_lsopts lso = {1e-4, 0.9, 25};
  if (rc) goto done;
  for (it = 0; it < max_iter; ++it) {
    double gn2 = sqrt(dotv(n, gv, gv));
    if (gn2 <= gtol) { status = 1; break; }
    double tol = (gn2 < 0.25 ? sqrt(gn2) : 0.5) * gn2;
    /* CG on (H_f) s = -g_f, starting from s = 0 */
    for (int q = 0; q < n; ++q) { sv[q] = 0.0; r[q] = -gv[q]; pv[q] = r[q]; }
    double rr = dotv(n, r, r);
    for (int j = 0; j < max_cg; ++j) {
      if (fit_hvp(&c, xv, pv, hp)) { rc = -1; goto done; }
      double curv = dotv(n, pv, hp);
      if (curv <= 0.0) {
        if (j == 0) for (int q = 0; q < n; ++q) sv[q] = -gv[q];
        break;
      }
      double alpha = rr / curv;
      for (int q = 0; q < n; ++q) { sv[q] += alpha * pv[q]; r[q] -= alpha * hp[q]; }
      double rr_new = dotv(n, r, r);
      if (sqrt(rr_new) <= tol) break;
      double beta = rr_new / rr;
      for (int q = 0; q < n; ++q) pv[q] = r[q] + beta * pv[q];
      rr = rr_new;
    }
    if (dotv(n, sv, gv) >= 0.0)
      for (int q = 0; q < n; ++q) sv[q] = -gv[q];
    double fn;
    double step = wolfe_search(&c, n, xv, f, gv, sv, 1.0, &lso, xn, &fn, gn);
    if (step == 0.0) { status = 2; break; }
    memcpy(xv, xn, sizeof(double) * n);
    memcpy(gv, gn, sizeof(double) * n);
    f = fn;
    if (phi_trace) phi_trace[it] = -f;
  }
  for (int i = 0; i < N - 1; ++i)
    for (int k = 0; k < K; ++k) theta_io[i * K + k] = xv[i * K + k];
  for (int k = 0; k < K; ++k) theta_io[(N - 1) * K + k] = 0.0;
  if (rep) {
    rep->iters = it;
    rep->evals = c.evals;
    rep->phi = -f;
    rep->gnorm = sqrt(dotv(n, gv, gv));
    rep->status = status;
  }
done:
  free(c.theta); free(c.gfull); free(xv); free(gv); free(xn); free(gn);
  free(sv); free(r); free(pv); free(hp);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Linear parameters -> physical parameters (Sec. 2.3, eqs. pd-lr-to-phys   */
/* and apd-lr-to-phys; Sec. 5.5.3).  The Legendre coefficients of degree    */
/* d in {1, 2} are first written in monomials by solving T theta_L =        */
/* theta_mono (T of or_mono_to_legendre is triangular: a monomial only      */
/* involves Legendre products of lower or equal multi-index, so back        */
/* substitution in the order of A_d solves it).  Then                       */
/*   d = 1:  y = -theta_x / 2,  w = |theta_x|^2 / 4 - theta_1;              */
/*   d = 2:  A_aa = theta_{x_a^2},  A_ab = theta_{x_a x_b} / 2,             */
/*           after the common shift A_i + lambda Id (which changes no cell  */
/*           boundary: it adds lambda |x|^2 to every h_i, Lemma 4.2),       */
/*           y = -A^-1 theta_x / 2,  w = theta_x . A^-1 theta_x / 4 -       */
/*           theta_1,                                                       */
/* with lambda = max(0, margin - min_i lambda_min(A_i)) so that every      */
/* shifted A_i has eigenvalues >= margin > 0 (the paper asks for lambda >   */
/* -min_i lambda_min(A_i)).  Eigenvalues of the symmetric A_i by cyclic      */
/* Jacobi rotations (textbook).  Outputs y [N][dim], w [N], A [N][dim][dim] */
/* (d = 2 only) and lambda.                                                 */
/* ------------------------------------------------------------------------ */
static double sym_min_eig(int dim, const double* A) {
  double a[3][3];
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) a[r][c] = A[r * dim + c];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int r = 0; r < dim; ++r)
      for (int c = r + 1; c < dim; ++c) off += a[r][c] * a[r][c];
    if (off == 0.0) break;
    for (int p = 0; p < dim; ++p)
      for (int q = p + 1; q < dim; ++q) {
        if (a[p][q] == 0.0) continue;
        /* rotation that zeroes a[p][q] */
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < dim; ++k) {
          double akp = a[k][p], akq = a[k][q];
          a[k][p] = cs * akp - sn * akq;
          a[k][q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < dim; ++k) {
          double apk = a[p][k], aqk = a[q][k];
          a[p][k] = cs * apk - sn * aqk;
          a[q][k] = sn * apk + cs * aqk;
        }
      }
  }
  double m = a[0][0];
  for (int r = 1; r < dim; ++r) m = a[r][r] < m ? a[r][r] : m;
  return m;
}

/* solve M z = b for symmetric positive definite M (dim <= 3) by Gaussian
 * elimination without pivoting (M is positive definite here) */
static void spd_solve(int dim, const double* M, const double* b, double* z) {
  double a[3][4];
  for (int r = 0; r < dim; ++r) {
    for (int c = 0; c < dim; ++c) a[r][c] = M[r * dim + c];
    a[r][dim] = b[r];
  }
  for (int k = 0; k < dim; ++k)
    for (int r = k + 1; r < dim; ++r) {
      double f = a[r][k] / a[k][k];
      for (int c = k; c <= dim; ++c) a[r][c] -= f * a[k][c];
    }
  for (int r = dim - 1; r >= 0; --r) {
    double v = a[r][dim];
    for (int c = r + 1; c < dim; ++c) v -= a[r][c] * z[c];
    z[r] = v / a[r][r];
  }
}

int or_theta_to_apd(int dim, int d, int N, const double* theta, double margin,
                    double* y, double* w, double* A, double* lambda_out) {
  if ((dim != 2 && dim != 3) || (d != 1 && d != 2) || N < 1 || !(margin > 0.0)) return -1;
  int K = or_K(dim, d);
  double* T = (double*)malloc(sizeof(double) * K * K);
  double* mono = (double*)malloc(sizeof(double) * N * K);
  or_mono_to_legendre(dim, d, T);
  /* back substitution: T is upper triangular in the order of A_d */
  for (int i = 0; i < N; ++i) {
    const double* tl = theta + (size_t)i * K;
    double* tm = mono + (size_t)i * K;
    for (int b = K - 1; b >= 0; --b) {
      double v = tl[b];
      for (int a = b + 1; a < K; ++a) v -= T[b * K + a] * tm[a];
      tm[b] = v / T[b * K + b];
    }
  }
  int e[3];
  double lambda = 0.0;
  if (d == 2) {
    /* A_i from the quadratic coefficients, then the common shift */
    double min_eig = INFINITY;
    for (int i = 0; i < N; ++i) {
      double* Ai = A + (size_t)i * dim * dim;
      for (int a = 0; a < dim; ++a)
        for (int b = a; b < dim; ++b) {
          for (int q = 0; q < dim; ++q) e[q] = 0;
          e[a] += 1; e[b] += 1;
          double c = mono[(size_t)i * K + alpha_index(dim, d, e)];
          Ai[a * dim + b] = Ai[b * dim + a] = (a == b) ? c : 0.5 * c;
        }
      double m = sym_min_eig(dim, Ai);
      if (m < min_eig) min_eig = m;
    }
    lambda = margin - min_eig > 0.0 ? margin - min_eig : 0.0;
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < dim; ++a) A[(size_t)i * dim * dim + a * dim + a] += lambda;
  }
  for (int i = 0; i < N; ++i) {
    double bx[3], z[3];
    for (int a = 0; a < dim; ++a) {
      for (int q = 0; q < dim; ++q) e[q] = 0;
      e[a] = 1;
      bx[a] = mono[(size_t)i * K + alpha_index(dim, d, e)];
    }
    for (int q = 0; q < dim; ++q) e[q] = 0;
    double t1 = mono[(size_t)i * K + alpha_index(dim, d, e)];
    if (d == 1) {
      /* eq. pd-lr-to-phys */
      double s = 0.0;
      for (int a = 0; a < dim; ++a) {
        y[(size_t)i * dim + a] = -0.5 * bx[a];
        s += 0.25 * bx[a] * bx[a];
      }
      w[i] = s - t1;
    } else {
      /* eq. apd-lr-to-phys: z = A^-1 b, y = -z/2, w = b.z/4 - theta_1 */
      spd_solve(dim, A + (size_t)i * dim * dim, bx, z);
      double s = 0.0;
      for (int a = 0; a < dim; ++a) {
        y[(size_t)i * dim + a] = -0.5 * z[a];
        s += 0.25 * bx[a] * z[a];
      }
      w[i] = s - t1;
    }
  }
  if (lambda_out) *lambda_out = lambda;
  free(T); free(mono);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Annealing of eps with stopping aligned with Err^G (Sec. 5.2 and Sec.     */
/* 5.5.4 leave both to future work; this is the build's reading).           */
/* Stages k = 0, 1, ...: eps_k = max(eps_min, eps0 factor^k); stage k runs  */
/* the ascent scheme (or_lbfgs_fit) at eps_k from the parameters the        */
/* previous stage ended with -- the same diagram F_theta, made sharper by   */
/* the smaller eps (Lemma 4.1: Phi_eps(theta) = Phi_1(theta / eps)) --, for  */
/* stage_iter iterations, or final_iter at eps_min.  After a stage above    */
/* eps_min and with err_stop, the schedule stops when the hard assignment   */
/* reconstructs G: Phi > -log 2 / |Omega| certifies Err^G = 0 (Cor. 4.10), */
/* else Err^G is computed by the arg-min assignment (Sec. 4).  Per stage:   */
/* eps, Phi, Err^G (-1 where the certificate made it unnecessary) and the   */
/* iterations; returns the number of stages (<= max_stages) or -1.          */
/* ------------------------------------------------------------------------ */
int or_anneal_fit(const or_grid* g, const int32_t* labels, int N, int d,
                  double eps0, double factor, double eps_min, int stage_iter,
                  int final_iter, int m, int err_stop, double* theta_io,
                  int max_stages, double* st_eps, double* st_phi,
                  double* st_err, int* st_iters) {
  if (!(eps_min > 0.0) || !(factor > 0.0 && factor < 1.0) || max_stages < 1) return -1;
  int K = or_K(g->dim, d);
  int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->P > 0 ? g->P : 1));
  double eps = eps0 > eps_min ? eps0 : eps_min;
  int k = 0;
  for (; k < max_stages; ++k) {
    int last = eps <= eps_min;
    if (last) eps = eps_min;
    or_fitreport rep;
    if (or_lbfgs_fit(g, labels, N, d, eps, theta_io, last ? final_iter : stage_iter, m, 0.0, NULL, &rep)) {
      free(lab);
      return -1;
    }
    st_eps[k] = eps;
    st_phi[k] = rep.phi;
    st_err[k] = -1.0;
    st_iters[k] = rep.iters;
    if (last) { ++k; break; }
    if (err_stop) {
      if (rep.phi > -log(2.0) / (double)g->P) { ++k; break; }  /* Cor. 4.10 */
      or_assign(g, N, d, 0, theta_io, lab, NULL);
      int64_t miss = 0;
      for (int64_t j = 0; j < g->P; ++j) miss += lab[j] != labels[j];
      st_err[k] = (double)miss / (double)g->P;
      if (miss == 0) { ++k; break; }
    }
    eps *= factor;
  }
  free(lab);
  (void)K;
  return k;
}


/* ------------------------------------------------------------------------ */
/* Learned warm start: a multilayer perceptron with two ReLU hidden layers, */
/*   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,           */
/* and the mean squared error L = (1/(B n_out)) sum (y - t)^2 with its      */
/* gradients by the chain rule (textbook back-propagation).  Weights are    */
/* row-major [n_out_of_layer][n_in_of_layer].  Not from the paper: this     */
/* restates the network that maps grain moments to warm-start parameters.   */
/* ------------------------------------------------------------------------ */
static void dense(int B, int n_in, int n_out, const double* X, const double* W,
                  const double* b, int relu, double* Y) {
  for (int r = 0; r < B; ++r)
    for (int o = 0; o < n_out; ++o) {
      double s = b[o];
      for (int i = 0; i < n_in; ++i) s += W[(size_t)o * n_in + i] * X[(size_t)r * n_in + i];
      Y[(size_t)r * n_out + o] = (relu && s < 0.0) ? 0.0 : s;
    }
}

int or_mlp_forward(int B, int n_in, int n_h1, int n_h2, int n_out, const double* X,
                   const double* W1, const double* b1, const double* W2,
                   const double* b2, const double* W3, const double* b3, double* Y) {
  double* h1 = (double*)malloc(sizeof(double) * (size_t)B * n_h1);
  double* h2 = (double*)malloc(sizeof(double) * (size_t)B * n_h2);
  dense(B, n_in, n_h1, X, W1, b1, 1, h1);
  dense(B, n_h1, n_h2, h1, W2, b2, 1, h2);
  dense(B, n_h2, n_out, h2, W3, b3, 0, Y);
  free(h1); free(h2);
  return 0;
}

double or_mlp_loss_grad(int B, int n_in, int n_h1, int n_h2, int n_out, const double* X,
                        const double* T, const double* W1, const double* b1,
                        const double* W2, const double* b2, const double* W3,
                        const double* b3, double* gW1, double* gb1, double* gW2,
                        double* gb2, double* gW3, double* gb3) {
  double* h1 = (double*)malloc(sizeof(double) * (size_t)B * n_h1);
  double* h2 = (double*)malloc(sizeof(double) * (size_t)B * n_h2);
  double* y = (double*)malloc(sizeof(double) * (size_t)B * n_out);
  double* dy = (double*)malloc(sizeof(double) * (size_t)B * n_out);
  double* d2 = (double*)malloc(sizeof(double) * (size_t)B * n_h2);
  double* d1 = (double*)malloc(sizeof(double) * (size_t)B * n_h1);
  dense(B, n_in, n_h1, X, W1, b1, 1, h1);
  dense(B, n_h1, n_h2, h1, W2, b2, 1, h2);
  dense(B, n_h2, n_out, h2, W3, b3, 0, y);
  const double scale = 1.0 / ((double)B * n_out);
  double loss = 0.0;
  for (size_t q = 0; q < (size_t)B * n_out; ++q) {
    const double e = y[q] - T[q];
    loss += e * e;
    dy[q] = 2.0 * e * scale;            /* dL/dy */
  }
  loss *= scale;
  /* layer 3 */
  for (int o = 0; o < n_out; ++o) {
    double sb = 0.0;
    for (int r = 0; r < B; ++r) sb += dy[(size_t)r * n_out + o];
    gb3[o] = sb;
    for (int i = 0; i < n_h2; ++i) {
      double s = 0.0;
      for (int r = 0; r < B; ++r) s += dy[(size_t)r * n_out + o] * h2[(size_t)r * n_h2 + i];
      gW3[(size_t)o * n_h2 + i] = s;
    }
  }
  for (int r = 0; r < B; ++r)
    for (int i = 0; i < n_h2; ++i) {
      double s = 0.0;
      for (int o = 0; o < n_out; ++o) s += W3[(size_t)o * n_h2 + i] * dy[(size_t)r * n_out + o];
      d2[(size_t)r * n_h2 + i] = h2[(size_t)r * n_h2 + i] > 0.0 ? s : 0.0;   /* relu' */
    }
  /* layer 2 */
  for (int o = 0; o < n_h2; ++o) {
    double sb = 0.0;
    for (int r = 0; r < B; ++r) sb += d2[(size_t)r * n_h2 + o];
    gb2[o] = sb;
    for (int i = 0; i < n_h1; ++i) {
      double s = 0.0;
      for (int r = 0; r < B; ++r) s += d2[(size_t)r * n_h2 + o] * h1[(size_t)r * n_h1 + i];
      gW2[(size_t)o * n_h1 + i] = s;
    }
  }
  for (int r = 0; r < B; ++r)
    for (int i = 0; i < n_h1; ++i) {
      double s = 0.0;
      for (int o = 0; o < n_h2; ++o) s += W2[(size_t)o * n_h1 + i] * d2[(size_t)r * n_h2 + o];
      d1[(size_t)r * n_h1 + i] = h1[(size_t)r * n_h1 + i] > 0.0 ? s : 0.0;
    }
  /* layer 1 */
  for (int o = 0; o < n_h1; ++o) {
    double sb = 0.0;
    for (int r = 0; r < B; ++r) sb += d1[(size_t)r * n_h1 + o];
    gb1[o] = sb;
    for (int i = 0; i < n_in; ++i) {
      double s = 0.0;
      for (int r = 0; r < B; ++r) s += d1[(size_t)r * n_h1 + o] * X[(size_t)r * n_in + i];
      gW1[(size_t)o * n_in + i] = s;
    }
  }
  free(h1); free(h2); free(y); free(dy); free(d2); free(d1);
  return loss;
}

/* Warm-start inputs of every grain: its degree-dm Legendre moments divided  */
/* by |G_i| (the first, psi_0 = 1, is the constant 1), followed by the same  */
/* vectors of its n_nb nearest grains by centroid distance (centroid = the   */
/* normalised psi_(1,0), psi_(0,1) moments, i.e. the mean pixel), nearest    */
/* first, ties to the smaller index; with fewer than n_nb other grains the   */
/* list is padded with the grain's own vector.  feat: [N][(1+n_nb) Kdm].     */
int or_mlp_features(const or_grid* g, const int32_t* labels, int N, int dm,
                    int n_nb, double* feat) {
  int Kd = or_K(g->dim, dm);
  double* mom = (double*)malloc(sizeof(double) * (size_t)N * Kd);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * N);
  int rc = or_grain_moments(g, labels, N, dm, mom, cnt);
  if (rc) { free(mom); free(cnt); return rc; }
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < Kd; ++k) mom[(size_t)i * Kd + k] = cnt[i] ? mom[(size_t)i * Kd + k] / (double)cnt[i] : 0.0;
  int F = (1 + n_nb) * Kd;
  int* nb = (int*)malloc(sizeof(int) * n_nb);
  double* dist = (double*)malloc(sizeof(double) * n_nb);
  for (int i = 0; i < N; ++i) {
    int have = 0;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double s = 0.0;
      for (int a = 0; a < g->dim; ++a) {
        double dx = mom[(size_t)j * Kd + 1 + a] - mom[(size_t)i * Kd + 1 + a];
        s += dx * dx;
      }
      /* insertion into the sorted list of the n_nb nearest */
      int pos = have;
      while (pos > 0 && dist[pos - 1] > s) --pos;
      if (pos >= n_nb) continue;
      int last = have < n_nb ? have : n_nb - 1;
      for (int q = last; q > pos; --q) { dist[q] = dist[q - 1]; nb[q] = nb[q - 1]; }
      dist[pos] = s; nb[pos] = j;
      if (have < n_nb) ++have;
    }
    for (int k = 0; k < Kd; ++k) feat[(size_t)i * F + k] = mom[(size_t)i * Kd + k];
    for (int q = 0; q < n_nb; ++q) {
      int j = q < have ? nb[q] : i;
      for (int k = 0; k < Kd; ++k) feat[(size_t)i * F + (1 + q) * Kd + k] = mom[(size_t)j * Kd + k];
    }
  }
  free(mom); free(cnt); free(nb); free(dist);
  return 0;
}
