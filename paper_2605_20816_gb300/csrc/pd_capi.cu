// pd_capi.cu -- the extern "C" entry points of libpd (declared in pd.h):
// argument checking, dispatch to the kernels, and the host-side helpers
// (multi-index table, physical-parameter conversion, moment heuristic).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "pd.h"
#include "pd_internal.h"

namespace pd {

int device_sm_count() {
  static std::mutex mu;
  static std::vector<int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
  if (cache[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 148;
    // keep freed scratch in the pool instead of returning it to the driver
    // at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  return cache[dev];
}

int validate_grid(const pd_grid* grid, Geom* g) {
  if (!grid) return PD_EINVAL;
  if (grid->dim != 2 && grid->dim != 3) return PD_EINVAL;
  if (grid->P < 0) return PD_EINVAL;
  if (grid->P == 0) {  // the empty pixel set
    g->n0 = g->n1 = g->n2 = 1;
    g->coords = grid->coords;
    g->P = 0;
    return PD_OK;
  }
  if (!grid->coords) {
    int64_t prod = 1;
    for (int a = 0; a < grid->dim; ++a) {
      if (grid->n[a] <= 0) return PD_EINVAL;
      if (prod > INT64_MAX / grid->n[a]) return PD_EINVAL;
      prod *= grid->n[a];
    }
    if (prod != grid->P) return PD_EINVAL;
  }
  g->n0 = grid->coords ? 1 : grid->n[0];
  g->n1 = grid->coords ? 1 : grid->n[1];
  g->n2 = (grid->coords || grid->dim < 3) ? 1 : grid->n[2];
  g->coords = grid->coords;
  g->P = grid->P;
  return PD_OK;
}

bool degree_ok(int dim, int d) {
  if (d < 1) return false;
  return dim == 2 ? d <= PD_MAX_DEGREE_2D : (dim == 3 ? d <= PD_MAX_DEGREE_3D : false);
}

// Multi-index table of A_d in library order (ascending degree, then
// descending alpha_1, then descending alpha_2).
static std::vector<int> alpha_table(int dim, int d) {
  std::vector<int> a;
  for (int g = 0; g <= d; ++g) {
    for (int a1 = g; a1 >= 0; --a1) {
      if (dim == 2) {
        a.push_back(a1);
        a.push_back(g - a1);
      } else {
        for (int a2 = g - a1; a2 >= 0; --a2) {
          a.push_back(a1);
          a.push_back(a2);
          a.push_back(g - a1 - a2);
        }
      }
    }
  }
  return a;
}

// Coefficient of P_m in the Legendre expansion of t^n (textbook closed form):
// t^n = sum_{m <= n, m = n mod 2} (2m+1) n! / (2^{(n-m)/2} ((n-m)/2)! (n+m+1)!!) P_m.
static double power_in_legendre(int n, int m) {
  if (m > n || ((n - m) & 1)) return 0.0;
  const int h = (n - m) / 2;
  double v = 2.0 * m + 1.0;
  for (int q = 2; q <= n; ++q) v *= q;                 // n!
  for (int q = 0; q < h; ++q) v /= 2.0;                // 2^h
  for (int q = 2; q <= h; ++q) v /= q;                 // h!
  for (int q = n + m + 1; q > 1; q -= 2) v /= q;       // (n+m+1)!!
  return v;
}

int theta_from_apd_host(int dim, int d, int N, const double* y, const double* w, const double* A,
                        double* theta_out) {
  if ((dim != 2 && dim != 3) || d < 1 || N < 1 || !y || !w || !theta_out) return PD_EINVAL;
  if (A && d < 2) return PD_EINVAL;
  const int K = basis_K(dim, d);
  const std::vector<int> al = alpha_table(dim, d);
  auto index_of = [&](int e0, int e1, int e2) {
    for (int k = 0; k < K; ++k)
      if (al[k * dim] == e0 && al[k * dim + 1] == e1 && (dim == 2 || al[k * dim + 2] == e2)) return k;
    return -1;
  };
  std::vector<double> mono(K);
  for (int i = 0; i < N; ++i) {
    double Ai[9];
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b) Ai[a * dim + b] = A ? A[(size_t)i * dim * dim + a * dim + b] : (a == b);
    std::fill(mono.begin(), mono.end(), 0.0);
    // cost (x - y).A(x - y) - w = x.Ax - 2(Ay).x + y.Ay - w in monomials
    double Ay[3] = {0, 0, 0}, yAy = 0.0;
    for (int a = 0; a < dim; ++a) {
      for (int b = 0; b < dim; ++b) Ay[a] += Ai[a * dim + b] * y[(size_t)i * dim + b];
      yAy += y[(size_t)i * dim + a] * Ay[a];
    }
    mono[index_of(0, 0, 0)] = yAy - w[i];
    for (int a = 0; a < dim; ++a) {
      int e[3] = {0, 0, 0};
      e[a] = 1;
      mono[index_of(e[0], e[1], e[2])] = -2.0 * Ay[a];
    }
    if (A) {  // the identity's |x|^2 is common to all grains and is omitted
      for (int a = 0; a < dim; ++a)
        for (int b = a; b < dim; ++b) {
          int e[3] = {0, 0, 0};
          e[a] += 1;
          e[b] += 1;
          mono[index_of(e[0], e[1], e[2])] = (a == b) ? Ai[a * dim + a] : 2.0 * Ai[a * dim + b];
        }
    }
    // to Legendre: x^alpha = prod_a sum_m c(alpha_a, m) P_m(x_a)
    for (int kb = 0; kb < K; ++kb) {
      double s = 0.0;
      for (int ka = 0; ka < K; ++ka) {
        if (mono[ka] == 0.0) continue;
        double c = 1.0;
        for (int ax = 0; ax < dim; ++ax) c *= power_in_legendre(al[ka * dim + ax], al[kb * dim + ax]);
        s += c * mono[ka];
      }
      theta_out[(size_t)i * K + kb] = s;
    }
  }
  return PD_OK;
}

}  // namespace pd

using namespace pd;

extern "C" {

int pd_K(int dim, int d) {
  if ((dim != 2 && dim != 3) || d < 0) return -1;
  return basis_K(dim, d);
}

int pd_alpha(int dim, int d, int* alpha_out) {
  if ((dim != 2 && dim != 3) || d < 0 || !alpha_out) return PD_EINVAL;
  const std::vector<int> a = alpha_table(dim, d);
  memcpy(alpha_out, a.data(), sizeof(int) * a.size());
  return basis_K(dim, d);
}

const char* pd_strerror(int code) {
  switch (code) {
    case PD_OK: return "success";
    case PD_EINVAL: return "invalid argument";
    case PD_ELABEL: return "label outside 0..N-1";
    case PD_ENAN: return "non-finite value";
    case PD_ENOMEM: return "scratch allocation failed";
    case PD_ECUDA: return "CUDA runtime error";
    case PD_ETIMEOUT: return "bounded device wait timed out";
    case PD_ENOTSUP: return "unsupported combination";
    case PD_ESCRATCH: return "problem exceeds the fixed scratch of the no-allocation entry point";
    default: return "unknown status";
  }
}

int pd_features(const pd_grid* grid, int d, int prec, void* eta_out, void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (!degree_ok(grid->dim, d)) return d < 1 ? PD_EINVAL : PD_ENOTSUP;
  if (prec != PD_FP64 && prec != PD_FP32) return PD_EINVAL;
  if (g.P > 0 && !eta_out) return PD_EINVAL;
  device_sm_count();
  return features_simt(g, grid->dim, d, prec, eta_out, (cudaStream_t)stream);
}

static int check_eval(const pd_grid* grid, int N, const double* theta, const pd_eval_opts* opts, Geom* g) {
  int rc = validate_grid(grid, g);
  if (rc) return rc;
  if (!opts || !theta || N < 2) return PD_EINVAL;
  if (!(opts->eps > 0.0) || !isfinite(opts->eps)) return PD_EINVAL;
  if (opts->d < 1) return PD_EINVAL;
  if (!degree_ok(grid->dim, opts->d)) return PD_ENOTSUP;
  if (opts->prec < PD_FP64 || opts->prec > PD_BF16X3) return PD_EINVAL;
  if (g->P < 1) return PD_EINVAL;
  return PD_OK;
}

int pd_objective_grad(const pd_grid* grid, const int32_t* labels, int N, const double* theta,
                      const pd_eval_opts* opts, double* obj_out, double* grad_out, void* stream) {
  Geom g;
  int rc = check_eval(grid, N, theta, opts, &g);
  if (rc) return rc;
  if (!labels || (!obj_out && !grad_out)) return PD_EINVAL;
  device_sm_count();
  EvalCall c{g, grid->dim, opts->d, N, opts->prec, opts->eps, labels, theta, nullptr, obj_out, grad_out, nullptr};
  if (opts->prec == PD_BF16 || opts->prec == PD_BF16X3) return eval_tc(c, (cudaStream_t)stream);
  return eval_simt(c, (cudaStream_t)stream);
}

int pd_hvp(const pd_grid* grid, const int32_t* labels, int N, const double* theta, const double* v,
           const pd_eval_opts* opts, double* hv_out, void* stream) {
  Geom g;
  int rc = check_eval(grid, N, theta, opts, &g);
  if (rc) return rc;
  if (!v || !hv_out) return PD_EINVAL;
  device_sm_count();
  EvalCall c{g, grid->dim, opts->d, N, opts->prec, opts->eps, labels, theta, v, nullptr, nullptr, hv_out};
  if (opts->prec == PD_BF16 || opts->prec == PD_BF16X3) return eval_tc(c, (cudaStream_t)stream);
  return eval_simt(c, (cudaStream_t)stream);
}

int pd_assign(const pd_grid* grid, int N, int d, const double* theta, int32_t* labels_out, double* gap_out,
              const int32_t* ref_labels, int64_t* mismatch_out, void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (N < 1 || d < 1) return PD_EINVAL;
  if (!degree_ok(grid->dim, d)) return PD_ENOTSUP;
  if (g.P > 0 && (!theta || !labels_out)) return PD_EINVAL;
  if (g.P > 0 && (ref_labels == nullptr) != (mismatch_out == nullptr)) return PD_EINVAL;
  device_sm_count();
  return assign_simt(g, grid->dim, d, N, theta, labels_out, gap_out, ref_labels, mismatch_out,
                     (cudaStream_t)stream);
}

int pd_moments(const pd_grid* grid, const int32_t* labels, int N, int dm, double* mom_out, int64_t* counts_out,
               void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (N < 1 || dm < 1 || !mom_out || !counts_out || (g.P > 0 && !labels)) return PD_EINVAL;
  if (dm > 4) return PD_ENOTSUP;
  device_sm_count();
  return moments_simt(g, grid->dim, dm, labels, N, mom_out, counts_out, (cudaStream_t)stream);
}

int pd_check_labels(const pd_grid* grid, const int32_t* labels, int N, void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (N < 1 || (g.P > 0 && !labels)) return PD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc(st);
  int* bad = sc.get<int>(1);
  if (!sc.ok()) return PD_ENOMEM;
  rc = check_labels_simt(labels, g.P, N, bad, st);
  if (rc) return rc;
  int hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PD_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PD_ECUDA;
  return hbad ? PD_ELABEL : PD_OK;
}

int pd_theta_from_apd(int dim, int d, int N, const double* y, const double* w, const double* A,
                      double* theta_out) {
  if ((dim == 2 && d > 64) || (dim == 3 && d > 64)) return PD_ENOTSUP;
  return theta_from_apd_host(dim, d, N, y, w, A, theta_out);
}

// Coefficient of t^n in P_m(t) (textbook closed form):
// P_m(t) = 2^-m sum_{k <= m/2} (-1)^k C(m, k) C(2m - 2k, m) t^(m - 2k).
static double legendre_power_coeff(int m, int n) {
  if (n > m || ((m - n) & 1)) return 0.0;
  const int k = (m - n) / 2;
  auto binom = [](int a, int b) {
    double v = 1.0;
    for (int q = 1; q <= b; ++q) v = v * (double)(a - b + q) / (double)q;
    return v;
  };
  double v = binom(m, k) * binom(2 * m - 2 * k, m);
  for (int q = 0; q < m; ++q) v *= 0.5;
  return (k & 1) ? -v : v;
}

// Smallest eigenvalue of a symmetric 2x2 or 3x3 matrix (closed forms: the
// quadratic's smaller root; the trigonometric solution of the cubic).
static double sym_lambda_min(int dim, const double* A) {
  if (dim == 2) {
    const double m = 0.5 * (A[0] + A[3]), h = 0.5 * (A[0] - A[3]);
    return m - sqrt(h * h + A[1] * A[1]);
  }
  const double p1 = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
  const double q = (A[0] + A[4] + A[8]) / 3.0;
  const double p2 = (A[0] - q) * (A[0] - q) + (A[4] - q) * (A[4] - q) + (A[8] - q) * (A[8] - q) + 2.0 * p1;
  if (p2 == 0.0) return q;
  const double p = sqrt(p2 / 6.0);
  double B[9];
  for (int r = 0; r < 9; ++r) B[r] = (A[r] - (r % 4 == 0 ? q : 0.0)) / p;
  const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
  double r = 0.5 * detB;
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  return q + 2.0 * p * cos(phi + 2.0 * M_PI / 3.0);
}

int pd_theta_to_apd(int dim, int d, int N, const double* theta, double margin, double* y, double* w, double* A,
                    double* lambda_out) {
  if ((dim != 2 && dim != 3) || N < 1 || !theta || !y || !w) return PD_EINVAL;
  if (d != 1 && d != 2) return PD_ENOTSUP;
  if (d == 2 && (!A || !(margin > 0.0) || !isfinite(margin))) return PD_EINVAL;
  const int K = basis_K(dim, d);
  const std::vector<int> al = alpha_table(dim, d);
  auto index_of = [&](int e0, int e1, int e2) {
    for (int k = 0; k < K; ++k)
      if (al[k * dim] == e0 && al[k * dim + 1] == e1 && (dim == 2 || al[k * dim + 2] == e2)) return k;
    return -1;
  };
  // monomial coefficients: h = sum_a theta_a prod_ax P_{a_ax}(x_ax)
  //                           = sum_b (sum_a theta_a prod_ax c(a_ax, b_ax)) x^b
  std::vector<double> mono((size_t)N * K, 0.0);
  for (int i = 0; i < N; ++i)
    for (int b = 0; b < K; ++b) {
      double v = 0.0;
      for (int a = 0; a < K; ++a) {
        double c = 1.0;
        for (int ax = 0; ax < dim && c != 0.0; ++ax) c *= legendre_power_coeff(al[a * dim + ax], al[b * dim + ax]);
        v += c * theta[(size_t)i * K + a];
      }
      mono[(size_t)i * K + b] = v;
    }
  for (double v : mono)
    if (!isfinite(v)) return PD_ENAN;
  double lambda = 0.0;
  if (d == 2) {
    double lmin = INFINITY;
    for (int i = 0; i < N; ++i) {
      double* Ai = A + (size_t)i * dim * dim;
      for (int a = 0; a < dim; ++a)
        for (int b = a; b < dim; ++b) {
          int e[3] = {0, 0, 0};
          e[a] += 1;
          e[b] += 1;
          const double c = mono[(size_t)i * K + index_of(e[0], e[1], e[2])];
          Ai[a * dim + b] = Ai[b * dim + a] = a == b ? c : 0.5 * c;
        }
      lmin = std::min(lmin, sym_lambda_min(dim, Ai));
    }
    // the common shift A_i + lambda Id of every grain leaves the diagram
    // unchanged (Lemma 4.2) and makes every A_i positive definite
    lambda = std::max(0.0, margin - lmin);
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < dim; ++a) A[(size_t)i * dim * dim + a * dim + a] += lambda;
  }
  for (int i = 0; i < N; ++i) {
    double bx[3], z[3];
    for (int a = 0; a < dim; ++a) {
      int e[3] = {0, 0, 0};
      e[a] = 1;
      bx[a] = mono[(size_t)i * K + index_of(e[0], e[1], e[2])];
    }
    const double t1 = mono[(size_t)i * K + index_of(0, 0, 0)];
    if (d == 1) {  // eq. pd-lr-to-phys
      double s = 0.0;
      for (int a = 0; a < dim; ++a) {
        y[(size_t)i * dim + a] = -0.5 * bx[a];
        s += 0.25 * bx[a] * bx[a];
      }
      w[i] = s - t1;
      continue;
    }
    // eq. apd-lr-to-phys: z = A^-1 b (adjugate over determinant), y = -z/2,
    // w = b.z / 4 - theta_1
    const double* M = A + (size_t)i * dim * dim;
    if (dim == 2) {
      const double det = M[0] * M[3] - M[1] * M[2];
      z[0] = (M[3] * bx[0] - M[1] * bx[1]) / det;
      z[1] = (-M[2] * bx[0] + M[0] * bx[1]) / det;
    } else {
      const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
      const double c11 = M[0] * M[8] - M[2] * M[6], c12 = M[1] * M[6] - M[0] * M[7], c22 = M[0] * M[4] - M[1] * M[3];
      const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
      // symmetric: the adjugate is symmetric too
      z[0] = (c00 * bx[0] + c01 * bx[1] + c02 * bx[2]) / det;
      z[1] = (c01 * bx[0] + c11 * bx[1] + c12 * bx[2]) / det;
      z[2] = (c02 * bx[0] + c12 * bx[1] + c22 * bx[2]) / det;
    }
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
      y[(size_t)i * dim + a] = -0.5 * z[a];
      s += 0.25 * bx[a] * z[a];
    }
    w[i] = s - t1;
  }
  if (lambda_out) *lambda_out = lambda;
  return PD_OK;
}

int pd_heuristic_init(const pd_grid* grid, const int32_t* labels, int N, int d, double* theta_out,
                      void* stream) {
  Geom g;
  int rc = validate_grid(grid, &g);
  if (rc) return rc;
  if (N < 1 || d < 1 || !theta_out || !labels || g.P < 1) return PD_EINVAL;
  if (!degree_ok(grid->dim, d)) return PD_ENOTSUP;
  const int dim = grid->dim;
  cudaStream_t st = (cudaStream_t)stream;
  const int K2 = basis_K(dim, 2);
  std::vector<double> mom((size_t)N * K2);
  std::vector<int64_t> cnt(N);
  {
    Scratch sc(st);
    double* dmom = sc.get<double>((size_t)N * K2);
    int64_t* dcnt = sc.get<int64_t>(N);
    if (!sc.ok()) return PD_ENOMEM;
    rc = moments_simt(g, dim, 2, labels, N, dmom, dcnt, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(mom.data(), dmom, sizeof(double) * mom.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return PD_ECUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return PD_ECUDA;
  // moments of degree <= 2 in library order: 1, x_a, then degree-2 entries
  const std::vector<int> al = alpha_table(dim, 2);
  auto idx = [&](int e0, int e1, int e2) {
    for (int k = 0; k < K2; ++k)
      if (al[k * dim] == e0 && al[k * dim + 1] == e1 && (dim == 2 || al[k * dim + 2] == e2)) return k;
    return 0;
  };
  const bool anis = d >= 2;
  const double vol = dim == 2 ? M_PI : 4.0 * M_PI / 3.0;
  std::vector<double> y((size_t)N * dim), w(N), A((size_t)N * dim * dim);
  for (int i = 0; i < N; ++i) {
    const double n = (double)cnt[i];
    const double* m = &mom[(size_t)i * K2];
    double Bm[9];
    for (int a = 0; a < dim; ++a) {
      int e[3] = {0, 0, 0};
      e[a] = 1;
      y[(size_t)i * dim + a] = n > 0 ? m[idx(e[0], e[1], e[2])] / n : 0.0;
    }
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b) {
        int e[3] = {0, 0, 0};
        e[a] += 1;
        e[b] += 1;
        // psi_{2 e_a} = P_2(x_a) = (3 x_a^2 - 1)/2  =>  x_a^2 = (2 P_2 + 1)/3
        double sxx = (a == b) ? (2.0 * m[idx(e[0], e[1], e[2])] + n) / 3.0 : m[idx(e[0], e[1], e[2])];
        Bm[a * dim + b] = n > 0 ? sxx / n - y[(size_t)i * dim + a] * y[(size_t)i * dim + b] : 0.0;
      }
    double det = dim == 2 ? Bm[0] * Bm[3] - Bm[1] * Bm[2]
                          : Bm[0] * (Bm[4] * Bm[8] - Bm[5] * Bm[7]) - Bm[1] * (Bm[3] * Bm[8] - Bm[5] * Bm[6]) +
                                Bm[2] * (Bm[3] * Bm[7] - Bm[4] * Bm[6]);
    double* Ai = &A[(size_t)i * dim * dim];
    if (!anis || n == 0 || !(det > 0.0) || !isfinite(det)) {
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) Ai[a * dim + b] = (a == b);
    } else if (dim == 2) {
      Ai[0] = Bm[3] / det; Ai[1] = -Bm[1] / det; Ai[2] = -Bm[2] / det; Ai[3] = Bm[0] / det;
    } else {
      // adjugate / det
      Ai[0] = (Bm[4] * Bm[8] - Bm[5] * Bm[7]) / det;
      Ai[1] = (Bm[2] * Bm[7] - Bm[1] * Bm[8]) / det;
      Ai[2] = (Bm[1] * Bm[5] - Bm[2] * Bm[4]) / det;
      Ai[3] = (Bm[5] * Bm[6] - Bm[3] * Bm[8]) / det;
      Ai[4] = (Bm[0] * Bm[8] - Bm[2] * Bm[6]) / det;
      Ai[5] = (Bm[2] * Bm[3] - Bm[0] * Bm[5]) / det;
      Ai[6] = (Bm[3] * Bm[7] - Bm[4] * Bm[6]) / det;
      Ai[7] = (Bm[1] * Bm[6] - Bm[0] * Bm[7]) / det;
      Ai[8] = (Bm[0] * Bm[4] - Bm[1] * Bm[3]) / det;
    }
    double detA = dim == 2 ? Ai[0] * Ai[3] - Ai[1] * Ai[2]
                           : Ai[0] * (Ai[4] * Ai[8] - Ai[5] * Ai[7]) - Ai[1] * (Ai[3] * Ai[8] - Ai[5] * Ai[6]) +
                                 Ai[2] * (Ai[3] * Ai[7] - Ai[4] * Ai[6]);
    w[i] = sqrt(detA) * n / ((double)g.P * vol);
  }
  const int K = basis_K(dim, d);
  std::vector<double> th((size_t)N * K);
  rc = theta_from_apd_host(dim, d, N, y.data(), w.data(), anis ? A.data() : nullptr, th.data());
  if (rc) return rc;
  if (cudaMemcpyAsync(theta_out, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PD_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? PD_OK : PD_ECUDA;
}

void pd_release(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  noalloc_forget_device();
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
  }
}

}  // extern "C"
