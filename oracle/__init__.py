"""Plain FP64 CPU oracle for polynomial-diagram fitting (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package.  The product
library never loads it and shares no code with it.

The arithmetic lives in ``pd_oracle.c`` (plain C, double precision, one
pixel and one grain at a time, in the order the paper writes its formulas);
this module compiles it with gcc on first use and marshals numpy arrays.
Each wrapper names the part of the paper it restates.

Parity status of each function (what pins it; see tests/test_oracle_*.py):
  features, legendre ........ closed forms, scipy/numpy Legendre routines,
                              Gauss-Legendre orthogonality
  objective_grad ............ Phi(0) = -log N, logsumexp brute force,
                              finite differences, invariances, eps->0 bound
  hvp, hessian .............. finite differences of the gradient, -Var form,
                              negative semidefiniteness, K-dim null space
  assign .................... brute-force numpy argmin, constructed ties
  mono_to_legendre .......... numpy poly2leg
  theta_from_apd ............ direct power-distance argmin, round trips
  heuristic_theta ........... printed formulas against numpy; its diagram
                              against numpy's (anisotropic) power diagram
                              of those parameters (d = 1, 2, 4)
  lbfgs_fit, newton_cg_fit .. scipy L-BFGS-B optimum on non-separable data,
                              recovery certificate (Cor. 4.10)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pd_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64 * 3),
                ("coords", C.POINTER(C.c_double)), ("P", C.c_int64)]


class FitReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("evals", C.c_int64), ("phi", C.c_double),
                ("gnorm", C.c_double), ("status", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
            gp = C.POINTER(_Grid)
            lib.or_K.argtypes = [C.c_int, C.c_int]
            lib.or_alpha.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
            lib.or_legendre.argtypes = [C.c_int, C.c_double]
            lib.or_legendre.restype = C.c_double
            lib.or_features.argtypes = [gp, C.c_int, C.c_int, dp]
            lib.or_objective_grad.argtypes = [gp, ip, C.c_int, C.c_int, C.c_int,
                                              C.c_double, dp, dp, dp]
            lib.or_pixel_terms.argtypes = [gp, ip, C.c_int, C.c_int, C.c_double, dp,
                                           C.c_int64, C.POINTER(C.c_int64), dp, dp]
            lib.or_hvp.argtypes = [gp, ip, C.c_int, C.c_int, C.c_double, dp, dp, dp]
            lib.or_hessian.argtypes = [gp, C.c_int, C.c_int, C.c_double, dp, dp]
            lib.or_assign.argtypes = [gp, C.c_int, C.c_int, C.c_int, dp, ip, dp]
            lib.or_grain_moments.argtypes = [gp, ip, C.c_int, C.c_int, dp,
                                             C.POINTER(C.c_int64)]
            lib.or_mono_to_legendre.argtypes = [C.c_int, C.c_int, dp]
            lib.or_theta_from_apd.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp]
            lib.or_heuristic_params.argtypes = [gp, ip, C.c_int, C.c_int, dp, dp, dp]
            lib.or_heuristic_theta.argtypes = [gp, ip, C.c_int, C.c_int, dp]
            lib.or_lbfgs_fit.argtypes = [gp, ip, C.c_int, C.c_int, C.c_double, dp,
                                         C.c_int, C.c_int, C.c_double, dp,
                                         C.POINTER(FitReport)]
            lib.or_newton_cg_fit.argtypes = [gp, ip, C.c_int, C.c_int, C.c_double, dp,
                                             C.c_int, C.c_int, C.c_double, dp,
                                             C.POINTER(FitReport)]
            lib.or_theta_to_apd.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_double, dp, dp, dp, dp]
            lib.or_anneal_fit.argtypes = [gp, ip, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                          C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_int, dp, dp, dp,
                                          C.POINTER(C.c_int)]
            lib.or_mlp_forward.argtypes = [C.c_int] * 5 + [dp] * 8
            lib.or_mlp_loss_grad.argtypes = [C.c_int] * 5 + [dp] * 14
            lib.or_mlp_loss_grad.restype = C.c_double
            lib.or_mlp_features.argtypes = [gp, ip, C.c_int, C.c_int, C.c_int, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


class Grid:
    """Pixel set: a structured grid of extents ``shape`` (axis 1 fastest) on
    [-1,1]^dim with pixel centres -1 + (2k+1)/n (Sec. 2.1), or an explicit
    [P, dim] point list."""

    def __init__(self, shape=None, coords=None):
        if coords is not None:
            self.coords = np.ascontiguousarray(coords, dtype=np.float64)
            self.dim = self.coords.shape[1]
            self.shape = None
            self.P = self.coords.shape[0]
        else:
            self.coords = None
            self.shape = tuple(int(s) for s in shape)
            self.dim = len(self.shape)
            self.P = int(np.prod(self.shape))
        n = list(self.shape) if self.shape else [0] * self.dim
        n = n + [1] * (3 - len(n))
        self._c = _Grid(self.dim, (C.c_int64 * 3)(*n),
                        _dp(self.coords), self.P)

    @property
    def ref(self):
        return C.byref(self._c)


def _labels(labels):
    return np.ascontiguousarray(labels, dtype=np.int32).reshape(-1)


def K(dim: int, d: int) -> int:
    """K_d = |A_d| (Sec. 3.1)."""
    return _load().or_K(dim, d)


def alpha(dim: int, d: int) -> np.ndarray:
    """Multi-indices of A_d in the fixed order, shape [K, dim]."""
    k = K(dim, d)
    out = np.zeros((k, dim), dtype=np.intc)
    _load().or_alpha(dim, d, out.ctypes.data_as(C.POINTER(C.c_int)))
    return out


def legendre(m: int, t: float) -> float:
    """P_m(t) by the three-term recurrence (Sec. 3.3)."""
    return _load().or_legendre(m, float(t))


def features(grid: Grid, d: int, basis: str = "legendre") -> np.ndarray:
    """Design matrix, pixel-major [P, K] (Sec. 3.2/3.3)."""
    out = np.empty((grid.P, K(grid.dim, d)), dtype=np.float64)
    rc = _load().or_features(grid.ref, d, 0 if basis == "legendre" else 1, _dp(out))
    assert rc == 0
    return out


def objective_grad(grid: Grid, labels, N: int, d: int, eps: float, theta,
                   basis: str = "legendre", want_grad: bool = True):
    """Phi (eqs. log-res-2, Phi) and grad Phi (eq. grad); theta is [N, K]."""
    lab = _labels(labels)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    phi = np.zeros(1)
    grad = np.empty_like(th) if want_grad else None
    rc = _load().or_objective_grad(grid.ref, _ip(lab), N, d,
                                   0 if basis == "legendre" else 1, float(eps),
                                   _dp(th), _dp(phi), _dp(grad))
    if rc != 0:
        raise ValueError("oracle: invalid arguments or labels")
    return (float(phi[0]), grad) if want_grad else float(phi[0])


def pixel_terms(grid: Grid, labels, N: int, d: int, eps: float, theta, idx):
    """Per-pixel r_x = l_G(x) - log S(x) and log S(x) for selected pixels."""
    lab = _labels(labels)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    r = np.empty(idx.size)
    lse = np.empty(idx.size)
    rc = _load().or_pixel_terms(grid.ref, _ip(lab), N, d, float(eps), _dp(th),
                                idx.size, idx.ctypes.data_as(C.POINTER(C.c_int64)),
                                _dp(r), _dp(lse))
    assert rc == 0
    return r, lse


def hvp(grid: Grid, labels, N: int, d: int, eps: float, theta, v):
    """Hessian-vector product from eq. (hess)."""
    lab = _labels(labels)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(th)
    rc = _load().or_hvp(grid.ref, _ip(lab), N, d, float(eps), _dp(th), _dp(vv), _dp(out))
    assert rc == 0
    return out


def hessian(grid: Grid, N: int, d: int, eps: float, theta):
    """Dense Hessian [N*K, N*K] from eq. (hess) (tiny problems only)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    n = th.size
    H = np.empty((n, n))
    rc = _load().or_hessian(grid.ref, N, d, float(eps), _dp(th), _dp(H))
    assert rc == 0
    return H


def assign(grid: Grid, N: int, d: int, theta, basis: str = "legendre"):
    """F_theta (smallest index on ties) and the top-two gap of h."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lab = np.empty(grid.P, dtype=np.int32)
    gap = np.empty(grid.P)
    rc = _load().or_assign(grid.ref, N, d, 0 if basis == "legendre" else 1,
                           _dp(th), _ip(lab), _dp(gap))
    assert rc == 0
    return lab, gap


def grain_moments(grid: Grid, labels, N: int, dm: int):
    """Per-grain sums of psi_alpha over the grain, degree dm; and counts."""
    lab = _labels(labels)
    mom = np.empty((N, K(grid.dim, dm)))
    cnt = np.empty(N, dtype=np.int64)
    rc = _load().or_grain_moments(grid.ref, _ip(lab), N, dm, _dp(mom),
                                  cnt.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ValueError("oracle: invalid labels")
    return mom, cnt


def mono_to_legendre(dim: int, d: int) -> np.ndarray:
    """T^(d) with theta_L = T theta_mono (Remark 3.1)."""
    k = K(dim, d)
    T = np.empty((k, k))
    assert _load().or_mono_to_legendre(dim, d, _dp(T)) == 0
    return T


def theta_from_apd(dim: int, d: int, y, w, A=None) -> np.ndarray:
    """(A, y, w) -> Legendre theta (Sec. 2.3); A=None is a power diagram."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    N = w.size
    Aa = None if A is None else np.ascontiguousarray(A, dtype=np.float64)
    th = np.empty((N, K(dim, d)))
    rc = _load().or_theta_from_apd(dim, d, N, _dp(y), _dp(w), _dp(Aa), _dp(th))
    if rc != 0:
        raise ValueError("oracle: bad conversion arguments")
    return th


def heuristic_params(grid: Grid, labels, N: int, anisotropic: bool):
    """(y', w', A') of the moment heuristic (Sec. 5.5.2)."""
    lab = _labels(labels)
    y = np.empty((N, grid.dim))
    w = np.empty(N)
    A = np.empty((N, grid.dim, grid.dim))
    rc = _load().or_heuristic_params(grid.ref, _ip(lab), N, int(anisotropic),
                                     _dp(y), _dp(w), _dp(A))
    assert rc == 0
    return y, w, A


def heuristic_theta(grid: Grid, labels, N: int, d: int) -> np.ndarray:
    """theta' of the moment heuristic, Legendre, degree d (Sec. 5.5.2)."""
    lab = _labels(labels)
    th = np.empty((N, K(grid.dim, d)))
    rc = _load().or_heuristic_theta(grid.ref, _ip(lab), N, d, _dp(th))
    assert rc == 0
    return th


def lbfgs_fit(grid: Grid, labels, N: int, d: int, eps: float, theta0,
              max_iter: int, m: int = 10, gtol: float = 0.0):
    """The ascent scheme of Sec. 5.2 (L-BFGS on -Phi, gauge theta_{N-1}=0).

    Returns (theta, report, phi_trace)."""
    lab = _labels(labels)
    th = np.array(theta0, dtype=np.float64, copy=True, order="C")
    trace = np.full(max_iter, np.nan)
    rep = FitReport()
    rc = _load().or_lbfgs_fit(grid.ref, _ip(lab), N, d, float(eps), _dp(th),
                              int(max_iter), int(m), float(gtol), _dp(trace),
                              C.byref(rep))
    assert rc == 0
    return th, rep, trace[:rep.iters]


def newton_cg_fit(grid: Grid, labels, N: int, d: int, eps: float, theta0,
                  max_iter: int, max_cg: int = 50, gtol: float = 0.0):
    """Truncated-Newton ascent with eq. (hess) products."""
    lab = _labels(labels)
    th = np.array(theta0, dtype=np.float64, copy=True, order="C")
    trace = np.full(max_iter, np.nan)
    rep = FitReport()
    rc = _load().or_newton_cg_fit(grid.ref, _ip(lab), N, d, float(eps), _dp(th),
                                  int(max_iter), int(max_cg), float(gtol),
                                  _dp(trace), C.byref(rep))
    assert rc == 0
    return th, rep, trace[:rep.iters]


def theta_to_apd(dim: int, d: int, theta, margin: float = 1e-3):
    """Legendre theta (d = 1 or 2) -> physical parameters (y, w, A, lambda)
    by eqs. pd-lr-to-phys / apd-lr-to-phys after the common shift A_i +
    lambda Id of Sec. 5.5.3 (A is None for d = 1)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    N = th.shape[0]
    y = np.empty((N, dim))
    w = np.empty(N)
    A = np.empty((N, dim, dim)) if d == 2 else None
    lam = C.c_double(0.0)
    rc = _load().or_theta_to_apd(dim, d, N, _dp(th), float(margin), _dp(y), _dp(w), _dp(A),
                                 C.cast(C.pointer(lam), C.POINTER(C.c_double)))
    if rc != 0:
        raise ValueError("oracle: bad recovery arguments")
    return y, w, A, lam.value


def anneal_fit(grid: Grid, labels, N: int, d: int, eps0: float, factor: float, eps_min: float,
               stage_iter: int, final_iter: int, theta0, m: int = 10, err_stop: bool = True,
               max_stages: int = 64):
    """eps annealing with Err^G-aligned stopping (the build's reading of the
    future-work schedule of Secs. 5.2 and 5.5.4).  Returns (theta, stages),
    stages a list of (eps, Phi, Err^G or -1, iterations)."""
    lab = _labels(labels)
    th = np.array(theta0, dtype=np.float64, copy=True, order="C")
    se, sp, sr = np.zeros(max_stages), np.zeros(max_stages), np.zeros(max_stages)
    si = np.zeros(max_stages, dtype=np.int32)
    n = _load().or_anneal_fit(grid.ref, _ip(lab), N, d, float(eps0), float(factor), float(eps_min),
                              int(stage_iter), int(final_iter), int(m), int(err_stop), _dp(th),
                              int(max_stages), _dp(se), _dp(sp), _dp(sr),
                              si.ctypes.data_as(C.POINTER(C.c_int)))
    assert n > 0
    return th, [(float(se[k]), float(sp[k]), float(sr[k]), int(si[k])) for k in range(n)]


# ---------------------------------------------------------------------------
# learned warm start (not from the paper): the MLP and its inputs
# ---------------------------------------------------------------------------
def mlp_forward(X, W1, b1, W2, b2, W3, b3):
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for every row of X."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    ws = [np.ascontiguousarray(w, dtype=np.float64) for w in (W1, b1, W2, b2, W3, b3)]
    B, n_in = X.shape
    n_h1, n_h2, n_out = ws[0].shape[0], ws[2].shape[0], ws[4].shape[0]
    Y = np.empty((B, n_out))
    _load().or_mlp_forward(B, n_in, n_h1, n_h2, n_out, _dp(X), *[_dp(w) for w in ws], _dp(Y))
    return Y


def mlp_loss_grad(X, T, W1, b1, W2, b2, W3, b3):
    """Mean squared error and its gradients (back-propagation)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    ws = [np.ascontiguousarray(w, dtype=np.float64) for w in (W1, b1, W2, b2, W3, b3)]
    B, n_in = X.shape
    n_h1, n_h2, n_out = ws[0].shape[0], ws[2].shape[0], ws[4].shape[0]
    gs = [np.empty_like(w) for w in ws]
    loss = _load().or_mlp_loss_grad(B, n_in, n_h1, n_h2, n_out, _dp(X), _dp(T), *[_dp(w) for w in ws],
                                    *[_dp(g) for g in gs])
    return loss, gs


def mlp_features(grid: Grid, labels, N: int, dm: int = 4, n_nb: int = 8):
    """[N, (1 + n_nb) K_dm] warm-start inputs: normalised grain moments and
    those of the n_nb nearest grains by centroid."""
    lab = _labels(labels)
    Kd = K(grid.dim, dm)
    F = np.empty((N, (1 + n_nb) * Kd))
    rc = _load().or_mlp_features(grid.ref, _ip(lab), N, dm, n_nb, _dp(F))
    if rc != 0:
        raise ValueError("oracle: invalid labels")
    return F
