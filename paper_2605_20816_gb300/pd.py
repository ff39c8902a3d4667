"""Thin Python binding of libpd (ctypes).

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors become device pointers, the current torch
CUDA stream becomes the stream argument, and a negative status code becomes
a ``PdError``.  All arithmetic happens inside libpd's CUDA kernels; there is
no CPU fallback.  If libpd.so is missing it is built from csrc/ with nvcc,
and any failure to build or load raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import torch

from . import build as _build

PD_OK, PD_EINVAL, PD_ELABEL, PD_ENAN, PD_ENOMEM, PD_ECUDA, PD_ETIMEOUT, PD_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
PD_ESCRATCH = -8
PD_NOALLOC_SCRATCH_BYTES = 32 << 20
PD_FP64, PD_FP32, PD_BF16, PD_BF16X3 = 0, 1, 2, 3
PD_INIT_GIVEN, PD_INIT_ZERO, PD_INIT_HEURISTIC = 0, 1, 2
PD_METHOD_LBFGS, PD_METHOD_NEWTON_CG = 0, 1
PREC = {"fp64": PD_FP64, "fp32": PD_FP32, "bf16": PD_BF16, "bf16x3": PD_BF16X3}


class PdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))


class pd_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64 * 3), ("coords", C.c_void_p), ("P", C.c_int64)]


class pd_eval_opts(C.Structure):
    _fields_ = [("d", C.c_int), ("eps", C.c_double), ("prec", C.c_int)]


class pd_fit_opts(C.Structure):
    _fields_ = [("d", C.c_int), ("eps", C.c_double), ("init", C.c_int), ("method", C.c_int),
                ("max_iter", C.c_int), ("lbfgs_m", C.c_int), ("max_cg", C.c_int), ("prec", C.c_int),
                ("refine_iter", C.c_int), ("gtol", C.c_double), ("target_phi", C.c_double),
                ("switch_rtol", C.c_double), ("anneal_eps0", C.c_double), ("anneal_factor", C.c_double),
                ("anneal_iter", C.c_int), ("err_stop", C.c_int)]


class pd_fit_report(C.Structure):
    _fields_ = [("phi", C.c_double), ("gnorm", C.c_double), ("err", C.c_double), ("iters", C.c_int),
                ("iters_phase1", C.c_int), ("evals", C.c_int64), ("hvps", C.c_int64), ("status", C.c_int),
                ("seconds", C.c_double), ("eps_final", C.c_double), ("stages", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pd_map(C.Structure):
    _fields_ = [("grid", pd_grid), ("labels", C.c_void_p), ("N", C.c_int), ("theta", C.c_void_p),
                ("obj_out", C.c_void_p), ("grad_out", C.c_void_p), ("target_phi", C.c_double)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load (building first if needed) the in-tree libpd.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, i64, dbl, ip = C.c_void_p, C.c_int64, C.c_double, C.c_int
            gp = C.POINTER(pd_grid)
            L.pd_K.argtypes = [ip, ip]
            L.pd_alpha.argtypes = [ip, ip, C.POINTER(C.c_int)]
            L.pd_strerror.argtypes = [ip]
            L.pd_strerror.restype = C.c_char_p
            L.pd_features.argtypes = [gp, ip, ip, vp, vp]
            L.pd_objective_grad.argtypes = [gp, vp, ip, vp, C.POINTER(pd_eval_opts), vp, vp, vp]
            L.pd_hvp.argtypes = [gp, vp, ip, vp, vp, C.POINTER(pd_eval_opts), vp, vp]
            L.pd_assign.argtypes = [gp, ip, ip, vp, vp, vp, vp, vp, vp]
            L.pd_moments.argtypes = [gp, vp, ip, ip, vp, vp, vp]
            L.pd_check_labels.argtypes = [gp, vp, ip, vp]
            L.pd_theta_from_apd.argtypes = [ip, ip, ip, vp, vp, vp, vp]
            L.pd_theta_to_apd.argtypes = [ip, ip, ip, vp, dbl, vp, vp, vp, C.POINTER(C.c_double)]
            L.pd_heuristic_init.argtypes = [gp, vp, ip, ip, vp, vp]
            L.pd_fit.argtypes = [gp, vp, ip, C.POINTER(pd_fit_opts), vp, C.POINTER(pd_fit_report), vp]
            L.pd_prof_enable.argtypes = [ip]
            L.pd_prof_read.argtypes = [ip, C.POINTER(C.c_char_p), C.POINTER(C.c_int64), C.POINTER(C.c_double)]
            L.pd_objective_grad_noalloc.argtypes = [gp, vp, ip, vp, C.POINTER(pd_eval_opts), vp, vp, vp]
            L.pd_microbench.argtypes = [ip, C.POINTER(C.c_double), vp]
            mp = C.POINTER(pd_map)
            L.pd_batch_create.argtypes = [ip, mp, C.POINTER(pd_eval_opts), ip, C.POINTER(vp)]
            L.pd_batch_eval.argtypes = [vp, vp]
            L.pd_batch_set_active.argtypes = [vp, C.POINTER(C.c_int32), vp]
            L.pd_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.pd_batch_destroy.argtypes = [vp]
            L.pd_batch_destroy.restype = None
            L.pd_fit_batched.argtypes = [ip, mp, C.POINTER(vp), C.POINTER(pd_fit_opts), C.POINTER(pd_fit_report), vp]
            L.pd_mlp_create.argtypes = [ip, ip, ip, ip, C.c_uint64, C.POINTER(vp)]
            L.pd_mlp_destroy.argtypes = [vp]
            L.pd_mlp_destroy.restype = None
            L.pd_mlp_num_params.argtypes = [vp]
            L.pd_mlp_num_params.restype = C.c_int64
            L.pd_mlp_get_params.argtypes = [vp, vp, ip]
            L.pd_mlp_set_params.argtypes = [vp, vp]
            L.pd_mlp_forward.argtypes = [vp, vp, ip, vp, vp]
            L.pd_mlp_loss_grad.argtypes = [vp, vp, vp, ip, vp, vp, vp]
            L.pd_mlp_train_step.argtypes = [vp, vp, vp, ip, C.c_float, vp, vp]
            L.pd_mlp_features.argtypes = [gp, vp, ip, vp, vp]
            L.pd_mlp_targets.argtypes = [vp, ip, ip, vp, vp]
            L.pd_warm_start.argtypes = [vp, gp, vp, ip, ip, C.c_double, ip, vp, C.POINTER(C.c_double), vp]
            L.pd_selftest_wait_timeout.argtypes = [C.c_double, C.POINTER(C.c_int), vp]
            L.pd_plan_create.argtypes = [gp, vp, ip, ip, ip, ip, C.POINTER(vp)]
            L.pd_plan_objective_grad.argtypes = [vp, vp, dbl, vp, vp, vp]
            L.pd_plan_hvp.argtypes = [vp, vp, vp, dbl, vp, vp]
            L.pd_plan_scratch_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
            L.pd_plan_destroy.argtypes = [vp]
            L.pd_plan_destroy.restype = None
            L.pd_release.argtypes = []
            L.pd_release.restype = None
            _lib = L
    return _lib


def lib_path() -> str:
    return _build.LIB


def strerror(code: int) -> str:
    try:
        return lib().pd_strerror(code).decode()
    except Exception:
        return "status %d" % code


def _check(rc: int, where: str):
    if rc != PD_OK:
        raise PdError(rc, where)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


class Grid:
    """Pixel set: structured grid ``shape`` = (n1, n2[, n3]) (axis 1
    fastest), or an explicit point list ``coords`` (CUDA float64 [P, dim])."""

    def __init__(self, shape=None, coords: torch.Tensor | None = None):
        if coords is not None:
            self.coords = coords.contiguous().to(torch.float64)
            self.dim = int(self.coords.shape[1])
            self.P = int(self.coords.shape[0])
            n = [0, 0, 0]
            ptr = self.coords.data_ptr()
        else:
            self.coords = None
            self.shape = tuple(int(s) for s in shape)
            self.dim = len(self.shape)
            self.P = int(math.prod(self.shape))
            n = list(self.shape) + [1] * (3 - self.dim)
            ptr = None
        self.c = pd_grid(self.dim, (C.c_int64 * 3)(*n), ptr, self.P)

    @property
    def ref(self):
        return C.byref(self.c)


def pd_K(dim: int, d: int) -> int:
    return lib().pd_K(dim, d)


def pd_alpha(dim: int, d: int):
    K = pd_K(dim, d)
    buf = (C.c_int * (K * dim))()
    rc = lib().pd_alpha(dim, d, buf)
    if rc < 0:
        raise PdError(rc, "pd_alpha")
    return [tuple(buf[k * dim:(k + 1) * dim]) for k in range(K)]


def pd_features(grid: Grid, d: int, prec: int = PD_FP64) -> torch.Tensor:
    K = pd_K(grid.dim, d)
    out = torch.empty((grid.P, K), dtype=torch.float64 if prec == PD_FP64 else torch.float32, device="cuda")
    _check(lib().pd_features(grid.ref, d, prec, _ptr(out), _stream()), "pd_features")
    return out


def pd_objective_grad(grid: Grid, labels: torch.Tensor, N: int, theta: torch.Tensor, d: int, eps: float,
                      prec: int = PD_FP64, want_grad: bool = True, obj_out=None, grad_out=None):
    """Returns (Phi as a 0-d CUDA float64 tensor, grad [N, K] or None)."""
    opts = pd_eval_opts(d, float(eps), int(prec))
    obj = obj_out if obj_out is not None else torch.empty((), dtype=torch.float64, device="cuda")
    grad = None
    if want_grad:
        grad = grad_out if grad_out is not None else torch.empty_like(theta, dtype=torch.float64)
    _check(lib().pd_objective_grad(grid.ref, _ptr(labels), N, _ptr(theta), C.byref(opts), _ptr(obj),
                                   _ptr(grad), _stream()), "pd_objective_grad")
    return obj, grad


def pd_objective_grad_noalloc(grid: Grid, labels: torch.Tensor, N: int, theta: torch.Tensor, d: int,
                              eps: float, prec: int = PD_FP32, obj_out=None, grad_out=None):
    """pd_objective_grad with all scratch in the library's fixed device
    array, for callers that cannot allocate device memory; the caller passes
    the output buffers (allocated here only when omitted)."""
    opts = pd_eval_opts(d, float(eps), int(prec))
    obj = obj_out if obj_out is not None else torch.empty((), dtype=torch.float64, device="cuda")
    grad = grad_out if grad_out is not None else torch.empty_like(theta, dtype=torch.float64)
    _check(lib().pd_objective_grad_noalloc(grid.ref, _ptr(labels), N, _ptr(theta), C.byref(opts), _ptr(obj),
                                           _ptr(grad), _stream()), "pd_objective_grad_noalloc")
    return obj, grad


def pd_hvp(grid: Grid, labels, N: int, theta: torch.Tensor, v: torch.Tensor, d: int, eps: float,
           prec: int = PD_FP64, out=None):
    opts = pd_eval_opts(d, float(eps), int(prec))
    hv = out if out is not None else torch.empty_like(theta, dtype=torch.float64)
    _check(lib().pd_hvp(grid.ref, _ptr(labels), N, _ptr(theta), _ptr(v), C.byref(opts), _ptr(hv), _stream()),
           "pd_hvp")
    return hv


def pd_assign(grid: Grid, N: int, d: int, theta: torch.Tensor, want_gap: bool = False,
              ref_labels: torch.Tensor | None = None, out: torch.Tensor | None = None,
              mismatch_out: torch.Tensor | None = None):
    """Returns (labels int32 [P], gap float64 [P] or None, mismatch int64 0-d or None)."""
    lab = out if out is not None else torch.empty(grid.P, dtype=torch.int32, device="cuda")
    gap = torch.empty(grid.P, dtype=torch.float64, device="cuda") if want_gap else None
    mis = None
    if ref_labels is not None:
        mis = mismatch_out if mismatch_out is not None else torch.empty((), dtype=torch.int64, device="cuda")
    _check(lib().pd_assign(grid.ref, N, d, _ptr(theta), _ptr(lab), _ptr(gap), _ptr(ref_labels), _ptr(mis),
                           _stream()), "pd_assign")
    return lab, gap, mis


def pd_moments(grid: Grid, labels: torch.Tensor, N: int, dm: int):
    K = pd_K(grid.dim, dm)
    mom = torch.empty((N, K), dtype=torch.float64, device="cuda")
    cnt = torch.empty(N, dtype=torch.int64, device="cuda")
    _check(lib().pd_moments(grid.ref, _ptr(labels), N, dm, _ptr(mom), _ptr(cnt), _stream()), "pd_moments")
    return mom, cnt


def pd_check_labels(grid: Grid, labels: torch.Tensor, N: int) -> int:
    """Returns the status code (PD_OK or PD_ELABEL); raises on other errors."""
    rc = lib().pd_check_labels(grid.ref, _ptr(labels), N, _stream())
    if rc not in (PD_OK, PD_ELABEL):
        raise PdError(rc, "pd_check_labels")
    return rc


def pd_theta_from_apd(dim: int, d: int, y, w, A=None):
    """Host conversion; y [N, dim], w [N], A [N, dim, dim] or None (numpy
    or CPU tensors).  Returns a CPU float64 tensor [N, K]."""
    y = torch.as_tensor(y, dtype=torch.float64).contiguous()
    w = torch.as_tensor(w, dtype=torch.float64).contiguous()
    Ah = None if A is None else torch.as_tensor(A, dtype=torch.float64).contiguous()
    N = int(w.numel())
    out = torch.empty((N, pd_K(dim, d)), dtype=torch.float64)
    rc = lib().pd_theta_from_apd(dim, d, N, C.c_void_p(y.data_ptr()), C.c_void_p(w.data_ptr()),
                                 None if Ah is None else C.c_void_p(Ah.data_ptr()), C.c_void_p(out.data_ptr()))
    _check(rc, "pd_theta_from_apd")
    return out


def pd_theta_to_apd(dim: int, d: int, theta, margin: float = 1e-3):
    """Host conversion of Legendre theta [N, K] (d = 1 or 2; numpy or CPU
    tensor) to physical parameters.  Returns (y [N, dim], w [N], A [N, dim,
    dim] or None, lambda) as CPU float64 tensors and a float."""
    th = torch.as_tensor(theta, dtype=torch.float64).contiguous()
    N = int(th.shape[0])
    y = torch.empty((N, dim), dtype=torch.float64)
    w = torch.empty(N, dtype=torch.float64)
    A = torch.empty((N, dim, dim), dtype=torch.float64) if d == 2 else None
    lam = C.c_double(0.0)
    rc = lib().pd_theta_to_apd(dim, d, N, C.c_void_p(th.data_ptr()), float(margin), C.c_void_p(y.data_ptr()),
                               C.c_void_p(w.data_ptr()), None if A is None else C.c_void_p(A.data_ptr()),
                               C.byref(lam))
    _check(rc, "pd_theta_to_apd")
    return y, w, A, lam.value


def pd_heuristic_init(grid: Grid, labels: torch.Tensor, N: int, d: int) -> torch.Tensor:
    out = torch.empty((N, pd_K(grid.dim, d)), dtype=torch.float64, device="cuda")
    _check(lib().pd_heuristic_init(grid.ref, _ptr(labels), N, d, _ptr(out), _stream()), "pd_heuristic_init")
    return out


def pd_fit(grid: Grid, labels: torch.Tensor, N: int, d: int, eps: float, theta: torch.Tensor | None = None,
           init: int = PD_INIT_ZERO, method: int = PD_METHOD_LBFGS, max_iter: int = 1000, lbfgs_m: int = 10,
           max_cg: int = 50, prec: int = PD_FP64, refine_iter: int = 0, gtol: float = 0.0,
           target_phi: float = -math.inf, switch_rtol: float = 0.0, anneal_eps0: float = 0.0,
           anneal_factor: float = 0.5, anneal_iter: int = 100, err_stop: bool = False):
    """Returns (theta [N, K] CUDA float64, report dict)."""
    K = pd_K(grid.dim, d)
    th = torch.zeros((N, K), dtype=torch.float64, device="cuda") if theta is None else theta.clone().contiguous()
    opts = pd_fit_opts(d, float(eps), init, method, max_iter, lbfgs_m, max_cg, prec, refine_iter, gtol,
                       target_phi, switch_rtol, float(anneal_eps0), float(anneal_factor), int(anneal_iter),
                       1 if err_stop else 0)
    rep = pd_fit_report()
    _check(lib().pd_fit(grid.ref, _ptr(labels), N, C.byref(opts), _ptr(th), C.byref(rep), _stream()), "pd_fit")
    return th, rep.as_dict()


PD_PLAN_HVP = 1


class Plan:
    """A pd_plan: repeated objective/gradient (and, with hvp=True,
    Hessian-vector) evaluations on one pixel set and label map, with all
    scratch allocated once.  The caller keeps grid and labels alive and
    unchanged while the plan is used."""

    def __init__(self, grid: Grid, labels: torch.Tensor, N: int, d: int, prec: int = PD_BF16X3,
                 hvp: bool = False):
        self._keep = (grid, labels)
        self.N, self.d, self.K = int(N), int(d), pd_K(grid.dim, d)
        h = C.c_void_p()
        _check(lib().pd_plan_create(grid.ref, _ptr(labels), self.N, self.d, int(prec),
                                    PD_PLAN_HVP if hvp else 0, C.byref(h)), "pd_plan_create")
        self.h = h

    def objective_grad(self, theta: torch.Tensor, eps: float, want_grad: bool = True, obj_out=None,
                       grad_out=None):
        """(Phi as a 0-d CUDA float64 tensor, grad [N, K] or None)."""
        obj = obj_out if obj_out is not None else torch.empty((), dtype=torch.float64, device="cuda")
        grad = None
        if want_grad:
            grad = grad_out if grad_out is not None else torch.empty_like(theta, dtype=torch.float64)
        _check(lib().pd_plan_objective_grad(self.h, _ptr(theta), float(eps), _ptr(obj), _ptr(grad), _stream()),
               "pd_plan_objective_grad")
        return obj, grad

    def hvp(self, theta: torch.Tensor, v: torch.Tensor, eps: float, out=None):
        hv = out if out is not None else torch.empty_like(theta, dtype=torch.float64)
        _check(lib().pd_plan_hvp(self.h, _ptr(theta), _ptr(v), float(eps), _ptr(hv), _stream()), "pd_plan_hvp")
        return hv

    def scratch_bytes(self) -> int:
        n = C.c_size_t()
        _check(lib().pd_plan_scratch_bytes(self.h, C.byref(n)), "pd_plan_scratch_bytes")
        return n.value

    def close(self):
        if self.h:
            lib().pd_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _map(grid: Grid, labels, N, theta=None, obj=None, grad=None, target_phi=math.nan):
    return pd_map(grid.c, _ptr(labels), int(N), _ptr(theta), _ptr(obj), _ptr(grad), float(target_phi))


class Batch:
    """A pd_batch plan over maps = [(grid, labels, N, theta, obj_out, grad_out)];
    the caller keeps the tensors alive while the plan is used."""

    def __init__(self, maps, d: int, eps: float, prec: int = PD_FP32, autotune: bool = True):
        self._keep = maps
        self.n = len(maps)
        arr = (pd_map * self.n)(*[_map(*m) for m in maps])
        opts = pd_eval_opts(d, float(eps), int(prec))
        h = C.c_void_p()
        _check(lib().pd_batch_create(self.n, arr, C.byref(opts), 1 if autotune else 0, C.byref(h)),
               "pd_batch_create")
        self.h = h

    def eval(self):
        _check(lib().pd_batch_eval(self.h, _stream()), "pd_batch_eval")

    def set_active(self, active):
        a = (C.c_int32 * self.n)(*[1 if x else 0 for x in active])
        self._active = a  # the copy is asynchronous: keep the source alive
        _check(lib().pd_batch_set_active(self.h, a, _stream()), "pd_batch_set_active")

    def info(self):
        cf, od, ms = C.c_int(), C.c_int(), C.c_double()
        _check(lib().pd_batch_info(self.h, C.byref(cf), C.byref(od), C.byref(ms)), "pd_batch_info")
        return {"chunk_factor": cf.value, "occ_div": od.value, "tuned_ms": ms.value}

    def close(self):
        if self.h:
            lib().pd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_fit_batched(maps, thetas, d: int, eps: float, init: int = PD_INIT_ZERO, max_iter: int = 1000,
                   lbfgs_m: int = 10, prec: int = PD_FP64, refine_iter: int = 0, gtol: float = 0.0,
                   target_phi: float = -math.inf, switch_rtol: float = 0.0, targets=None,
                   anneal_eps0: float = 0.0, anneal_factor: float = 0.5, anneal_iter: int = 100):
    """maps = [(grid, labels, N)], thetas = [CUDA float64 [N, K]] (in/out),
    targets = per-map objective targets (None: target_phi for all).
    Returns the list of per-map report dicts."""
    n = len(maps)
    tg = [math.nan] * n if targets is None else [float(t) for t in targets]
    arr = (pd_map * n)(*[_map(g, lab, N, target_phi=t) for (g, lab, N), t in zip(maps, tg)])
    ths = (C.c_void_p * n)(*[t.data_ptr() for t in thetas])
    opts = pd_fit_opts(d, float(eps), init, PD_METHOD_LBFGS, max_iter, lbfgs_m, 50, prec, refine_iter, gtol,
                       target_phi, switch_rtol, float(anneal_eps0), float(anneal_factor), int(anneal_iter), 0)
    reps = (pd_fit_report * n)()
    _check(lib().pd_fit_batched(n, arr, ths, C.byref(opts), reps, _stream()), "pd_fit_batched")
    return [r.as_dict() for r in reps]


class MLP:
    """The warm-start network (pd_mlp_*)."""

    def __init__(self, n_in=135, n_h1=256, n_h2=256, n_out=15, seed=1):
        h = C.c_void_p()
        _check(lib().pd_mlp_create(n_in, n_h1, n_h2, n_out, seed, C.byref(h)), "pd_mlp_create")
        self.h = h
        self.dims = (n_in, n_h1, n_h2, n_out)
        self.n_params = int(lib().pd_mlp_num_params(h))

    def params(self, rounded=True):
        out = torch.empty(self.n_params, dtype=torch.float32)
        _check(lib().pd_mlp_get_params(self.h, C.c_void_p(out.data_ptr()), 1 if rounded else 0), "pd_mlp_get_params")
        return out

    def set_params(self, flat):
        flat = torch.as_tensor(flat, dtype=torch.float32).contiguous()
        _check(lib().pd_mlp_set_params(self.h, C.c_void_p(flat.data_ptr())), "pd_mlp_set_params")

    def unflatten(self, flat):
        n_in, h1, h2, o = self.dims
        sizes = [(h1, n_in), (h1,), (h2, h1), (h2,), (o, h2), (o,)]
        out, q = [], 0
        for sz in sizes:
            n = int(math.prod(sz))
            out.append(flat[q:q + n].reshape(sz))
            q += n
        return out

    def forward(self, X):
        Y = torch.empty((X.shape[0], self.dims[3]), dtype=torch.float32, device="cuda")
        _check(lib().pd_mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), _stream()), "pd_mlp_forward")
        return Y

    def loss_grad(self, X, T):
        loss = torch.empty((), dtype=torch.float32, device="cuda")
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().pd_mlp_loss_grad(self.h, _ptr(X), _ptr(T), X.shape[0], _ptr(loss), _ptr(g), _stream()),
               "pd_mlp_loss_grad")
        return loss, g

    def train_step(self, X, T, lr):
        loss = torch.empty((), dtype=torch.float32, device="cuda")
        _check(lib().pd_mlp_train_step(self.h, _ptr(X), _ptr(T), X.shape[0], C.c_float(lr), _ptr(loss), _stream()),
               "pd_mlp_train_step")
        return loss

    def close(self):
        if self.h:
            lib().pd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_mlp_features(grid: Grid, labels, N: int):
    Kd = pd_K(grid.dim, 4)
    out = torch.empty((N, 9 * Kd), dtype=torch.float32, device="cuda")
    _check(lib().pd_mlp_features(grid.ref, _ptr(labels), N, _ptr(out), _stream()), "pd_mlp_features")
    return out


def pd_mlp_targets(theta: torch.Tensor):
    N, K = theta.shape
    out = torch.empty((N, K), dtype=torch.float32, device="cuda")
    _check(lib().pd_mlp_targets(_ptr(theta), N, K, _ptr(out), _stream()), "pd_mlp_targets")
    return out


def pd_warm_start(net: MLP, grid: Grid, labels, N: int, d: int, eps: float, prec: int = PD_FP32):
    """Returns (theta [N, K] CUDA float64, chosen scale)."""
    th = torch.empty((N, pd_K(grid.dim, d)), dtype=torch.float64, device="cuda")
    s = C.c_double()
    _check(lib().pd_warm_start(net.h, grid.ref, _ptr(labels), N, d, float(eps), prec, _ptr(th), C.byref(s),
                               _stream()), "pd_warm_start")
    return th, s.value


def pd_prof_enable(on: bool):
    _check(lib().pd_prof_enable(1 if on else 0), "pd_prof_enable")


def pd_prof_read():
    """{kernel name: (launches, total device ms)} of the traced launches."""
    cap = 64
    names = (C.c_char_p * cap)()
    cnt = (C.c_int64 * cap)()
    ms = (C.c_double * cap)()
    n = lib().pd_prof_read(cap, names, cnt, ms)
    if n < 0:
        raise PdError(n, "pd_prof_read")
    return {names[q].decode(): (int(cnt[q]), float(ms[q])) for q in range(min(n, cap))}


def pd_microbench(kind: int) -> float:
    """Operations per second of one unit: 0 FP32 FMA, 1 MUFU ex2, 2 FP64 FMA."""
    v = C.c_double()
    _check(lib().pd_microbench(kind, C.byref(v), _stream()), "pd_microbench")
    return v.value


def pd_selftest_wait_timeout(seconds: float) -> int:
    """Runs the bounded-wait self-test; returns the status the kernel recorded."""
    st = C.c_int(0)
    _check(lib().pd_selftest_wait_timeout(float(seconds), C.byref(st), _stream()), "pd_selftest_wait_timeout")
    return st.value


def pd_release():
    lib().pd_release()
