"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (derived from the arithmetic):
  FP64 mode: Phi within 1e-10 relative; gradient and Hessian-vector
             product within 1e-10 in ||.||_2 relative to the oracle's norm.
  FP32 mode: every logit of a 128-pixel tile is kept relative to the
             tile's reference logit (centre parts in float-float, rounded
             once), so the float quantities are small; Phi and the gradient
             (and the Hessian-vector product) within 1e-5 relative (norm),
             the bound the method's reduced-precision form is held to.
  labels:    bit-exact wherever the oracle's top-two gap is >= 1e-9.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth
from helpers import poly_problem, power_problem, rel

pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_eval(shape_or_coords, lab, N, th, d, eps, prec):
    if isinstance(shape_or_coords, tuple):
        grid = pd.Grid(shape_or_coords)
    else:
        grid = pd.Grid(coords=dev(shape_or_coords))
    obj, grad = pd.pd_objective_grad(grid, dev(lab), N, dev(th), d, eps, prec=prec)
    torch.cuda.synchronize()
    return float(obj.item()), grad.cpu().numpy()


CASES = [
    # (shape, N, d, eps, theta scale) -- ragged pixel and grain tails
    ((64, 64), 8, 2, 1e-2, 0.02),
    ((37, 29), 131, 3, 5e-2, 0.05),
    ((100, 3), 2, 1, 1e-1, 0.3),
    ((9, 7, 5), 3, 2, 2e-2, 0.02),
    ((13, 11, 6), 40, 4, 5e-2, 0.05),
    ((31, 17), 260, 7, 5e-2, 0.01),
    ((1, 1), 5, 2, 1e-1, 0.5),
]


@pytest.mark.parametrize("shape,N,d,eps,scale", CASES)
def test_objective_grad_fp64(shape, N, d, eps, scale):
    g = O.Grid(shape)
    lab = synth.random_labels(11, g.P, N)
    th = synth.random_theta(12, N, O.K(len(shape), d), scale)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = gpu_eval(shape, lab, N, th, d, eps, pd.PD_FP64)
    assert abs(phi - phi_o) <= 1e-10 * abs(phi_o)
    assert rel(grad, grad_o) <= 1e-10


@pytest.mark.parametrize("shape,N,d,eps,scale", CASES)
def test_objective_grad_fp32(shape, N, d, eps, scale):
    g = O.Grid(shape)
    lab = synth.random_labels(13, g.P, N)
    th = synth.random_theta(14, N, O.K(len(shape), d), scale)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = gpu_eval(shape, lab, N, th, d, eps, pd.PD_FP32)
    print("fp32 %s N=%d d=%d: phi %.2e grad %.2e" % (shape, N, d, abs(phi - phi_o) / abs(phi_o), rel(grad, grad_o)))
    assert abs(phi - phi_o) <= 1e-5 * abs(phi_o)
    assert rel(grad, grad_o) <= 1e-5


def test_fully_ambiguous_exact():
    # theta = 0: Phi = -log N (Sec. 2.1), in both precisions
    shape, N = (50, 41), 300
    lab = synth.random_labels(3, 50 * 41, N)
    for prec, tol in ((pd.PD_FP64, 1e-15), (pd.PD_FP32, 1e-7)):
        phi, grad = gpu_eval(shape, lab, N, np.zeros((N, 6)), 2, 1e-2, prec)
        assert abs(phi + math.log(N)) <= tol * math.log(N)


def test_structured_grid_equals_point_list():
    shape, N, d = (23, 19), 17, 3
    g = O.Grid(shape)
    lab = synth.random_labels(5, g.P, N)
    th = synth.random_theta(6, N, O.K(2, d), 0.1)
    xs = -1.0 + (2.0 * np.arange(shape[0]) + 1.0) / shape[0]
    ys = -1.0 + (2.0 * np.arange(shape[1]) + 1.0) / shape[1]
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    pts = np.stack([X.reshape(-1), Y.reshape(-1)], 1)
    a = gpu_eval(shape, lab, N, th, d, 0.05, pd.PD_FP64)
    b = gpu_eval(pts, lab, N, th, d, 0.05, pd.PD_FP64)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_bitwise_reproducible():
    shape, N, d = (200, 150), 300, 4
    lab = synth.random_labels(8, 200 * 150, N)
    th = synth.random_theta(9, N, O.K(2, d), 0.05)
    for prec in (pd.PD_FP64, pd.PD_FP32):
        r1 = gpu_eval(shape, lab, N, th, d, 1e-2, prec)
        r2 = gpu_eval(shape, lab, N, th, d, 1e-2, prec)
        assert r1[0] == r2[0]
        np.testing.assert_array_equal(r1[1], r2[1])


@pytest.mark.parametrize("shape,N,d,eps,scale", CASES[:5])
def test_hvp(shape, N, d, eps, scale):
    g = O.Grid(shape)
    lab = synth.random_labels(15, g.P, N)
    K = O.K(len(shape), d)
    th = synth.random_theta(16, N, K, scale)
    v = synth.random_theta(17, N, K, 1.0)
    hv_o = O.hvp(g, lab, N, d, eps, th, v)
    grid = pd.Grid(shape)
    for prec, tol in ((pd.PD_FP64, 1e-10), (pd.PD_FP32, 1e-5)):
        hv = pd.pd_hvp(grid, dev(lab), N, dev(th), dev(v), d, eps, prec=prec).cpu().numpy()
        print("hvp prec %d %s: %.2e" % (prec, shape, rel(hv, hv_o)))
        assert rel(hv, hv_o) <= tol, (prec, rel(hv, hv_o))


@pytest.mark.parametrize("shape,N,d", [((64, 64), 8, 2), ((57, 43), 200, 4), ((11, 9, 7), 30, 3),
                                        ((5, 1), 3, 1), ((40, 30), 150, 7)])
def test_assign(shape, N, d):
    g = O.Grid(shape)
    th = synth.random_theta(21, N, O.K(len(shape), d), 1.0)
    th[1] = th[0]  # an exact duplicate: ties must go to the smaller index
    lab_o, gap_o = O.assign(g, N, d, th)
    ref = synth.random_labels(22, g.P, N)
    lab, gap, mis = pd.pd_assign(pd.Grid(shape), N, d, dev(th), want_gap=True, ref_labels=dev(ref))
    lab, gap = lab.cpu().numpy(), gap.cpu().numpy()
    sure = gap_o >= 1e-9
    np.testing.assert_array_equal(lab[sure], lab_o[sure])
    assert np.all(lab != 1)
    np.testing.assert_allclose(gap, gap_o, rtol=0, atol=1e-10 * max(1.0, np.abs(gap_o).max()))
    assert int(mis.item()) == int(np.sum(lab != ref))


@pytest.mark.parametrize("shape,d,prec", [((17, 13), 5, "fp64"), ((6, 5, 4), 3, "fp64"), ((17, 13), 7, "fp32"),
                                           ((9, 8, 7), 4, "fp32")])
def test_features(shape, d, prec):
    eta_o = O.features(O.Grid(shape), d)
    eta = pd.pd_features(pd.Grid(shape), d, pd.PREC[prec]).double().cpu().numpy()
    tol = 1e-14 if prec == "fp64" else 2e-6
    np.testing.assert_allclose(eta, eta_o, rtol=0, atol=tol)


@pytest.mark.parametrize("shape,N,dm", [((64, 48), 9, 2), ((30, 20, 10), 12, 4), ((100, 100), 40, 4)])
def test_moments(shape, N, dm):
    g, lab, N = power_problem(shape, N, seed=4)
    mom_o, cnt_o = O.grain_moments(g, lab, N, dm)
    mom, cnt = pd.pd_moments(pd.Grid(shape), dev(lab), N, dm)
    np.testing.assert_array_equal(cnt.cpu().numpy(), cnt_o)
    np.testing.assert_allclose(mom.cpu().numpy(), mom_o, rtol=0, atol=1e-9 * g.P)


@pytest.mark.parametrize("shape,N,d", [((64, 64), 12, 1), ((64, 64), 12, 2), ((24, 20, 16), 10, 2)])
def test_heuristic_init(shape, N, d):
    g, lab, N = power_problem(shape, N, seed=9)
    th_o = O.heuristic_theta(g, lab, N, d)
    th = pd.pd_heuristic_init(pd.Grid(shape), dev(lab), N, d).cpu().numpy()
    # fixed-point moments and the E[xx] - yy form differ from the oracle's
    # two-pass moments by rounding only
    np.testing.assert_allclose(th, th_o, rtol=1e-6, atol=1e-8 * np.abs(th_o).max())


def test_theta_from_apd_matches_oracle():
    for dim, d in ((2, 2), (2, 5), (3, 2), (3, 4)):
        y, w, A = synth.apd_params(30 + d, 7, dim=dim)
        np.testing.assert_allclose(pd.pd_theta_from_apd(dim, d, y, w, A).numpy(),
                                   O.theta_from_apd(dim, d, y, w, A), rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(pd.pd_theta_from_apd(dim, d, y, w).numpy(),
                                   O.theta_from_apd(dim, d, y, w), rtol=1e-13, atol=1e-13)


def test_errors_and_edge_cases():
    grid = pd.Grid((8, 8))
    lab = torch.zeros(64, dtype=torch.int32, device="cuda")
    th = torch.zeros((3, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PdError) as e:
        pd.pd_objective_grad(grid, lab, 1, th[:1], 2, 0.1)           # N < 2
    assert e.value.code == pd.PD_EINVAL
    with pytest.raises(pd.PdError) as e:
        pd.pd_objective_grad(grid, lab, 3, th, 2, 0.0)               # eps <= 0
    assert e.value.code == pd.PD_EINVAL
    with pytest.raises(pd.PdError) as e:
        pd.pd_objective_grad(grid, lab, 3, torch.zeros((3, 45), dtype=torch.float64, device="cuda"), 8, 0.1)
    assert e.value.code == pd.PD_ENOTSUP
    bad = lab.clone()
    bad[17] = 3
    assert pd.pd_check_labels(grid, bad, 3) == pd.PD_ELABEL
    assert pd.pd_check_labels(grid, lab, 3) == pd.PD_OK
    # empty pixel set: assignment and features are no-ops
    empty = pd.Grid(coords=torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
    l0, _, mis = pd.pd_assign(empty, 3, 2, th, ref_labels=torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert l0.numel() == 0 and int(mis.item()) == 0
    # a single pixel
    one = pd.Grid((1, 1))
    obj, grad = pd.pd_objective_grad(one, lab[:1], 3, th, 2, 0.1)
    assert abs(obj.item() + math.log(3)) < 1e-15


@pytest.mark.slow
def test_config2_full_size_fp32_and_fp64():
    # 1024 x 1024, N = 500 degree-4 diagram with 2% boundary noise, fit
    # degree 4 (K = 15), eps = 1e-3: one evaluation at the generating theta
    shape, d, eps = (1024, 1024), 4, 1e-3
    g, lab, N, th = poly_problem(shape, 500, d, seed=synth.SEED_BASE + 1, noise=0.02)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi64, grad64 = gpu_eval(shape, lab, N, th, d, eps, pd.PD_FP64)
    assert abs(phi64 - phi_o) <= 1e-10 * abs(phi_o)
    assert rel(grad64, grad_o) <= 1e-10
    phi32, grad32 = gpu_eval(shape, lab, N, th, d, eps, pd.PD_FP32)
    print("config2 fp32 rel err: phi %.3e grad %.3e" % (abs(phi32 - phi_o) / abs(phi_o), rel(grad32, grad_o)))
    assert abs(phi32 - phi_o) <= 1e-5 * abs(phi_o)
    assert rel(grad32, grad_o) <= 1e-5


@pytest.mark.parametrize("shape,N,d,scale", [((64, 64), 8, 2, 1.0), ((57, 43), 200, 4, 1.0), ((11, 9, 7), 30, 3, 1.0),
                                             ((40, 30), 150, 7, 1.0), ((200, 190), 300, 4, 0.01),
                                             ((20, 20), 40, 2, 0.0)])
def test_assign_fast_path_equals_double(shape, N, d, scale, monkeypatch):
    # labels without the gap take the fp32 pass with a certified margin and
    # double precision only where the margin is not met: every label must
    # equal the double-precision kernel's, ties (a duplicate grain, theta = 0)
    # included, and so must the mismatch count
    th = synth.random_theta(23, N, O.K(len(shape), d), scale)
    if N > 2:
        th[2] = th[1]
    g = O.Grid(shape)
    ref = synth.random_labels(24, g.P, N)
    grid = pd.Grid(shape)
    lab, _, mis = pd.pd_assign(grid, N, d, dev(th), ref_labels=dev(ref))
    monkeypatch.setenv("PD_ASSIGN_FP64", "1")
    lab64, _, mis64 = pd.pd_assign(grid, N, d, dev(th), ref_labels=dev(ref))
    monkeypatch.delenv("PD_ASSIGN_FP64")
    np.testing.assert_array_equal(lab.cpu().numpy(), lab64.cpu().numpy())
    assert int(mis.item()) == int(mis64.item())
    lab_o, gap_o = O.assign(g, N, d, th)
    sure = gap_o >= 1e-9
    np.testing.assert_array_equal(lab.cpu().numpy()[sure], lab_o[sure])


@pytest.mark.slow
def test_assign_fast_path_config2_full_size(monkeypatch):
    # 1024 x 1024, N = 485 degree-4 diagram: the fast assignment against the
    # double-precision kernel on every pixel, and its time
    shape, d = (1024, 1024), 4
    g, lab_ref, N, th = poly_problem(shape, 500, d, seed=synth.SEED_BASE + 1, noise=0.02)
    grid, dth, dref = pd.Grid(shape), dev(th), dev(lab_ref)
    lab, _, mis = pd.pd_assign(grid, N, d, dth, ref_labels=dref)
    monkeypatch.setenv("PD_ASSIGN_FP64", "1")
    lab64, _, mis64 = pd.pd_assign(grid, N, d, dth, ref_labels=dref)
    monkeypatch.delenv("PD_ASSIGN_FP64")
    assert torch.equal(lab, lab64)
    assert int(mis.item()) == int(mis64.item())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        pd.pd_assign(grid, N, d, dth, ref_labels=dref)
    e1.record()
    torch.cuda.synchronize()
    print("config2 fast assignment: %.3f ms, mismatch %d" % (e0.elapsed_time(e1) / 5, int(mis.item())))
