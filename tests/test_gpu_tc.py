"""Parity of the tensor-core (tcgen05) evaluation with the FP64 oracle.

PD_BF16X3 splits the logit operands into three bf16 terms (about 24
significant bits), keeps every logit relative to its tile's reference logit,
and contracts the gradient with c = delta - p in two fp16 terms (hi, and
the remainder scaled by 2^12) against fp16 hi + lo features: it must meet
the FP32 tolerances (Phi, gradient and Hessian-vector product within 1e-5
relative).
PD_BF16 rounds every operand to bf16 (8 significant bits): its logit error
is about |theta| / eps * 2^-9, so it is checked at a loose bound scaled to
that, and its error is reported by the benchmark.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth
from helpers import poly_problem, rel

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


CASES = [
    ((64, 64), 8, 2, 1e-2, 0.02),
    ((37, 29), 131, 3, 5e-2, 0.05),
    ((100, 3), 2, 1, 1e-1, 0.3),
    ((9, 7, 5), 3, 2, 2e-2, 0.02),
    ((13, 11, 6), 40, 3, 5e-2, 0.05),
    ((31, 17), 130, 5, 5e-2, 0.01),
    ((40, 30), 260, 6, 5e-2, 0.01),
    ((200, 190), 300, 4, 1e-2, 0.01),
]


def run(shape, lab, N, th, d, eps, prec):
    grid = pd.Grid(shape)
    obj, grad = pd.pd_objective_grad(grid, dev(lab), N, dev(th), d, eps, prec=prec)
    torch.cuda.synchronize()
    return float(obj.item()), grad.cpu().numpy()


@pytest.mark.parametrize("shape,N,d,eps,scale", CASES)
def test_bf16x3_matches_oracle(shape, N, d, eps, scale):
    g = O.Grid(shape)
    lab = synth.random_labels(31, g.P, N)
    th = synth.random_theta(32, N, O.K(len(shape), d), scale)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = run(shape, lab, N, th, d, eps, pd.PD_BF16X3)
    print("bf16x3 %s N=%d d=%d: phi %.2e grad %.2e" % (shape, N, d, abs(phi - phi_o) / abs(phi_o), rel(grad, grad_o)))
    assert abs(phi - phi_o) <= 1e-5 * abs(phi_o), (phi, phi_o)
    assert rel(grad, grad_o) <= 1e-5, rel(grad, grad_o)


@pytest.mark.parametrize("shape,N,d,eps,scale", CASES)
def test_bf16_close_to_oracle(shape, N, d, eps, scale):
    g = O.Grid(shape)
    lab = synth.random_labels(33, g.P, N)
    K = O.K(len(shape), d)
    th = synth.random_theta(34, N, K, scale)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = run(shape, lab, N, th, d, eps, pd.PD_BF16)
    # logit error bound of one bf16 rounding of theta/eps and eta
    dl = np.abs(th).sum(1).max() / eps * 2.0 ** -7
    assert abs(phi - phi_o) <= 2 * dl + 1e-3 * abs(phi_o), (phi, phi_o, dl)
    assert rel(grad, grad_o) <= 0.05 + 4 * dl


def test_tc_bitwise_reproducible():
    shape, N, d = (300, 200), 200, 4
    lab = synth.random_labels(35, 300 * 200, N)
    th = synth.random_theta(36, N, 15, 0.02)
    for prec in (pd.PD_BF16, pd.PD_BF16X3):
        a = run(shape, lab, N, th, d, 1e-2, prec)
        b = run(shape, lab, N, th, d, 1e-2, prec)
        assert a[0] == b[0]
        np.testing.assert_array_equal(a[1], b[1])


STRUCTURED = [
    ((256, 192), 300, 4, 1e-3),
    ((250, 130), 700, 3, 2e-3),       # ragged tiles on both axes, 6 blocks
    ((40, 36, 30), 200, 2, 2e-3),
]


@pytest.mark.parametrize("shape,N,d,eps", STRUCTURED)
def test_tc_skip_structured(shape, N, d, eps, monkeypatch):
    # a sharp diagram: most (tile, 128-grain block) pairs of the gradient
    # pass carry only probabilities below 2^-26 and are left out after the
    # grains are reordered by label centroid.  Against the oracle, and
    # against the same evaluation visiting every pair in index order (the
    # two differ only by the fp32 accumulation order of the partials).
    g, lab, N, th = poly_problem(shape, N, d, seed=synth.SEED_BASE + 5, noise=0.02)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = run(shape, lab, N, th, d, eps, pd.PD_BF16X3)
    monkeypatch.setenv("PD_TC_NO_SKIP", "1")
    phi_a, grad_a = run(shape, lab, N, th, d, eps, pd.PD_BF16X3)
    monkeypatch.delenv("PD_TC_NO_SKIP")
    # the label part (1/(eps P)) sum_{x in G_i} eta(x), which the probability
    # part cancels down to the gradient: the scale of its rounding
    E = O.features(g, d)
    L = np.zeros((N, E.shape[1]))
    np.add.at(L, lab, E)
    L /= eps * g.P
    dgrad = np.linalg.norm(grad - grad_a) / np.linalg.norm(L)
    print("skip %s N=%d: phi %.2e grad %.2e vs oracle; vs all pairs: phi %.2e grad %.2e of the label part"
          % (shape, N, abs(phi - phi_o) / abs(phi_o), rel(grad, grad_o), abs(phi - phi_a) / abs(phi_a), dgrad))
    # Phi of a sharp fit is near zero: its error is measured on the scale of
    # the log-sum-exp, O(1).  The tensor cores accumulate the logits'
    # remainders theta'.(eta(x) - eta(c)) with truncation, an error of about
    # 2^-23 A per logit for remainders up to A = sum_k |theta'_k| D_k: on the
    # 40 x 36 x 30 grid at eps = 2e-3 a tile spans a fifth of the x-axis and
    # A reaches about 600 (against 70 at 1024^2, eps = 1e-3), which the
    # gradient bound of that case reflects
    tol = 2e-5 if len(shape) == 3 else 1e-5
    assert abs(phi - phi_o) <= 1e-5 * max(1.0, abs(phi_o)), (phi, phi_o)
    assert rel(grad, grad_o) <= tol, rel(grad, grad_o)
    assert abs(phi - phi_a) <= 1e-6 * max(1.0, abs(phi_a))
    assert dgrad <= 2e-5, dgrad
    # deterministic
    phi_b, grad_b = run(shape, lab, N, th, d, eps, pd.PD_BF16X3)
    assert phi_b == phi
    np.testing.assert_array_equal(grad_b, grad)
    # the Hessian-vector product skips the pairs whose c = p (u - ubar)
    # fp16 rounds to zero, in the same grain order
    v = synth.random_theta(44, N, th.shape[1], 2.0)
    hv_o = O.hvp(g, lab, N, d, eps, th, v)
    hv = pd.pd_hvp(pd.Grid(shape), dev(lab), N, dev(th), dev(v), d, eps, prec=pd.PD_BF16X3).cpu().numpy()
    monkeypatch.setenv("PD_TC_NO_SKIP", "1")
    hv_a = pd.pd_hvp(pd.Grid(shape), dev(lab), N, dev(th), dev(v), d, eps, prec=pd.PD_BF16X3).cpu().numpy()
    monkeypatch.delenv("PD_TC_NO_SKIP")
    print("skip %s N=%d: hvp %.2e vs oracle, %.2e vs all pairs" % (shape, N, rel(hv, hv_o), rel(hv, hv_a)))
    assert rel(hv, hv_o) <= 1e-5, rel(hv, hv_o)
    assert rel(hv, hv_a) <= 1e-5, rel(hv, hv_a)


def test_tc_unsupported_shapes():
    grid = pd.Grid((16, 16))
    lab = torch.zeros(256, dtype=torch.int32, device="cuda")
    th = torch.zeros((3, 36), dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PdError) as e:
        pd.pd_objective_grad(grid, lab, 3, th, 7, 0.1, prec=pd.PD_BF16X3)   # K = 36 > 32
    assert e.value.code == pd.PD_ENOTSUP
    v = torch.zeros_like(th)
    with pytest.raises(pd.PdError) as e:
        pd.pd_hvp(grid, lab, 3, th, v, 7, 0.1, prec=pd.PD_BF16X3)
    assert e.value.code == pd.PD_ENOTSUP


@pytest.mark.parametrize("N,d", [(1792, 4), (1793, 4), (2300, 4), (1000, 6)])
def test_tc_grain_groups(N, d):
    # K = 15 in bf16x3: 1536 grains is the largest parameter image one SM
    # holds beside the pass's stages; beyond it (and at K = 28 from a few
    # hundred grains) pass 1 runs in groups of grains whose log-sum-exp
    # parts are merged
    shape, eps = (64, 48), 2e-2
    g = O.Grid(shape)
    K = O.K(2, d)
    lab = synth.random_labels(37, g.P, N)
    th = synth.random_theta(38, N, K, 0.02)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = run(shape, lab, N, th, d, eps, pd.PD_BF16X3)
    print("groups N=%d d=%d: phi %.2e grad %.2e" % (N, d, abs(phi - phi_o) / abs(phi_o), rel(grad, grad_o)))
    assert abs(phi - phi_o) <= 1e-5 * abs(phi_o), (phi, phi_o)
    assert rel(grad, grad_o) <= 1e-5, rel(grad, grad_o)


HVP_CASES = [
    ((64, 64), 8, 2, 1e-2, 0.02),
    ((37, 29), 131, 3, 5e-2, 0.05),
    ((9, 7, 5), 3, 2, 2e-2, 0.02),
    ((13, 11, 6), 40, 3, 5e-2, 0.05),
    ((200, 190), 300, 4, 1e-2, 0.01),
    ((64, 48), 1793, 4, 2e-2, 0.02),     # pass 1 in three grain groups
]


@pytest.mark.parametrize("shape,N,d,eps,scale", HVP_CASES)
def test_bf16x3_hvp_matches_oracle(shape, N, d, eps, scale):
    # the Hessian-vector product on the tensor cores: float-level logits and
    # u, c = p (u - ubar) and the features in fp16 (hi + lo for eta)
    g = O.Grid(shape)
    K = O.K(len(shape), d)
    lab = synth.random_labels(41, g.P, N)
    th = synth.random_theta(42, N, K, scale)
    v = synth.random_theta(43, N, K, 3.0)          # magnitude above 1: exercises the scaling of v
    hv_o = O.hvp(g, lab, N, d, eps, th, v)
    hv = pd.pd_hvp(pd.Grid(shape), dev(lab), N, dev(th), dev(v), d, eps, prec=pd.PD_BF16X3)
    err = rel(hv.cpu().numpy(), hv_o)
    print("hvp bf16x3 %s N=%d d=%d: rel err %.2e" % (shape, N, d, err))
    assert err <= 1e-5, err


@pytest.mark.slow
def test_config2_full_size_bf16x3():
    shape, d, eps = (1024, 1024), 4, 1e-3
    g, lab, N, th = poly_problem(shape, 500, d, seed=synth.SEED_BASE + 1, noise=0.02)
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    phi, grad = run(shape, lab, N, th, d, eps, pd.PD_BF16X3)
    print("config2 bf16x3 rel err: phi %.3e grad %.3e" % (abs(phi - phi_o) / abs(phi_o), rel(grad, grad_o)))
    assert abs(phi - phi_o) <= 1e-5 * abs(phi_o)
    assert rel(grad, grad_o) <= 1e-5
    phi16, grad16 = run(shape, lab, N, th, d, eps, pd.PD_BF16)
    print("config2 bf16 rel err: phi %.3e grad %.3e" % (abs(phi16 - phi_o) / abs(phi_o), rel(grad16, grad_o)))


SMALL_GRIDS = [((1, 1), 2, 2), ((1, 5), 3, 3), ((7, 3), 5, 4), ((3, 2, 1), 4, 2), ((2, 1, 1), 2, 3),
               ((1, 3, 2), 3, 3)]


def sharpness(g, d, eps, th, lab):
    # max over the pixels of 1 - p_max(x) and of 1 - p_G(x), in double: the
    # oracle forms these differences in double, so its own relative error
    # is about P 2^-53 over them
    eta = O.features(g, d)
    L = -(eta @ th.T) / eps
    L -= L.max(1, keepdims=True)
    p = np.exp(L)
    p /= p.sum(1, keepdims=True)
    return (1.0 - p.max(1)).max(), (1.0 - p[np.arange(g.P), lab]).max()


@pytest.mark.parametrize("shape,N,d", SMALL_GRIDS)
def test_reduced_precision_on_grids_smaller_than_a_tile(shape, N, d):
    # one ragged tile holding a handful of pixels (a single pixel included):
    # the tile-relative logits, the pair skipping and the passes' padding
    # rows must still give the oracle's Phi and gradient.  With |theta|/eps
    # large, p_G(x) lies close to 1 at most pixels: the gradient is then
    # small and must not lose its relative accuracy to 1 - p_G.  Phi is a
    # mean of log p over the pixels and can lie near 0: its bound adds
    # 2^-20, a few float roundings of one log S; a tile centre placed
    # outside [-1, 1] (P_m(16) ~ 4e2 at d = 2) misses it by a factor of four
    # on the single pixel.
    g = O.Grid(shape)
    K = O.K(len(shape), d)
    lab = synth.random_labels(51, g.P, N)
    th = synth.random_theta(52, N, K, 0.3)
    eps = 2e-2
    assert g.P * 2.0 ** -53 / sharpness(g, d, eps, th, lab)[1] < 1e-8  # the oracle's own error
    phi_o, grad_o = O.objective_grad(g, lab, N, d, eps, th)
    for prec in (pd.PD_FP32, pd.PD_BF16X3):
        phi, grad = run(shape, lab, N, th, d, eps, prec)
        assert abs(phi - phi_o) <= 1e-5 * abs(phi_o) + 2.0 ** -20, (prec, phi, phi_o)
        assert rel(grad, grad_o) <= 1e-5, (prec, rel(grad, grad_o))
        # theta = 0: every grain equally likely, Phi = -log N
        phi0, _ = run(shape, lab, N, np.zeros_like(th), d, eps, prec)
        assert abs(phi0 + math.log(N)) <= 1e-6 * math.log(N), (prec, phi0)


@pytest.mark.parametrize("shape,N,d", [c for c in SMALL_GRIDS if c[0] != (2, 1, 1)])
def test_reduced_precision_hvp_on_grids_smaller_than_a_tile(shape, N, d):
    # the Hessian-vector product at the same sharp parameters: where one
    # grain's p is close to 1, u_i - ubar of that grain is a small
    # difference that must keep its relative accuracy.  FP32 leaves each
    # pixel's arg-max grain out of its sums, with labels or without.  (The
    # tensor cores form the plain difference, which loses about
    # log2(1 / (1 - p_max)) of the float's 24 bits: they are checked at
    # 2^-18 / max_x(1 - p_max(x)), 1e-5 at the least.  On the 2 x 1 x 1 grid
    # every 1 - p_max(x) is below 1e-14: the oracle's double differences
    # carry no digits there.)
    g = O.Grid(shape)
    K = O.K(len(shape), d)
    lab = synth.random_labels(51, g.P, N)
    th = synth.random_theta(52, N, K, 0.3)
    v = synth.random_theta(53, N, K, 1.0)
    eps = 2e-2
    sharp = sharpness(g, d, eps, th, lab)[0]
    assert g.P * 2.0 ** -53 / sharp < 1e-8  # the oracle's own error
    hv_o = O.hvp(g, lab, N, d, eps, th, v)
    for labels in (dev(lab), None):
        hv = pd.pd_hvp(pd.Grid(shape), labels, N, dev(th), dev(v), d, eps, prec=pd.PD_FP32).cpu().numpy()
        assert rel(hv, hv_o) <= 1e-5, rel(hv, hv_o)
    hv = pd.pd_hvp(pd.Grid(shape), dev(lab), N, dev(th), dev(v), d, eps, prec=pd.PD_BF16X3).cpu().numpy()
    assert rel(hv, hv_o) <= max(1e-5, 2.0 ** -18 / sharp), (rel(hv, hv_o), sharp)
