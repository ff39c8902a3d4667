"""Pins of the oracle's objective and gradient (Sec. 2.2 and Sec. 4)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy.special import expit, logsumexp

from paper_2605_20816_gb300 import synth


def problem(oracle, shape=(11, 9), N=5, d=2, seed=0, scale=1.0):
    g = oracle.Grid(shape)
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, N, g.P).astype(np.int32)
    th = scale * rng.standard_normal((N, oracle.K(len(shape), d)))
    return g, lab, th


def np_features(shape, d, oracle):
    # independent design matrix via numpy's Legendre series evaluation
    axes = [-1.0 + (2.0 * np.arange(n) + 1.0) / n for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([m.transpose(tuple(range(len(shape)))[::-1]).reshape(-1) for m in mesh], 1)
    a = oracle.alpha(len(shape), d)
    cols = []
    for al in a:
        v = np.ones(pts.shape[0])
        for ax, e in enumerate(al):
            c = np.zeros(e + 1); c[e] = 1.0
            v = v * npleg.legval(pts[:, ax], c)
        cols.append(v)
    return np.stack(cols, 1)


def test_fully_ambiguous_value(oracle):
    # theta = 0 gives p = 1/N everywhere (Sec. 2.1), hence Phi = -log N exactly
    for N in (2, 3, 8, 50):
        g = oracle.Grid((9, 7))
        lab = np.arange(g.P, dtype=np.int32) % N
        phi, _ = oracle.objective_grad(g, lab, N, 2, 0.01, np.zeros((N, 6)))
        assert abs(phi - (-math.log(N))) < 4e-16 * math.log(N) + 1e-16


def test_gradient_at_zero_closed_form(oracle):
    # eq. (grad) at theta = 0: -(1/(eps|Omega|)) (sum_{x in G_i} eta - (1/N) sum_x eta)
    shape, N, d, eps = (10, 8), 4, 3, 0.02
    g = oracle.Grid(shape)
    lab = (np.arange(g.P) * 7 % N).astype(np.int32)
    eta = np_features(shape, d, oracle)
    _, grad = oracle.objective_grad(g, lab, N, d, eps, np.zeros((N, eta.shape[1])))
    tot = eta.sum(0)
    for i in range(N):
        want = -(eta[lab == i].sum(0) - tot / N) / (eps * g.P)
        np.testing.assert_allclose(grad[i], want, rtol=1e-13, atol=1e-12)


def test_brute_force_logsumexp(oracle):
    shape, N, d, eps = (6, 5), 4, 2, 0.3
    g, lab, th = problem(oracle, shape, N, d, seed=1)
    eta = np_features(shape, d, oracle)
    L = -(eta @ th.T) / eps
    lse = logsumexp(L, axis=1)
    phi_want = np.mean(L[np.arange(g.P), lab] - lse)
    P = np.exp(L - lse[:, None])
    Y = np.eye(N)[lab]
    grad_want = -((Y - P).T @ eta) / (eps * g.P)
    phi, grad = oracle.objective_grad(g, lab, N, d, eps, th)
    assert abs(phi - phi_want) < 1e-13 * abs(phi_want)
    np.testing.assert_allclose(grad, grad_want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_finite_differences(oracle, dim):
    shape = (7, 6) if dim == 2 else (4, 3, 5)
    N, d, eps = 3, 2, 0.5
    g, lab, th = problem(oracle, shape, N, d, seed=2, scale=0.5)
    _, grad = oracle.objective_grad(g, lab, N, d, eps, th)
    h = 1e-5
    fd = np.zeros_like(th)
    for i in range(N):
        for k in range(th.shape[1]):
            tp, tm = th.copy(), th.copy()
            tp[i, k] += h; tm[i, k] -= h
            fd[i, k] = (oracle.objective_grad(g, lab, N, d, eps, tp, want_grad=False)
                        - oracle.objective_grad(g, lab, N, d, eps, tm, want_grad=False)) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-7, atol=1e-8)


def test_gauge_invariance(oracle):
    # Lemma 4.2: adding the same c to every theta_i changes nothing
    g, lab, th = problem(oracle, (9, 8), 6, 3, seed=4)
    c = np.random.default_rng(9).standard_normal(th.shape[1])
    p0, g0 = oracle.objective_grad(g, lab, 6, 3, 0.1, th)
    p1, g1 = oracle.objective_grad(g, lab, 6, 3, 0.1, th + c)
    assert abs(p0 - p1) < 1e-13 * abs(p0)
    np.testing.assert_allclose(g0, g1, rtol=1e-9, atol=1e-11)
    l0, gap = oracle.assign(g, 6, 3, th)
    l1, _ = oracle.assign(g, 6, 3, th + c)
    sure = gap > 1e-9
    np.testing.assert_array_equal(l0[sure], l1[sure])
    # gradient sums to zero over grains (the gauge direction is flat)
    _, gr = oracle.objective_grad(g, lab, 6, 3, 0.1, th)
    assert np.abs(gr.sum(0)).max() < 1e-10 * np.abs(gr).max()


def test_eps_scaling(oracle):
    # Lemma 4.1: Phi_eps(theta) = Phi_1(theta / eps); F_{lambda theta} = F_theta
    g, lab, th = problem(oracle, (8, 8), 4, 2, seed=5, scale=0.05)
    for eps in (1e-3, 0.02, 3.0):
        a = oracle.objective_grad(g, lab, 4, 2, eps, th, want_grad=False)
        b = oracle.objective_grad(g, lab, 4, 2, 1.0, th / eps, want_grad=False)
        assert abs(a - b) < 1e-12 * abs(a)
    l0, gap = oracle.assign(g, 4, 2, th)
    l1, _ = oracle.assign(g, 4, 2, 17.0 * th)
    sure = gap > 1e-9
    np.testing.assert_array_equal(l0[sure], l1[sure])


def test_eps_to_zero_bound(oracle):
    # Prop. 4.7: 0 <= -eps Phi_eps - E_0 <= eps log N
    shape, N, d = (10, 9), 6, 2
    g, lab, th = problem(oracle, shape, N, d, seed=6)
    eta = np_features(shape, d, oracle)
    h = eta @ th.T
    E0 = np.mean(h[np.arange(g.P), lab] - h.min(1))
    for eps in (1e-3, 1e-2, 0.3, 5.0):
        phi = oracle.objective_grad(g, lab, N, d, eps, th, want_grad=False)
        gapv = -eps * phi - E0
        assert -1e-12 <= gapv <= eps * math.log(N) + 1e-12


def test_negative_and_misassignment_penalty(oracle):
    # Prop. 4.8: Phi < 0 for finite theta; Lemma 4.9: Phi <= -(log 2) Err
    for seed in range(5):
        g, lab, th = problem(oracle, (9, 9), 5, 2, seed=seed)
        for eps in (0.01, 0.3):
            phi = oracle.objective_grad(g, lab, 5, 2, eps, th, want_grad=False)
            F, _ = oracle.assign(g, 5, 2, th)
            err = np.mean(F != lab)
            assert phi < 0.0
            assert phi <= -math.log(2.0) * err + 1e-15


def test_two_grains_is_binary_logistic(oracle):
    # N = 2: log p_{G(x)} = log sigma(+-(h_1 - h_0)/eps), the textbook
    # binary logistic log-likelihood with weight theta_1 - theta_0
    shape, d, eps = (7, 7), 2, 0.2
    g, lab, th = problem(oracle, shape, 2, d, seed=8)
    eta = np_features(shape, d, oracle)
    z = eta @ (th[1] - th[0]) / eps          # = l_0 - l_1
    s = np.where(lab == 0, z, -z)
    want = np.mean(np.log(expit(s)))
    got = oracle.objective_grad(g, lab, 2, d, eps, th, want_grad=False)
    assert abs(got - want) < 1e-13 * abs(want)


def test_concavity_along_lines(oracle):
    # concavity (Prop. 4.4): Phi(mid) >= mean of endpoint values
    g, lab, th = problem(oracle, (9, 7), 4, 2, seed=10)
    th2 = np.random.default_rng(11).standard_normal(th.shape)
    for t in (0.25, 0.5, 0.75):
        f = lambda x: oracle.objective_grad(g, lab, 4, 2, 0.2, x, want_grad=False)
        assert f((1 - t) * th + t * th2) >= (1 - t) * f(th) + t * f(th2) - 1e-14


def test_invalid_labels_rejected(oracle):
    g = oracle.Grid((4, 4))
    lab = np.zeros(16, dtype=np.int32)
    lab[3] = 5
    with pytest.raises(ValueError):
        oracle.objective_grad(g, lab, 3, 1, 0.1, np.zeros((3, 3)))


def test_point_list_objective_matches_grid(oracle):
    shape = (8, 6)
    g, lab, th = problem(oracle, shape, 4, 3, seed=12)
    axes = [-1.0 + (2.0 * np.arange(n) + 1.0) / n for n in shape]
    xs, ys = np.meshgrid(axes[0], axes[1], indexing="xy")
    gl = oracle.Grid(coords=np.stack([xs.reshape(-1), ys.reshape(-1)], 1))
    a = oracle.objective_grad(g, lab, 4, 3, 0.1, th)
    b = oracle.objective_grad(gl, lab, 4, 3, 0.1, th)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])


def test_pixel_terms_sum_to_objective(oracle):
    g, lab, th = problem(oracle, (9, 6), 5, 2, seed=13)
    r, lse = oracle.pixel_terms(g, lab, 5, 2, 0.05, th, np.arange(g.P))
    phi = oracle.objective_grad(g, lab, 5, 2, 0.05, th, want_grad=False)
    assert abs(np.mean(r) - phi) < 1e-13 * abs(phi)
