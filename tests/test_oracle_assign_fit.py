"""Pins of the oracle's arg-min assignment, parameter conversions,
initialisation and ascent scheme (Sec. 2.1, 2.3, 4, 5.2, 5.5)."""
import math

import numpy as np
import pytest
import scipy.optimize as so

from paper_2605_20816_gb300 import synth


def centres_2d(shape):
    n1, n2 = shape
    xs, ys = np.meshgrid(-1.0 + (2.0 * np.arange(n1) + 1.0) / n1,
                         -1.0 + (2.0 * np.arange(n2) + 1.0) / n2, indexing="xy")
    return np.stack([xs.reshape(-1), ys.reshape(-1)], 1)


def test_assign_brute_force(oracle):
    g = oracle.Grid((13, 11))
    rng = np.random.default_rng(0)
    N, d = 7, 3
    th = rng.standard_normal((N, oracle.K(2, d)))
    eta = oracle.features(g, d)
    h = eta @ th.T
    lab, gap = oracle.assign(g, N, d, th)
    np.testing.assert_array_equal(lab, np.argmin(h, axis=1))  # first minimum
    hs = np.sort(h, axis=1)
    np.testing.assert_allclose(gap, hs[:, 1] - hs[:, 0], rtol=0, atol=1e-12)


def test_assign_ties_go_to_smallest_index(oracle):
    # eq. (Li_def): a tie is assigned to the smallest index
    g = oracle.Grid((9, 9))
    rng = np.random.default_rng(1)
    th = rng.standard_normal((5, 6))
    th[3] = th[1]          # exact duplicate: grain 3 can never win
    lab, gap = oracle.assign(g, 5, 2, th)
    assert not np.any(lab == 3)
    assert np.all(gap[lab == 1] == 0.0)
    # fully ambiguous diagram (Sec. 2.1): everything goes to grain 0
    lab0, gap0 = oracle.assign(g, 4, 2, np.tile(th[0], (4, 1)))
    assert np.all(lab0 == 0) and np.all(gap0 == 0.0)


def test_power_diagram_conversion(oracle):
    # Sec. 2.3: theta = (-2y, |y|^2 - w) reproduces argmin |x-y_i|^2 - w_i
    shape, N = (40, 36), 9
    y, w = synth.power_params(5, N)
    th = oracle.theta_from_apd(2, 1, y, w)
    lab, gap = oracle.assign(oracle.Grid(shape), N, 1, th)
    X = centres_2d(shape)
    cost = ((X[:, None, :] - y[None]) ** 2).sum(-1) - w[None]
    sure = gap > 1e-9
    np.testing.assert_array_equal(lab[sure], np.argmin(cost, 1)[sure])
    # round trip with eq. (pd-lr-to-phys): degree-1 Legendre = monomial here
    # up to order; the constant is index 0 and x1, x2 are indices 1, 2
    y_back = -0.5 * th[:, 1:3]
    w_back = 0.25 * (th[:, 1] ** 2 + th[:, 2] ** 2) - th[:, 0]
    np.testing.assert_allclose(y_back, y, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w_back, w, rtol=0, atol=1e-15)


def test_apd_conversion_round_trip(oracle):
    shape, N = (32, 30), 6
    y, w, A = synth.apd_params(6, N)
    th = oracle.theta_from_apd(2, 2, y, w, A)
    X = centres_2d(shape)
    D = X[:, None, :] - y[None]
    cost = np.einsum("pna,nab,pnb->pn", D, A, D) - w[None]
    lab, gap = oracle.assign(oracle.Grid(shape), N, 2, th)
    sure = gap > 1e-9
    np.testing.assert_array_equal(lab[sure], np.argmin(cost, 1)[sure])
    # back to monomials, then eq. (apd-lr-to-phys) with the paper's ordering
    T = oracle.mono_to_legendre(2, 2)
    mono = np.linalg.solve(T, th.T).T     # our order: 1, x1, x2, x1^2, x1x2, x2^2
    for i in range(N):
        Ai = np.array([[mono[i, 3], 0.5 * mono[i, 4]], [0.5 * mono[i, 4], mono[i, 5]]])
        yi = -0.5 * np.linalg.solve(Ai, mono[i, 1:3])
        wi = yi @ Ai @ yi - mono[i, 0]
        np.testing.assert_allclose(Ai, A[i], atol=1e-13)
        np.testing.assert_allclose(yi, y[i], atol=1e-12)
        assert abs(wi - w[i]) < 1e-12


def test_apd_conversion_3d(oracle):
    shape, N = (10, 9, 8), 5
    y, w, A = synth.apd_params(7, N, dim=3)
    th = oracle.theta_from_apd(3, 2, y, w, A)
    n1, n2, n3 = shape
    c = [-1.0 + (2.0 * np.arange(n) + 1.0) / n for n in shape]
    Z, Y, Xg = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    X = np.stack([Xg.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1)
    D = X[:, None, :] - y[None]
    cost = np.einsum("pna,nab,pnb->pn", D, A, D) - w[None]
    lab, gap = oracle.assign(oracle.Grid(shape), N, 2, th)
    sure = gap > 1e-9
    np.testing.assert_array_equal(lab[sure], np.argmin(cost, 1)[sure])


def test_grain_moments(oracle):
    g = oracle.Grid((12, 10))
    lab = (np.arange(g.P) % 4).astype(np.int32)
    mom, cnt = oracle.grain_moments(g, lab, 4, 4)
    eta = oracle.features(g, 4)
    for i in range(4):
        assert cnt[i] == np.sum(lab == i)
        np.testing.assert_allclose(mom[i], eta[lab == i].sum(0), rtol=1e-14, atol=1e-13)


def test_heuristic_formulas(oracle):
    # eqs. (centroid-guess), (cov-guess), (A-guess), (w-guess)
    shape, N = (30, 28), 5
    y0, w0 = synth.power_params(8, N)
    g = oracle.Grid(shape)
    lab, _ = oracle.assign(g, N, 1, oracle.theta_from_apd(2, 1, y0, w0))
    lab, N, _ = synth.compact(lab)
    X = centres_2d(shape)
    y, w, A = oracle.heuristic_params(g, lab, N, anisotropic=True)
    for i in range(N):
        Xi = X[lab == i]
        np.testing.assert_allclose(y[i], Xi.mean(0), atol=1e-14)
        B = np.cov(Xi.T, bias=True)
        np.testing.assert_allclose(A[i], np.linalg.inv(B), rtol=1e-10)
        want_w = math.sqrt(np.linalg.det(np.linalg.inv(B))) * len(Xi) / (g.P * math.pi)
        assert abs(w[i] - want_w) < 1e-12 * want_w
    y1, w1, A1 = oracle.heuristic_params(g, lab, N, anisotropic=False)
    np.testing.assert_array_equal(A1, np.broadcast_to(np.eye(2), A1.shape))
    np.testing.assert_allclose(w1, np.bincount(lab) / (g.P * math.pi), rtol=1e-14)


def noisy_problem(oracle, shape=(24, 22), N=5, d=1, seed=3, noise=0.15):
    g = oracle.Grid(shape)
    y, w = synth.power_params(seed, N)
    lab, _ = oracle.assign(g, N, 1, oracle.theta_from_apd(2, 1, y, w))
    lab, N, _ = synth.compact(lab)
    flip = synth.rng(seed + 1).random(g.P) < noise
    lab = np.where(flip, synth.random_labels(seed + 2, g.P, N), lab).astype(np.int32)
    return g, lab, N


def scipy_reference(oracle, g, lab, N, d, eps, x0):
    K = oracle.K(2, d)

    def fg(x):
        th = np.vstack([x.reshape(N - 1, K), np.zeros((1, K))])
        phi, gr = oracle.objective_grad(g, lab, N, d, eps, th)
        return -phi, -gr[: N - 1].reshape(-1)

    r = so.minimize(fg, x0, jac=True, method="L-BFGS-B",
                    options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12, maxcor=20))
    return -r.fun, r.x


@pytest.mark.parametrize("method", ["lbfgs", "newton"])
def test_fit_reaches_scipy_optimum_on_nonseparable_data(oracle, method):
    # Prop. 4.11: with label noise a unique gauge-fixed maximiser exists;
    # the ascent scheme must reach the optimum found by scipy's L-BFGS-B
    g, lab, N = noisy_problem(oracle)
    d, eps = 2, 0.1
    K = oracle.K(2, d)
    phi_ref, x_ref = scipy_reference(oracle, g, lab, N, d, eps, np.zeros((N - 1) * K))
    th0 = np.zeros((N, K))
    if method == "lbfgs":
        th, rep, tr = oracle.lbfgs_fit(g, lab, N, d, eps, th0, 500, gtol=1e-11)
    else:
        th, rep, tr = oracle.newton_cg_fit(g, lab, N, d, eps, th0, 60, gtol=1e-11)
    assert abs(rep.phi - phi_ref) <= 1e-10 * abs(phi_ref)
    np.testing.assert_allclose(th[: N - 1].reshape(-1), x_ref, rtol=0, atol=1e-4 * np.abs(x_ref).max())
    assert np.all(th[N - 1] == 0.0)
    assert np.all(np.diff(tr) >= -1e-15)   # ascent: Phi never decreases


def test_degree1_power_diagram_recovery(oracle):
    # Sec. 5.4 / Cor. 4.10: fit a PD-generated map at degree 1 from theta = 0;
    # Phi > -log2/|Omega| certifies Err = 0, and Err is checked directly
    shape, N0 = (48, 48), 6
    g = oracle.Grid(shape)
    y, w = synth.power_params(1, N0)
    lab, _ = oracle.assign(g, N0, 1, oracle.theta_from_apd(2, 1, y, w))
    lab, N, _ = synth.compact(lab)
    th, rep, _ = oracle.lbfgs_fit(g, lab, N, 1, 1e-2, np.zeros((N, 3)), 2000)
    assert rep.phi > -math.log(2.0) / g.P
    F, _ = oracle.assign(g, N, 1, th)
    assert np.all(F == lab)


def test_degree2_anisotropic_recovery(oracle):
    shape, N0 = (48, 48), 6
    g = oracle.Grid(shape)
    y, w, A = synth.apd_params(2, N0)
    lab, _ = oracle.assign(g, N0, 2, oracle.theta_from_apd(2, 2, y, w, A))
    lab, N, _ = synth.compact(lab)
    th, rep, _ = oracle.lbfgs_fit(g, lab, N, 2, 1e-2, np.zeros((N, 6)), 2000)
    assert rep.phi > -math.log(2.0) / g.P
    F, _ = oracle.assign(g, N, 2, th)
    assert np.all(F == lab)


def test_nested_degrees(oracle):
    # Sec. 5.5.1: a degree-d fit padded with zeros is admissible at degree
    # d+1, so the degree-(d+1) optimum is at least as good
    g, lab, N = noisy_problem(oracle, seed=11)
    eps = 0.1
    th1, r1, _ = oracle.lbfgs_fit(g, lab, N, 1, eps, np.zeros((N, 3)), 300, gtol=1e-10)
    pad = np.zeros((N, 6))
    pad[:, :3] = th1          # degrees <= 1 come first in the fixed order
    phi_pad = oracle.objective_grad(g, lab, N, 2, eps, pad, want_grad=False)
    assert abs(phi_pad - r1.phi) < 1e-13
    th2, r2, _ = oracle.lbfgs_fit(g, lab, N, 2, eps, pad, 300, gtol=1e-10)
    assert r2.phi >= r1.phi - 1e-14


@pytest.mark.parametrize("d", [1, 2, 4])
def test_heuristic_theta_diagram(oracle, d):
    # the heuristic's parameters (Sec. 5.5.2), computed here from their
    # printed formulas in numpy, define a (d = 1: isotropic, d >= 2:
    # anisotropic) power diagram; heuristic_theta must rasterise to exactly
    # that diagram, whatever the degree its higher terms are padded to
    shape, N = (36, 30), 7
    y0, w0 = synth.power_params(11, N)
    g = oracle.Grid(shape)
    lab, _ = oracle.assign(g, N, 1, oracle.theta_from_apd(2, 1, y0, w0))
    lab, N, _ = synth.compact(lab)
    X = centres_2d(shape)
    ys, ws, As = [], [], []
    for i in range(N):
        Xi = X[lab == i]
        y = Xi.mean(0)
        A = np.linalg.inv(np.cov(Xi.T, bias=True)) if d >= 2 else np.eye(2)
        ys.append(y)
        As.append(A)
        ws.append(math.sqrt(np.linalg.det(A)) * len(Xi) / (g.P * math.pi))
    ys, ws, As = np.array(ys), np.array(ws), np.array(As)
    D = X[:, None, :] - ys[None]
    cost = np.einsum("pna,nab,pnb->pn", D, As, D) - ws[None]
    th = oracle.heuristic_theta(g, lab, N, d)
    assert th.shape == (N, oracle.K(2, d))
    got, gap = oracle.assign(g, N, d, th)
    sure = gap > 1e-9
    assert sure.mean() > 0.99
    np.testing.assert_array_equal(got[sure], np.argmin(cost, 1)[sure])


def centres_3d(shape):
    n0, n1, n2 = shape
    idx = np.arange(n0 * n1 * n2)
    k = [idx % n0, (idx // n0) % n1, idx // (n0 * n1)]
    return np.stack([-1.0 + (2.0 * k[a] + 1.0) / shape[a] for a in range(3)], 1)


def test_heuristic_formulas_3d(oracle):
    # the 3-D branch of the heuristic (the paper states it in 2-D; the
    # reading: A' = B'^-1 of the 3x3 central second moments, w' = sqrt(det
    # A') |G_i| / (|Omega| 4 pi / 3), the ellipsoid volume in place of pi),
    # against numpy's mean, covariance, inverse and determinant
    shape, N = (14, 12, 10), 6
    y0, w0, A0 = synth.apd_params(17, N, dim=3)
    g = oracle.Grid(shape)
    lab, _ = oracle.assign(g, N, 2, oracle.theta_from_apd(3, 2, y0, w0, A0))
    lab, N, _ = synth.compact(lab)
    X = centres_3d(shape)
    y, w, A = oracle.heuristic_params(g, lab, N, anisotropic=True)
    for i in range(N):
        Xi = X[lab == i]
        np.testing.assert_allclose(y[i], Xi.mean(0), atol=1e-14)
        B = np.cov(Xi.T, bias=True)
        np.testing.assert_allclose(A[i], np.linalg.inv(B), rtol=1e-9, atol=1e-9 * np.abs(np.linalg.inv(B)).max())
        want_w = math.sqrt(np.linalg.det(np.linalg.inv(B))) * len(Xi) / (g.P * 4.0 * math.pi / 3.0)
        assert abs(w[i] - want_w) < 1e-10 * want_w
    # a collinear grain (B' singular) falls back to A' = Id (Sec. 5.5.2: "if B' is invertible")
    lab2 = np.zeros(g.P, dtype=np.int32)
    line = (X[:, 1] == X[0, 1]) & (X[:, 2] == X[0, 2])      # one row of voxels along x
    lab2[line] = 1
    _, _, A2 = oracle.heuristic_params(g, lab2, 2, anisotropic=True)
    np.testing.assert_array_equal(A2[1], np.eye(3))


def test_heuristic_theta_diagram_3d(oracle):
    # the 3-D heuristic's parameters computed here from the formulas in numpy
    # define an anisotropic power diagram; heuristic_theta (degree 2) must
    # rasterise to it, which pins the 3-D conversion to Legendre as well
    shape, N = (16, 14, 12), 7
    y0, w0, A0 = synth.apd_params(19, N, dim=3)
    g = oracle.Grid(shape)
    lab, _ = oracle.assign(g, N, 2, oracle.theta_from_apd(3, 2, y0, w0, A0))
    lab, N, _ = synth.compact(lab)
    X = centres_3d(shape)
    ys, ws, As = [], [], []
    for i in range(N):
        Xi = X[lab == i]
        A = np.linalg.inv(np.cov(Xi.T, bias=True))
        ys.append(Xi.mean(0))
        As.append(A)
        ws.append(math.sqrt(np.linalg.det(A)) * len(Xi) / (g.P * 4.0 * math.pi / 3.0))
    ys, ws, As = np.array(ys), np.array(ws), np.array(As)
    D = X[:, None, :] - ys[None]
    cost = np.einsum("pna,nab,pnb->pn", D, As, D) - ws[None]
    th = oracle.heuristic_theta(g, lab, N, 2)
    got, gap = oracle.assign(g, N, 2, th)
    sure = gap > 1e-9
    assert sure.mean() > 0.99
    np.testing.assert_array_equal(got[sure], np.argmin(cost, 1)[sure])
