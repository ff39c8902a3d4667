"""Pins of the oracle's Hessian-vector product and dense Hessian (eq. hess,
Prop. 4.4/4.5)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg


def np_features(shape, d, oracle):
    axes = [-1.0 + (2.0 * np.arange(n) + 1.0) / n for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([m.transpose(tuple(range(len(shape)))[::-1]).reshape(-1) for m in mesh], 1)
    cols = []
    for al in oracle.alpha(len(shape), d):
        v = np.ones(pts.shape[0])
        for ax, e in enumerate(al):
            c = np.zeros(e + 1); c[e] = 1.0
            v = v * npleg.legval(pts[:, ax], c)
        cols.append(v)
    return np.stack(cols, 1)


def setup(oracle, shape=(7, 6), N=4, d=2, seed=0):
    g = oracle.Grid(shape)
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, N, g.P).astype(np.int32)
    K = oracle.K(len(shape), d)
    th = 0.4 * rng.standard_normal((N, K))
    v = rng.standard_normal((N, K))
    u = rng.standard_normal((N, K))
    return g, lab, th, v, u


@pytest.mark.parametrize("dim", [2, 3])
def test_hvp_vs_finite_difference_of_gradient(oracle, dim):
    shape = (7, 6) if dim == 2 else (4, 4, 3)
    N, d, eps = 4, 2, 0.5
    g, lab, th, v, _ = setup(oracle, shape, N, d, seed=1)
    hv = oracle.hvp(g, lab, N, d, eps, th, v)
    h = 1e-5
    _, gp = oracle.objective_grad(g, lab, N, d, eps, th + h * v)
    _, gm = oracle.objective_grad(g, lab, N, d, eps, th - h * v)
    np.testing.assert_allclose(hv, (gp - gm) / (2 * h), rtol=1e-6, atol=1e-8)


def test_quadratic_form_is_minus_variance(oracle):
    # proof of Prop. 4.5: v'Hv = -(1/(eps^2|Omega|)) sum_x Var_{P_x}(v_i . eta(x))
    shape, N, d, eps = (8, 7), 5, 2, 0.3
    g, lab, th, v, _ = setup(oracle, shape, N, d, seed=2)
    eta = np_features(shape, d, oracle)
    L = -(eta @ th.T) / eps
    P = np.exp(L - L.max(1, keepdims=True)); P /= P.sum(1, keepdims=True)
    U = eta @ v.T
    var = (P * U**2).sum(1) - (P * U).sum(1) ** 2
    want = -var.sum() / (eps**2 * g.P)
    got = np.sum(v * oracle.hvp(g, lab, N, d, eps, th, v))
    assert abs(got - want) < 1e-11 * abs(want)


def test_hvp_symmetric(oracle):
    g, lab, th, v, u = setup(oracle, (9, 5), 4, 3, seed=3)
    a = np.sum(u * oracle.hvp(g, lab, 4, 3, 0.2, th, v))
    b = np.sum(v * oracle.hvp(g, lab, 4, 3, 0.2, th, u))
    assert abs(a - b) < 1e-11 * max(abs(a), abs(b))


def test_dense_hessian_nsd_with_gauge_null_space(oracle):
    # Prop. 4.4/4.5: H is negative semidefinite; its null space is exactly
    # {(c, ..., c)} (K-dimensional) when {eta(x)} spans R^K
    shape, N, d, eps = (6, 6), 4, 2, 0.5
    g, lab, th, v, _ = setup(oracle, shape, N, d, seed=4)
    H = oracle.hessian(g, N, d, eps, th)
    K = th.shape[1]
    assert np.allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    scale = np.abs(ev).max()
    assert ev.max() <= 1e-12 * scale
    assert np.sum(np.abs(ev) <= 1e-10 * scale) == K
    c = np.random.default_rng(5).standard_normal(K)
    np.testing.assert_allclose(H @ np.tile(c, N), 0.0, atol=1e-11 * scale)
    # the dense matrix and the matrix-free product agree
    np.testing.assert_allclose(H @ v.reshape(-1), oracle.hvp(g, lab, N, d, eps, th, v).reshape(-1),
                               rtol=1e-11, atol=1e-12 * scale)


def test_gauge_fixed_hessian_negative_definite(oracle):
    shape, N, d, eps = (6, 5), 3, 1, 0.4
    g, lab, th, _, _ = setup(oracle, shape, N, d, seed=6)
    H = oracle.hessian(g, N, d, eps, th)
    K = th.shape[1]
    Hf = H[: (N - 1) * K, : (N - 1) * K]
    assert np.linalg.eigvalsh(0.5 * (Hf + Hf.T)).max() < 0.0
