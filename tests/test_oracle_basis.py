"""Pins of the oracle's design functions against closed forms and library
routines (Sec. 3 of the paper)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly
from scipy.special import comb, eval_legendre

HERE = os.path.dirname(os.path.abspath(__file__))


def centres(n):
    # pixel centres of Sec. 2.1 with n = 2M: (-1) + (k - 1/2)/M, k = 1..2M
    M = n / 2.0
    return -1.0 + (np.arange(1, n + 1) - 0.5) / M


def test_legendre_closed_forms(oracle):
    # textbook closed forms of P_2, P_3, P_4
    for t in np.linspace(-1, 1, 41):
        assert oracle.legendre(0, t) == 1.0
        assert oracle.legendre(1, t) == t
        assert abs(oracle.legendre(2, t) - (3 * t**2 - 1) / 2) < 1e-15
        assert abs(oracle.legendre(3, t) - (5 * t**3 - 3 * t) / 2) < 1e-15
        assert abs(oracle.legendre(4, t) - (35 * t**4 - 30 * t**2 + 3) / 8) < 1e-15


def test_legendre_vs_scipy(oracle):
    for m in range(0, 12):
        for t in np.linspace(-1, 1, 37):
            assert abs(oracle.legendre(m, t) - eval_legendre(m, t)) < 1e-13


@pytest.mark.parametrize("d", [1, 3, 7])
def test_legendre_orthogonality(oracle, d):
    # Gauss-Legendre with d+1 nodes integrates degree <= 2d+1 exactly
    x, w = npleg.leggauss(d + 1)
    for m in range(d + 1):
        for n in range(d + 1):
            s = sum(wi * oracle.legendre(m, xi) * oracle.legendre(n, xi) for xi, wi in zip(x, w))
            want = 2.0 / (2 * n + 1) if m == n else 0.0
            assert abs(s - want) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_multi_index_set(oracle, dim):
    for d in range(0, 8):
        K = oracle.K(dim, d)
        want = (d + 1) * (d + 2) // 2 if dim == 2 else int(comb(d + 3, 3, exact=True))
        assert K == want
        a = oracle.alpha(dim, d)
        assert a.shape == (K, dim)
        tot = a.sum(axis=1)
        assert np.all(tot <= d) and np.all(np.diff(tot) >= 0)   # graded
        assert len({tuple(r) for r in a}) == K                  # distinct
    assert oracle.alpha(2, 2).tolist() == [[0, 0], [1, 0], [0, 1], [2, 0], [1, 1], [0, 2]]
    assert oracle.K(3, 2) == 10 and oracle.K(3, 3) == 20 and oracle.K(2, 4) == 15


@pytest.mark.parametrize("shape,d", [((7, 5), 3), ((4, 6, 3), 2)])
def test_features_vs_numpy_legval(oracle, shape, d):
    g = oracle.Grid(shape)
    eta = oracle.features(g, d)
    a = oracle.alpha(len(shape), d)
    axes = [centres(n) for n in shape]
    # linear index j = k1 + n1 (k2 + n2 k3): axis 1 fastest
    mesh = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([m.transpose(tuple(range(len(shape)))[::-1]).reshape(-1) for m in mesh], 1)
    for k, al in enumerate(a):
        v = np.ones(g.P)
        for ax, e in enumerate(al):
            c = np.zeros(e + 1); c[e] = 1.0
            v = v * npleg.legval(pts[:, ax], c)
        np.testing.assert_allclose(eta[:, k], v, rtol=0, atol=1e-14)


def test_point_list_matches_grid(oracle):
    g = oracle.Grid((6, 4))
    xs, ys = np.meshgrid(centres(6), centres(4), indexing="xy")
    pts = np.stack([xs.reshape(-1), ys.reshape(-1)], 1)
    gl = oracle.Grid(coords=pts)
    np.testing.assert_array_equal(oracle.features(g, 3), oracle.features(gl, 3))


def test_monomial_features(oracle):
    g = oracle.Grid((5, 3))
    eta = oracle.features(g, 3, basis="monomial")
    a = oracle.alpha(2, 3)
    xs, ys = np.meshgrid(centres(5), centres(3), indexing="xy")
    x1, x2 = xs.reshape(-1), ys.reshape(-1)
    for k, (e1, e2) in enumerate(a):
        np.testing.assert_allclose(eta[:, k], x1**e1 * x2**e2, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("dim,d", [(2, 1), (2, 2), (2, 4), (2, 7), (3, 3)])
def test_mono_to_legendre_vs_poly2leg(oracle, dim, d):
    T = oracle.mono_to_legendre(dim, d)
    a = oracle.alpha(dim, d)
    idx = {tuple(r): k for k, r in enumerate(a)}
    for col, al in enumerate(a):
        # x^alpha as a tensor product of 1-D Legendre series (numpy poly2leg)
        series = []
        for e in al:
            c = np.zeros(e + 1); c[e] = 1.0
            series.append(npleg.poly2leg(c))
        want = np.zeros(len(a))
        for combo in np.ndindex(*[len(s) for s in series]):
            coef = np.prod([series[ax][combo[ax]] for ax in range(dim)])
            if coef != 0.0:
                want[idx[tuple(combo)]] += coef
        np.testing.assert_allclose(T[:, col], want, rtol=0, atol=1e-14)


def test_basis_change_preserves_objective(oracle):
    # Remark 3.1: both bases span the same space, so Phi_mono(th) = Phi_Leg(T th)
    g = oracle.Grid((12, 10))
    N, d, eps = 5, 3, 0.05
    rng = np.random.default_rng(3)
    lab = rng.integers(0, N, g.P).astype(np.int32)
    th_m = 0.2 * rng.standard_normal((N, oracle.K(2, d)))
    T = oracle.mono_to_legendre(2, d)
    th_l = th_m @ T.T
    pm = oracle.objective_grad(g, lab, N, d, eps, th_m, basis="monomial", want_grad=False)
    pl = oracle.objective_grad(g, lab, N, d, eps, th_l, want_grad=False)
    assert abs(pm - pl) < 1e-12 * abs(pl)
    lm, _ = oracle.assign(g, N, d, th_m, basis="monomial")
    ll, gap = oracle.assign(g, N, d, th_l)
    sure = gap > 1e-9
    np.testing.assert_array_equal(lm[sure], ll[sure])


def test_compression_table(oracle):
    # Table 1 (Sec. 5.5.1): Compr = K_d N / (3 |Omega|), printed in percent
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table1_compression.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for name, N, Om, *vals in rows:
        for d, v in enumerate(vals, start=1):
            c = 100.0 * oracle.K(2, d) * int(N) / (3.0 * int(Om))
            assert abs(round(c, 2) - float(v)) < 1e-9, (name, d, c, v)
