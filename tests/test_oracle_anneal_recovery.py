"""Pins of the oracle's physical-parameter recovery (Sec. 2.3, eqs.
pd-lr-to-phys and apd-lr-to-phys, with the common shift of Sec. 5.5.3) and
of its eps annealing with Err^G-aligned stopping (the schedule Secs. 5.2 and
5.5.4 leave to future work, in this build's reading).

The recovery is checked against the forward relations of Sec. 2.3 written
out in numpy (exact round trips), against numpy's direct power-distance
arg-min (the recovered parameters draw the same diagram as theta, Lemma 4.2)
and against numpy's eigenvalues (every shifted A_i positive definite).  The
annealing is checked against numpy's arg-min of the returned parameters
(Err^G = 0 on a separable map), Cor. 4.10 (the certificate implies Err^G =
0) and Prop. 4.7."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2605_20816_gb300 import synth


def legendre_design(grid_pts, dim, d):
    """eta(x) by numpy's Legendre series, in the library order of A_d."""
    al = O.alpha(dim, d)
    cols = []
    for a in al:
        v = np.ones(len(grid_pts))
        for ax in range(dim):
            c = np.zeros(a[ax] + 1)
            c[a[ax]] = 1.0
            v = v * np.polynomial.legendre.legval(grid_pts[:, ax], c)
        cols.append(v)
    return np.stack(cols, 1)


def grid_points(shape):
    axes = [-1.0 + (2.0 * np.arange(n) + 1.0) / n for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    # linear index j = k0 + n0 (k1 + n1 k2): axis 0 fastest
    return np.stack([m.transpose().reshape(-1) for m in mesh], 1) if len(shape) == 2 else \
        np.stack([m.transpose(2, 1, 0).reshape(-1) for m in mesh], 1)


def power_argmin(pts, y, w, A):
    """argmin_i |x - y_i|^2_{A_i} - w_i (A None: identity), smallest i on ties."""
    cost = []
    for i in range(len(w)):
        z = pts - y[i]
        Ai = np.eye(pts.shape[1]) if A is None else A[i]
        cost.append(np.einsum("pa,ab,pb->p", z, Ai, z) - w[i])
    return np.argmin(np.stack(cost, 1), 1)


def test_pd_round_trip_eq_pd_lr_to_phys():
    for dim in (2, 3):
        y, w = synth.power_params(11 + dim, 9, dim=dim)
        th = O.theta_from_apd(dim, 1, y, w)
        y2, w2, A2, lam = O.theta_to_apd(dim, 1, th)
        assert A2 is None and lam == 0.0
        np.testing.assert_allclose(y2, y, rtol=0, atol=1e-13)
        np.testing.assert_allclose(w2, w, rtol=0, atol=1e-13)
        # eq. pd-lr-to-phys written out: monomial theta = (-2 y, |y|^2 - w)
        th_mono = np.concatenate([-2.0 * y, (np.sum(y * y, 1) - w)[:, None]], 1)
        T = O.mono_to_legendre(dim, 1)
        order = [dim] + list(range(dim))   # library order: constant, then x_1..x_dim
        np.testing.assert_allclose(th, th_mono[:, order] @ T.T, rtol=0, atol=1e-13)


def test_apd_round_trip_eq_apd_lr_to_phys():
    for dim in (2, 3):
        y, w, A = synth.apd_params(21 + dim, 7, dim=dim)
        assert np.linalg.eigvalsh(A).min() > 0.4          # eigenvalues in [0.5, 2]
        th = O.theta_from_apd(dim, 2, y, w, A)
        y2, w2, A2, lam = O.theta_to_apd(dim, 2, th, margin=1e-3)
        assert lam == 0.0                                  # already positive definite
        np.testing.assert_allclose(A2, A, rtol=0, atol=1e-12)
        np.testing.assert_allclose(y2, y, rtol=0, atol=1e-11)
        np.testing.assert_allclose(w2, w, rtol=0, atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_shift_enforces_positive_definite_and_keeps_the_diagram(dim):
    shape = (40, 36) if dim == 2 else (14, 12, 10)
    y, w, A = synth.apd_params(31 + dim, 8, dim=dim)
    th = O.theta_from_apd(dim, 2, y, w, A)
    # a common shift (Lemma 4.2) that leaves some A_i indefinite, as the
    # gauge theta_{N-1} = 0 of a fit does: subtract the last grain's block
    th_g = th - th[-1]
    g = O.Grid(shape)
    lab, gap = O.assign(g, 8, 2, th_g)
    margin = 1e-2
    y2, w2, A2, lam = O.theta_to_apd(dim, 2, th_g, margin=margin)
    ev = np.linalg.eigvalsh(A2)
    assert lam > 0.0
    assert ev.min() >= margin * (1 - 1e-9)                 # every A_i + lambda Id positive definite
    assert ev.min() <= margin * (1 + 1e-9)                 # lambda is the smallest such shift
    lab2 = power_argmin(grid_points(shape), y2, w2, A2)
    sure = gap >= 1e-9
    np.testing.assert_array_equal(lab2[sure], lab[sure])


def test_recovery_rejects_bad_arguments():
    th = np.zeros((3, 10))
    with pytest.raises(ValueError):
        O.theta_to_apd(2, 3, th)                           # only degrees 1 and 2
    with pytest.raises(ValueError):
        O.theta_to_apd(2, 2, np.zeros((3, 6)), margin=0.0)  # the shift needs a positive margin


def test_single_stage_is_the_plain_ascent():
    g, lab, N = _pd_problem()
    th0 = np.zeros((N, O.K(2, 2)))
    th_a, stages = O.anneal_fit(g, lab, N, 2, eps0=1e-2, factor=0.5, eps_min=1e-2, stage_iter=5,
                                final_iter=30, theta0=th0)
    th_p, rep, _ = O.lbfgs_fit(g, lab, N, 2, 1e-2, th0, 30)
    assert len(stages) == 1 and stages[0][0] == 1e-2
    np.testing.assert_array_equal(th_a, th_p)


def _pd_problem():
    shape, N = (64, 64), 8
    g = O.Grid(shape)
    y, w = synth.power_params(synth.SEED_BASE, N, dim=2)
    lab, _ = O.assign(g, N, 1, O.theta_from_apd(2, 1, y, w))
    lab, N, _ = synth.compact(lab)
    return g, lab.astype(np.int32), N


def test_annealing_reconstructs_a_power_diagram():
    # a separable map (Prop. 4.8): annealing from theta = 0 must reach a
    # parameter whose hard assignment is G itself; the schedule stops there
    g, lab, N = _pd_problem()
    th0 = np.zeros((N, O.K(2, 2)))
    th, stages = O.anneal_fit(g, lab, N, 2, eps0=1e-1, factor=0.5, eps_min=1e-4, stage_iter=200,
                              final_iter=200, theta0=th0)
    eps = [s[0] for s in stages]
    # the geometric schedule, clamped at eps_min
    assert all(abs(b - max(1e-4, a * 0.5)) <= 1e-15 * a for a, b in zip(eps, eps[1:]))
    assert stages[-1][0] > 1e-4                            # stopped by Err^G = 0 before eps_min
    # the hard assignment of the result, by numpy
    E = legendre_design(grid_points((64, 64)), 2, 2)
    lab_np = np.argmin(E @ th.T, 1)
    assert np.array_equal(lab_np, lab)
    last = stages[-1]
    if last[2] < 0:
        # stopped by the certificate of Cor. 4.10
        assert last[1] > -math.log(2.0) / g.P
    else:
        assert last[2] == 0.0 or last[0] == 1e-4
    # Prop. 4.7 at the stage's eps: 0 <= -eps Phi - E_0 <= eps log N
    h = E @ th.T
    E0 = np.mean(h[np.arange(g.P), lab] - h.min(1))
    gap = -last[0] * last[1] - E0
    assert -1e-12 <= gap <= last[0] * math.log(N) + 1e-12
