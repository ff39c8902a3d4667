"""Pins of the oracle's warm-start network and its inputs (not from the
paper): back-propagation against finite differences, a network with
identity layers against its closed form, and the moment features against
numpy."""
import numpy as np
import pytest


def small_net(rng, dims=(7, 6, 5, 3)):
    n_in, h1, h2, out = dims
    return [rng.standard_normal((h1, n_in)) * 0.5, rng.standard_normal(h1) * 0.1,
            rng.standard_normal((h2, h1)) * 0.5, rng.standard_normal(h2) * 0.1,
            rng.standard_normal((out, h2)) * 0.5, rng.standard_normal(out) * 0.1]


def test_identity_network_closed_form(oracle):
    # with identity weights, zero biases and non-negative inputs the ReLUs
    # pass everything: y = x
    X = np.abs(np.random.default_rng(0).standard_normal((5, 4)))
    I = np.eye(4)
    Y = oracle.mlp_forward(X, I, np.zeros(4), I, np.zeros(4), I, np.zeros(4))
    np.testing.assert_array_equal(Y, X)
    # a negative pre-activation is cut by the first ReLU
    Y = oracle.mlp_forward(-X, I, np.zeros(4), I, np.zeros(4), I, np.ones(4))
    np.testing.assert_array_equal(Y, np.ones_like(X))


def test_backprop_vs_finite_differences(oracle):
    rng = np.random.default_rng(1)
    ws = small_net(rng)
    X = rng.standard_normal((9, 7))
    T = rng.standard_normal((9, 3))
    loss, gs = oracle.mlp_loss_grad(X, T, *ws)
    Y = oracle.mlp_forward(X, *ws)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-14
    h = 1e-6
    for w, gw in zip(ws, gs):
        for idx in list(np.ndindex(w.shape))[:12]:
            old = w[idx]
            w[idx] = old + h
            lp = oracle.mlp_loss_grad(X, T, *ws)[0]
            w[idx] = old - h
            lm = oracle.mlp_loss_grad(X, T, *ws)[0]
            w[idx] = old
            assert abs((lp - lm) / (2 * h) - gw[idx]) <= 1e-7 * max(1.0, abs(gw[idx]))


def test_features(oracle):
    from paper_2605_20816_gb300 import synth
    g = oracle.Grid((40, 36))
    y, w = synth.power_params(5, 12)
    lab, _ = oracle.assign(g, 12, 1, oracle.theta_from_apd(2, 1, y, w))
    lab, N, _ = synth.compact(lab)
    F = oracle.mlp_features(g, lab, N, dm=4, n_nb=3)
    eta = oracle.features(g, 4)
    mom = np.stack([eta[lab == i].mean(0) for i in range(N)])
    np.testing.assert_allclose(F[:, :15], mom, rtol=1e-13, atol=1e-14)
    cen = mom[:, 1:3]
    for i in range(N):
        d = ((cen - cen[i]) ** 2).sum(1)
        d[i] = np.inf
        order = np.argsort(d, kind="stable")[:3]
        for q, j in enumerate(order):
            np.testing.assert_allclose(F[i, 15 * (q + 1):15 * (q + 2)], mom[j], rtol=1e-13, atol=1e-14)
