"""The learned warm start: the network's own forward and backward kernels
against the oracle's back-propagation (same bf16-rounded weights, so the
difference is fp32 accumulation only), the features against the oracle, and
what the trained network gains over the ascent scheme from theta = 0."""
import math
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth, warmstart
from helpers import poly_problem, rel

pytestmark = pytest.mark.gpu


def test_forward_and_gradients_match_oracle():
    net = pd.MLP(135, 256, 256, 15, seed=3)
    g = torch.Generator().manual_seed(0)
    X = (0.5 * torch.randn(300, 135, generator=g)).float()
    T = torch.randn(300, 15, generator=g).float()
    W = net.unflatten(net.params(rounded=True).double().numpy())
    Y = net.forward(X.cuda()).cpu().numpy()
    Yo = O.mlp_forward(X.double().numpy(), *W)
    assert rel(Y, Yo) <= 1e-5
    loss, gr = net.loss_grad(X.cuda(), T.cuda())
    loss_o, gs_o = O.mlp_loss_grad(X.double().numpy(), T.double().numpy(), *W)
    assert abs(loss.item() - loss_o) <= 1e-5 * loss_o
    for got, want in zip(net.unflatten(gr.cpu().double().numpy()), gs_o):
        assert rel(got, want) <= 1e-4, rel(got, want)
    net.close()


def test_features_match_oracle():
    g, lab, N, _ = poly_problem((160, 144), 120, 4, seed=11)
    F = pd.pd_mlp_features(pd.Grid((160, 144)), torch.from_numpy(lab).cuda(), N).cpu().numpy()
    Fo = O.mlp_features(g, lab, N, dm=4, n_nb=8)
    np.testing.assert_allclose(F, Fo, rtol=0, atol=2e-6)


def test_training_reduces_loss():
    X, T = warmstart.dataset(12, seed0=77, side=128, grains=(30, 120))
    net = pd.MLP(135, 256, 256, 15, seed=4)
    losses = warmstart.train(net, X, T, epochs=25, batch=512, lr=2e-3)
    print("training loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]
    net.close()


def iters_to(grid, lab, N, d, eps, theta0, target, budget):
    init = pd.PD_INIT_ZERO if theta0 is None else pd.PD_INIT_GIVEN
    t = time.perf_counter()
    _, rep = pd.pd_fit(grid, lab, N, d, eps, theta=theta0, init=init, max_iter=budget, target_phi=target)
    return rep, time.perf_counter() - t


@pytest.mark.slow
def test_warm_start_gain():
    # train on 256^2 degree-4 diagrams (N uniform in [50, 400]); evaluate on
    # 512^2, N = 300 degree-4 diagrams: iterations and time of the plain
    # FP64 ascent to the objective the plain fit reaches in 1000 iterations
    # from theta = 0, with and without the warm start
    X, T = warmstart.dataset(300, seed0=5_000_000, side=256, grains=(50, 400))
    net = pd.MLP(135, 256, 256, 15, seed=1)
    losses = warmstart.train(net, X, T, epochs=40, batch=4096, lr=1e-3)
    print("warm-start training: %d grains, loss %.4f -> %.4f" % (X.shape[0], losses[0], losses[-1]))
    d, eps = 4, 1e-3
    rows = []
    for s in range(2):
        grid, lab, N, th = warmstart.diagram(6_000_000 + s, (512, 512), 300, d)
        _, ref = pd.pd_fit(grid, lab, N, d, eps, max_iter=1000)
        target = ref["phi"] - 1e-8 * abs(ref["phi"])
        plain, t_plain = iters_to(grid, lab, N, d, eps, None, target, 1000)
        t0 = time.perf_counter()
        th0, scale = pd.pd_warm_start(net, grid, lab, N, d, eps, prec=pd.PD_FP64)
        t_ws = time.perf_counter() - t0
        phi0 = pd.pd_objective_grad(grid, lab, N, th0, d, eps, want_grad=False)[0].item()
        warm, t_warm = iters_to(grid, lab, N, d, eps, th0, target, 1000)
        rows.append((plain["iters"], warm["iters"], t_plain, t_ws + t_warm))
        print("map %d: N=%d Phi_ref=%.6e; plain %d iters %.2fs; warm start Phi0=%.4e (scale %.3g), %d iters "
              "%.2fs (+%.2fs prediction), reached=%s" % (s, N, ref["phi"], plain["iters"], t_plain, phi0, scale,
                                                         warm["iters"], t_warm, t_ws, warm["status"] == 3))
        assert phi0 > -math.log(N)          # better than the fully ambiguous start
        # the gain: the warm-started ascent reaches the plain fit's objective,
        # in fewer iterations and less wall time (prediction included)
        assert warm["status"] == 3, warm
        assert warm["iters"] < plain["iters"], (warm["iters"], plain["iters"])
        assert t_ws + t_warm < t_plain, (t_ws + t_warm, t_plain)
    print("iterations plain / warm: %s" % [(r[0], r[1]) for r in rows])
    net.close()
