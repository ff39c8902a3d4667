"""Batched evaluation of many grain maps (one persistent launch per pass,
replayed as a CUDA graph; on the tensor cores one graph of the maps'
single-map evaluations on parallel chains) against single-map calls and
the oracle, and the lockstep batched fit against single-map fits."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth
from helpers import poly_problem, power_problem

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def make_maps(n, d=3, seed=0, small=False):
    shapes = synth.batched_shapes(seed, n, side=(16, 96) if small else (40, 300), grains=(2, 300))
    maps = []
    for q, (n1, n2, N) in enumerate(shapes):
        g = O.Grid((n1, n2))
        lab = synth.random_labels(seed + 100 + q, g.P, N)
        th = synth.random_theta(seed + 200 + q, N, O.K(2, d), 0.05)
        maps.append(((n1, n2), lab, N, th))
    return maps


# on the tensor cores a map's evaluation in the batch is the single-map
# evaluation itself: bitwise equal
@pytest.mark.parametrize("prec,tol", [(pd.PD_FP64, 1e-12), (pd.PD_FP32, 1e-6), (pd.PD_BF16, 0.0),
                                      (pd.PD_BF16X3, 0.0)])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_map_calls(prec, tol, autotune):
    d, eps = 3, 2e-2
    raw = make_maps(12, d=d, seed=1)
    keep, specs = [], []
    for shape, lab, N, th in raw:
        grid = pd.Grid(shape)
        lt, tt = dev(lab), dev(th)
        obj = torch.empty((), dtype=torch.float64, device="cuda")
        grad = torch.empty_like(tt)
        keep.append((grid, lt, N, tt, obj, grad))
    b = pd.Batch(keep, d, eps, prec=prec, autotune=autotune)
    for rep in range(2):
        b.eval()
        torch.cuda.synchronize()
        for grid, lt, N, tt, obj, grad in keep:
            o1, g1 = pd.pd_objective_grad(grid, lt, N, tt, d, eps, prec=prec)
            torch.cuda.synchronize()
            assert abs(obj.item() - o1.item()) <= tol * abs(o1.item())
            gw = g1.cpu().numpy()
            assert np.linalg.norm(grad.cpu().numpy() - gw) <= tol * np.linalg.norm(gw)
    b.close()


def test_batch_matches_oracle_and_is_reproducible():
    d, eps = 2, 5e-2
    raw = make_maps(5, d=d, seed=7, small=True)
    keep = []
    for shape, lab, N, th in raw:
        tt = dev(th)
        keep.append((pd.Grid(shape), dev(lab), N, tt, torch.empty((), dtype=torch.float64, device="cuda"),
                     torch.empty_like(tt)))
    b = pd.Batch(keep, d, eps, prec=pd.PD_FP64, autotune=False)
    b.eval()
    torch.cuda.synchronize()
    first = [(o.item(), g.cpu().numpy().copy()) for *_, o, g in keep]
    for (shape, lab, N, th), (phi, grad) in zip(raw, first):
        phi_o, grad_o = O.objective_grad(O.Grid(shape), lab, N, d, eps, th)
        assert abs(phi - phi_o) <= 1e-10 * abs(phi_o)
        assert np.linalg.norm(grad - grad_o) <= 1e-10 * np.linalg.norm(grad_o)
    b.eval()
    torch.cuda.synchronize()
    for (phi, grad), (*_, o, g) in zip(first, keep):
        assert o.item() == phi
        np.testing.assert_array_equal(g.cpu().numpy(), grad)
    b.close()


@pytest.mark.parametrize("prec", [pd.PD_FP32, pd.PD_BF16X3])
def test_reduced_precision_batch_matches_oracle(prec):
    # within the reduced-precision bound of the single-map tests
    d, eps = 3, 2e-2
    raw = make_maps(6, d=d, seed=9, small=True)
    keep = []
    for shape, lab, N, th in raw:
        tt = dev(th)
        keep.append((pd.Grid(shape), dev(lab), N, tt, torch.empty((), dtype=torch.float64, device="cuda"),
                     torch.empty_like(tt)))
    b = pd.Batch(keep, d, eps, prec=prec, autotune=True)
    b.eval()
    torch.cuda.synchronize()
    if prec == pd.PD_BF16X3:
        assert b.info()["chunk_factor"] in (1, 2, 4, 8)
    for (shape, lab, N, th), (*_, o, g) in zip(raw, keep):
        phi_o, grad_o = O.objective_grad(O.Grid(shape), lab, N, d, eps, th)
        assert abs(o.item() - phi_o) <= 1e-6 * abs(phi_o)
        assert np.linalg.norm(g.cpu().numpy() - grad_o) <= 1e-5 * np.linalg.norm(grad_o)
    b.close()


@pytest.mark.parametrize("prec", [pd.PD_FP32, pd.PD_BF16X3])
def test_inactive_maps_untouched(prec):
    d, eps = 2, 5e-2
    raw = make_maps(4, d=d, seed=3, small=True)
    keep = []
    for shape, lab, N, th in raw:
        tt = dev(th)
        keep.append((pd.Grid(shape), dev(lab), N, tt, torch.full((), 7.0, dtype=torch.float64, device="cuda"),
                     torch.full_like(tt, 7.0)))
    b = pd.Batch(keep, d, eps, prec=prec, autotune=False)
    b.set_active([1, 0, 1, 0])
    b.eval()
    torch.cuda.synchronize()
    for q, (*_, o, g) in enumerate(keep):
        if q % 2:
            assert o.item() == 7.0 and bool(torch.all(g == 7.0))
        else:
            assert o.item() != 7.0
    # all active again: the graph evaluates every map
    b.set_active([1, 1, 1, 1])
    b.eval()
    torch.cuda.synchronize()
    assert all(o.item() != 7.0 for *_, o, g in keep)
    b.close()


def test_fit_batched_reaches_single_map_optima():
    # non-separable maps (label noise): unique maxima (Prop. 4.11)
    d, eps = 2, 0.05
    maps, thetas, single = [], [], []
    for q in range(4):
        g, lab, N = power_problem((40 + 8 * q, 36), 5 + q, seed=50 + q)
        flip = synth.rng(60 + q).random(g.P) < 0.1
        lab = np.where(flip, synth.random_labels(70 + q, g.P, N), lab).astype(np.int32)
        grid = pd.Grid((40 + 8 * q, 36))
        lt = dev(lab)
        maps.append((grid, lt, N))
        thetas.append(torch.zeros((N, 6), dtype=torch.float64, device="cuda"))
        _, rep = pd.pd_fit(grid, lt, N, d, eps, max_iter=600, gtol=1e-12)
        single.append(rep)
    reps = pd.pd_fit_batched(maps, thetas, d, eps, max_iter=600, gtol=1e-12)
    for r, s in zip(reps, single):
        assert abs(r["phi"] - s["phi"]) <= 1e-9 * abs(s["phi"]), (r, s)
    # FP32 phase + FP64 refinement reaches the same optima
    thetas2 = [torch.zeros_like(t) for t in thetas]
    reps2 = pd.pd_fit_batched(maps, thetas2, d, eps, max_iter=300, prec=pd.PD_FP32, refine_iter=600,
                              switch_rtol=1e-7, gtol=1e-12)
    for r, s in zip(reps2, single):
        assert abs(r["phi"] - s["phi"]) <= 1e-8 * abs(s["phi"]), (r, s)
    # a BF16X3 phase on the tensor cores + FP64 refinement, warm-started from
    # a short FP64 run: the same optima
    thetas3 = [torch.zeros_like(t) for t in thetas]
    pd.pd_fit_batched(maps, thetas3, d, eps, max_iter=20)
    reps3 = pd.pd_fit_batched(maps, thetas3, d, eps, init=pd.PD_INIT_GIVEN, max_iter=300, prec=pd.PD_BF16X3,
                              refine_iter=600, switch_rtol=1e-7, gtol=1e-12)
    for r, s in zip(reps3, single):
        assert abs(r["phi"] - s["phi"]) <= 1e-8 * abs(s["phi"]), (r, s)
    # with eps-annealing (0.2, 0.1, then eps = 0.05): the same optima
    thetas4 = [torch.zeros_like(t) for t in thetas]
    reps4 = pd.pd_fit_batched(maps, thetas4, d, eps, max_iter=300, prec=pd.PD_BF16X3, refine_iter=600,
                              switch_rtol=1e-7, gtol=1e-12, anneal_eps0=0.2, anneal_factor=0.5, anneal_iter=30)
    for r, s in zip(reps4, single):
        assert r["stages"] == 3 and r["eps_final"] == eps, r
        assert abs(r["phi"] - s["phi"]) <= 1e-8 * abs(s["phi"]), (r, s)
