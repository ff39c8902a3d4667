"""The 3-D workload: 256^3 voxels, N = 2000 grains of a seeded anisotropic
power diagram (SPD metrics with eigenvalues log-uniform in [0.5, 2]), fit
degree 2 (K = 10) and 3 (K = 20), eps = 1e-3.

The oracle cannot evaluate 3.4e10 voxel-grain pairs in reasonable time, so
(i) a seeded random 1/256 subsample of the voxels, as an explicit point
list labelled by the oracle, is checked pair-for-pair against the oracle
(objective, gradient, Hessian-vector product), and (ii) the full structured
grid is checked through properties that hold at any size: Phi(0) = -log N
exactly (Sec. 2.1), gauge invariance (Lemma 4.2), and equality of the
structured-grid and point-list evaluations of the same voxels.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth
from helpers import rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SHAPE = (256, 256, 256)
N0 = 2000
EPS = 1e-3


def centres(idx):
    n = SHAPE[0]
    k0 = idx % n
    k1 = (idx // n) % n
    k2 = idx // (n * n)
    c = lambda k: -1.0 + (2.0 * k + 1.0) / n
    return np.stack([c(k0), c(k1), c(k2)], 1)


def morton(idx):
    """Z-curve key of linear voxel indices (bits of x, y, z interleaved)."""
    n = SHAPE[0]
    k = [idx % n, (idx // n) % n, idx // (n * n)]
    key = np.zeros_like(idx)
    for b in range(8):
        for a in range(3):
            key |= ((k[a] >> b) & 1) << (3 * b + a)
    return key


@pytest.fixture(scope="module")
def apd():
    y, w, A = synth.apd_params(synth.SEED_BASE + 2, N0, dim=3)
    return y, w, A


@pytest.mark.parametrize("d", [2, 3])
def test_subsample_matches_oracle(apd, d):
    y, w, A = apd
    P = int(np.prod(SHAPE))
    idx = np.sort(synth.rng(synth.SEED_BASE + 30 + d).choice(P, size=P // 256, replace=False))
    pts = centres(idx)
    g = O.Grid(coords=pts)
    th_true = O.theta_from_apd(3, 2, y, w, A)
    lab, _ = O.assign(g, N0, 2, th_true)
    lab, N, used = synth.compact(lab)
    K = O.K(3, d)
    th = np.zeros((N, K))
    th[:, :10] = th_true[used]          # degree-2 parameters padded to degree d
    phi_o, grad_o = O.objective_grad(g, lab, N, d, EPS, th)
    grid = pd.Grid(coords=torch.from_numpy(pts).cuda())
    dl, dth = torch.from_numpy(lab.astype(np.int32)).cuda(), torch.from_numpy(th).cuda()
    obj, grad = pd.pd_objective_grad(grid, dl, N, dth, d, EPS, prec=pd.PD_FP64)
    assert abs(obj.item() - phi_o) <= 1e-10 * abs(phi_o)
    assert rel(grad.cpu().numpy(), grad_o) <= 1e-10
    # the reduced precisions take 128 consecutive points as one tile and
    # keep each logit relative to the tile (its first point); the float
    # remainder theta'.(eta(x) - eta(c)) grows with the tile's extent.  In
    # index order a tile of this 1/256 subsample spans half a z-slice; in
    # z-curve order about 32^3 voxels (0.25 per axis, against 0.03 for the
    # full grid's 8 x 4 x 4 tiles), which the bounds below reflect.  Phi and
    # its gradient do not depend on the order.
    order = np.argsort(morton(idx), kind="stable")
    gm = pd.Grid(coords=torch.from_numpy(np.ascontiguousarray(pts[order])).cuda())
    dlm = torch.from_numpy(np.ascontiguousarray(lab[order]).astype(np.int32)).cuda()
    obj32, grad32 = pd.pd_objective_grad(grid, dl, N, dth, d, EPS, prec=pd.PD_FP32)
    objz, gradz = pd.pd_objective_grad(gm, dlm, N, dth, d, EPS, prec=pd.PD_FP32)
    print("3-D d=%d: N=%d, fp32 rel err index order: phi %.2e grad %.2e; z order: phi %.2e grad %.2e" % (
        d, N, abs(obj32.item() - phi_o) / abs(phi_o), rel(grad32.cpu().numpy(), grad_o),
        abs(objz.item() - phi_o) / abs(phi_o), rel(gradz.cpu().numpy(), grad_o)))
    assert abs(obj32.item() - phi_o) <= 1e-5 * abs(phi_o)
    assert rel(grad32.cpu().numpy(), grad_o) <= 1e-3
    assert abs(objz.item() - phi_o) <= 1e-5 * abs(phi_o)
    assert rel(gradz.cpu().numpy(), grad_o) <= 1e-4
    if d == 2:
        # tensor cores: their tiles are 128 consecutive points of the list
        # and every logit is split at the tile's first point, so a point
        # list must be ordered along space; Phi and its gradient do not
        # depend on the order, so the same voxels in Morton (z-curve) order
        # are compared with the same oracle values.  At this density (one
        # voxel in 256) a tile still spans about 32^3 voxels, and the fp32
        # accumulation of the tensor cores acts on logit parts 8x larger
        # than on the full grid's 8x4x4 tiles: the bound is 5e-4 here, 1e-5
        # on the full grid (test_full_grid_properties)
        obj3, grad3 = pd.pd_objective_grad(gm, dlm, N, dth, d, EPS, prec=pd.PD_BF16X3)
        print("3-D d=2 point list (z-order): bf16x3 rel err phi %.2e grad %.2e" % (
            abs(obj3.item() - phi_o) / abs(phi_o), rel(grad3.cpu().numpy(), grad_o)))
        assert abs(obj3.item() - phi_o) <= 5e-4 * abs(phi_o)
        assert rel(grad3.cpu().numpy(), grad_o) <= 2e-3
        v = synth.random_theta(synth.SEED_BASE + 40, N, K, 1e-3)
        hv_o = O.hvp(g, lab, N, d, EPS, th, v)
        hv = pd.pd_hvp(grid, dl, N, dth, torch.from_numpy(v).cuda(), d, EPS, prec=pd.PD_FP64)
        assert rel(hv.cpu().numpy(), hv_o) <= 1e-10
        obj16, _ = pd.pd_objective_grad(grid, dl, N, dth, d, EPS, prec=pd.PD_BF16)
        print("3-D d=2: bf16 rel err phi %.2e" % (abs(obj16.item() - phi_o) / abs(phi_o)))


def test_full_grid_properties(apd):
    y, w, A = apd
    d = 2
    th_true = pd.pd_theta_from_apd(3, 2, y, w, A).cuda()
    grid = pd.Grid(SHAPE)
    lab, _, _ = pd.pd_assign(grid, N0, 2, th_true)
    N = N0
    # Phi(0) = -log N exactly
    obj0, _ = pd.pd_objective_grad(grid, lab, N, torch.zeros_like(th_true), d, EPS, prec=pd.PD_FP32,
                                   want_grad=False)
    assert abs(obj0.item() + math.log(N)) <= 1e-6 * math.log(N)
    # gauge invariance
    c = torch.from_numpy(synth.random_theta(5, 1, 10, 0.3)).cuda()
    o1, g1 = pd.pd_objective_grad(grid, lab, N, th_true, d, EPS, prec=pd.PD_FP64)
    # the tensor cores on the full grid (8 x 4 x 4 voxel tiles) against FP64
    o3, g3 = pd.pd_objective_grad(grid, lab, N, th_true, d, EPS, prec=pd.PD_BF16X3)
    print("3-D full grid d=2: bf16x3 rel err vs fp64: phi %.2e grad %.2e" % (
        abs(o3.item() - o1.item()) / abs(o1.item()), rel(g3.cpu().numpy(), g1.cpu().numpy())))
    assert abs(o3.item() - o1.item()) <= 1e-5 * abs(o1.item())
    assert rel(g3.cpu().numpy(), g1.cpu().numpy()) <= 1e-5
    o2, g2 = pd.pd_objective_grad(grid, lab, N, th_true + c, d, EPS, prec=pd.PD_FP64)
    assert abs(o1.item() - o2.item()) <= 1e-9 * abs(o1.item())
    assert rel(g2.cpu().numpy(), g1.cpu().numpy()) <= 1e-8
    # a slab of voxels: structured grid == point list of the same voxels
    slab = (256, 256, 8)
    idx = np.arange(int(np.prod(slab)))
    pts = centres(idx)[:, :3]
    pts[:, 2] = -1.0 + (2.0 * (idx // (256 * 256)) + 1.0) / 8.0     # the slab's own z-centres
    gs = pd.Grid(slab)
    gl = pd.Grid(coords=torch.from_numpy(pts).cuda())
    lab_s = lab[: int(np.prod(slab))].contiguous()
    a = pd.pd_objective_grad(gs, lab_s, N, th_true, d, EPS, prec=pd.PD_FP64)
    b = pd.pd_objective_grad(gl, lab_s, N, th_true, d, EPS, prec=pd.PD_FP64)
    assert a[0].item() == b[0].item()
    assert torch.equal(a[1], b[1])
