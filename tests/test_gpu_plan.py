"""Plans (pd_plan_*): repeated evaluations on one pixel set and label map
with the scratch allocated once and the centre features and grain order
computed by the first call.  A plan evaluation runs the same kernels on the
same inputs as the one-off call, so the results must be bitwise equal to
pd_objective_grad / pd_hvp -- on the first call, which fills the cached
data, and on every later one, which reuses it -- and no call after the
plan's creation may allocate device memory."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth

from helpers import USED_MEM_CURRENT, USED_MEM_HIGH, DefaultPool, poly_problem

pytestmark = pytest.mark.gpu

PRECS = [pd.PD_FP64, pd.PD_FP32, pd.PD_BF16, pd.PD_BF16X3]


def _setup(shape, N, d, seed):
    g, lab, N_eff, th = poly_problem(shape, N, d, seed)
    dim = len(shape)
    lab_t = torch.from_numpy(lab).cuda()
    # a parameter near the generating one (so that the gradient pass keeps
    # few tile/grain pairs) and a direction for the Hessian
    rng = np.random.default_rng(seed + 5)
    th = th - th[-1]
    th_t = torch.from_numpy(th + 0.01 * rng.standard_normal(th.shape)).cuda()
    v_t = torch.from_numpy(rng.standard_normal(th.shape)).cuda()
    return pd.Grid(shape), lab_t, N_eff, th_t, v_t, O.K(dim, d)


def _same(a, b):
    return torch.equal(a, b) and a.dtype == b.dtype


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,N,d", [((200, 190), 60, 4), ((24, 20, 18), 20, 2)])
def test_plan_equals_one_off_calls(prec, shape, N, d):
    grid, lab, N, th, v, K = _setup(shape, N, d, 11)
    plan = pd.Plan(grid, lab, N, d, prec=prec, hvp=True)
    assert plan.scratch_bytes() > 0
    for eps in (2e-2, 5e-3, 2e-2):          # eps may change between calls
        for rep in range(2):                # the second call reuses the cached data
            th_r = th * (1.0 + 0.1 * rep)
            want_o, want_g = pd.pd_objective_grad(grid, lab, N, th_r, d, eps, prec=prec)
            got_o, got_g = plan.objective_grad(th_r, eps)
            assert _same(got_o, want_o), (eps, rep, got_o.item(), want_o.item())
            assert _same(got_g, want_g), (eps, rep)
            # objective only, as the one-off objective-only call (on tensor
            # cores that call keeps the grains in index order, so its Phi may
            # differ from the gradient call's in the last bits)
            want_oo, _ = pd.pd_objective_grad(grid, lab, N, th_r, d, eps, prec=prec, want_grad=False)
            only_o, none = plan.objective_grad(th_r, eps, want_grad=False)
            assert none is None and _same(only_o, want_oo), (only_o.item(), want_oo.item())
            want_h = pd.pd_hvp(grid, lab, N, th_r, v, d, eps, prec=prec)
            got_h = plan.hvp(th_r, v, eps)
            assert _same(got_h, want_h), (eps, rep)
    plan.close()


@pytest.mark.parametrize("prec", [pd.PD_FP32, pd.PD_BF16X3])
def test_plan_calls_allocate_nothing(prec):
    grid, lab, N, th, v, K = _setup((256, 256), 90, 6, 23)
    plan = pd.Plan(grid, lab, N, 6, prec=prec, hvp=True)
    obj = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty((N, K), dtype=torch.float64, device="cuda")
    hv = torch.empty((N, K), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    pool = DefaultPool()
    used0 = pool.get(USED_MEM_CURRENT)
    pool.reset_high()
    torch_allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        plan.objective_grad(th, 1e-2, obj_out=obj, grad_out=grad)
        plan.hvp(th, v, 1e-2, out=hv)
    torch.cuda.synchronize()
    assert pool.get(USED_MEM_HIGH) <= used0, (pool.get(USED_MEM_HIGH), used0)
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == torch_allocs0
    assert np.isfinite(obj.item()) and torch.isfinite(grad).all() and torch.isfinite(hv).all()
    plan.close()


def test_plan_argument_errors():
    grid, lab, N, th, v, K = _setup((64, 60), 12, 2, 31)
    plan = pd.Plan(grid, lab, N, 2, prec=pd.PD_FP32)        # no Hessian scratch
    with pytest.raises(pd.PdError) as e:
        plan.hvp(th, v, 1e-2)
    assert e.value.code == pd.PD_EINVAL
    for eps in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(pd.PdError) as e:
            plan.objective_grad(th, eps)
        assert e.value.code == pd.PD_EINVAL
    plan.close()
    plan.close()                                             # closing twice is a no-op
    with pytest.raises(pd.PdError) as e:
        pd.Plan(grid, lab, N, 2, prec=7)
    assert e.value.code == pd.PD_EINVAL
    with pytest.raises(pd.PdError) as e:
        pd.Plan(grid, lab, 1, 2)
    assert e.value.code == pd.PD_EINVAL
    with pytest.raises(pd.PdError) as e:
        pd.Plan(grid, lab, N, 9)                             # above the 2-D maximum degree
    assert e.value.code == pd.PD_ENOTSUP


@pytest.mark.parametrize("prec", PRECS)
def test_plan_graph_replay_follows_theta(prec):
    # the calls of a fit: the same buffers every time, theta rewritten in
    # place; from the second call on the plan replays a recorded graph,
    # which must read the current theta and v
    grid, lab, N, th0, v, K = _setup((200, 190), 60, 4, 17)
    plan = pd.Plan(grid, lab, N, 4, prec=prec, hvp=True)
    th = th0.clone()
    obj = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty_like(th)
    hv = torch.empty_like(th)
    vv = v.clone()
    for rep in range(4):
        th.copy_(th0 * (1.0 + 0.05 * rep))
        vv.copy_(v * (1.0 - 0.1 * rep))
        want_o, want_g = pd.pd_objective_grad(grid, lab, N, th, 4, 1e-2, prec=prec)
        want_h = pd.pd_hvp(grid, lab, N, th, vv, 4, 1e-2, prec=prec)
        plan.objective_grad(th, 1e-2, obj_out=obj, grad_out=grad)
        plan.hvp(th, vv, 1e-2, out=hv)
        torch.cuda.synchronize()
        assert _same(obj, want_o) and _same(grad, want_g), rep
        assert _same(hv, want_h), rep
    plan.close()
