"""pd_objective_grad_noalloc: the objective/gradient evaluation for callers
that cannot allocate device memory (their memory is reserved up front by
another allocator, or allocation is forbidden after start-up).  Its scratch
is a fixed array inside the library, so it must give the same results as
pd_objective_grad, call after call, even though every call reuses the same
array.  This file is collected last so that a failure here does not stop a
`-x` run before the other tests have run."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_20816_gb300 import pd, synth

from helpers import USED_MEM_CURRENT, USED_MEM_HIGH, DefaultPool

pytestmark = pytest.mark.gpu

def _problem(seed, shape, N, d, scale):
    g = O.Grid(shape)
    lab = torch.from_numpy(synth.random_labels(seed, g.P, N)).cuda()
    th = torch.from_numpy(synth.random_theta(seed + 1, N, O.K(2, d), scale)).cuda()
    return lab, th


@pytest.mark.parametrize("prec,tol_phi,tol_grad", [(pd.PD_FP64, 1e-12, 1e-12), (pd.PD_FP32, 1e-6, 1e-5)])
def test_noalloc_matches_objective_grad_twice(prec, tol_phi, tol_grad):
    shape, N, d, eps = (300, 257), 140, 4, 1e-2
    grid = pd.Grid(shape)
    obj = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty((N, O.K(2, d)), dtype=torch.float64, device="cuda")
    for call, seed in enumerate((3, 40)):   # two calls in a row on the shared array
        lab, th = _problem(seed, shape, N, d, 0.02)
        want_obj, want_grad = pd.pd_objective_grad(grid, lab, N, th, d, eps, prec=prec)
        torch.cuda.synchronize()
        # the entry point's defining property: no device allocation, neither
        # from the driver's default pool nor from torch's allocator
        pool = DefaultPool()
        used0 = pool.get(USED_MEM_CURRENT)
        pool.reset_high()
        torch_allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        pd.pd_objective_grad_noalloc(grid, lab, N, th, d, eps, prec=prec, obj_out=obj, grad_out=grad)
        torch.cuda.synchronize()
        assert pool.get(USED_MEM_HIGH) <= used0, (pool.get(USED_MEM_HIGH), used0)
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == torch_allocs0
        a, b = obj.item(), want_obj.item()
        assert abs(a - b) <= tol_phi * abs(b), (call, a, b)
        gw = want_grad.cpu().numpy()
        assert np.linalg.norm(grad.cpu().numpy() - gw) <= tol_grad * np.linalg.norm(gw), call


def test_noalloc_rejects_problems_beyond_its_scratch():
    # 4096 x 4096 pixels need 64 MiB of log S in FP32: more than the array
    shape, N, d = (4096, 4096), 3, 1
    grid = pd.Grid(shape)
    lab = torch.zeros(shape[0] * shape[1], dtype=torch.int32, device="cuda")
    th = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PdError) as e:
        pd.pd_objective_grad_noalloc(grid, lab, N, th, d, 0.1, prec=pd.PD_FP32)
    assert e.value.code == pd.PD_ESCRATCH
    # an out-of-range precision is an invalid argument, as for pd_objective_grad
    small = pd.Grid((16, 16))
    with pytest.raises(pd.PdError) as e:
        pd.pd_objective_grad_noalloc(small, lab[:256], N, th, d, 0.1, prec=7)
    assert e.value.code == pd.PD_EINVAL
