"""Failure detection without a GPU fault: a bounded device wait on an
mbarrier that nothing completes gives up, reports PD_ETIMEOUT, and leaves
the context usable; host-side errors come back as status codes."""
import math

import numpy as np
import pytest
import torch

from paper_2605_20816_gb300 import pd

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    assert pd.pd_selftest_wait_timeout(0.05) == pd.PD_ETIMEOUT
    # the context still works
    grid = pd.Grid((32, 32))
    lab = (torch.arange(1024, dtype=torch.int32, device="cuda") % 5).contiguous()
    th = torch.zeros((5, 6), dtype=torch.float64, device="cuda")
    for prec in (pd.PD_FP64, pd.PD_BF16X3):
        obj, _ = pd.pd_objective_grad(grid, lab, 5, th, 2, 0.1, prec=prec)
        torch.cuda.synchronize()
        assert abs(obj.item() + math.log(5)) < 1e-6


def test_selftest_argument_checks():
    with pytest.raises(pd.PdError) as e:
        pd.pd_selftest_wait_timeout(5.0)
    assert e.value.code == pd.PD_EINVAL


def test_nonfinite_parameters_reported_by_fit():
    grid = pd.Grid((16, 16))
    lab = (torch.arange(256, dtype=torch.int32, device="cuda") % 3).contiguous()
    th = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    th[0, 0] = float("nan")
    with pytest.raises(pd.PdError) as e:
        pd.pd_fit(grid, lab, 3, 1, 0.1, theta=th, init=pd.PD_INIT_GIVEN, max_iter=3)
    assert e.value.code == pd.PD_ENAN
