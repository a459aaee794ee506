"""The gather kernels' bounded waits, exercised without a fault: with the
plan's test hook (ctis_plan_set_debug, CTIS_DEBUG_DROP_COPIES) every copy
barrier is armed but no copy is issued, so each warp's wait runs out after
about a second; the kernel records the failure and returns, ctis_plan_check
reports CTIS_ERR_TIMEOUT, and the same plan then projects and reconstructs
correctly once the hook is cleared (the context stayed usable)."""
import time

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CtisError, Plan
from tests.helpers import floored_rel, problem

pytestmark = pytest.mark.gpu

CTIS_ERR_TIMEOUT = -5


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_waits_that_run_out_report_a_timeout_and_the_plan_recovers():
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 101)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        ft = torch.from_numpy(f).cuda()
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        plan.set_debug(True)
        t0 = time.monotonic()
        plan.forward(ft)                       # raw forward: one launch
        with pytest.raises(CtisError) as e:
            plan.check()
        assert e.value.code == CTIS_ERR_TIMEOUT
        plan.reconstruct(gt, 1, init="ones", stats=True)   # the EM graph: both kernels
        with pytest.raises(CtisError) as e:
            plan.check()
        assert e.value.code == CTIS_ERR_TIMEOUT
        assert time.monotonic() - t0 < 60.0    # each wait gave up after about a second
        plan.set_debug(False)
        hf = plan.forward(ft).cpu().numpy().ravel()
        out, _ = plan.reconstruct(gt, 3, init="ones")
        plan.check()                           # the flag was cleared by the last check
    assert floored_rel(hf, H.forward(f.ravel())) <= 1e-5
    ref, _ = O.mlem(H, g, 3)
    assert floored_rel(out.cpu().numpy().ravel(), ref) <= 3e-5


def test_the_hook_takes_only_known_flags():
    wl = synth.TINY
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl)) as plan:
        from paper_2006_01573_gb300 import load
        import ctypes
        assert load().ctis_plan_set_debug(plan._h, 4) != 0
        assert load().ctis_plan_set_debug(plan._h, 2) == 0
        assert load().ctis_plan_set_debug(plan._h, 0) == 0
