"""ctis_forward_static_scratch: the forward projection with its scratch in a
fixed array inside the library, for callers that cannot call cudaMalloc when
they project (allocation-free real-time loops, code whose device memory all
belongs to its own pool, code running under a stream capture that rejects
allocation). It must give the same H f as ctis_forward, call after call, even
though every call reuses the array the previous call left behind.

Runs last (file name) so that a failure here does not stop the rest of a
"-x" run; it also passes alone in a fresh process, where the first call sets
up the array's device address."""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
import synth
from paper_2006_01573_gb300 import Plan, load
from tests.helpers import floored_rel

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the projector tolerance of the parity tests

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _forward_static(plan, f, out):
    lib = load()
    return lib.ctis_forward_static_scratch(
        plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("wl", [synth.TINY, RAGGED, synth.MODEL_A, synth.REALISTIC],
                         ids=lambda w: w.name)
def test_static_scratch_forward_matches_forward_on_consecutive_calls(wl):
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl)) as plan:
        for seed in (101, 102):   # two calls in a row, different inputs
            f = torch.from_numpy(synth.random_positive((wl.w, wl.alpha, wl.a), seed)).cuda()
            ref = plan.forward(f)
            out = torch.full_like(ref, float("nan"))
            assert _forward_static(plan, f, out) == 0, load().ctis_last_error()
            plan.check()
            got = out.cpu().numpy()
            want = ref.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert floored_rel(got, want) <= TOL
            # same kernel, same tables, same summation order
            assert np.array_equal(got, want)


def test_static_scratch_rejects_plans_it_cannot_hold():
    wl = synth.LARGE   # its shifted copies of f alone need about 136 MB
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl)) as plan:
        f = torch.ones((wl.w, wl.alpha, wl.a), device="cuda")
        out = torch.empty((wl.xi, wl.gamma), device="cuda")
        rc = _forward_static(plan, f, out)
        assert rc == -6   # CTIS_ERR_UNSUPPORTED
        assert b"static scratch" in load().ctis_last_error()
