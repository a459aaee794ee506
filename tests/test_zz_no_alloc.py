"""ctis_forward_static_scratch: the forward projection with its scratch in a
fixed array inside the library, for callers that cannot call cudaMalloc when
they project (allocation-free real-time loops, code whose device memory all
belongs to its own pool, code running under a stream capture that rejects
allocation). It must give the FP64 oracle's H f within the projector
tolerance, and ctis_forward's H f bit for bit, call after call, even though
every call reuses the array the previous call left behind; and a call must
allocate nothing.

Runs last (file name) so that a failure here does not stop the rest of a
"-x" run; it also passes alone in a fresh process, where the first call sets
up the array's device address."""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import Plan, load
from tests.helpers import floored_rel, geometry

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the projector tolerance of the parity tests

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 3)
@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _forward_static(plan, f, out, stream=None):
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream()
    return lib.ctis_forward_static_scratch(
        plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(st.cuda_stream))


def _edge_psf(wl, boundary):
    """The grating PSF of wl moved so that light leaves the FPA: shifted
    left and down under clip (footprints cross the edges and are cut), to
    the FPA's last column and row under wrap (shifted copies re-enter)."""
    ptr, x, y, v = synth.make_psf(wl)
    if boundary == "clip":
        x, y = x - 7, y + 6
    elif boundary == "wrap":
        x, y = x + wl.gamma - 1 - x.max(), y + wl.xi - 1 - y.max()
    return ptr, x.astype(np.int32), y.astype(np.int32), v


def _case(wl, dtype, boundary, seed):
    psf = _edge_psf(wl, boundary) if boundary != "reject" else synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf, boundary)
    if dtype == "bf16":
        taps = O.with_values(taps, O.round_bf16(taps.v))
    f = synth.random_positive((wl.w, wl.alpha, wl.a), seed)
    if dtype == "bf16":
        f = O.round_bf16(f).astype(np.float32)
    return psf, O.BlockH(geom, taps), f


CASES = [(synth.TINY, "f32", "reject", "32x32"), (RAGGED, "f32", "reject", "32x32"),
         (synth.MODEL_A, "f32", "reject", "32x32"), (synth.REALISTIC, "f32", "reject", "32x32"),
         (RAGGED, "bf16", "reject", "32x32"), (RAGGED, "f32", "clip", "32x32"),
         (synth.TINY, "f32", "wrap", "32x32"), (RAGGED, "bf16", "clip", "32x32"),
         (RAGGED, "f32", "reject", "32x16"), (synth.MODEL_A, "bf16", "clip", "32x16")]


@pytest.mark.parametrize("wl,dtype,boundary,tile", CASES,
                         ids=[f"{w.name}-{d}-{b}-{t}" for w, d, b, t in CASES])
def test_static_scratch_forward_matches_oracle_and_forward_on_consecutive_calls(wl, dtype, boundary,
                                                                               tile):
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    psf = _edge_psf(wl, boundary) if boundary != "reject" else synth.make_psf(wl)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype=dtype, boundary=boundary,
              forward_tile=tile) as plan:
        for seed in (101, 102):   # two calls in a row, different inputs
            _, H, f = _case(wl, dtype, boundary, seed)
            ft = torch.from_numpy(f).to(tdt).cuda()
            ref = plan.forward(ft)
            out = torch.full_like(ref, float("nan"))
            assert _forward_static(plan, ft, out) == 0, load().ctis_last_error()
            plan.check()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert floored_rel(got, H.forward(f.ravel())) <= TOL
            # same kernel, same tables, same summation order
            assert np.array_equal(got, ref.cpu().numpy())


def test_static_scratch_call_allocates_nothing():
    """After the first call on the device (which looks up the array's
    address), a call leaves the device's free memory and torch's allocator
    counters unchanged, and it can be recorded in a stream capture whose mode
    rejects allocation (torch.cuda.graph captures in global mode); the
    replayed graph gives the same H f."""
    wl = synth.MODEL_A
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl)) as plan:
        _, H, f = _case(wl, "f32", "reject", 103)
        ft = torch.from_numpy(f).cuda()
        out = torch.empty((wl.xi, wl.gamma), device="cuda")
        assert _forward_static(plan, ft, out) == 0, load().ctis_last_error()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        stats0 = {k: v for k, v in torch.cuda.memory_stats().items() if "allocation" in k}
        for _ in range(3):
            assert _forward_static(plan, ft, out) == 0, load().ctis_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert {k: v for k, v in torch.cuda.memory_stats().items() if "allocation" in k} == stats0
        want = out.cpu().numpy().copy()
        assert floored_rel(want, H.forward(f.ravel())) <= TOL

        out2 = torch.full_like(out, float("nan"))
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s, capture_error_mode="global"):
                rc = _forward_static(plan, ft, out2, s)
        assert rc == 0, load().ctis_last_error()
        graph.replay()
        torch.cuda.synchronize()
        plan.check()
        assert np.array_equal(out2.cpu().numpy(), want)
        del graph


def test_static_scratch_rejects_plans_it_cannot_hold():
    wl = synth.LARGE   # its shifted copies of f alone need about 136 MB
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl)) as plan:
        f = torch.ones((wl.w, wl.alpha, wl.a), device="cuda")
        out = torch.empty((wl.xi, wl.gamma), device="cuda")
        rc = _forward_static(plan, f, out)
        assert rc == -6   # CTIS_ERR_UNSUPPORTED
        assert b"static scratch" in load().ctis_last_error()
