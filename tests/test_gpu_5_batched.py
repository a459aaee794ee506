"""GPU tests of the batched form: many frames of several plans in one call
(one CUDA graph), each frame reconstructed exactly as a single-frame call
would, and against the FP64 oracle.

A frame of a batch runs the same kernels over the same work lists, tables and
summation order as a single-frame reconstruction (only the warps that run its
items differ, and partial sums are still added in chunk order), so its result
and statistics must be bit-identical to ctis_reconstruct's."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CtisError, Plan, reconstruct_batched
from tests.helpers import floored_rel, geometry, rel_l2

pytestmark = pytest.mark.gpu

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _plan(wl, dtype="f32", forward_tile="32x32"):
    return Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl), dtype=dtype,
                forward_tile=forward_tile)


def _frame_g(plan, wl, seed):
    """A per-frame measurement: Poisson counts of H f_scene(seed)."""
    f = torch.from_numpy(synth.make_scene(wl, seed)).cuda()
    if plan.dtype == 1:
        f = f.to(torch.bfloat16)
    g, _ = synth.make_measurement(plan.forward(f).cpu().numpy(), wl.peak, seed)
    return torch.from_numpy(g).cuda()


@pytest.mark.parametrize("init", ["ones", "htg", None])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_frames_equal_single_frame_reconstructions(init, dtype):
    wls = [synth.TINY, RAGGED]
    plans = [_plan(wl, dtype) for wl in wls]
    try:
        plan_idx = [0, 1, 0, 0, 1, 0, 1, 0]     # interleaved, 5 + 3 frames
        gs = [_frame_g(plans[i], wls[i], 100 + n) for n, i in enumerate(plan_idx)]
        k = 7
        f0 = None
        if init is None:
            f0 = [torch.from_numpy(synth.random_positive((wls[i].w, wls[i].alpha, wls[i].a), 200 + n))
                  .to(plans[i]._f_dtype()).cuda() for n, i in enumerate(plan_idx)]
            fs = [f.clone() for f in f0]
        else:
            fs = None
        fs, st = reconstruct_batched(plans, plan_idx, gs, k, fs=fs, init=init, stats=True)
        for p in plans:
            p.check()
        for n, i in enumerate(plan_idx):
            f1 = f0[n].clone() if init is None else None
            ref, ref_st = plans[i].reconstruct(gs[n], k=k, f=f1, init=init, stats=True)
            plans[i].check()
            assert torch.equal(fs[n], ref), f"frame {n}"
            assert torch.equal(st[n], ref_st), f"frame {n} statistics"
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batched_plans_of_different_forward_tiles(dtype):
    """Plans of one batch may use different forward tile shapes (each plan's
    frames run on its own launches): every frame equals its single-frame
    reconstruction bit for bit, statistics included."""
    wls = [synth.TINY, RAGGED]
    plans = [_plan(wls[0], dtype, "32x16"), _plan(wls[1], dtype, "32x32")]
    try:
        assert [p.forward_tile() for p in plans] == ["32x16", "32x32"]
        plan_idx = [1, 0, 0, 1, 0]
        gs = [_frame_g(plans[i], wls[i], 300 + n) for n, i in enumerate(plan_idx)]
        k = 5
        fs, st = reconstruct_batched(plans, plan_idx, gs, k, init="ones", stats=True)
        for p in plans:
            p.check()
        for n, i in enumerate(plan_idx):
            ref, ref_st = plans[i].reconstruct(gs[n], k=k, init="ones", stats=True)
            plans[i].check()
            assert torch.equal(fs[n], ref), f"frame {n}"
            assert torch.equal(st[n], ref_st), f"frame {n} statistics"
    finally:
        for p in plans:
            p.close()


def test_batched_against_oracle_and_replay():
    wl = synth.TINY
    geom = geometry(wl)
    psf = synth.make_psf(wl)
    H = O.build_H(geom, psf)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gs = []
        for n in range(3):
            f_true = synth.make_scene(wl, 300 + n).ravel()
            g, _ = synth.make_measurement(H.forward(f_true), wl.peak, 300 + n)
            gs.append(g)
        gt = [torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda() for g in gs]
        fs, st = reconstruct_batched([plan], [0, 0, 0], gt, wl.k, stats=True)
        first = [f.clone() for f in fs]
        fs, st2 = reconstruct_batched([plan], [0, 0, 0], gt, wl.k, fs=fs, stats=st)  # cached graph
        plan.check()
        for n in range(3):
            ref, hist = O.mlem(H, gs[n], wl.k)
            got = fs[n].cpu().numpy().ravel()
            assert torch.equal(first[n], fs[n])
            assert floored_rel(got, ref) <= wl.k * 1e-5
            assert rel_l2(got, ref) <= 1e-5 * np.sqrt(wl.k)
            for t in (0, wl.k):
                assert abs(float(st2[n, t, 2]) - hist[t]["loglik"]) <= 1e-5 * abs(hist[t]["loglik"])


def test_batched_rejects_bad_arguments():
    wl = synth.TINY
    with _plan(wl) as plan:
        g = torch.ones((wl.xi, wl.gamma), device="cuda")
        with pytest.raises((CtisError, ValueError)):
            reconstruct_batched([plan], [1], [g], 2)
        with pytest.raises(CtisError):
            reconstruct_batched([plan, plan], [0, 1], [g, g], 2)


def test_batched_full_size_mixed_frames():
    """The 256-frame workload (192 frames of 64x64x32 -> 512x512 and 64 of
    128x128x64 -> 1024x1024, seeds 1000 + i, plans in a 3:1 mix) in the
    launch configuration of the benchmark, for 2 iterations; sampled frames
    must equal their single-frame reconstructions bit for bit."""
    wls = [synth.MODEL_A, synth.MODEL_B]
    plans = [_plan(wl) for wl in wls]
    try:
        plan_idx = [1 if i % 4 == 3 else 0 for i in range(256)]
        proto = [_frame_g(plans[0], wls[0], 1000), _frame_g(plans[1], wls[1], 1003)]
        gs = []
        for i, p in enumerate(plan_idx):
            gs.append(_frame_g(plans[p], wls[p], 1000 + i) if i in (0, 3, 128, 255) else proto[p])
        k = 2
        fs, st = reconstruct_batched(plans, plan_idx, gs, k, stats=True)
        for p in plans:
            p.check()
        for i in (0, 3, 128, 255):
            ref, ref_st = plans[plan_idx[i]].reconstruct(gs[i], k=k, init="ones", stats=True)
            plans[plan_idx[i]].check()
            assert torch.equal(fs[i], ref) and torch.equal(st[i], ref_st), f"frame {i}"
    finally:
        for p in plans:
            p.close()
