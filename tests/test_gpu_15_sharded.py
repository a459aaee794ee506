"""GPU parity of the wavelength-sharded EM reconstruction
(ctis_reconstruct_sharded; Eq. 8's sum over wavelength blocks split into
slices, one plan per slice). On one GPU the ranks are two host threads, each
with its own plan, stream and slice of the datacube; their reduction
callback waits for its own partial image, meets the other thread at a host
barrier and adds the two images in rank order (what an all-reduce of the
partial images does across GPUs). No kernel waits on another: the threads
synchronise on the host between launches. The gathered slices must match
the FP64 oracle's EM and the single-plan reconstruction within the EM
bounds (k * 1e-5 floored-relative, 1e-5 * sqrt(k) relative L2), and both
threads must return the same statistics, within 1e-5 of the oracle's."""
import math
import threading

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CtisError, Plan, shard_wavelengths, slice_psf
from tests.helpers import floored_rel, geometry, problem, rel_l2

pytestmark = pytest.mark.gpu

STAT_KEYS = ("flux_hf", "flux_g_covered", "loglik", "resid2")
RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 500.0, 6)


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


class _PairSum:
    """The all-reduce of `world` host threads' partial images, in rank order."""

    def __init__(self, world):
        self.world = world
        self.slots = [None] * world
        self.barrier = threading.Barrier(world, timeout=120)

    def reduce_of(self, rank, stream):
        def reduce(q):
            stream.synchronize()                  # this slice's image is complete
            self.slots[rank] = q.clone()
            self.barrier.wait()
            total = self.slots[0].clone()
            for r in range(1, self.world):
                total += self.slots[r]
            self.barrier.wait()                   # every rank has read every slot
            q.copy_(total)
            stream.synchronize()
        return reduce


def _sharded(wl, psf, g, k, world, init="ones", f0=None, forward_tile="32x32"):
    bounds = [shard_wavelengths(wl.w, world, r) for r in range(world)]
    red = _PairSum(world)
    out, errs = [None] * world, []

    def run(rank):
        try:
            s0, s1 = bounds[rank]
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                plan = Plan(wl.a, wl.alpha, s1 - s0, wl.gamma, wl.xi, slice_psf(psf, s0, s1),
                            forward_tile=forward_tile)
                gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
                f = None
                if f0 is not None:
                    f = torch.from_numpy(f0.reshape(wl.w, wl.alpha, wl.a)[s0:s1].copy()).cuda()
                f, stt = plan.reconstruct_sharded(gt, k, f=f, init=init, stats=True,
                                                  reduce=red.reduce_of(rank, st), stream=st)
                st.synchronize()
                plan.check()
                out[rank] = (f.double().cpu().numpy().ravel(), stt.cpu().numpy())
                plan.close()
        except BaseException as e:   # noqa: BLE001 - reported below
            errs.append(e)
            red.barrier.abort()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errs, errs
    return np.concatenate([o[0] for o in out]), [o[1] for o in out]


@pytest.mark.parametrize("wl,k,tile", [(synth.TINY, 10, "32x32"), (RAGGED, 6, "32x32"),
                                       (synth.MODEL_A, 4, "32x32"), (RAGGED, 6, "32x16")],
                         ids=["tiny", "ragged", "model_a", "ragged-32x16"])
def test_two_slices_reconstruct_like_the_whole_plan(wl, k, tile):
    geom, psf, H, _, g = problem(wl)
    f_ref, hist = O.mlem(H, g, k)
    f, stats = _sharded(wl, psf, g, k, 2, forward_tile=tile)
    floor = 1e-6 * np.abs(f_ref).max()
    assert np.max(np.abs(f - f_ref) / np.maximum(np.abs(f_ref), floor)) <= k * 1e-5
    assert rel_l2(f, f_ref) <= 1e-5 * math.sqrt(k)
    assert np.array_equal(stats[0], stats[1])
    for it in range(k + 1):
        for j, key in enumerate(STAT_KEYS):
            ref = hist[it][key]
            assert abs(stats[0][it, j] - ref) <= 1e-5 * abs(ref), (it, key)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        whole, _ = plan.reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), k,
                                    init="ones")
    assert floored_rel(f, whole.double().cpu().numpy().ravel()) <= 2 * k * 1e-5


def test_three_slices_from_a_given_iterate():
    wl = RAGGED
    geom, psf, H, _, g = problem(wl)
    f0 = synth.random_positive(geom.m, 5).astype(np.float32).astype(np.float64)
    k = 3
    f_ref, _ = O.mlem(H, g, k, f0=f0)
    f, stats = _sharded(wl, psf, g, k, 3, init="given", f0=f0.astype(np.float32))
    assert floored_rel(f, f_ref) <= k * 1e-5
    assert np.array_equal(stats[0], stats[2])


def test_one_slice_without_reduction_is_the_whole_em():
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)
    k = 8
    f_ref, hist = O.mlem(H, g, k, init="htg")
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        f, st = plan.reconstruct_sharded(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), k,
                                         init="htg", stats=True)
        plan.check()
    assert floored_rel(f.double().cpu().numpy().ravel(), f_ref) <= k * 1e-5
    assert abs(float(st[k, 2]) - hist[k]["loglik"]) <= 1e-5 * abs(hist[k]["loglik"])


def test_a_failing_reduction_is_reported():
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)

    def bad(q):
        raise RuntimeError("the exchange failed")

    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        with pytest.raises(CtisError, match="reduction callback"):
            plan.reconstruct_sharded(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), 2,
                                     reduce=bad)
        torch.cuda.synchronize()
        plan.check()
