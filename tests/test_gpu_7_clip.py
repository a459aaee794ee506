"""GPU parity of the clipped FPA boundary (CTIS_BOUNDARY_CLIP) against the
FP64 oracle's clip reading: shifted PSF nonzeros that leave the FPA are
dropped, so h = H^T 1 varies per voxel (Eq. 2's normaliser).

Workloads: the synthetic PSFs of the parity suite shifted so that some
diffraction orders spill past the FPA edges (and, for k5, some nonzeros miss
it for every voxel), plus the hand-made PSF of the oracle pins. Tolerances
as in the EM and projector suites."""
import math

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CTIS_BOUNDARY_CLIP, CtisError, Plan, reconstruct_batched
from tests.helpers import floored_rel, geometry, rel_l2

pytestmark = pytest.mark.gpu

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 500.0, 6)
K5 = synth.Workload("k5", 20, 24, 6, 120, 110, 3, 36.0, 1.2, 5, 1.2, "segmentation", 800.0, 6)
CASES = [(RAGGED, (-9, 4)), (K5, (30, -20)), (synth.MODEL_A, (-40, 35))]
STAT_KEYS = ("flux_hf", "flux_g_covered", "loglik", "resid2")


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _psf(wl, shift):
    ptr, x, y, v = synth.make_psf(wl)
    return ptr, (x + shift[0]).astype(np.int32), (y + shift[1]).astype(np.int32), v


@pytest.fixture(scope="module", params=CASES, ids=lambda c: c[0].name)
def prob(request):
    wl, shift = request.param
    geom = geometry(wl)
    psf = _psf(wl, shift)
    H = O.build_H(geom, psf, boundary="clip")
    f_true = synth.make_scene(wl).ravel()
    g, _ = synth.make_measurement(H.forward(f_true), wl.peak, wl.seed)
    return wl, geom, psf, H, g


def _plan(wl, psf, **kw):
    return Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, boundary="clip", **kw)


def test_reject_refuses_a_psf_that_leaves_the_fpa(prob):
    wl, geom, psf, H, g = prob
    with pytest.raises(CtisError):
        Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf)


def test_projectors_match_the_clipped_oracle(prob):
    wl, geom, psf, H, g = prob
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 71)
    r = synth.random_positive((wl.xi, wl.gamma), 72)
    with _plan(wl, psf) as plan:
        assert plan.info()["boundary"] == CTIS_BOUNDARY_CLIP
        hf = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy()
        ht = plan.adjoint(torch.from_numpy(r).cuda()).cpu().numpy()
        plan.check()
    assert floored_rel(hf.ravel(), H.forward(f.ravel())) <= 1e-5
    assert floored_rel(ht.ravel(), H.adjoint(r.ravel())) <= 1e-5


def test_em_iterations_and_statistics(prob):
    """k EM updates with h per voxel: the iterates and the per-iteration
    statistics against the oracle's mlem on the clipped H."""
    wl, geom, psf, H, g = prob
    k = wl.k
    ref, hist = O.mlem(H, g, k)
    with _plan(wl, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        out, st = plan.reconstruct(gt, k=k, init="ones", stats=True)
        plan.check()
        got, st = out.cpu().numpy().ravel(), st.cpu().numpy()
    assert floored_rel(got, ref) <= k * 1e-5
    assert rel_l2(got, ref) <= 1e-5 * math.sqrt(k)
    for t in range(k + 1):
        for q, key in enumerate(STAT_KEYS):
            assert abs(st[t, q] - hist[t][key]) <= 1e-5 * abs(hist[t][key]), (t, key)


def test_pinned_hand_made_psf():
    """The oracle pins' PSF (nonzeros over every edge, a duplicate, one off the
    FPA altogether), one EM update from a random iterate."""
    ptr = np.array([0, 4, 9], np.int32)
    x = np.array([-2, 7, 3, 1, -1, 5, 5, 20, 6], np.int32)
    y = np.array([1, 6, 2, -2, -1, 0, 0, 3, 7], np.int32)
    v = np.array([0.5, 1.5, 1.0, 0.25, 0.7, 0.3, 0.2, 2.0, 0.9], np.float32)
    geom = O.Geometry(4, 3, 2, 9, 8)
    H = O.build_H(geom, (ptr, x, y, v), boundary="clip")
    f0 = synth.random_positive(geom.m, 73).astype(np.float32)
    g = synth.random_positive(geom.n, 74).astype(np.float32) * 10
    ref = O.em_step(H, g, f0.astype(np.float64))
    with Plan(4, 3, 2, 9, 8, (ptr, x, y, v), boundary="clip") as plan:
        f = torch.from_numpy(f0.reshape(2, 3, 4)).cuda()
        out, _ = plan.reconstruct(torch.from_numpy(g.reshape(8, 9)).cuda(), k=1, f=f, init=None)
        plan.check()
    assert floored_rel(out.cpu().numpy().ravel(), ref) <= 1e-5


def test_set_values_recomputes_h_per_voxel():
    wl, shift = CASES[0]
    geom = geometry(wl)
    psf = _psf(wl, shift)
    with _plan(wl, psf) as plan:
        s, x, y, v, _ = plan.export_taps()
        v2 = (np.asarray(v) * synth.random_positive(len(v), 75) * 2).astype(np.float32)
        plan.set_values(v2)
        # the oracle with the new values on the same merged taps
        H = O.build_H(geom, (np.searchsorted(s, np.arange(wl.w + 1)).astype(np.int32), x, y, v2),
                      boundary="clip")
        g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
        ref, _ = O.mlem(H, g, 3)
        out, _ = plan.reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), k=3,
                                  init="ones")
        plan.check()
    assert floored_rel(out.cpu().numpy().ravel(), ref) <= 3e-5


def test_batched_clipped_frames_equal_single_frame_reconstructions():
    wl, shift = CASES[0]
    psf = _psf(wl, shift)
    H = O.build_H(geometry(wl), psf, boundary="clip")
    with _plan(wl, psf) as plan:
        gs = []
        for i in range(4):
            g, _ = synth.make_measurement(H.forward(synth.make_scene(wl, 200 + i).ravel()),
                                          wl.peak, 200 + i)
            gs.append(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda())
        fs, st = reconstruct_batched([plan], [0] * 4, gs, 5, stats=True)
        for i in range(4):
            ref, ref_st = plan.reconstruct(gs[i], k=5, init="ones", stats=True)
            assert torch.equal(fs[i], ref) and torch.equal(st[i], ref_st), i
        plan.check()


@pytest.mark.parametrize("k", [0, 1, 3])
def test_unrolled_gradient_with_h_per_voxel(k):
    """The NLL after k EM updates under clipping and its gradient in the tap
    values (h per voxel depends on the taps that land for each voxel),
    against the oracle's NLL and central differences of it."""
    wl, shift = CASES[0]
    geom = geometry(wl)
    psf = _psf(wl, shift)
    taps = O.merge_psf(geom, psf, "clip")
    taps = O.with_values(taps, taps.v.astype(np.float32).astype(np.float64))
    H = O.BlockH(geom, taps)
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    f0 = np.ones(geom.m)
    with _plan(wl, psf) as plan:
        nll, dval, _ = plan.unrolled_nll_grad(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), k)
        plan.check()
        nll, dval = float(nll), dval.cpu().numpy()
    ref = O.unrolled_nll(geom, taps, g, f0, k)
    assert abs(nll - ref) <= 1e-5 * abs(ref)
    idx = np.random.default_rng(20 + k).choice(taps.v.size, 24, replace=False)
    fd = np.zeros(len(idx))
    for n, t in enumerate(idx):
        eps = 1e-4 * max(taps.v[t], 1e-3)
        vp, vm = taps.v.copy(), taps.v.copy()
        vp[t] += eps
        vm[t] -= eps
        fd[n] = (O.unrolled_nll(geom, O.with_values(taps, vp), g, f0, k) -
                 O.unrolled_nll(geom, O.with_values(taps, vm), g, f0, k)) / (2 * eps)
    assert np.all(np.abs(dval[idx] - fd) <= 2e-3 * np.abs(fd).max()), (dval[idx], fd)


def test_batched_frames_read_zeros_past_their_fpa_edges():
    """In a batch, an adjoint window past the FPA's first or last row reads
    zeros, not the neighbouring frame's image: a PSF spilling over all four
    FPA edges, frames with light in their first and last rows, each frame
    equal to its single-frame reconstruction and to the oracle."""
    wl = RAGGED.with_(pitch=20.0)
    geom = geometry(wl)
    psf = synth.make_psf(wl)
    ptr, x, y, v = psf
    assert y.min() < 0 and y.max() + wl.alpha - 1 >= wl.xi
    assert x.min() < 0 and x.max() + wl.a - 1 >= wl.gamma
    H = O.build_H(geom, psf, boundary="clip")
    with _plan(wl, psf) as plan:
        gs, refs = [], []
        for i in range(3):
            g, _ = synth.make_measurement(H.forward(synth.make_scene(wl, 400 + i).ravel()),
                                          wl.peak, 400 + i)
            img = g.reshape(wl.xi, wl.gamma)
            assert img[0].sum() > 0 and img[-1].sum() > 0
            gs.append(torch.from_numpy(img).cuda())
            refs.append(O.mlem(H, g, 4)[0])
        fs, _ = reconstruct_batched([plan], [0] * 3, gs, 4)
        for i in range(3):
            single, _ = plan.reconstruct(gs[i], k=4, init="ones")
            assert torch.equal(fs[i], single), i
            assert floored_rel(fs[i].cpu().numpy().ravel(), refs[i]) <= 4e-5, i
        plan.check()
