"""GPU parity of the wrap FPA boundary (CTIS_BOUNDARY_WRAP, Eq. 7's circulant
taken literally: a shifted nonzero past the right edge re-enters at the left
of the next FPA row, one past the last row at the top) against the FP64
oracle's wrap reading, for the gather projectors (stored as the clip reading
of the PSF and its wrapped images) and the FFT form (circular by
construction). The PSFs of the parity workloads are moved to the FPA's last
column and row, so many shifted copies wrap. Tolerances as in the clip, EM
and FFT suites."""
import math

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CTIS_BOUNDARY_WRAP, CtisError, Plan, reconstruct_batched
from tests.helpers import floored_rel, geometry, rel_l2

pytestmark = pytest.mark.gpu

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 500.0, 6)
K5 = synth.Workload("k5", 20, 24, 6, 120, 110, 3, 36.0, 1.2, 5, 1.2, "segmentation", 800.0, 6)
WORKLOADS = [synth.TINY, RAGGED, K5, synth.MODEL_A]
STAT_KEYS = ("flux_hf", "flux_g_covered", "loglik", "resid2")
FFT_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _to_edges(wl):
    ptr, x, y, v = synth.make_psf(wl)
    return (ptr, (x + wl.gamma - 1 - x.max()).astype(np.int32),
            (y + wl.xi - 1 - y.max()).astype(np.int32), v)


@pytest.fixture(scope="module", params=WORKLOADS, ids=lambda w: w.name)
def prob(request):
    wl = request.param
    geom = geometry(wl)
    psf = _to_edges(wl)
    H = O.build_H(geom, psf, boundary="wrap")
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    return wl, geom, psf, H, g


def _plan(wl, psf, **kw):
    return Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, boundary="wrap", **kw)


def _normwise(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_gather_and_fft_projectors_match_the_wrapped_oracle(prob):
    wl, geom, psf, H, g = prob
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 91)
    r = synth.random_positive((wl.xi, wl.gamma), 92)
    with _plan(wl, psf) as plan:
        assert plan.info()["boundary"] == CTIS_BOUNDARY_WRAP
        ft, rt = torch.from_numpy(f).cuda(), torch.from_numpy(r).cuda()
        hf = plan.forward(ft).cpu().numpy()
        ht = plan.adjoint(rt).cpu().numpy()
        hf_fft = plan.fft_forward(ft).cpu().numpy()
        ht_fft = plan.fft_adjoint(rt).cpu().numpy()
        plan.check()
    ref_f, ref_t = H.forward(f.ravel()), H.adjoint(r.ravel())
    assert floored_rel(hf.ravel(), ref_f) <= 1e-5
    assert floored_rel(ht.ravel(), ref_t) <= 1e-5
    assert _normwise(hf_fft, ref_f) <= FFT_TOL and _normwise(ht_fft, ref_t) <= FFT_TOL
    assert _normwise(hf_fft, hf) <= FFT_TOL and _normwise(ht_fft, ht) <= FFT_TOL


def test_em_iterations_and_statistics(prob):
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


def test_fft_em_iterations_match_the_wrapped_oracle():
    wl = RAGGED
    geom = geometry(wl)
    psf = _to_edges(wl)
    H = O.build_H(geom, psf, boundary="wrap")
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    ref, _ = O.mlem(H, g, wl.k)
    with _plan(wl, psf) as plan:
        f = plan.fft_reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), wl.k)
        plan.check()
    assert rel_l2(f.cpu().numpy().ravel(), ref) <= 2 * FFT_TOL * math.sqrt(wl.k)


def test_h_is_the_total_psf_value_and_values_are_fixed():
    """Nothing is lost under the wrap reading: h per wavelength is the sum of
    the caller's nonzeros; the stored table lists the images too; new values
    and the PSF-value gradient are refused."""
    wl = RAGGED
    psf = _to_edges(wl)
    ptr, x, y, v = psf
    with _plan(wl, psf) as plan:
        s, xs, ys, vs, h = plan.export_taps()
        assert len(vs) > len(v) and (xs < 0).any() and (ys < 0).any()
        for q in range(wl.w):
            want = float(np.sum(v[ptr[q]:ptr[q + 1]], dtype=np.float64))
            assert abs(h[q] - want) <= 1e-6 * want
        with pytest.raises(CtisError):
            plan.set_values(vs)
        f = torch.ones((wl.w, wl.alpha, wl.a), device="cuda")
        with pytest.raises(CtisError):
            plan.psf_grad(f, torch.ones((wl.xi, wl.gamma), device="cuda"))
        with pytest.raises(CtisError):
            plan.unrolled_nll_grad(torch.ones((wl.xi, wl.gamma), device="cuda"), 1)


def test_batched_wrapped_frames_equal_single_frame_reconstructions():
    wl = RAGGED
    psf = _to_edges(wl)
    H = O.build_H(geometry(wl), psf, boundary="wrap")
    with _plan(wl, psf) as plan:
        gs = []
        for i in range(3):
            g, _ = synth.make_measurement(H.forward(synth.make_scene(wl, 300 + i).ravel()),
                                          wl.peak, 300 + i)
            gs.append(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda())
        fs, st = reconstruct_batched([plan], [0] * 3, gs, 4, stats=True)
        for i in range(3):
            ref, ref_st = plan.reconstruct(gs[i], k=4, init="ones", stats=True)
            assert torch.equal(fs[i], ref) and torch.equal(st[i], ref_st), i
        plan.check()
