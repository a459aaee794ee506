"""Degenerate plans on the GPU against the oracle and closed forms: a
wavelength without calibration nonzeros (h = 0 there, so EM zeroes it), a
PSF with no nonzeros at all, a field stop as large as the FPA with one
nonzero (H = v I: one EM, SART or SMART step from ones gives g / v), and a
one-pixel field stop (the columns of H are the calibration images)."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import Plan
from tests.helpers import floored_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _run(geom, psf, g, k, tile="32x32"):
    with Plan(geom.a, geom.alpha, geom.w, geom.gamma, geom.xi, psf, forward_tile=tile) as plan:
        f = torch.from_numpy(synth.random_positive(geom.m, 95).reshape(geom.w, geom.alpha, geom.a)).cuda()
        r = torch.from_numpy(synth.random_positive(geom.n, 96).reshape(geom.xi, geom.gamma)).cuda()
        hf = plan.forward(f).cpu().numpy().ravel()
        ht = plan.adjoint(r).cpu().numpy().ravel()
        out, st = plan.reconstruct(torch.from_numpy(g.reshape(geom.xi, geom.gamma)).cuda(), k,
                                   init="ones", stats=True)
        plan.check()
        return (f.cpu().numpy().ravel(), r.cpu().numpy().ravel(), hf, ht,
                out.cpu().numpy().ravel(), st.cpu().numpy())


def _compare(geom, psf, g, k=5, tile="32x32"):
    H = O.build_H(geom, psf)
    f, r, hf, ht, out, st = _run(geom, psf, g, k, tile)
    assert floored_rel(hf, H.forward(f)) <= 1e-5 if np.any(H.forward(f)) else not np.any(hf)
    assert floored_rel(ht, H.adjoint(r)) <= 1e-5 if np.any(H.adjoint(r)) else not np.any(ht)
    ref, hist = O.mlem(H, g, k)
    if np.any(ref):
        assert floored_rel(out, ref) <= k * 1e-5
    else:
        assert not np.any(out)
    for t in range(k + 1):
        for q, key in enumerate(("flux_hf", "flux_g_covered", "loglik", "resid2")):
            assert abs(st[t, q] - hist[t][key]) <= 1e-5 * abs(hist[t][key]), (t, key)
    return out


TILES = pytest.mark.parametrize("tile", ["32x32", "32x16"])


@TILES
def test_a_wavelength_without_nonzeros(tile):
    geom = O.Geometry(12, 9, 3, 40, 33)
    ptr = np.array([0, 4, 4, 7], np.int32)   # wavelength 1 has no calibration nonzeros
    x = np.array([2, 3, 20, 21, 5, 15, 27], np.int32)
    y = np.array([1, 1, 10, 11, 20, 3, 22], np.int32)
    v = np.array([0.5, 0.3, 0.9, 0.2, 0.6, 0.4, 0.8], np.float32)
    g = synth.random_positive(geom.n, 97).astype(np.float32) * 20
    out = _compare(geom, (ptr, x, y, v), g, tile=tile)
    assert not np.any(out.reshape(3, -1)[1])    # h = 0: EM sets that wavelength to 0


@TILES
def test_a_psf_without_nonzeros(tile):
    geom = O.Geometry(6, 5, 2, 20, 18)
    psf = (np.zeros(3, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32))
    g = synth.random_positive(geom.n, 98).astype(np.float32)
    f, r, hf, ht, out, st = _run(geom, psf, g, 3, tile)
    assert not np.any(hf) and not np.any(ht) and not np.any(out) and not np.any(st)


@TILES
@pytest.mark.parametrize("solver", ["em", "sart", "smart"])
def test_field_stop_as_large_as_the_fpa(solver, tile):
    """a = gamma, alpha = xi, one nonzero v at (0, 0): H = v I, and one update
    of any of the solvers from f = 1 gives g / v (exactly for EM and SART on
    integer counts with v = 2; SMART to a few ulp)."""
    geom = O.Geometry(40, 35, 1, 40, 35)
    psf = (np.array([0, 1], np.int32), np.array([0], np.int32), np.array([0], np.int32),
           np.array([2.0], np.float32))
    g = np.floor(synth.random_positive(geom.n, 99) * 50).astype(np.float32) + 1
    with Plan(40, 35, 1, 40, 35, psf, forward_tile=tile) as plan:
        out, _ = plan.reconstruct(torch.from_numpy(g.reshape(35, 40)).cuda(), 1, init="ones",
                                  solver=solver)
        plan.check()
    got = out.cpu().numpy().ravel()
    if solver == "smart":
        np.testing.assert_allclose(got, g / 2, rtol=2e-6)
    else:
        assert np.array_equal(got, g / 2)


@TILES
def test_one_pixel_field_stop(tile):
    geom = O.Geometry(1, 1, 2, 7, 5)
    psf = (np.array([0, 3, 6], np.int32), np.array([0, 6, 3, 1, 2, 2], np.int32),
           np.array([0, 4, 2, 1, 1, 1], np.int32),
           np.array([1.0, 0.5, 0.25, 0.75, 0.5, 0.5], np.float32))   # a duplicate in s = 1
    g = synth.random_positive(geom.n, 100).astype(np.float32) * 10
    _compare(geom, psf, g, tile=tile)
