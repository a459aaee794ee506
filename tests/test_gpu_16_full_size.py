"""Full-size parity against the FP64 oracle, element by element, in the
launch configuration bench.py times (autotuned schedules):

* realistic workload (128x128x64 -> 1024^2, 225 nonzeros per image): both
  projectors on every pixel and voxel, one EM step from a float32 iterate,
  and the benchmarked reconstruction of k = 100 updates from ones on every
  voxel and every one of its 101 statistics rows (the oracle's sparse H of
  all 64 wavelength blocks);
* large workload (256x256x128 -> 2048^2, 625 nonzeros): both projectors and
  k = 3 EM updates on every element, against the oracle's shifted-sum
  projectors (its sparse H would not fit in host memory);
* the autograd form at its stated size (10 unrolled updates, realistic):
  the NLL and the gradient in the tap values along two random directions
  against central differences of the oracle's float64 NLL.

Inputs are the oracle's: g is Poisson noise on the oracle's own image of the
seeded scene. Tolerances are those of the smaller parity suites: 1e-5
floored-relative per projection and per step, k * 1e-5 floored-relative and
1e-5 * sqrt(k) relative L2 after k steps, 1e-5 for the statistics, 2e-3 of
the gradient's scale for the unrolled gradient."""
import math

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import Plan
from tests.helpers import floored_rel, geometry, rel_l2

pytestmark = pytest.mark.gpu

STAT_KEYS = ("flux_hf", "flux_g_covered", "loglik", "resid2")


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.fixture(scope="module")
def realistic():
    wl = synth.REALISTIC
    geom = geometry(wl)
    psf = synth.make_psf(wl)
    H = O.build_H(geom, psf)
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    return wl, geom, psf, H, np.asarray(g, dtype=np.float64)


def _tuned_plan(wl, psf, g):
    plan = Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf)
    plan.autotune(torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda())
    return plan


def test_realistic_projectors_every_element(realistic):
    wl, geom, psf, H, g = realistic
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 201)
    u = synth.random_positive((wl.xi, wl.gamma), 202)
    with _tuned_plan(wl, psf, g) as plan:
        hf = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy()
        hu = plan.adjoint(torch.from_numpy(u).cuda()).cpu().numpy()
        plan.check()
    assert floored_rel(hf, H.forward(f.ravel())) <= 1e-5
    assert floored_rel(hu, H.adjoint(u.ravel())) <= 1e-5


def test_realistic_one_step_every_voxel(realistic):
    wl, geom, psf, H, g = realistic
    f5, _ = O.mlem(H, g, 5)
    f5 = f5.astype(np.float32)
    ref = O.em_step(H, g, f5.astype(np.float64))
    with _tuned_plan(wl, psf, g) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda()
        out, _ = plan.reconstruct(gt, k=1, f=torch.from_numpy(f5.reshape(wl.w, wl.alpha, wl.a)).cuda(),
                                  init=None)
        plan.check()
    assert floored_rel(out.cpu().numpy(), ref) <= 1e-5


def test_realistic_benchmarked_reconstruction_every_voxel_and_statistic(realistic):
    wl, geom, psf, H, g = realistic
    k = wl.k
    f_ref, hist = O.mlem(H, g, k)
    with _tuned_plan(wl, psf, g) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda()
        f, st = plan.reconstruct(gt, k=k, init="ones", stats=True)
        plan.check()
        f, st = f.double().cpu().numpy().ravel(), st.cpu().numpy()
    err, l2 = floored_rel(f, f_ref), rel_l2(f, f_ref)
    print(f"realistic k={k}: max floored-rel {err:.3e}, rel L2 {l2:.3e}")
    assert err <= k * 1e-5
    assert l2 <= 1e-5 * math.sqrt(k)
    worst = 0.0
    for t in range(k + 1):
        for q, key in enumerate(STAT_KEYS):
            e = abs(st[t, q] - hist[t][key]) / abs(hist[t][key])
            worst = max(worst, e)
            assert e <= 1e-5, (t, key, e)
    print(f"realistic k={k}: worst statistic relative error {worst:.3e}")


@pytest.fixture(scope="module")
def large():
    wl = synth.LARGE
    geom = geometry(wl)
    psf = synth.make_psf(wl)
    taps = O.merge_psf(geom, psf)
    g, _ = synth.make_measurement(O.forward_shifts(geom, taps, synth.make_scene(wl).ravel()),
                                  wl.peak, wl.seed)
    return wl, geom, psf, taps, np.asarray(g, dtype=np.float64)


def test_large_projectors_and_three_updates_every_element(large):
    wl, geom, psf, taps, g = large
    k = 3
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 203)
    u = synth.random_positive((wl.xi, wl.gamma), 204)
    f_ref, hist = O.mlem_shifts(geom, taps, g, k)
    with _tuned_plan(wl, psf, g) as plan:
        hf = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy()
        hu = plan.adjoint(torch.from_numpy(u).cuda()).cpu().numpy()
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda()
        fk, st = plan.reconstruct(gt, k=k, init="ones", stats=True)
        plan.check()
        fk, st = fk.double().cpu().numpy().ravel(), st.cpu().numpy()
    assert floored_rel(hf, O.forward_shifts(geom, taps, f.ravel())) <= 1e-5
    assert floored_rel(hu, O.adjoint_shifts(geom, taps, u.ravel())) <= 1e-5
    assert floored_rel(fk, f_ref) <= k * 1e-5
    assert rel_l2(fk, f_ref) <= 1e-5 * math.sqrt(k)
    for t in range(k + 1):
        for q, key in enumerate(STAT_KEYS):
            assert abs(st[t, q] - hist[t][key]) <= 1e-5 * abs(hist[t][key]), (t, key)


def test_autograd_form_at_its_stated_size(realistic):
    """Config 5: the Poisson NLL after 10 unrolled EM updates of the realistic
    workload and its gradient in the tap values, along two random directions,
    against central differences of the oracle's float64 NLL (shifted-sum
    projectors, values perturbed along the direction)."""
    wl, geom, psf, H, g = realistic
    taps = O.merge_psf(geom, psf)
    taps = O.with_values(taps, taps.v.astype(np.float32).astype(np.float64))
    k = 10
    f0 = np.ones(geom.m)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda()
        nll, dval, _ = plan.unrolled_nll_grad(gt, k)
        plan.check()
        nll, dval = float(nll), dval.cpu().numpy().astype(np.float64)
    ref = O.unrolled_nll_shifts(geom, taps, g, f0, k)
    assert abs(nll - ref) <= 1e-5 * abs(ref)
    rng = np.random.default_rng(11)
    for _ in range(2):
        d = rng.standard_normal(taps.v.size) * taps.v
        eps = 1e-4
        lp = O.unrolled_nll_shifts(geom, O.with_values(taps, taps.v + eps * d), g, f0, k)
        lm = O.unrolled_nll_shifts(geom, O.with_values(taps, taps.v - eps * d), g, f0, k)
        fd = (lp - lm) / (2 * eps)
        got = float(dval @ d)
        scale = float(np.abs(dval) @ np.abs(d))
        print(f"autograd full size: directional derivative {got:.6e} vs central difference {fd:.6e}")
        assert abs(got - fd) <= 2e-3 * scale
