"""GPU parity of the differentiable form: the PSF-value gradient, replacing the
tap values, the autograd wrappers and the gradient of the Poisson NLL through
unrolled EM updates, against the FP64 oracle.

The PSF-value gradient of <r, H f> is a sum of products f_s(p, r) r(.) over the
field stop (float32, fixed order): for nonnegative inputs its worst-case
relative rounding error is below 6e-8 times the number of terms added
sequentially (32 per lane, then a 5-level warp tree and one term per voxel
tile), far below the 1e-5 used here; with signed r the bound applies relative
to sum |f| |r|. The unrolled gradient is checked against central differences
of the oracle's float64 NLL (which add an O(eps^2) truncation error) with a
tolerance of 2e-3 of the gradient's scale: every step of the float32 backward
pass carries the projectors' 1e-5 error, and k steps compound it."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CtisError, Plan
from paper_2006_01573_gb300.autograd import project, unrolled_nll
from tests.helpers import floored_rel, geometry, problem

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _cases():
    wl5 = synth.Workload("k5", 20, 24, 6, 120, 110, 3, 36.0, 1.2, 5, 1.2, "segmentation", 100.0, 3)
    deep = synth.Workload("deep", 24, 20, 40, 140, 130, 3, 40.0, 0.5, 3, 0.8, "segmentation", 100.0, 3)
    ragged = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 3)
    return {w.name: w for w in (synth.TINY, wl5, deep, ragged)}


CASES = _cases()


def _plan(wl, psf, dtype="f32", forward_tile="32x32"):
    return Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype=dtype, forward_tile=forward_tile)


@pytest.mark.parametrize("name", sorted(CASES))
def test_psf_grad_parity(name):
    wl = CASES[name]
    psf = synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 71)
    r = synth.random_positive((wl.xi, wl.gamma), 72)
    rs = (r - 0.5).astype(np.float32)          # signed: cancellation inside the sums
    with _plan(wl, psf) as plan:
        ft = torch.from_numpy(f).cuda()
        got = plan.psf_grad(ft, torch.from_numpy(r).cuda()).cpu().numpy()
        got_s = plan.psf_grad(ft, torch.from_numpy(rs).cuda()).cpu().numpy()
        plan.check()
    assert floored_rel(got, O.psf_value_grad(geom, taps, f, r)) <= TOL
    ref_s = O.psf_value_grad(geom, taps, f, rs)
    scale = O.psf_value_grad(geom, taps, np.abs(f), np.abs(rs))
    assert np.all(np.abs(got_s - ref_s) <= TOL * scale)


def test_psf_grad_bf16_plan():
    wl = CASES["ragged"]
    psf = synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    f = O.round_bf16(synth.random_positive((wl.w, wl.alpha, wl.a), 73))
    r = synth.random_positive((wl.xi, wl.gamma), 74)
    with _plan(wl, psf, "bf16") as plan:
        got = plan.psf_grad(torch.from_numpy(f).to(torch.bfloat16).cuda(),
                            torch.from_numpy(r).cuda()).cpu().numpy()
    assert floored_rel(got, O.psf_value_grad(geom, taps, f, r)) <= TOL


def test_psf_grad_full_size_sampled():
    wl = synth.REALISTIC
    psf = synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    f = synth.make_scene(wl)
    r = synth.random_positive((wl.xi, wl.gamma), 75)
    with _plan(wl, psf) as plan:
        got = plan.psf_grad(torch.from_numpy(f).cuda(), torch.from_numpy(r).cuda()).cpu().numpy()
        plan.check()
    pick = np.random.default_rng(2).choice(taps.v.size, 300, replace=False)
    sub = O.Taps(taps.s[pick], taps.x[pick], taps.y[pick], taps.v[pick], None)
    assert floored_rel(got[pick], O.psf_value_grad(geom, sub, f, r)) <= TOL


def test_set_values_replaces_taps_and_h():
    wl = CASES["k5"]
    psf = synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    new = (synth.random_positive(taps.v.size, 76) + 0.1).astype(np.float32)
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 77)
    with _plan(wl, psf) as plan:
        plan.set_values(new)
        s, x, y, v, h = plan.export_taps()
        hf = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy()
        with pytest.raises(CtisError):
            plan.set_values(np.full(taps.v.size, -1.0, np.float32))
    assert np.array_equal(v, new)
    t2 = O.with_values(taps, new.astype(np.float64))
    H2 = O.BlockH(geom, t2)
    np.testing.assert_allclose(h, H2.h().reshape(geom.w, -1)[:, 0], rtol=1.2e-7, atol=0)
    assert floored_rel(hf, H2.forward(f.ravel())) <= TOL


def test_project_autograd_matches_adjoint_and_psf_grad():
    wl = CASES["ragged"]
    psf = synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 78)
    gy = synth.random_positive((wl.xi, wl.gamma), 79)
    with _plan(wl, psf) as plan:
        ft = torch.from_numpy(f).cuda().requires_grad_(True)
        vt = torch.from_numpy(taps.v.astype(np.float32)).cuda().requires_grad_(True)
        out = project(plan, ft, vt)
        (out * torch.from_numpy(gy).cuda()).sum().backward()
        df, dv = ft.grad.cpu().numpy(), vt.grad.cpu().numpy()
    H = O.BlockH(geom, taps)
    assert floored_rel(out.detach().cpu().numpy(), H.forward(f.ravel())) <= TOL
    assert floored_rel(df, H.adjoint(gy.ravel())) <= TOL
    assert floored_rel(dv, O.psf_value_grad(geom, taps, f, gy)) <= TOL


def test_two_live_projections_with_different_values_on_one_plan():
    """Two project() calls on one plan with different tap values, both
    pending when backward runs: each df must be H^T gy of its own values."""
    wl = CASES["ragged"]
    psf = synth.make_psf(wl)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    v2 = (taps.v * (1.0 + synth.random_positive(taps.v.size, 80))).astype(np.float32)
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 81)
    gy1 = synth.random_positive((wl.xi, wl.gamma), 82)
    gy2 = synth.random_positive((wl.xi, wl.gamma), 83)
    with _plan(wl, psf) as plan:
        f1 = torch.from_numpy(f).cuda().requires_grad_(True)
        f2 = torch.from_numpy(f).cuda().requires_grad_(True)
        out1 = project(plan, f1, torch.from_numpy(taps.v.astype(np.float32)).cuda())
        out2 = project(plan, f2, torch.from_numpy(v2).cuda())
        loss = (out1 * torch.from_numpy(gy1).cuda()).sum() + (out2 * torch.from_numpy(gy2).cuda()).sum()
        loss.backward()
        df1, df2 = f1.grad.cpu().numpy(), f2.grad.cpu().numpy()
        # and the other order of the two backward passes
        f1.grad, f2.grad = None, None
        out1 = project(plan, f1, torch.from_numpy(taps.v.astype(np.float32)).cuda())
        out2 = project(plan, f2, torch.from_numpy(v2).cuda())
        (out2 * torch.from_numpy(gy2).cuda()).sum().backward()
        (out1 * torch.from_numpy(gy1).cuda()).sum().backward()
        df1b, df2b = f1.grad.cpu().numpy(), f2.grad.cpu().numpy()
        plan.check()
    H1 = O.BlockH(geom, taps)
    H2 = O.BlockH(geom, O.with_values(taps, v2.astype(np.float64)))
    for a, b in ((df1, df1b), (df2, df2b)):
        assert np.array_equal(a, b)
    assert floored_rel(df1, H1.adjoint(gy1.ravel())) <= TOL
    assert floored_rel(df2, H2.adjoint(gy2.ravel())) <= TOL


def _fd_grad(geom, taps, g, f0, k, idx, rel_eps=1e-4):
    """Central differences of the oracle's float64 unrolled NLL in tap values."""
    out = np.zeros(len(idx))
    for n, t in enumerate(idx):
        eps = rel_eps * max(taps.v[t], 1e-3)
        vp, vm = taps.v.copy(), taps.v.copy()
        vp[t] += eps
        vm[t] -= eps
        lp = O.unrolled_nll(geom, O.with_values(taps, vp), g, f0, k)
        lm = O.unrolled_nll(geom, O.with_values(taps, vm), g, f0, k)
        out[n] = (lp - lm) / (2 * eps)
    return out


@pytest.mark.parametrize("k,tile", [(0, "32x32"), (1, "32x32"), (3, "32x32"), (3, "32x16")])
def test_unrolled_nll_gradient_against_oracle_differences(k, tile):
    wl = synth.TINY
    geom, psf, _, _, g = problem(wl)
    taps = O.merge_psf(geom, psf)
    taps = O.with_values(taps, taps.v.astype(np.float32).astype(np.float64))
    f0 = np.ones(geom.m)
    with _plan(wl, psf, forward_tile=tile) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        nll, dval, df0 = plan.unrolled_nll_grad(gt, k, f0=torch.ones((wl.w, wl.alpha, wl.a),
                                                                     device="cuda"), want_df0=True)
        plan.check()
        nll, dval, df0 = float(nll), dval.cpu().numpy(), df0.cpu().numpy().ravel()
    ref = O.unrolled_nll(geom, taps, g, f0, k)
    assert abs(nll - ref) <= 1e-5 * abs(ref)
    idx = np.random.default_rng(k).choice(taps.v.size, 24, replace=False)
    fd = _fd_grad(geom, taps, g, f0, k, idx)
    scale = np.abs(fd).max()
    assert np.all(np.abs(dval[idx] - fd) <= 2e-3 * scale), (dval[idx], fd)
    # dL/df0 on a few voxels, same way
    H = O.BlockH(geom, taps)
    vox = np.random.default_rng(10 + k).choice(geom.m, 12, replace=False)
    fdf = np.zeros(len(vox))
    for n, j in enumerate(vox):
        e = 1e-4
        fp, fm = f0.copy(), f0.copy()
        fp[j] += e
        fm[j] -= e
        lp = O.poisson_nll(H.forward(_em(H, g, fp, k)), g)
        lm = O.poisson_nll(H.forward(_em(H, g, fm, k)), g)
        fdf[n] = (lp - lm) / (2 * e)
    assert np.all(np.abs(df0[vox] - fdf) <= 2e-3 * max(np.abs(fdf).max(), 1e-12)), (df0[vox], fdf)


def _em(H, g, f, k):
    for _ in range(k):
        f = O.em_step(H, g, f)
    return f


def test_unrolled_nll_autograd_wrapper():
    wl = synth.TINY
    geom, psf, _, _, g = problem(wl)
    taps = O.merge_psf(geom, psf)
    with _plan(wl, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        vt = torch.from_numpy(taps.v.astype(np.float32)).cuda().requires_grad_(True)
        loss = unrolled_nll(plan, vt, gt, 2)
        loss.backward()
        nll, dval, _ = plan.unrolled_nll_grad(gt, 2)
        assert float(loss.detach()) == float(nll)
        assert torch.equal(vt.grad, dval)


def test_unrolled_nll_directional_derivative_model_a():
    """64x64x32 -> 512x512 workload, 10 unrolled updates: the NLL against the
    oracle's, and the gradient along a random direction of the tap values
    against a central difference of the oracle's float64 NLL along it."""
    wl = synth.MODEL_A
    geom, psf, _, _, g = problem(wl)
    taps = O.merge_psf(geom, psf)
    taps = O.with_values(taps, taps.v.astype(np.float32).astype(np.float64))
    k = 10
    f0 = np.ones(geom.m)
    with _plan(wl, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma).astype(np.float32)).cuda()
        nll, dval, _ = plan.unrolled_nll_grad(gt, k)
        plan.check()
        nll, dval = float(nll), dval.cpu().numpy().astype(np.float64)
    ref = O.unrolled_nll(geom, taps, g, f0, k)
    assert abs(nll - ref) <= 1e-5 * abs(ref)
    d = np.random.default_rng(3).standard_normal(taps.v.size) * taps.v
    eps = 1e-4
    lp = O.unrolled_nll(geom, O.with_values(taps, taps.v + eps * d), g, f0, k)
    lm = O.unrolled_nll(geom, O.with_values(taps, taps.v - eps * d), g, f0, k)
    fd = (lp - lm) / (2 * eps)
    got = float(dval @ d)
    assert abs(got - fd) <= 2e-3 * abs(fd), (got, fd)


def test_unrolled_nll_full_size_matches_reconstruction_statistics():
    """Realistic 128x128x64 -> 1024x1024 workload, 10 unrolled updates at full
    size: the NLL equals minus the log-likelihood that the reconstruction
    reports for the same 10 updates, and the gradient is finite."""
    wl = synth.REALISTIC
    psf = synth.make_psf(wl)
    k = 10
    with _plan(wl, psf) as plan:
        f_true = torch.from_numpy(synth.make_scene(wl)).cuda()
        hf = plan.forward(f_true)
        g, _ = synth.make_measurement(hf.cpu().numpy(), wl.peak, wl.seed)
        gt = torch.from_numpy(g).cuda()
        nll, dval, _ = plan.unrolled_nll_grad(gt, k)
        _, stats = plan.reconstruct(gt, k=k, init="ones", stats=True)
        plan.check()
        nll = float(nll)
        loglik = float(stats[k, 2])
        dval = dval.cpu().numpy()
    assert abs(nll + loglik) <= 1e-6 * abs(loglik)
    assert np.all(np.isfinite(dval))


def test_unrolled_gradient_rejects_bf16_plans():
    wl = synth.TINY
    psf = synth.make_psf(wl)
    with _plan(wl, psf, "bf16") as plan:
        g = torch.ones((wl.xi, wl.gamma), device="cuda")
        with pytest.raises(CtisError) as e:
            plan.unrolled_nll_grad(g, 1)
    assert e.value.code == -6
