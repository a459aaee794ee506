"""GPU parity of the bfloat16 storage form against the FP64 oracle.

In this form the plan stores the PSF values and the datacube in bfloat16 and
accumulates in float32; g, u and every sum stay float32 (statistics float64).
A product of two bfloat16 values is exact in float32, so the projectors of the
form, given the same bfloat16 inputs, meet the float32 bound 1e-5 against the
oracle evaluated on the rounded values (round_bf16, pinned to PyTorch's cast).
An EM step stores its float32 result in bfloat16, one rounding of at most half
a bfloat16 unit (2^-9 relative); over k steps the error is reported against the
float64 EM, with a loose bound rather than one derived a priori."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import Plan
from tests.helpers import floored_rel, geometry, problem, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5
BF16_ULP = 2.0 ** -8   # spacing of bfloat16 values in [1, 2), relative


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


def _bf16_H(wl, psf):
    """Oracle H on the plan's stored values: merged in float64, rounded to
    float32, then to bfloat16."""
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    stored = O.round_bf16(taps.v.astype(np.float32)).astype(np.float64)
    return geom, O.with_values(taps, stored)


def _plan(wl, psf, forward_tile="32x32"):
    return Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype="bf16", forward_tile=forward_tile)


def _bf16_cube(wl, seed):
    f = O.round_bf16(synth.random_positive((wl.w, wl.alpha, wl.a), seed))
    return f, torch.from_numpy(f).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("name", sorted(CASES))
def test_bf16_tables_hold_rounded_values(name):
    wl = CASES[name]
    psf = synth.make_psf(wl)
    geom, taps = _bf16_H(wl, psf)
    with _plan(wl, psf) as plan:
        s, x, y, v, h = plan.export_taps()
    assert np.array_equal(v, taps.v.astype(np.float32))
    assert np.array_equal(s, taps.s) and np.array_equal(x, taps.x) and np.array_equal(y, taps.y)
    h_ref = O.BlockH(geom, taps).h().reshape(geom.w, -1)[:, 0]
    np.testing.assert_allclose(h, h_ref, rtol=1.2e-7, atol=0)


@pytest.mark.parametrize("tile", ["32x32", "32x16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bf16_forward_parity(name, tile):
    wl = CASES[name]
    psf = synth.make_psf(wl)
    geom, taps = _bf16_H(wl, psf)
    f, ft = _bf16_cube(wl, 61)
    with _plan(wl, psf, tile) as plan:
        assert plan.forward_tile() == tile
        hf = plan.forward(ft)
        plan.check()
        hf = hf.cpu().numpy()
    ref = O.BlockH(geom, taps).forward(f.ravel())
    assert floored_rel(hf, ref) <= TOL
    assert np.all(hf.ravel()[ref == 0] == 0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_bf16_adjoint_parity(name):
    wl = CASES[name]
    psf = synth.make_psf(wl)
    geom, taps = _bf16_H(wl, psf)
    r = synth.random_positive((wl.xi, wl.gamma), 62)
    with _plan(wl, psf) as plan:
        out = plan.adjoint(torch.from_numpy(r).cuda())
        plan.check()
        out = out.cpu().numpy()
    assert floored_rel(out, O.BlockH(geom, taps).adjoint(r.ravel())) <= TOL


@pytest.mark.parametrize("name", [synth.TINY.name, "ragged", "deep"])
def test_bf16_single_em_step(name):
    """From the same bfloat16 iterate, one GPU EM step lies within one
    bfloat16 unit of the float64 step, and nearly every element is exactly
    the float64 step rounded to bfloat16 (the rest sit on a rounding tie
    that the float32 arithmetic resolves the other way)."""
    wl = CASES[name]
    psf = synth.make_psf(wl)
    geom, taps = _bf16_H(wl, psf)
    H = O.BlockH(geom, taps)
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    f, ft = _bf16_cube(wl, 63)
    with _plan(wl, psf) as plan:
        out, _ = plan.reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), k=1,
                                  f=ft, init=None)
        plan.check()
        got = out.float().cpu().numpy().ravel()
    ref = O.em_step(H, g, f.ravel())
    assert floored_rel(got, ref) <= BF16_ULP
    same = got == O.round_bf16(ref.astype(np.float32))
    assert same.mean() >= 0.99


def test_bf16_em_iterations_against_stored_and_float64_em():
    """k bfloat16 EM iterations against the oracle EM that stores every
    iterate the same way, and against the float64 EM (the error of the form).
    The bounds are loose, stated limits for the reported errors."""
    wl = synth.TINY
    geom, psf, _, _, g = problem(wl)
    geom, taps = _bf16_H(wl, psf)
    H = O.BlockH(geom, taps)
    k = wl.k
    f_stored = np.ones(geom.m)
    store = lambda z: O.round_bf16(z.astype(np.float32))   # noqa: E731
    for _ in range(k):
        f_stored = O.em_step_stored(H, g, f_stored, store)
    f64, _ = O.mlem(H, g, k)
    with _plan(wl, psf) as plan:
        out, _ = plan.reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), k=k,
                                  init="ones")
        plan.check()
        got = out.float().cpu().numpy().ravel()
    assert np.all(np.isfinite(got)) and np.all(got >= 0)
    err_stored = rel_l2(got, f_stored)
    err_f64 = rel_l2(got, f64)
    print(f"bf16 EM k={k}: rel L2 vs stored-bf16 oracle {err_stored:.2e}, vs float64 EM {err_f64:.2e}")
    assert err_stored <= 4 * BF16_ULP
    assert err_f64 <= 8 * BF16_ULP


def test_bf16_full_size_sampled_outputs():
    """The realistic workload at full size in the bfloat16 form, checked on
    sampled outputs that the oracle evaluates one by one."""
    wl = synth.REALISTIC
    psf = synth.make_psf(wl)
    geom, taps = _bf16_H(wl, psf)
    f = O.round_bf16(synth.make_scene(wl))
    rng = np.random.default_rng(1)
    with _plan(wl, psf) as plan:
        hf = plan.forward(torch.from_numpy(f).to(torch.bfloat16).cuda())
        r = torch.from_numpy(synth.random_positive((wl.xi, wl.gamma), 8)).cuda()
        z = plan.adjoint(r)
        plan.check()
        hf, z, r = hf.cpu().numpy(), z.cpu().numpy(), r.cpu().numpy()
    cov = np.argwhere(hf > 0)
    pick = cov[rng.choice(len(cov), 300, replace=False)]
    xs = np.concatenate([pick[:, 1], rng.integers(0, wl.gamma, 100)])
    ys = np.concatenate([pick[:, 0], rng.integers(0, wl.xi, 100)])
    assert floored_rel(hf[ys, xs], O.forward_at(geom, taps, f.ravel(), xs, ys)) <= TOL
    ss = rng.integers(0, wl.w, 200)
    ps = rng.integers(0, wl.a, 200)
    rs = rng.integers(0, wl.alpha, 200)
    assert floored_rel(z[ss, rs, ps], O.adjoint_at(geom, taps, r.ravel(), ss, ps, rs)) <= TOL


@pytest.mark.parametrize("boundary", ["clip", "wrap"])
def test_bf16_under_the_other_boundaries(boundary):
    """bfloat16 storage under the clip (h per voxel) and wrap (stored images)
    boundaries: projectors on the rounded inputs within the float32 bound,
    one EM step within one bfloat16 unit of the float64 step from the same
    stored iterate."""
    wl = CASES["ragged"]
    ptr, x, y, v = synth.make_psf(wl)
    if boundary == "clip":
        x, y = x - 9, y + 4
    else:
        x, y = x + wl.gamma - 1 - x.max(), y + wl.xi - 1 - y.max()
    psf = (ptr, x.astype(np.int32), y.astype(np.int32), v)
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf, boundary)
    taps = O.with_values(taps, O.round_bf16(taps.v.astype(np.float32)).astype(np.float64))
    H = O.BlockH(geom, taps)
    f, ft = _bf16_cube(wl, 71)
    r = synth.random_positive((wl.xi, wl.gamma), 72)
    g = (synth.random_positive(geom.n, 73) * 100).astype(np.float32)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype="bf16", boundary=boundary) as plan:
        hf = plan.forward(ft).cpu().numpy().ravel()
        ht = plan.adjoint(torch.from_numpy(r).cuda()).cpu().numpy().ravel()
        f1, _ = plan.reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), 1,
                                 f=ft.clone(), init=None)
        plan.check()
        f1 = f1.float().cpu().numpy().ravel()
    assert floored_rel(hf, H.forward(f.ravel())) <= TOL
    assert floored_rel(ht, H.adjoint(r.ravel())) <= TOL
    step = O.em_step(H, g, f.ravel().astype(np.float64))
    assert floored_rel(f1, step) <= BF16_ULP
