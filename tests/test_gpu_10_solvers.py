"""GPU parity of the other solvers on the projector pair (ctis_reconstruct_solver:
SART and SMART, the simultaneous ART and MART) against the FP64 oracle's
sart_step / smart_step, fused into the same forward and adjoint launches as
EM. Tolerances: SMART is multiplicative like EM and takes the EM suite's
bounds (k updates: k * 1e-5 floored-relative); SART adds signed terms, so an
element's float32 error is a few eps times |f| + |step|, which cancellation
can leave far above the new value: its bound is normwise, max |error| <=
k * 1e-5 * max |f|. Both: relative L2 <= 1e-5 sqrt(k), statistics 1e-5
relative. SMART's log and exp are the fast intrinsics (a few ulp each, far
inside the bound)."""
import math

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CtisError, Plan
from tests.helpers import floored_rel, geometry, problem, rel_l2

pytestmark = pytest.mark.gpu

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 500.0, 6)
K5 = synth.Workload("k5", 20, 24, 6, 120, 110, 3, 36.0, 1.2, 5, 1.2, "segmentation", 800.0, 6)
STAT_KEYS = ("flux_hf", "flux_g_covered", "loglik", "resid2")
K = 6


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _check(got, st, ref, hist, k, solver):
    if solver == "sart":
        assert np.max(np.abs(got - ref)) <= k * 1e-5 * np.max(np.abs(ref))
    else:
        assert floored_rel(got, ref) <= k * 1e-5
    assert rel_l2(got, ref) <= 1e-5 * math.sqrt(k)
    for t in range(k + 1):
        for q, key in enumerate(STAT_KEYS):
            assert abs(st[t, q] - hist[t][key]) <= 1e-5 * abs(hist[t][key]) + 1e-9, (t, key)


@pytest.mark.parametrize("wl", [synth.TINY, RAGGED, K5, synth.MODEL_A], ids=lambda w: w.name)
@pytest.mark.parametrize("solver,lam", [("sart", 1.0), ("sart", 1.7), ("smart", 1.0), ("smart", 0.5)])
def test_solver_iterations_and_statistics(wl, solver, lam):
    geom, psf, H, _, g = problem(wl)
    ref, hist = O.solve(H, g, K, solver, lam)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        out, st = plan.reconstruct(gt, K, init="ones", stats=True, solver=solver, relax=lam)
        plan.check()
        got, st = out.cpu().numpy().ravel(), st.cpu().numpy()
    _check(got, st, ref, hist, K, solver)
    if solver == "sart":
        assert got.min() >= 0.0


@pytest.mark.parametrize("wl", [RAGGED, synth.MODEL_A], ids=lambda w: w.name)
@pytest.mark.parametrize("solver", ["sart", "smart"])
def test_solvers_on_32x16_forward_tiles(wl, solver):
    """The solvers' ratio rules (SART's row-sum weighted residual, SMART's
    log ratio) in the epilogue of the 32 x 16 forward tiles."""
    geom, psf, H, _, g = problem(wl)
    ref, hist = O.solve(H, g, K, solver, 1.0)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, forward_tile="32x16") as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        out, st = plan.reconstruct(gt, K, init="ones", stats=True, solver=solver, relax=1.0)
        plan.check()
        got, st = out.cpu().numpy().ravel(), st.cpu().numpy()
    _check(got, st, ref, hist, K, solver)


@pytest.mark.parametrize("boundary", ["clip", "wrap"])
@pytest.mark.parametrize("solver", ["sart", "smart"])
def test_solvers_under_the_other_boundaries(boundary, solver):
    """Per-voxel h (clip) and the stored wrapped images (wrap) feed the
    same updates."""
    wl = RAGGED
    ptr, x, y, v = synth.make_psf(wl)
    if boundary == "clip":
        x, y = x - 9, y + 4
    else:
        x, y = x + wl.gamma - 1 - x.max(), y + wl.xi - 1 - y.max()
    psf = (ptr, x.astype(np.int32), y.astype(np.int32), v)
    H = O.build_H(geometry(wl), psf, boundary=boundary)
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    ref, hist = O.solve(H, g, K, solver, 1.0)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, boundary=boundary) as plan:
        out, st = plan.reconstruct(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda(), K,
                                   init="ones", stats=True, solver=solver)
        plan.check()
    _check(out.cpu().numpy().ravel(), st.cpu().numpy(), ref, hist, K, solver)


def test_one_step_from_a_given_iterate():
    """From the oracle's own iterate, one more update equals its step."""
    wl = synth.MODEL_A
    geom, psf, H, _, g = problem(wl)
    f0 = O.solve(H, g, 3, "sart")[0].astype(np.float32)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        for solver, step in (("sart", O.sart_step), ("smart", O.smart_step)):
            f = torch.from_numpy(f0.reshape(wl.w, wl.alpha, wl.a)).cuda()
            out, _ = plan.reconstruct(gt, 1, f=f, init=None, solver=solver, relax=0.8)
            want = step(H, g, f0.astype(np.float64), 0.8)
            err = np.abs(out.cpu().numpy().ravel() - want)
            if solver == "sart":
                assert err.max() <= 1e-5 * np.abs(want).max(), solver
            else:
                assert floored_rel(out.cpu().numpy().ravel(), want) <= 1e-5, solver
        plan.check()


def test_graph_cache_and_new_values():
    """Switching solver or relaxation re-captures; repeating a call replays
    bit for bit; new PSF values rebuild SART's row sums."""
    wl = RAGGED
    geom, psf, H, _, g = problem(wl)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        f = torch.empty((wl.w, wl.alpha, wl.a), device="cuda")
        runs = {}
        for solver, lam in (("em", 1.0), ("sart", 1.0), ("sart", 0.5), ("smart", 1.0),
                            ("sart", 1.0), ("em", 1.0)):
            plan.reconstruct(gt, 4, f=f, init="ones", solver=solver, relax=lam)
            key = (solver, lam)
            if key in runs:
                assert torch.equal(runs[key], f), key
            runs[key] = f.clone()
        assert not torch.equal(runs[("sart", 1.0)], runs[("sart", 0.5)])
        s, x, y, v, _ = plan.export_taps()
        v2 = (np.asarray(v) * synth.random_positive(len(v), 93) * 2).astype(np.float32)
        plan.set_values(v2)
        out, _ = plan.reconstruct(gt, 3, f=f, init="ones", solver="sart")
        plan.check()
    H2 = O.build_H(geom, (np.searchsorted(s, np.arange(wl.w + 1)).astype(np.int32), x, y, v2))
    want = O.solve(H2, g, 3, "sart")[0]
    assert np.max(np.abs(out.cpu().numpy().ravel() - want)) <= 3e-5 * np.abs(want).max()


def test_bf16_storage_runs_the_solvers():
    """bfloat16 datacube storage: the same updates, the iterate re-rounded
    each time; within 2e-2 relative L2 of the float32 run."""
    wl = RAGGED
    geom, psf, H, _, g = problem(wl)
    gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
    for solver in ("sart", "smart"):
        with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as p32, \
                Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype="bf16") as p16:
            a, _ = p32.reconstruct(gt, K, init="ones", solver=solver)
            b, _ = p16.reconstruct(gt, K, init="ones", solver=solver)
            p16.check()
            assert rel_l2(b.float().cpu().numpy(), a.cpu().numpy()) <= 2e-2, solver


def test_bad_solver_arguments_are_refused():
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        for lam in (0.0, -1.0, 2.5, float("nan")):
            with pytest.raises(CtisError):
                plan.reconstruct(gt, 2, solver="sart", relax=lam)
        with pytest.raises(KeyError):
            plan.reconstruct(gt, 2, solver="mart")


@pytest.mark.parametrize("solver", ["sart", "smart"])
def test_batched_frames_equal_single_frame_solver_runs(solver):
    """ctis_reconstruct_batched_solver: frames of two geometries, each equal
    bit for bit to its single-frame ctis_reconstruct_solver run."""
    from paper_2006_01573_gb300 import reconstruct_batched
    wls = [synth.TINY, RAGGED]
    plans = [Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl)) for wl in wls]
    try:
        plan_idx = [0, 1, 1, 0, 1]
        gs = []
        for n, i in enumerate(plan_idx):
            wl = wls[i]
            H = O.build_H(geometry(wl), synth.make_psf(wl))
            g, _ = synth.make_measurement(H.forward(synth.make_scene(wl, 500 + n).ravel()),
                                          wl.peak, 500 + n)
            gs.append(torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda())
        fs, st = reconstruct_batched(plans, plan_idx, gs, 5, stats=True, solver=solver, relax=0.9)
        for p in plans:
            p.check()
        for n, i in enumerate(plan_idx):
            ref, ref_st = plans[i].reconstruct(gs[n], 5, init="ones", stats=True, solver=solver,
                                               relax=0.9)
            assert torch.equal(fs[n], ref) and torch.equal(st[n], ref_st), n
    finally:
        for p in plans:
            p.close()
