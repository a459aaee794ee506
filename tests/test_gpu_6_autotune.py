"""GPU tests of the schedule autotuner: it keeps a schedule from its candidate
set, and reconstructions on the tuned plan still meet the parity bounds and
stay bit-reproducible (the schedule only regroups the chunk partial sums)."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import Plan
from tests.helpers import floored_rel, problem, rel_l2

pytestmark = pytest.mark.gpu

CANDIDATES = ({("chunk", c, 0) for c in (16, 24, 32, 48, 64, 96, 128, 192)}
              | {("split", q, 0) for q in (2, 4, 8, 12, 16, 24)}
              | {("chunk", c, s) for c in (64, 96, 128) for s in (100, 200, 300)}
              | {("split", q, s) for q in (12, 16, 20) for s in (100, 200, 300)})


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def test_autotuned_plan_matches_oracle_and_is_reproducible():
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)
    ref, _ = O.mlem(H, g, wl.k)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        model_choice = plan.schedules()
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        fc, ac = plan.autotune(gt)
        assert fc in CANDIDATES | {model_choice[0]} and ac in CANDIDATES | {model_choice[1]}
        assert plan.forward_tile() in ("32x32", "32x16")
        a, _ = plan.reconstruct(gt, k=wl.k, init="ones")
        a = a.clone()
        b, _ = plan.reconstruct(gt, k=wl.k, init="ones")
        plan.check()
        got = b.cpu().numpy().ravel()
    assert torch.equal(a, b)
    assert floored_rel(got, ref) <= wl.k * 1e-5
    assert rel_l2(got, ref) <= 1e-5 * np.sqrt(wl.k)


def test_autotune_full_size_stays_within_tolerance_of_untuned():
    wl = synth.REALISTIC
    psf = synth.make_psf(wl)
    k = 10
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as p1, \
            Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as p2:
        hf = p1.forward(torch.from_numpy(synth.make_scene(wl)).cuda())
        g, _ = synth.make_measurement(hf.cpu().numpy(), wl.peak, wl.seed)
        gt = torch.from_numpy(g).cuda()
        p2.autotune(gt)
        a, sa = p1.reconstruct(gt, k=k, init="ones", stats=True)
        b, sb = p2.reconstruct(gt, k=k, init="ones", stats=True)
        p1.check()
        p2.check()
        a, b = a.cpu().numpy(), b.cpu().numpy()
        sa, sb = sa.cpu().numpy(), sb.cpu().numpy()
    # two float32 reconstructions that differ only in the grouping of sums
    assert floored_rel(b, a) <= 2 * k * 1e-5
    assert np.all(np.abs(sb - sa) <= 2e-5 * np.abs(sa))


@pytest.mark.parametrize("opts", [dict(tasks_per_item=24), dict(item_overhead_q=2),
                                  dict(item_overhead_q=24),
                                  dict(tasks_per_item=16, cta_skew_permille=300),
                                  dict(item_overhead_q=4, cta_skew_permille=500)])
def test_forced_schedules_match_oracle(opts):
    """Every schedule form (chunks assigned longest first; the balanced split,
    whose runs cut tiles into chunks on consecutive CTAs) gives the EM
    iterates within the parity bounds, on the tiny and the ragged workloads."""
    for wl in (synth.TINY, synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7,
                                          "mask_spectra", 100.0, 5)):
        geom, psf, H, _, g = problem(wl)
        ref, _ = O.mlem(H, g, wl.k)
        with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, **opts) as plan:
            kind = "chunk" if "tasks_per_item" in opts else "split"
            skew = opts.get("cta_skew_permille", 0)
            assert all(s[0] == kind and s[2] == skew for s in plan.schedules())
            gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
            got, _ = plan.reconstruct(gt, k=wl.k, init="ones")
            plan.check()
            got = got.cpu().numpy().ravel()
        assert floored_rel(got, ref) <= wl.k * 1e-5, wl.name
        assert rel_l2(got, ref) <= 1e-5 * np.sqrt(wl.k), wl.name


def test_schedule_options_are_exclusive():
    from paper_2006_01573_gb300 import CtisError
    wl = synth.TINY
    with pytest.raises(CtisError):
        Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl), tasks_per_item=16,
             item_overhead_q=4)
    with pytest.raises(CtisError):
        Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, synth.make_psf(wl), cta_skew_permille=901)


def test_set_schedule_reapplies_a_schedule():
    """A schedule set on a plan is the one it reports, and the plan's
    reconstructions stay within the parity bounds and bit-reproducible."""
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)
    ref, _ = O.mlem(H, g, wl.k)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        for fwd, adj in ((("chunk", 16, 300), ("split", 8, 0)), (("split", 4, 100), ("chunk", 24, 0))):
            plan.set_schedule(True, fwd)
            plan.set_schedule(False, adj)
            assert plan.schedules() == (fwd, adj)
            a, _ = plan.reconstruct(gt, k=wl.k, init="ones")
            a = a.clone()
            b, _ = plan.reconstruct(gt, k=wl.k, init="ones")
            plan.check()
            assert torch.equal(a, b)
            got = b.cpu().numpy().ravel()
            assert floored_rel(got, ref) <= wl.k * 1e-5
        with pytest.raises(ValueError):
            plan.set_schedule(True, ("lpt", 16, 0))
        from paper_2006_01573_gb300 import CtisError
        with pytest.raises(CtisError):
            plan.set_schedule(True, ("chunk", 16, 901))


STAT_KEYS = ("flux_hf", "flux_g_covered", "loglik", "resid2")


@pytest.mark.parametrize("tile", ["32x16"])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_other_forward_tiles_in_em_and_statistics(dtype, tile):
    """EM on 32 x 16 forward tiles (the fused ratio and the per-tile
    statistics over twice as many tiles). float32: iterates and statistics
    within the parity bounds of the oracle. bfloat16: iterates within the
    bound of the oracle EM that stores every iterate in bfloat16, and the
    same statistics as the 32 x 32 run up to the rounding of a few iterate
    elements (the tiles regroup float32 partial sums, so an element may round
    to the neighbouring bfloat16 value)."""
    for wl in (synth.TINY, synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7,
                                          "mask_spectra", 100.0, 5)):
        geom, psf, H, _, g = problem(wl)
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        runs = {}
        for t in ("32x32", tile):
            with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype=dtype,
                      forward_tile=t) as plan:
                assert plan.forward_tile() == t
                got, st = plan.reconstruct(gt, k=wl.k, init="ones", stats=True)
                plan.check()
                runs[t] = (got.float().cpu().numpy().ravel(), st.cpu().numpy())
        got, st = runs[tile]
        if dtype == "f32":
            ref, hist = O.mlem(H, g, wl.k)
            assert floored_rel(got, ref) <= wl.k * 1e-5, wl.name
            assert rel_l2(got, ref) <= 1e-5 * np.sqrt(wl.k), wl.name
            for t in range(wl.k + 1):
                for q, key in enumerate(STAT_KEYS):
                    assert abs(st[t, q] - hist[t][key]) <= 1e-5 * abs(hist[t][key]), (wl.name, t, key)
        else:
            taps = O.merge_psf(geom, psf)
            stored = O.round_bf16(taps.v.astype(np.float32)).astype(np.float64)
            Hb = O.BlockH(geom, O.with_values(taps, stored))
            store = lambda z: O.round_bf16(z.astype(np.float32))   # noqa: E731
            f_stored = np.ones(geom.m)
            for _ in range(wl.k):
                f_stored = O.em_step_stored(Hb, g, f_stored, store)
            assert rel_l2(got, f_stored) <= 4 * 2.0 ** -8, wl.name
            base = runs["32x32"][1]
            assert np.all(np.abs(st - base) <= 1e-3 * np.abs(base)), wl.name


def test_autotune_on_a_small_field_stop_keeps_parity():
    """A 20x20 field stop with many wavelengths, where 32 x 16 forward tiles
    compute far less of the footprints' empty rows than 32 x 32 ones (the
    autotuner keeps them on the GPU of this project): after autotuning,
    whichever shape it kept, the EM iterates and every statistic meet the
    parity bounds, and the plan's forward tile count is the one its shape's
    work lists have (switching shape regrows the tile tickets and
    statistics)."""
    from paper_2006_01573_gb300._native import tables_inspect
    wl = synth.Workload("fs20", 20, 20, 24, 192, 192, 5, 30.0, 1.0, 3, 0.8, "segmentation",
                        2000.0, 6)
    geom, psf, H, _, g = problem(wl)
    ref, hist = O.mlem(H, g, wl.k)
    with Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf) as plan:
        gt = torch.from_numpy(g.reshape(wl.xi, wl.gamma)).cuda()
        plan.autotune(gt)
        tile = plan.forward_tile()
        assert tile in ("32x32", "32x16")
        t = tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, True, 608, forward_tile=tile)
        assert int(plan.info()["fwd_tiles"]) == t["tiles"]
        got, st = plan.reconstruct(gt, k=wl.k, init="ones", stats=True)
        plan.check()
        got, st = got.cpu().numpy().ravel(), st.cpu().numpy()
    assert floored_rel(got, ref) <= wl.k * 1e-5
    assert rel_l2(got, ref) <= 1e-5 * np.sqrt(wl.k)
    for it in range(wl.k + 1):
        for q, key in enumerate(STAT_KEYS):
            assert abs(st[it, q] - hist[it][key]) <= 1e-5 * abs(hist[it][key]), (it, key)
