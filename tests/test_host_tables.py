"""Host logic of the plan, checked on the CPU (ctis_tables_inspect: the plan's
table builder and schedulers without a device).

The work lists are checked against definitions written out here: a forward
task (FPA tile, spot cluster) exists exactly when the cluster's footprint
(its K x K box swept over the a x alpha field stop, Eqs. 8 and 12) meets the
tile; an adjoint voxel tile of wavelength s has one task per cluster of s
(Eq. 14). Every schedule form must run every task exactly once, with the
CTA's warps sharing each item and each tile's chunks numbered in order; the
probed CTA-to-SM map may only change which CTA runs which list."""
import numpy as np
import pytest

import synth
from paper_2006_01573_gb300 import CtisError, tables_inspect

RAGGED = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 3)
K5 = synth.Workload("k5", 20, 24, 6, 120, 110, 3, 36.0, 1.2, 5, 1.2, "segmentation", 100.0, 3)
WORKLOADS = [synth.TINY, RAGGED, K5, synth.MODEL_A]
# clipped boundary: the PSF shifted so that some orders spill past FPA edges
CLIPPED = [(RAGGED, (-9, 4)), (synth.MODEL_A, (-40, 35)), (K5, (30, -20))]


def _psf(wl, shift=None):
    ptr, x, y, v = synth.make_psf(wl)
    if shift is not None:
        x, y = x + shift[0], y + shift[1]
    return ptr, x, y, v


def _inspect(wl, forward, n_ctas, shift=None, **kw):
    if shift is not None:
        kw["boundary"] = "clip"
    return tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, _psf(wl, shift), forward,
                          n_ctas, **kw)


def _tile_tasks(t):
    ptr = t["tile_task_ptr"]
    return {tuple(t["tile_xyp"][i]): sorted(t["task_cluster"][ptr[i]:ptr[i + 1]].tolist())
            for i in range(t["tiles"])}


CASES = [(wl, None) for wl in WORKLOADS] + CLIPPED


def _case_id(c):
    return c[0].name + ("" if c[1] is None else f"_clip{c[1][0]}_{c[1][1]}")


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_clusters_cover_every_psf_nonzero(case):
    wl, shift = case
    ptr, x, y, _ = _psf(wl, shift)
    t = _inspect(wl, True, 8, shift)
    K = t["cluster_k"]
    cl = t["cluster_sxy"]
    for s in range(wl.w):
        mine = cl[cl[:, 0] == s]
        for k in range(ptr[s], ptr[s + 1]):
            inside = ((mine[:, 1] <= x[k]) & (x[k] < mine[:, 1] + K)
                      & (mine[:, 2] <= y[k]) & (y[k] < mine[:, 2] + K))
            assert inside.any(), (s, x[k], y[k])
    # every cluster box holds at least one nonzero of its wavelength
    for s, X, Y in cl:
        xs, ys = x[ptr[s]:ptr[s + 1]], y[ptr[s]:ptr[s + 1]]
        assert np.any((X <= xs) & (xs < X + K) & (Y <= ys) & (ys < Y + K))


@pytest.mark.parametrize("tile", ["32x32", "32x16"])
@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_forward_tasks_are_the_footprint_overlaps(case, tile):
    """A forward task exists exactly when the cluster's footprint meets an FPA
    tile (under clipping only its part on the FPA counts), for either forward
    tile shape."""
    wl, shift = case
    t = _inspect(wl, True, 8, shift, forward_tile=tile)
    K, TW, TH = t["cluster_k"], t["tile_w"], t["tile_h"]
    assert (TW, TH) == ((32, 32) if tile == "32x32" else (32, 16))
    expect = {}
    for c, (s, X, Y) in enumerate(t["cluster_sxy"]):
        # the footprint's part on the FPA: [x0, x1) x [y0, y1)
        x0, x1 = max(X, 0), min(X + wl.a + K - 1, wl.gamma)
        y0, y1 = max(Y, 0), min(Y + wl.alpha + K - 1, wl.xi)
        if x0 >= x1 or y0 >= y1:
            continue
        for ty in range(0, wl.xi, TH):
            for tx in range(0, wl.gamma, TW):
                if tx < x1 and x0 < tx + TW and ty < y1 and y0 < ty + TH:
                    expect.setdefault((tx, ty, 0), []).append(c)
    got = _tile_tasks(t)
    assert got == {k: sorted(v) for k, v in expect.items()}   # no tile without a task


@pytest.mark.parametrize("case", CASES, ids=_case_id)
def test_adjoint_tasks_are_the_clusters_of_the_plane(case):
    """A voxel tile of wavelength s lists the clusters of s; under clipping
    only those whose window (tile plus the K - 1 halo, at the cluster's
    offset) meets the FPA."""
    wl, shift = case
    t = _inspect(wl, False, 8, shift)
    TW, TH, K = t["tile_w"], t["tile_h"], t["cluster_k"]
    cl = t["cluster_sxy"]
    expect = {}
    for s in range(wl.w):
        for ty in range(0, wl.alpha, TH):
            for tx in range(0, wl.a, TW):
                expect[(tx, ty, s)] = sorted(
                    c for c in np.nonzero(cl[:, 0] == s)[0].tolist()
                    if shift is None or (cl[c, 1] + tx < wl.gamma and cl[c, 2] + ty < wl.xi and
                                         cl[c, 1] + tx + TW + K - 1 > 0 and
                                         cl[c, 2] + ty + TH + K - 1 > 0))
    assert _tile_tasks(t) == expect


def _check_schedule(t):
    """Every task once; CTA warps share items; chunks numbered in order."""
    nw, wb = t["warps_per_cta"], t["warp_begin"]
    ptr = t["tile_task_ptr"]
    covered = np.zeros(t["tasks"], np.int64)
    chunks = {}
    lists = []
    for cta in range(t["warps"] // nw):
        ws = range(cta * nw, (cta + 1) * nw)
        counts = {wb[w + 1] - wb[w] for w in ws}
        assert len(counts) == 1, "the CTA's warps walk parallel lists"
        items = []
        for k in range(counts.pop()):
            idx = [wb[w] + k for w in ws]
            tiles = {t["item_tile"][i] for i in idx}
            chk = {tuple(t["item_chunk"][i]) for i in idx}
            assert len(tiles) == 1 and len(chk) == 1
            tile, (chunk, nch) = tiles.pop(), chk.pop()
            rs = [tuple(t["item_range"][i]) for i in idx]
            for a, b in zip(rs, rs[1:]):      # warp w runs the w-th consecutive part
                assert a[1] == b[0]
            b0, e0 = rs[0][0], rs[-1][1]
            assert ptr[tile] <= b0 <= e0 <= ptr[tile + 1]
            covered[b0:e0] += 1
            chunks.setdefault(tile, []).append((chunk, nch, b0, e0))
            items.append((tile, chunk, b0, e0))
        lists.append(tuple(items))
    assert np.all(covered == 1), "every task runs exactly once"
    assert set(chunks) == set(range(t["tiles"])), "every tile is an item"
    for tile, cs in chunks.items():
        cs.sort()
        nch = cs[0][1]
        assert [c[0] for c in cs] == list(range(nch)) and all(c[1] == nch for c in cs)
        assert cs[0][2] == ptr[tile] and cs[-1][3] == ptr[tile + 1]
        for a, b in zip(cs, cs[1:]):          # chunk order is task order
            assert a[3] == b[2]
    return lists


SCHEDULES = [dict(), dict(tasks_per_item=16), dict(tasks_per_item=256), dict(item_overhead_q=2),
             dict(item_overhead_q=24), dict(tasks_per_item=32, cta_skew_permille=300),
             dict(item_overhead_q=8, cta_skew_permille=500)]


def _sm_map(n_ctas, per_sm, seed):
    """A CTA-to-SM map with per_sm CTAs on each SM, SM ids in a shuffled order."""
    nsm = n_ctas // per_sm
    ids = np.random.default_rng(seed).permutation(4 * nsm)[:nsm]
    return np.array([ids[b % nsm] for b in range(n_ctas)], np.int32)


@pytest.mark.parametrize("opts", SCHEDULES, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "model")
@pytest.mark.parametrize("forward", [True, False], ids=["fwd", "adj"])
def test_every_schedule_runs_every_task_once(opts, forward):
    for wl, n_ctas in ((synth.TINY, 8), (RAGGED, 12), (synth.MODEL_A, 64)):
        t = _inspect(wl, forward, n_ctas, **opts)
        _check_schedule(t)
        if "tasks_per_item" in opts:
            assert t["chunk"] == opts["tasks_per_item"] and t["split_q"] == 0
        if "item_overhead_q" in opts:
            assert t["split_q"] == opts["item_overhead_q"] and t["chunk"] == 0
        assert t["skew_pm"] == opts.get("cta_skew_permille", 0)


@pytest.mark.parametrize("opts", [dict(tasks_per_item=64), dict(item_overhead_q=12)],
                         ids=["chunks", "split"])
def test_sm_map_only_moves_lists_between_ctas(opts):
    wl = synth.REALISTIC
    base = _check_schedule(_inspect(wl, True, 608, **opts))
    for seed, per_sm in ((1, 4), (2, 4), (3, 3)):   # 3 per SM: an uneven, unexpected map
        sm = _sm_map(608, per_sm, seed)
        mapped = _check_schedule(_inspect(wl, True, 608, block_sm=sm, **opts))
        assert sorted(mapped) == sorted(base)


def test_sm_map_balances_the_sms():
    """With the map, the lists (longest first) go to the least-loaded SM:
    the SMs' task totals are closer than with the map-blind placement."""
    wl = synth.REALISTIC
    sm = _sm_map(608, 4, 7)

    def sm_totals(t):
        nw, wb = t["warps_per_cta"], t["warp_begin"]
        tot = {}
        for cta in range(t["warps"] // nw):
            n = sum(int(r[1] - r[0]) for w in range(cta * nw, (cta + 1) * nw)
                    for r in t["item_range"][wb[w]:wb[w + 1]])
            tot[sm[cta]] = tot.get(sm[cta], 0) + n
        return np.array(list(tot.values()))

    for forward in (True, False):
        blind = sm_totals(_inspect(wl, forward, 608, tasks_per_item=96))
        aware = sm_totals(_inspect(wl, forward, 608, tasks_per_item=96, block_sm=sm))
        assert blind.sum() == aware.sum()
        assert aware.max() - aware.min() <= blind.max() - blind.min()
        assert aware.max() <= 1.1 * aware.mean()


def test_clip_is_needed_for_a_psf_that_leaves_the_fpa():
    wl, shift = CLIPPED[0]
    with pytest.raises(CtisError):
        tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, _psf(wl, shift), True, 8)
    t = _inspect(wl, True, 8, shift)
    _check_schedule(t)


def test_inspect_rejects_bad_arguments():
    wl = synth.TINY
    psf = synth.make_psf(wl)
    with pytest.raises(CtisError):
        tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, True, 0)
    with pytest.raises(CtisError):
        tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, True, 4,
                       block_sm=np.array([0, 1, 4096, 2], np.int32))
    with pytest.raises(CtisError):
        tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, True, 4, tasks_per_item=16,
                       item_overhead_q=4)


def _to_edges(wl):
    """The workload's PSF moved so that its last nonzeros sit in the FPA's last
    column and row: every nonzero stays on the FPA, many shifted copies pass
    the right edge, the last row, or both."""
    ptr, x, y, v = synth.make_psf(wl)
    return (ptr, (x + wl.gamma - 1 - x.max()).astype(np.int32),
            (y + wl.xi - 1 - y.max()).astype(np.int32), v)


def _images_meeting_the_fpa(wl, psf):
    """Each nonzero (x, y) plus its images (x - gamma, y + 1), (x, y - xi),
    (x - gamma, y + 1 - xi) whose footprint [X, X + a) x [Y, Y + alpha)
    meets the FPA, wavelength by wavelength."""
    ptr, x, y, v = psf
    P, X, Y, V = [0], [], [], []
    for s in range(wl.w):
        for k in range(int(ptr[s]), int(ptr[s + 1])):
            for dx, dy in ((0, 0), (-wl.gamma, 1), (0, -wl.xi), (-wl.gamma, 1 - wl.xi)):
                xx, yy = int(x[k]) + dx, int(y[k]) + dy
                if xx + wl.a > 0 and yy + wl.alpha > 0 and xx < wl.gamma and yy < wl.xi:
                    X.append(xx)
                    Y.append(yy)
                    V.append(v[k])
        P.append(len(X))
    return (np.array(P, np.int32), np.array(X, np.int32), np.array(Y, np.int32),
            np.array(V, np.float32))


@pytest.mark.parametrize("wl", [synth.TINY, RAGGED, K5, synth.MODEL_A], ids=lambda w: w.name)
@pytest.mark.parametrize("forward", [True, False], ids=["fwd", "adj"])
def test_wrap_tables_are_the_clip_tables_of_the_images(wl, forward):
    """The wrap boundary (Eq. 7 literally) is stored as the clip reading of
    the PSF and its wrapped images: the work lists and schedules are those of
    a clip plan given that PSF."""
    psf = _to_edges(wl)
    tw = tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, forward, 12, boundary="wrap")
    tc = tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, _images_meeting_the_fpa(wl, psf),
                        forward, 12, boundary="clip")
    assert tw["clusters"] > _inspect(wl, forward, 12, (0, 0))["clusters"]   # images were added
    for key, val in tc.items():
        assert np.array_equal(np.asarray(tw[key]), np.asarray(val)), key
    _check_schedule(tw)


def test_wrap_needs_every_nonzero_on_the_fpa():
    wl = RAGGED
    ptr, x, y, v = _to_edges(wl)
    tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, (ptr, x, y, v), True, 8, boundary="wrap")
    for bad in ((x + 1, y), (x, y + 1), (x - x.min() - 1, y)):
        with pytest.raises(CtisError):
            tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, (ptr, *bad, v), True, 8,
                           boundary="wrap")
    with pytest.raises(CtisError):   # and the reject rule refuses the copies past the edges
        tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, (ptr, x, y, v), True, 8)


@pytest.mark.parametrize("seed", range(30))
@pytest.mark.parametrize("forward", [True, False], ids=["fwd", "adj"])
def test_random_wrap_tables_are_the_clip_tables_of_the_images(seed, forward):
    """Random small geometries, including a field stop as wide or as tall as
    the FPA and nonzeros in the last column and row: the wrap plan's lists are
    the clip plan's lists of the images that meet the FPA."""
    rng = np.random.default_rng(7000 + seed)
    a, al = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    ga = a + int(rng.integers(0, 3)) * int(rng.integers(0, 40))
    xi = al + int(rng.integers(0, 3)) * int(rng.integers(0, 40))
    w = int(rng.integers(1, 4))
    wl = synth.Workload("r", a, al, w, ga, xi, 1, 0.0, 0.0, 1, 1.0, "mask_spectra", 1.0, 1)
    ptr, xs, ys, vs = [0], [], [], []
    for _ in range(w):
        n = int(rng.integers(0, 12))
        xs += rng.integers(0, ga, n).tolist()
        ys += rng.integers(0, xi, n).tolist()
        vs += rng.uniform(0.1, 1.0, n).tolist()
        ptr.append(len(xs))
    xs.append(ga - 1)                                   # the last pixel, in the last wavelength
    ys.append(xi - 1)
    vs.append(0.5)
    ptr[-1] += 1
    psf = (np.array(ptr, np.int32), np.array(xs, np.int32), np.array(ys, np.int32),
           np.array(vs, np.float32))
    tw = tables_inspect(a, al, w, ga, xi, psf, forward, 6, boundary="wrap")
    tc = tables_inspect(a, al, w, ga, xi, _images_meeting_the_fpa(wl, psf), forward, 6,
                        boundary="clip")
    for key, val in tc.items():
        assert np.array_equal(np.asarray(tw[key]), np.asarray(val)), key
    _check_schedule(tw)


def _random_case(seed, boundary):
    rng = np.random.default_rng(8000 + seed)
    a, al = int(rng.integers(1, 50)), int(rng.integers(1, 50))
    ga, xi = a + int(rng.integers(0, 90)), al + int(rng.integers(0, 90))
    w = int(rng.integers(1, 4))
    wl = synth.Workload("r", a, al, w, ga, xi, 1, 0.0, 0.0, 1, 1.0, "mask_spectra", 1.0, 1)
    ptr, xs, ys, vs = [0], [], [], []
    for _ in range(w):
        for _ in range(int(rng.integers(0, 4))):   # blobs of side 1..5
            side = int(rng.integers(1, 6))
            if boundary == "clip":
                x0, y0 = int(rng.integers(-a - 6, ga + 2)), int(rng.integers(-al - 6, xi + 2))
            else:
                x0, y0 = int(rng.integers(0, ga - a + 1)), int(rng.integers(0, xi - al + 1))
            for dy in range(side):
                for dx in range(side):
                    x, y = x0 + dx, y0 + dy
                    if boundary == "reject" and (x + a > ga or y + al > xi):
                        continue
                    xs.append(x)
                    ys.append(y)
                    vs.append(float(rng.uniform(0.1, 1.0)))
        ptr.append(len(xs))
    psf = (np.array(ptr, np.int32), np.array(xs, np.int32), np.array(ys, np.int32),
           np.array(vs, np.float32))
    return wl, psf


@pytest.mark.parametrize("seed", range(20))
@pytest.mark.parametrize("boundary", ["reject", "clip"])
@pytest.mark.parametrize("tile", ["32x32", "32x16"])
def test_random_work_lists_follow_their_definitions(seed, boundary, tile):
    """Random geometries and blob PSFs: forward tasks are exactly the
    (tile, cluster) pairs whose footprint (its part on the FPA) meets the
    tile; adjoint tiles list the clusters of their plane whose window meets
    the FPA; every schedule runs every task once."""
    wl, psf = _random_case(seed, boundary)
    tf = tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, True, 6, boundary=boundary,
                        forward_tile=tile)
    K, TW, TH = tf["cluster_k"], tf["tile_w"], tf["tile_h"]
    expect = {}
    for c, (s, X, Y) in enumerate(tf["cluster_sxy"]):
        x0, x1 = max(X, 0), min(X + wl.a + K - 1, wl.gamma)
        y0, y1 = max(Y, 0), min(Y + wl.alpha + K - 1, wl.xi)
        for ty in range(0, wl.xi, TH):
            for tx in range(0, wl.gamma, TW):
                if x0 < x1 and y0 < y1 and tx < x1 and x0 < tx + TW and ty < y1 and y0 < ty + TH:
                    expect.setdefault((tx, ty, 0), []).append(c)
    assert _tile_tasks(tf) == {k: sorted(v) for k, v in expect.items()}
    _check_schedule(tf)
    ta = tables_inspect(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, False, 6, boundary=boundary)
    TW, TH = ta["tile_w"], ta["tile_h"]
    cl = ta["cluster_sxy"]
    expect = {}
    for s in range(wl.w):
        for ty in range(0, wl.alpha, TH):
            for tx in range(0, wl.a, TW):
                expect[(tx, ty, s)] = sorted(
                    c for c in np.nonzero(cl[:, 0] == s)[0].tolist()
                    if boundary == "reject" or (cl[c, 1] + tx < wl.gamma and cl[c, 2] + ty < wl.xi and
                                                cl[c, 1] + tx + TW + K - 1 > 0 and
                                                cl[c, 2] + ty + TH + K - 1 > 0))
    assert _tile_tasks(ta) == expect
    _check_schedule(ta)
