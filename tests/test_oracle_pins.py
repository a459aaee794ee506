"""Pins for the FP64 oracle: each check compares it with something other than
itself (hand-worked values, a dense H assembled from Eqs. 5-7, the FFT form of
Eqs. 13/17, SciPy's 2-D convolution, brute-force loops, EM invariants)."""
import json
import os

import numpy as np
import pytest
import scipy.signal

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _geom(a, al, w, ga, xi):
    return O.Geometry(a, al, w, ga, xi)


def _tiny_psf(geom, nnz, seed, dup=0):
    return synth.random_sparse_psf(geom.w, nnz, geom.gamma - geom.a, geom.xi - geom.alpha,
                                   seed, duplicates=dup)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# --- hand-worked values -------------------------------------------------------

def test_golden_index_map():
    gold = json.load(open(os.path.join(GOLDEN, "hand_worked_a2_alpha2_gamma4_xi3.json")))
    g = gold["index_map"]["geometry"]
    geom = _geom(g["a"], g["alpha"], g["w"], g["gamma"], g["xi"])
    assert O.index_map(geom).tolist() == gold["index_map"]["i_of_j"]


def test_golden_projector_and_em_step():
    gold = json.load(open(os.path.join(GOLDEN, "hand_worked_a2_alpha2_gamma4_xi3.json")))["projector"]
    g = gold["geometry"]
    geom = _geom(g["a"], g["alpha"], g["w"], g["gamma"], g["xi"])
    p = gold["psf"]
    psf = (np.array(p["ptr"]), np.array(p["x"]), np.array(p["y"]), np.array(p["val"], np.float32))
    H = O.build_H(geom, psf)
    f = np.array(gold["f_r_p"]).ravel()
    hf = H.forward(f)
    assert np.array_equal(hf, np.array(gold["hf_y_x"]).ravel())
    assert np.array_equal(H.adjoint(hf), np.array(gold["adjoint_of_hf_r_p"]).ravel())
    assert np.all(H.h() == gold["h"])
    em = gold["em_from_ones"]
    assert np.array_equal(H.forward(np.ones(geom.m)), np.array(em["hf1_y_x"]).ravel())
    f2, _ = O.mlem(H, hf, 1)
    assert np.allclose(f2, np.array(em["f2_r_p"]).ravel(), rtol=0, atol=1e-15)


def _golden_stats_case():
    gold = json.load(open(os.path.join(GOLDEN, "hand_worked_a2_alpha2_gamma4_xi3.json")))["projector"]
    q = np.array(gold["hf_y_x"], dtype=np.float64).ravel()
    st = gold["stats"]
    g = np.array(st["g_y_x"], dtype=np.float64).ravel()
    c2, c3, c0 = st["loglik_ln2_ln3_const"]
    want = {"flux_hf": st["flux_hf"], "flux_g_covered": st["flux_g_covered"],
            "loglik": c2 * np.log(2.0) + c3 * np.log(3.0) + c0, "resid2": st["resid2"]}
    return q, g, want


def _matches_golden(got, want):
    return all(abs(got[k] - want[k]) <= 1e-14 * max(1.0, abs(want[k])) for k in want)


def test_golden_statistics():
    """stats() against the hand-worked sums of Eq. 2's likelihood over the
    support of H f, with a g > 0 pixel off the support and a g = 0 pixel on it."""
    gold = json.load(open(os.path.join(GOLDEN, "hand_worked_a2_alpha2_gamma4_xi3.json")))["projector"]
    p = gold["psf"]
    geom = _geom(2, 2, 1, 4, 3)
    psf = (np.array(p["ptr"]), np.array(p["x"]), np.array(p["y"]), np.array(p["val"], np.float32))
    H = O.build_H(geom, psf)
    q, g, want = _golden_stats_case()
    assert np.array_equal(H.forward(np.array(gold["f_r_p"]).ravel()), q)
    assert _matches_golden(O.stats(q, g), want)


def _mutant_stats(q, g, kind):
    """stats() with one plausible mistake planted."""
    pos = q > 0
    out = dict(O.stats(q, g))
    if kind == "all_pixels_resid":      # residual over every pixel, not the support
        out["resid2"] = float(np.sum((g - q) ** 2))
    elif kind == "all_pixels_flux_g":   # covered flux over every pixel
        out["flux_g_covered"] = float(g.sum())
    elif kind == "unsquared_resid":
        out["resid2"] = float(np.sum(np.abs(g[pos] - q[pos])))
    elif kind == "resid_sign_dropped":  # (g + q)^2
        out["resid2"] = float(np.sum((g[pos] + q[pos]) ** 2))
    elif kind == "log10":
        out["loglik"] = float(np.sum(g[pos] * np.log10(q[pos])) - q[pos].sum())
    elif kind == "missing_q_term":
        out["loglik"] = float(np.sum(g[pos] * np.log(q[pos])))
    elif kind == "g_zero_pixels_dropped":   # a g = 0 pixel still adds -q
        on = pos & (g > 0)
        out["loglik"] = float(np.sum(g[on] * np.log(q[on])) - q[on].sum())
    elif kind == "flux_is_g":
        out["flux_hf"] = float(g[pos].sum())
    elif kind == "swapped_log_args":   # q log g - g
        on = pos & (g > 0)
        out["loglik"] = float(np.sum(q[on] * np.log(g[on])) - g[pos].sum())
    return out


@pytest.mark.parametrize("kind", ["all_pixels_resid", "all_pixels_flux_g", "unsquared_resid",
                                  "resid_sign_dropped", "log10", "missing_q_term",
                                  "g_zero_pixels_dropped", "flux_is_g", "swapped_log_args"])
def test_planted_statistics_mistakes_are_caught_by_golden_pin(kind):
    q, g, want = _golden_stats_case()
    assert not _matches_golden(_mutant_stats(q, g, kind), want)


# --- index map and E ------------------------------------------------------------

@pytest.mark.parametrize("dims", [(2, 2, 2, 4, 3), (3, 2, 3, 5, 4), (4, 3, 2, 7, 6), (1, 1, 1, 1, 1)])
def test_index_map_is_the_embedding_E(dims):
    """Sec. 3 map equals the nonzero row of each column of I_w kron E (Eqs. 5-6)."""
    geom = _geom(*dims)
    a, al, ga, n = geom.a, geom.alpha, geom.gamma, geom.n
    Q = np.vstack([np.eye(a), np.zeros((ga - a, a))])
    top = np.kron(np.eye(al), Q)
    E = np.vstack([top, np.zeros((n - top.shape[0], a * al))])
    big = np.kron(np.eye(geom.w), E)
    rows = np.argmax(big, axis=0)
    assert np.all(big.sum(axis=0) == 1)
    assert np.array_equal(rows, O.index_map(geom))


# --- dense brute force (Eqs. 5-7) -------------------------------------------------

@pytest.mark.parametrize("dims,nnz,dup,seed", [
    ((3, 2, 2, 6, 5), 3, 0, 1),
    ((4, 3, 3, 9, 7), 5, 2, 2),
    ((2, 4, 2, 5, 9), 4, 1, 3),
    ((5, 5, 1, 8, 8), 6, 0, 4),
])
def test_sparse_H_equals_dense_circulant_form(dims, nnz, dup, seed):
    geom = _geom(*dims)
    psf = _tiny_psf(geom, nnz, seed, dup)
    D = O.dense_H(geom, psf)
    S = O.build_H(geom, psf).as_csr().toarray()
    assert D.shape == (geom.n, geom.m)
    np.testing.assert_allclose(S, D, rtol=1e-15, atol=0)
    assert np.array_equal(S != 0, D != 0)


def test_dense_form_on_synthetic_grating_psf():
    wl = synth.Workload("t", 4, 3, 3, 22, 20, 3, 6.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 3)
    psf = synth.make_psf(wl)
    geom = _geom(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    np.testing.assert_allclose(O.build_H(geom, psf).as_csr().toarray(), O.dense_H(geom, psf),
                               rtol=1e-15, atol=0)


# --- FFT form of the paper (Eqs. 13 and 17) ----------------------------------------

def test_fft_forms_match_sparse_projectors_tiny_workload():
    wl = synth.TINY
    geom = _geom(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    psf = synth.make_psf(wl)
    H = O.build_H(geom, psf)
    f = synth.make_scene(wl).ravel()
    u = synth.random_positive(geom.n, seed=7)
    assert _rel(O.fft_forward(geom, psf, f), H.forward(f)) < 1e-12
    assert _rel(O.fft_adjoint(geom, psf, u), H.adjoint(u)) < 1e-12


# --- adjoint identity --------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_identity(seed):
    geom = _geom(7, 5, 4, 19, 17)
    psf = _tiny_psf(geom, 9, seed, dup=3)
    H = O.build_H(geom, psf)
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(geom.m)
    r = rng.standard_normal(geom.n)
    lhs = np.dot(H.forward(f), r)
    rhs = np.dot(f, H.adjoint(r))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


# --- special cases ---------------------------------------------------------------

def test_single_wavelength_is_2d_convolution():
    geom = _geom(6, 5, 1, 16, 14)
    psf = _tiny_psf(geom, 7, 11)
    H = O.build_H(geom, psf)
    taps = O.merge_psf(geom, psf)
    img = np.zeros((geom.xi, geom.gamma))
    img[taps.y, taps.x] = taps.v
    f = synth.random_positive((geom.alpha, geom.a), 3).astype(np.float64)
    conv = scipy.signal.convolve2d(img, f, mode="full")[:geom.xi, :geom.gamma]
    np.testing.assert_allclose(H.forward(f.ravel()).reshape(geom.xi, geom.gamma), conv,
                               rtol=1e-13, atol=1e-13)
    u = synth.random_positive((geom.xi, geom.gamma), 4).astype(np.float64)
    # (H^T u)(p, r) = sum_k v_k u(x_k + p, y_k + r): correlate u with the PSF image
    corr = scipy.signal.correlate2d(u, img, mode="full")
    # full-mode index of lag (r, p) is (r + xi - 1, p + gamma - 1)
    ref = corr[geom.xi - 1:geom.xi - 1 + geom.alpha, geom.gamma - 1:geom.gamma - 1 + geom.a]
    np.testing.assert_allclose(H.adjoint(u.ravel()).reshape(geom.alpha, geom.a), ref,
                               rtol=1e-13, atol=1e-13)


def test_delta_psf_paste_crop_and_exact_em_recovery():
    geom = _geom(5, 4, 3, 12, 11)
    x0 = [2, 0, 7]
    y0 = [1, 6, 3]
    psf = (np.arange(4, dtype=np.int32), np.array(x0, np.int32), np.array(y0, np.int32),
           np.ones(3, np.float32))
    H = O.build_H(geom, psf)
    f = synth.random_positive(geom.m, 5).astype(np.float64)
    hf = H.forward(f).reshape(geom.xi, geom.gamma)
    expect = np.zeros_like(hf)
    fr = f.reshape(geom.w, geom.alpha, geom.a)
    for s in range(geom.w):
        expect[y0[s]:y0[s] + geom.alpha, x0[s]:x0[s] + geom.a] += fr[s]
    assert np.array_equal(hf, expect)
    u = synth.random_positive(geom.n, 6).astype(np.float64).reshape(geom.xi, geom.gamma)
    crop = np.stack([u[y0[s]:y0[s] + geom.alpha, x0[s]:x0[s] + geom.a] for s in range(geom.w)])
    assert np.array_equal(H.adjoint(u.ravel()), crop.ravel())
    # disjoint footprints: one EM step from ones on noiseless data gives f exactly
    geom1 = _geom(5, 4, 1, 12, 11)
    psf1 = (np.array([0, 1], np.int32), np.array([3], np.int32), np.array([2], np.int32),
            np.ones(1, np.float32))
    H1 = O.build_H(geom1, psf1)
    f1 = synth.random_positive(geom1.m, 8).astype(np.float64)
    f2, _ = O.mlem(H1, H1.forward(f1), 1)
    np.testing.assert_allclose(f2, f1, rtol=1e-15, atol=0)


# --- merging and bounds ---------------------------------------------------------------

def test_merge_matches_bruteforce_dict():
    geom = _geom(3, 3, 4, 10, 9)
    psf = _tiny_psf(geom, 12, 21, dup=6)
    taps = O.merge_psf(geom, psf)
    ptr, x, y, v = psf
    for s in range(geom.w):
        d = {}
        for k in range(ptr[s], ptr[s + 1]):
            key = (int(y[k]), int(x[k]))
            d[key] = d.get(key, 0.0) + float(v[k])
        keys = sorted(d)
        tx, ty, tv = taps.of(s)
        assert [(int(b), int(a)) for a, b in zip(tx, ty)] == keys
        np.testing.assert_allclose(tv, [d[k] for k in keys], rtol=1e-15)


def test_bounds_rejects_off_fpa():
    geom = _geom(4, 4, 1, 10, 10)
    ok = (np.array([0, 1]), np.array([6]), np.array([6]), np.ones(1, np.float32))
    O.check_bounds(geom, ok)
    for x, y in [(7, 0), (0, 7), (-1, 0), (0, -1)]:
        bad = (np.array([0, 1]), np.array([x]), np.array([y]), np.ones(1, np.float32))
        with pytest.raises(O.OutOfBounds):
            O.check_bounds(geom, bad)


# --- pointwise evaluators ---------------------------------------------------------

def test_pointwise_evaluators_match_full_projectors():
    wl = synth.TINY
    geom = _geom(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    psf = synth.make_psf(wl)
    H = O.build_H(geom, psf)
    taps = O.merge_psf(geom, psf)
    f = synth.make_scene(wl).ravel()
    u = synth.random_positive(geom.n, 9)
    rng = np.random.default_rng(0)
    xs = rng.integers(0, geom.gamma, 200)
    ys = rng.integers(0, geom.xi, 200)
    full = H.forward(f).reshape(geom.xi, geom.gamma)
    np.testing.assert_allclose(O.forward_at(geom, taps, f, xs, ys), full[ys, xs], rtol=1e-13, atol=1e-13)
    ss = rng.integers(0, geom.w, 100)
    ps = rng.integers(0, geom.a, 100)
    rs = rng.integers(0, geom.alpha, 100)
    adj = H.adjoint(u).reshape(geom.w, geom.alpha, geom.a)
    np.testing.assert_allclose(O.adjoint_at(geom, taps, u, ss, ps, rs), adj[ss, rs, ps], rtol=1e-13)


# --- EM invariants ----------------------------------------------------------------

def _tiny_problem(noisy=True):
    wl = synth.TINY
    geom = _geom(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    psf = synth.make_psf(wl)
    H = O.build_H(geom, psf)
    f_true = synth.make_scene(wl).ravel().astype(np.float64)
    q = H.forward(f_true)
    if noisy:
        g, scale = synth.make_measurement(q, wl.peak, wl.seed)
    else:
        g, scale = q * (wl.peak / q.max()), wl.peak / q.max()
    return geom, H, g.astype(np.float64), f_true * scale


@pytest.mark.parametrize("noisy", [False, True])
def test_em_invariants(noisy):
    geom, H, g, _ = _tiny_problem(noisy)
    f, hist = O.mlem(H, g, 20)
    assert np.all(f >= 0)
    h = H.h()
    f_t = np.ones(geom.m)
    for t in range(20):
        q = H.forward(f_t)
        f_t = O.em_update(f_t, H.adjoint(O.ratio(g, q)), h)
        covered = g[q > 0].sum()
        # flux: sum_i (H f')_i = sum_j h_j f'_j = <Hf, u> = sum_{q>0} g
        assert abs(H.forward(f_t).sum() - covered) <= 1e-10 * covered
    lls = [s["loglik"] for s in hist]
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(lls, lls[1:]))


def test_noiseless_loglik_rises_toward_its_maximum():
    geom, H, g, _ = _tiny_problem(noisy=False)
    _, hist = O.mlem(H, g, 40)
    pos = g > 0
    ll_max = float(np.sum(g[pos] * np.log(g[pos])) - g.sum())
    lls = [s["loglik"] for s in hist]
    assert lls[-1] <= ll_max + 1e-9 * abs(ll_max)
    gap0, gap = ll_max - lls[0], ll_max - lls[-1]
    assert gap < 0.05 * gap0


def test_htg_initial_guess_is_adjoint_of_g():
    geom, H, g, _ = _tiny_problem(noisy=True)
    f, hist = O.mlem(H, g, 0, init="htg")
    np.testing.assert_allclose(f, H.adjoint(g), rtol=0, atol=0)


# --- gradients ------------------------------------------------------------------------

def test_psf_value_grad_matches_finite_differences_of_dense_H():
    geom = _geom(4, 3, 2, 9, 8)
    psf = _tiny_psf(geom, 4, 31)
    taps = O.merge_psf(geom, psf)
    rng = np.random.default_rng(1)
    f = rng.uniform(0.1, 1, geom.m)
    gy = rng.standard_normal(geom.n)
    grad = O.psf_value_grad(geom, taps, f, gy)
    eps = 1e-6
    for t in range(taps.v.size):
        def loss(delta):
            v = taps.v.copy()
            v[t] += delta
            p = (taps.ptr, taps.x, taps.y, v)
            return gy @ (O.dense_H(geom, p) @ f)
        fd = (loss(eps) - loss(-eps)) / (2 * eps)
        assert abs(fd - grad[t]) <= 1e-7 * max(1.0, abs(grad[t]))


def test_nll_gradient_wrt_f_is_Ht_of_one_minus_ratio():
    """d/df sum(Hf - g log Hf) = H^T(1 - g/Hf): central differences on dense H."""
    geom = _geom(3, 3, 2, 8, 7)
    psf = _tiny_psf(geom, 4, 5)
    D = O.dense_H(geom, psf)
    H = O.build_H(geom, psf)
    rng = np.random.default_rng(2)
    f = rng.uniform(0.5, 1.5, geom.m)
    g = rng.poisson(D @ f * 10) / 10.0
    q = H.forward(f)
    grad = H.adjoint(1.0 - O.ratio(g, q))
    eps = 1e-6
    for j in range(0, geom.m, 3):
        e = np.zeros(geom.m)
        e[j] = eps
        fd = (O.poisson_nll(D @ (f + e), g) - O.poisson_nll(D @ (f - e), g)) / (2 * eps)
        assert abs(fd - grad[j]) <= 1e-6 * max(1.0, abs(grad[j]))


# --- planted mistakes: the pins above must catch plausible oracle bugs -----------

def _mutant_forward(geom, taps, f, kind):
    fr = f.reshape(geom.w, geom.alpha, geom.a)
    out = np.zeros((geom.xi, geom.gamma))
    for s in range(geom.w):
        xs, ys, vs = taps.of(s)
        for x, y, v in zip(xs, ys, vs):
            if kind == "transposed_shift":
                # wrong: field-stop row shifts the FPA column
                for r in range(geom.alpha):
                    for p in range(geom.a):
                        xx, yy = x + r, y + p
                        if xx < geom.gamma and yy < geom.xi:
                            out[yy, xx] += v * fr[s, r, p]
            elif kind == "flipped_psf":
                out[y:y + geom.alpha, x:x + geom.a] += v * fr[s, ::-1, ::-1]
            elif kind == "wrong_wavelength":
                out[y:y + geom.alpha, x:x + geom.a] += v * fr[(s + 1) % geom.w]
    return out.ravel()


@pytest.mark.parametrize("kind", ["transposed_shift", "flipped_psf", "wrong_wavelength"])
def test_planted_mistakes_are_caught_by_dense_pin(kind):
    geom = _geom(4, 3, 2, 10, 9)
    psf = _tiny_psf(geom, 5, 41)
    taps = O.merge_psf(geom, psf)
    f = synth.random_positive(geom.m, 12).astype(np.float64)
    D = O.dense_H(geom, psf)
    assert not np.allclose(_mutant_forward(geom, taps, f, kind), D @ f, rtol=1e-6)


# --- bfloat16 storage rounding ---------------------------------------------------

def test_round_bf16_matches_torch_conversion():
    """round_bf16 against PyTorch's float32 -> bfloat16 cast (round to nearest
    even) on random magnitudes, exact ties of both parities and values that
    are already bfloat16."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = (rng.uniform(0, 1, 4000) * 10.0 ** rng.integers(-30, 30, 4000)).astype(np.float32)
    # upper 16 bits below 0x7f80: finite, positive (exponent field < 255)
    ties = (rng.integers(1, 0x7F80, 2000).astype(np.uint32) << 16 | 0x8000).view(np.float32)
    exact = (rng.integers(1, 0x7F80, 500).astype(np.uint32) << 16).view(np.float32)
    for v in (x, ties, exact):
        want = torch.from_numpy(v.copy()).to(torch.bfloat16).to(torch.float32).numpy()
        assert np.array_equal(O.round_bf16(v).view(np.uint32), want.view(np.uint32))
    assert np.array_equal(O.round_bf16(exact), exact)


def test_round_bf16_ties_go_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (kept last bit even: down);
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6 (odd: up)
    v = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20], np.float32)
    assert O.round_bf16(v).tolist() == [1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7]


def test_em_step_stored_with_exact_store_is_em_step():
    geom = _geom(5, 4, 3, 14, 12)
    psf = _tiny_psf(geom, 6, 44)
    H = O.build_H(geom, psf)
    f = synth.random_positive(geom.m, 45).astype(np.float64)
    g = H.forward(synth.random_positive(geom.m, 46))
    assert np.array_equal(O.em_step_stored(H, g, f, lambda z: z), O.em_step(H, g, f))
    stored = O.em_step_stored(H, g, f, lambda z: O.round_bf16(z.astype(np.float32)))
    assert np.array_equal(stored, O.round_bf16(O.em_step(H, g, f).astype(np.float32)))


# --- the clip boundary reading (shifted nonzeros off the FPA are dropped) -------

CLIP_GEOM = (4, 3, 2, 9, 8)
# nonzeros spilling over every FPA edge, a duplicate, and one wholly off the FPA
CLIP_PSF = (np.array([0, 4, 9], np.int32),
            np.array([-2, 7, 3, 1, -1, 5, 5, 20, 6], np.int32),
            np.array([1, 6, 2, -2, -1, 0, 0, 3, 7], np.int32),
            np.array([0.5, 1.5, 1.0, 0.25, 0.7, 0.3, 0.2, 2.0, 0.9], np.float32))


def _clip_bruteforce_dense(geom, psf):
    """H by four nested loops over wavelengths, nonzeros and field-stop pixels,
    keeping a term only when its shifted pixel is on the FPA."""
    ptr, x, y, v = psf
    D = np.zeros((geom.n, geom.m))
    for s in range(geom.w):
        for k in range(int(ptr[s]), int(ptr[s + 1])):
            for r in range(geom.alpha):
                for p in range(geom.a):
                    X, Y = int(x[k]) + p, int(y[k]) + r
                    if 0 <= X < geom.gamma and 0 <= Y < geom.xi:
                        D[X + geom.gamma * Y, s * geom.ell + r * geom.a + p] += float(v[k])
    return D


def test_clip_reading_matches_bruteforce_and_reject_refuses_it():
    geom = _geom(*CLIP_GEOM)
    with pytest.raises(O.OutOfBounds):
        O.build_H(geom, CLIP_PSF)
    H = O.build_H(geom, CLIP_PSF, boundary="clip")
    D = _clip_bruteforce_dense(geom, CLIP_PSF)
    assert np.array_equal(H.as_csr().toarray(), D)
    # h = column sums: smaller at the voxels whose light partly leaves the FPA
    assert np.allclose(H.h(), D.sum(axis=0))
    assert len(np.unique(H.h()[:geom.ell])) > 1


def test_clip_reading_is_the_reject_reading_when_nothing_leaves():
    geom = _geom(4, 3, 2, 10, 9)
    psf = _tiny_psf(geom, 5, 43, dup=2)
    a = O.build_H(geom, psf).as_csr().toarray()
    b = O.build_H(geom, psf, boundary="clip").as_csr().toarray()
    assert np.array_equal(a, b)
    assert np.allclose(a, O.dense_H(geom, psf))


def test_clip_pointwise_evaluators_and_psf_grad():
    geom = _geom(*CLIP_GEOM)
    taps = O.merge_psf(geom, CLIP_PSF, "clip")
    H = O.BlockH(geom, taps)
    D = _clip_bruteforce_dense(geom, CLIP_PSF)
    f = synth.random_positive(geom.m, 61).astype(np.float64)
    u = synth.random_positive(geom.n, 62).astype(np.float64)
    xs, ys = np.meshgrid(np.arange(geom.gamma), np.arange(geom.xi))
    assert _rel(O.forward_at(geom, taps, f, xs.ravel(), ys.ravel()), D @ f) < 1e-14
    s, r, p = np.unravel_index(np.arange(geom.m), (geom.w, geom.alpha, geom.a))
    assert _rel(O.adjoint_at(geom, taps, u, s, p, r), D.T @ u) < 1e-14
    # d <u, H f> / d v_t against the derivative of the brute-force H
    grad = O.psf_value_grad(geom, taps, f, u)
    for t in range(taps.v.size):
        ptr = np.zeros(geom.w + 1, np.int32)
        ptr[int(taps.s[t]) + 1:] = 1
        Dt = _clip_bruteforce_dense(geom, (ptr, taps.x[t:t + 1], taps.y[t:t + 1],
                                           np.ones(1, np.float32)))
        assert abs(grad[t] - u @ (Dt @ f)) <= 1e-12 * max(1.0, abs(grad[t]))


def test_clip_em_invariants():
    """Under clipping h varies per voxel; EM still conserves the flux
    sum_j h_j f_j^(t+1) = sum of g over the support of H f^(t), and keeps f >= 0."""
    geom = _geom(*CLIP_GEOM)
    H = O.build_H(geom, CLIP_PSF, boundary="clip")
    g = synth.random_positive(geom.n, 63).astype(np.float64) * 50
    f = np.ones(geom.m)
    h = H.h()
    for _ in range(5):
        q = H.forward(f)
        f_next = O.em_step(H, g, f)
        assert np.all(f_next >= 0)
        assert abs(np.dot(h, f_next) - g[q > 0].sum()) <= 1e-9 * g.sum()
        f = f_next


# --- the wrap boundary reading (Eq. 7 taken literally: rows mod n) ---------------

# nonzeros whose shifted copies pass the right edge, the last row, and both
WRAP_PSF = (np.array([0, 4, 8], np.int32),
            np.array([7, 2, 8, 0, 5, 5, 6, 1], np.int32),
            np.array([1, 6, 7, 0, 5, 5, 2, 7], np.int32),
            np.array([0.5, 1.5, 1.0, 0.25, 0.7, 0.3, 2.0, 0.9], np.float32))


def _wrap_images(geom, psf):
    """The PSF plus, for each nonzero (x, y), its images at (x - gamma, y + 1),
    (x, y - xi) and (x - gamma, y + 1 - xi), wavelength by wavelength."""
    ptr, x, y, v = psf
    P, X, Y, V = [0], [], [], []
    for s in range(geom.w):
        lo, hi = int(ptr[s]), int(ptr[s + 1])
        for dx, dy in ((0, 0), (-geom.gamma, 1), (0, -geom.xi), (-geom.gamma, 1 - geom.xi)):
            X.append(x[lo:hi] + dx)
            Y.append(y[lo:hi] + dy)
            V.append(v[lo:hi])
        P.append(P[-1] + 4 * (hi - lo))
    return (np.array(P, np.int32), np.concatenate(X).astype(np.int32),
            np.concatenate(Y).astype(np.int32), np.concatenate(V).astype(np.float32))


def test_wrap_reading_is_the_literal_circulant_of_eq7():
    """Under the wrap reading H equals the dense C_s E of Eqs. 5-7 (columns of
    C_s are c_s rolled), for a PSF whose shifted copies pass every edge; the
    reject rule refuses that PSF, and wrap refuses a nonzero off the FPA."""
    geom = _geom(*CLIP_GEOM)
    with pytest.raises(O.OutOfBounds):
        O.build_H(geom, WRAP_PSF)
    H = O.build_H(geom, WRAP_PSF, boundary="wrap")
    np.testing.assert_allclose(H.as_csr().toarray(), O.dense_H(geom, WRAP_PSF), rtol=1e-15, atol=0)
    ptr, x, y, v = WRAP_PSF
    with pytest.raises(O.OutOfBounds):
        O.build_H(geom, (ptr, np.where(np.arange(len(x)) == 3, 9, x).astype(np.int32), y, v),
                  boundary="wrap")
    # nothing is lost: h_j is the wavelength's total PSF value for every voxel
    h = H.h().reshape(geom.w, geom.ell)
    for s in range(geom.w):
        assert np.allclose(h[s], float(np.sum(v[ptr[s]:ptr[s + 1]], dtype=np.float64)), rtol=1e-15)


def test_wrap_reading_matches_the_fft_form():
    """The FFT form (Eqs. 13, 17) is circular by construction: it equals the
    wrap reading's sparse projectors."""
    geom = _geom(*CLIP_GEOM)
    H = O.build_H(geom, WRAP_PSF, boundary="wrap")
    f = synth.random_positive(geom.m, 64).astype(np.float64)
    u = synth.random_positive(geom.n, 65).astype(np.float64)
    assert _rel(O.fft_forward(geom, WRAP_PSF, f, boundary="wrap"), H.forward(f)) < 1e-13
    assert _rel(O.fft_adjoint(geom, WRAP_PSF, u, boundary="wrap"), H.adjoint(u)) < 1e-13
    with pytest.raises(ValueError):
        O.fft_forward(geom, WRAP_PSF, f, boundary="clip")


def test_wrap_pointwise_evaluators_and_psf_grad():
    geom = _geom(*CLIP_GEOM)
    taps = O.merge_psf(geom, WRAP_PSF, "wrap")
    D = O.dense_H(geom, WRAP_PSF)
    f = synth.random_positive(geom.m, 66).astype(np.float64)
    u = synth.random_positive(geom.n, 67).astype(np.float64)
    xs, ys = np.meshgrid(np.arange(geom.gamma), np.arange(geom.xi))
    assert _rel(O.forward_at(geom, taps, f, xs.ravel(), ys.ravel()), D @ f) < 1e-14
    s, r, p = np.unravel_index(np.arange(geom.m), (geom.w, geom.alpha, geom.a))
    assert _rel(O.adjoint_at(geom, taps, u, s, p, r), D.T @ u) < 1e-14
    grad = O.psf_value_grad(geom, taps, f, u)
    for t in range(taps.v.size):
        ptr = np.zeros(geom.w + 1, np.int32)
        ptr[int(taps.s[t]) + 1:] = 1
        Dt = O.dense_H(geom, (ptr, taps.x[t:t + 1], taps.y[t:t + 1], np.ones(1, np.float32)))
        assert abs(grad[t] - u @ (Dt @ f)) <= 1e-12 * max(1.0, abs(grad[t]))


def test_wrap_is_the_clip_reading_of_the_psf_and_its_images():
    """Each shifted copy (x + p, y + r) of a nonzero on the FPA re-enters at
    exactly one of (x + p - gamma, y + r + 1), (x + p, y + r - xi) and
    (x + p - gamma, y + r + 1 - xi) when it leaves, so the wrap reading is the
    clip reading of the PSF together with those three images."""
    for dims, psf in ((CLIP_GEOM, WRAP_PSF),
                      ((3, 4, 3, 7, 6), synth.random_sparse_psf(3, 6, 6, 5, 91, duplicates=2)),
                      ((5, 2, 2, 6, 9), synth.random_sparse_psf(2, 7, 5, 8, 92))):
        geom = _geom(*dims)
        a = O.build_H(geom, psf, boundary="wrap").as_csr().toarray()
        b = O.build_H(geom, _wrap_images(geom, psf), boundary="clip").as_csr().toarray()
        np.testing.assert_allclose(a, b, rtol=1e-15, atol=0)
        np.testing.assert_allclose(a, O.dense_H(geom, psf), rtol=1e-15, atol=0)


def test_wrap_em_invariants():
    """With nothing lost, EM under the wrap reading conserves sum_j h_j f_j
    (= the sum of g over the support of H f) and keeps f >= 0."""
    geom = _geom(*CLIP_GEOM)
    H = O.build_H(geom, WRAP_PSF, boundary="wrap")
    g = synth.random_positive(geom.n, 68).astype(np.float64) * 50
    f = np.ones(geom.m)
    h = H.h()
    for _ in range(5):
        q = H.forward(f)
        f_next = O.em_step(H, g, f)
        assert np.all(f_next >= 0)
        assert abs(np.dot(h, f_next) - g[q > 0].sum()) <= 1e-9 * g.sum()
        f = f_next


# --- the shifted-sum projectors (large workloads) -----------------------------------

@pytest.mark.parametrize("boundary,shift", [("reject", (0, 0)), ("clip", (-5, 4)), ("clip", (9, -7))])
def test_shifted_sum_projectors_equal_the_sparse_and_dense_H(boundary, shift):
    """forward_shifts / adjoint_shifts (pasting the field stop per tap) against
    the sparse BlockH (indices of Sec. 2's shifted columns) and, under the
    reject reading, the dense C_s E of Eqs. 5-7; random PSFs with duplicates."""
    for seed, dims in ((3, (4, 3, 2, 10, 9)), (4, (5, 6, 3, 17, 13)), (5, (7, 2, 4, 12, 20))):
        geom = _geom(*dims)
        ptr, x, y, v = _tiny_psf(geom, 5, seed, dup=2)
        psf = (ptr, (x + shift[0]).astype(np.int32), (y + shift[1]).astype(np.int32), v)
        taps = O.merge_psf(geom, psf, boundary)
        H = O.BlockH(geom, taps)
        f = synth.random_positive(geom.m, seed + 10).astype(np.float64)
        u = synth.random_positive(geom.n, seed + 20).astype(np.float64)
        np.testing.assert_allclose(O.forward_shifts(geom, taps, f), H.forward(f), rtol=1e-14, atol=0)
        np.testing.assert_allclose(O.adjoint_shifts(geom, taps, u), H.adjoint(u), rtol=1e-14, atol=0)
        np.testing.assert_allclose(O.h_shifts(geom, taps), H.h(), rtol=1e-14, atol=0)
        if boundary == "reject":
            D = O.dense_H(geom, psf)
            np.testing.assert_allclose(O.forward_shifts(geom, taps, f), D @ f, rtol=1e-13, atol=1e-13)


def test_shifted_sum_em_equals_sparse_em():
    geom, H, g, _ = _tiny_problem(noisy=True)
    taps = H.taps
    f1, h1 = O.mlem(H, g, 7)
    f2, h2 = O.mlem_shifts(geom, taps, g, 7)
    np.testing.assert_allclose(f2, f1, rtol=1e-12, atol=0)
    for a, b in zip(h1, h2):
        for key in a:
            assert b[key] == pytest.approx(a[key], rel=1e-12)


@pytest.mark.parametrize("kind", ["transposed_shift", "flipped_psf", "wrong_wavelength"])
def test_planted_mistakes_fail_the_shifted_sum_pin(kind):
    geom = _geom(4, 3, 2, 10, 9)
    psf = _tiny_psf(geom, 5, 41)
    taps = O.merge_psf(geom, psf)
    f = synth.random_positive(geom.m, 12).astype(np.float64)
    assert not np.allclose(_mutant_forward(geom, taps, f, kind), O.forward_shifts(geom, taps, f),
                           rtol=1e-6)


def test_unrolled_nll_shifts_equals_unrolled_nll():
    geom, H, g, _ = _tiny_problem(noisy=True)
    f0 = synth.random_positive(geom.m, 9).astype(np.float64)
    for k in (0, 1, 4):
        assert O.unrolled_nll_shifts(geom, H.taps, g, f0, k) == pytest.approx(
            O.unrolled_nll(geom, H.taps, g, f0, k), rel=1e-12)
