"""Pins for the oracle's other solvers on the projector pair (SART and
SMART, the simultaneous forms of the ART and MART the paper lists in Sec. 2):
closed forms worked by hand, brute-force loops over a dense H, fixed points
at consistent data, and the monotone objectives their convergence theory
gives (SART: the row-weighted residual; SMART: KL(H f, g))."""
import math

import numpy as np
import pytest

import oracle as O
import synth


def _one_by_one(v):
    """a = alpha = w = gamma = xi = 1: H is the 1 x 1 matrix [v]."""
    geom = O.Geometry(1, 1, 1, 1, 1)
    psf = (np.array([0, 1], np.int32), np.array([0], np.int32), np.array([0], np.int32),
           np.array([v], np.float32))
    return O.build_H(geom, psf)


def test_scalar_closed_forms():
    # r = h = v: SART gives (1 - lam) f + lam g / v, SMART f (g / (v f))^lam
    H = _one_by_one(0.5)
    g, f = np.array([3.0]), np.array([2.0])
    assert O.sart_step(H, g, f, 1.0)[0] == pytest.approx(6.0, rel=1e-15)
    assert O.sart_step(H, g, f, 0.5)[0] == pytest.approx(4.0, rel=1e-15)
    assert O.smart_step(H, g, f, 1.0)[0] == pytest.approx(6.0, rel=1e-14)
    assert O.smart_step(H, g, f, 0.5)[0] == pytest.approx(2.0 * math.sqrt(3.0), rel=1e-14)
    # SART clips at zero: g = 0 with lam = 1.5 would give -1
    assert O.sart_step(H, np.array([0.0]), f, 1.5)[0] == 0.0


def test_hand_worked_two_voxel_step():
    """a = 2, alpha = w = 1 on a 3 x 1 FPA, nonzeros 1 at x = 0 and 2 at x = 1:
    H = [[1, 0], [2, 1], [0, 2]], r = (1, 3, 2), h = (3, 3). From f = (1, 1)
    with g = (2, 3, 4): H f = (1, 3, 2); SART's u = (1, 0, 1), H^T u = (1, 2),
    f' = (4/3, 5/3); SMART's u = (ln 2, 0, ln 2), H^T u = (ln 2, 2 ln 2),
    f' = (2^(1/3), 2^(2/3))."""
    geom = O.Geometry(2, 1, 1, 3, 1)
    psf = (np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([0, 0], np.int32),
           np.array([1.0, 2.0], np.float32))
    H = O.build_H(geom, psf)
    assert np.array_equal(H.as_csr().toarray(), [[1, 0], [2, 1], [0, 2]])
    g, f = np.array([2.0, 3.0, 4.0]), np.ones(2)
    np.testing.assert_allclose(O.sart_step(H, g, f), [4 / 3, 5 / 3], rtol=1e-15)
    np.testing.assert_allclose(O.smart_step(H, g, f), [2 ** (1 / 3), 2 ** (2 / 3)], rtol=1e-14)


def _dense_step(D, g, f, lam, kind):
    """One step by explicit loops over the dense matrix D (n x m)."""
    n, m = D.shape
    r = [sum(D[i, j] for j in range(m)) for i in range(n)]
    h = [sum(D[i, j] for i in range(n)) for j in range(m)]
    q = [sum(D[i, j] * f[j] for j in range(m)) for i in range(n)]
    out = np.empty(m)
    for j in range(m):
        z = 0.0
        for i in range(n):
            if D[i, j] == 0:
                continue
            if kind == "sart" and r[i] > 0:
                z += D[i, j] * (g[i] - q[i]) / r[i]
            elif kind == "smart" and g[i] > 0 and q[i] > 0:
                z += D[i, j] * math.log(g[i] / q[i])
        step = z / h[j] if h[j] > 0 else 0.0
        out[j] = max(f[j] + lam * step, 0.0) if kind == "sart" else f[j] * math.exp(lam * step)
    return out


@pytest.mark.parametrize("kind", ["sart", "smart"])
@pytest.mark.parametrize("lam", [1.0, 0.6])
def test_step_matches_bruteforce_loops(kind, lam):
    geom = O.Geometry(3, 2, 2, 7, 6)
    psf = synth.random_sparse_psf(2, 4, 4, 4, 77, duplicates=1)
    H = O.build_H(geom, psf)
    D = O.dense_H(geom, psf)
    f = synth.random_positive(geom.m, 78).astype(np.float64)
    g = synth.random_positive(geom.n, 79).astype(np.float64) * 5
    g[::5] = 0.0                                      # zero counts on some pixels
    step = O.sart_step if kind == "sart" else O.smart_step
    np.testing.assert_allclose(step(H, g, f, lam), _dense_step(D, g, f, lam, kind),
                               rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("kind", ["sart", "smart"])
def test_consistent_data_is_a_fixed_point(kind):
    wl = synth.TINY
    geom = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    H = O.build_H(geom, synth.make_psf(wl))
    f_true = synth.random_positive(geom.m, 80).astype(np.float64) + 0.1
    g = H.forward(f_true)
    step = O.sart_step if kind == "sart" else O.smart_step
    np.testing.assert_allclose(step(H, g, f_true, 1.0), f_true, rtol=1e-12)


def _problem(seed):
    wl = synth.TINY
    geom = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    H = O.build_H(geom, synth.make_psf(wl))
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), 200.0, seed)
    return H, np.asarray(g, np.float64)


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.9])
def test_sart_decreases_the_row_weighted_residual(lam):
    """SART is a projected gradient step on sum_i (g_i - q_i)^2 / r_i in the
    h-weighted metric, whose Lipschitz constant is at most 1, so for
    0 < lam < 2 that objective never rises (noisy data, clipping active)."""
    H, g = _problem(81)
    r = O.row_sums(H)
    on = r > 0
    obj = lambda f: float(np.sum((g[on] - H.forward(f)[on]) ** 2 / r[on]))
    f = np.ones(H.geom.m)
    prev = obj(f)
    for _ in range(15):
        f = O.sart_step(H, g, f, lam)
        cur = obj(f)
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    assert f.min() >= 0.0


def test_smart_decreases_kl_of_the_model_from_the_data():
    """SMART decreases KL(H f, g) = sum q log(q / g) + g - q when g > 0 on
    the support of H."""
    H, g = _problem(82)
    g = g + 1.0                                       # positive counts everywhere
    r = O.row_sums(H)
    on = r > 0

    def kl(f):
        q = H.forward(f)[on]
        return float(np.sum(q * np.log(q / g[on]) + g[on] - q))

    f = np.ones(H.geom.m)
    prev = kl(f)
    for _ in range(15):
        f = O.smart_step(H, g, f, 1.0)
        cur = kl(f)
        assert cur <= prev * (1 + 1e-12)
        prev = cur


def test_solve_runs_the_steps_and_records_statistics():
    H, g = _problem(83)
    for kind in ("em", "sart", "smart"):
        f, hist = O.solve(H, g, 3, kind, 0.8)
        ref = np.ones(H.geom.m)
        for _ in range(3):
            ref = {"em": lambda x: O.em_step(H, g, x),
                   "sart": lambda x: O.sart_step(H, g, x, 0.8),
                   "smart": lambda x: O.smart_step(H, g, x, 0.8)}[kind](ref)
        np.testing.assert_array_equal(f, ref)
        assert len(hist) == 4 and hist[-1] == O.stats(H.forward(f), g)
