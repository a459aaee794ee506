"""Plain FP64 CPU oracle for shift-invariant CTIS EM reconstruction.

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The GPU product path (the C-ABI library and its Python binding) never
imports, links or calls it, and shares no code with it.

It follows White, Bell and Haygood, "Accelerating computed tomographic imaging
spectrometer reconstruction using a parallel algorithm exploiting spatial
shift-invariance":

* Eq. 1: the imaging model ``g = H f``.
* Sec. 2: one calibration image per wavelength (point source at field-stop pixel
  (0,0)) vectorised into a column of H; every other column of that wavelength is
  the same image shifted by the field-stop offset (shift-invariance).
* Eq. 2: the EM update ``f <- (f / h) * H^T (g / H f)`` with ``h_j = sum_i H_ij``.
* Eqs. 3-7: ``H = (H_1 ... H_w)`` and ``H_i = C_i E`` with circulant ``C_i`` and
  the 0/1 embedding ``E`` built from ``Q = [I_a; 0]`` (used by :func:`dense_H`).
* Sec. 3 index map ``i = j - s l + (gamma - a) floor((j - s l)/a) + s n``
  (:func:`index_map`).
* Eq. 13 (forward) and Eq. 17 (back projection) in their FFT form
  (:func:`fft_forward`, :func:`fft_adjoint`).
* The bfloat16 storage form (datacube and PSF values kept in bfloat16, sums in
  wider precision) is not in the paper; :func:`round_bf16` states the storage
  rounding and :func:`em_step_stored` applies it to an EM step.
* Sec. 2 names ART and MART among the usual solvers without defining them;
  :func:`sart_step` and :func:`smart_step` are their simultaneous forms from
  the literature the paper cites (SART, SMART), on the same projector pair.

Everything is float64. Inputs given as float32 (datacube, PSF values, counts)
are promoted exactly. Readings of points the paper leaves open:

* vectorisation: ``i = x + gamma*y`` on the FPA and ``j = s*a*alpha + r*a + p``
  in the datacube (the index map pairs the fast FPA axis with the fast
  field-stop axis);
* boundary: every shifted nonzero must stay on the FPA (checked by
  :func:`check_bounds`); then the circulant form of Eq. 7 and the 2-D shift agree.
  The optional clip reading (``boundary="clip"``) keeps the physical 2-D shift
  and drops the shifted nonzeros that leave the FPA (the light is lost), so
  ``h`` then varies from voxel to voxel; the wrap reading (``boundary="wrap"``)
  is Eq. 7 taken literally: row ``(x + p + gamma (y + r)) mod n``, so a
  shifted nonzero past the right edge re-enters at the left of the next FPA
  row and one past the last row re-enters at the top;
* ``u_i = 0`` where ``(Hf)_i = 0`` and ``f_j = 0`` where ``h_j = 0`` (Eq. 2 leaves
  both divisions undefined);
* duplicate PSF entries at one FPA position add up (H is a sum of responses);
* ``k`` iterations means ``k`` EM updates from the initial guess.

The shifted-sum projectors (:func:`forward_shifts`, :func:`adjoint_shifts`,
:func:`mlem_shifts`, :func:`unrolled_nll_shifts`) apply the same H without
building it (Sec. 2's columns pasted tap by tap), for the workloads whose
sparse H would not fit in host memory; they are pinned to the sparse and
dense forms.

Pins (tests/test_oracle_*.py): every function here is checked against something
other than itself - a dense H assembled literally from Eqs. 5-7, the FFT form of
Eqs. 13/17 through numpy's FFT, the adjoint identity, 2-D convolution from SciPy
for w = 1, brute-force Python loops on tiny inputs, hand-worked values in
tests/golden/, the EM invariants (nonnegativity, flux, monotone likelihood),
finite differences of a dense H, and PyTorch's float32 -> bfloat16 conversion
for :func:`round_bf16`. The wrap reading is pinned to the literal circulant of
Eq. 7 (:func:`dense_H`) and to the FFT form; the solvers
(tests/test_oracle_solvers.py) to hand-worked steps, brute-force loops over a
dense H, fixed points at consistent data and their monotone objectives.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass(frozen=True)
class Geometry:
    a: int        # field-stop columns (fast axis)
    alpha: int    # field-stop rows
    w: int        # wavelengths
    gamma: int    # FPA columns (fast axis)
    xi: int       # FPA rows

    @property
    def ell(self) -> int:
        return self.a * self.alpha

    @property
    def m(self) -> int:
        return self.a * self.alpha * self.w

    @property
    def n(self) -> int:
        return self.gamma * self.xi


@dataclasses.dataclass
class Taps:
    """Merged PSF nonzeros, sorted by (s, y, x); values in float64."""

    s: np.ndarray
    x: np.ndarray
    y: np.ndarray
    v: np.ndarray
    ptr: np.ndarray   # [w+1] start of each wavelength's taps
    wrap: bool = False   # boundary "wrap": shifted positions taken mod n (Eq. 7)

    def of(self, s: int):
        lo, hi = int(self.ptr[s]), int(self.ptr[s + 1])
        return self.x[lo:hi], self.y[lo:hi], self.v[lo:hi]


class OutOfBounds(ValueError):
    pass


def check_bounds(geom: Geometry, psf, boundary: str = "reject") -> None:
    """Reject a PSF whose shifted copies would leave the FPA (``boundary=
    "reject"``); with ``boundary="clip"`` such nonzeros are allowed and the
    projectors drop the shifted positions off the FPA; with ``boundary=
    "wrap"`` every nonzero must lie on the FPA (it is an entry of the length-n
    first column ``c_s`` of Eq. 7) and its shifted copies wrap mod n.

    Column j = (p, r, s) of H holds the calibration image of wavelength s shifted
    by (p, r) (Sec. 2). Every shifted nonzero must satisfy ``0 <= x + p < gamma``
    and ``0 <= y + r < xi`` for all p < a, r < alpha; otherwise the 1-D circulant
    of Eq. 7 would wrap it into another FPA row while a physical shift would
    lose it, and the two readings differ.
    """
    ptr, x, y, _ = psf
    if len(ptr) != geom.w + 1:
        raise ValueError("psf_ptr must have w+1 entries")
    if boundary not in ("reject", "clip", "wrap"):
        raise ValueError(boundary)
    if boundary == "clip":
        return
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    if boundary == "wrap":
        if x.size and (x.min() < 0 or y.min() < 0 or x.max() >= geom.gamma or
                       y.max() >= geom.xi):
            raise OutOfBounds("PSF nonzero off the FPA (c_s has n entries)")
        return
    if x.size and (x.min() < 0 or y.min() < 0 or
                   x.max() + geom.a - 1 >= geom.gamma or
                   y.max() + geom.alpha - 1 >= geom.xi):
        raise OutOfBounds("PSF nonzero shifted off the FPA")


def merge_psf(geom: Geometry, psf, boundary: str = "reject") -> Taps:
    """Sort each wavelength's nonzeros by (y, x) and add up duplicates (float64)."""
    check_bounds(geom, psf, boundary)
    ptr, x, y, v = psf
    ptr = np.asarray(ptr, dtype=np.int64)
    S, X, Y, V, P = [], [], [], [], [0]
    for s in range(geom.w):
        lo, hi = ptr[s], ptr[s + 1]
        xs = np.asarray(x[lo:hi], dtype=np.int64)
        ys = np.asarray(y[lo:hi], dtype=np.int64)
        vs = np.asarray(v[lo:hi], dtype=np.float64)
        yx = np.stack([ys, xs], axis=1).reshape(-1, 2)
        uniq, inv = np.unique(yx, axis=0, return_inverse=True)   # sorted by (y, x)
        acc = np.zeros(len(uniq))
        np.add.at(acc, np.asarray(inv).ravel(), vs)
        S.append(np.full(len(uniq), s, dtype=np.int64))
        X.append(uniq[:, 1])
        Y.append(uniq[:, 0])
        V.append(acc)
        P.append(P[-1] + len(uniq))
    cat = lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt)
    return Taps(cat(S, np.int64), cat(X, np.int64), cat(Y, np.int64),
                cat(V, np.float64), np.asarray(P, dtype=np.int64), boundary == "wrap")


def index_map(geom: Geometry) -> np.ndarray:
    """Zero-based position in ``v = (I_w kron E) f`` of each datacube entry j.

    Sec. 3, Eq. 11: ``s = floor(j / l)`` and
    ``i = j - s l + (gamma - a) floor((j - s l) / a) + s n``.
    """
    j = np.arange(geom.m, dtype=np.int64)
    s = j // geom.ell
    q = j - s * geom.ell
    return q + (geom.gamma - geom.a) * (q // geom.a) + s * geom.n


class BlockH:
    """The system matrix kept as its wavelength blocks ``H = (H_1 ... H_w)`` (Eq. 3).

    Each block ``H_s`` (n x l, CSR, float64) is built straight from Sec. 2:
    column ``r*a + p`` is the calibration image of wavelength s shifted by
    (p, r), i.e. nonzero ``(x_k, y_k, v_k)`` lands in row
    ``(x_k + p) + gamma*(y_k + r)``. A shifted nonzero off the FPA (possible
    only under the clip reading) is dropped; under the wrap reading the row is
    taken mod n instead (Eq. 7's circulant).
    """

    def __init__(self, geom: Geometry, taps: Taps, wavelengths=None):
        self.geom = geom
        self.taps = taps
        self.wavelengths = list(range(geom.w)) if wavelengths is None else list(wavelengths)
        a, al, ga = geom.a, geom.alpha, geom.gamma
        P, R = np.meshgrid(np.arange(a), np.arange(al))     # [alpha][a]
        col = (R * a + P).ravel()
        shift = (P + ga * R).ravel()
        self.blocks = {}
        Pf, Rf = P.ravel(), R.ravel()
        for s in self.wavelengths:
            xs, ys, vs = taps.of(s)
            px = xs[:, None] + Pf[None, :]
            py = ys[:, None] + Rf[None, :]
            if taps.wrap:
                on = np.ones(px.shape, dtype=bool)
                rows = ((px + ga * py) % geom.n).ravel()
            else:
                on = (px >= 0) & (px < ga) & (py >= 0) & (py < geom.xi)
                rows = (px + ga * py)[on]
            cols = np.broadcast_to(col[None, :], on.shape)[on]
            vals = np.broadcast_to(vs[:, None], on.shape)[on]
            self.blocks[s] = sp.csr_matrix((vals, (rows, cols)), shape=(geom.n, geom.ell))

    def forward(self, f: np.ndarray) -> np.ndarray:
        """``H f = sum_s H_s f_s`` (Eq. 1 with the partition of Eq. 3)."""
        f = np.asarray(f, dtype=np.float64).reshape(self.geom.w, -1)
        out = np.zeros(self.geom.n)
        for s in self.wavelengths:
            out += self.blocks[s] @ f[s]
        return out

    def adjoint(self, r: np.ndarray) -> np.ndarray:
        """``H^T r`` stacked over the wavelength blocks."""
        r = np.asarray(r, dtype=np.float64).ravel()
        out = np.zeros((self.geom.w, self.geom.ell))
        for s in self.wavelengths:
            out[s] = self.blocks[s].T @ r
        return out.ravel()

    def h(self) -> np.ndarray:
        """``h_j = sum_i H_ij`` (the normaliser of Eq. 2)."""
        out = np.zeros((self.geom.w, self.geom.ell))
        for s in self.wavelengths:
            out[s] = np.asarray(self.blocks[s].sum(axis=0)).ravel()
        return out.ravel()

    def as_csr(self) -> sp.csr_matrix:
        return sp.hstack([self.blocks[s] for s in range(self.geom.w)]).tocsr()


def build_H(geom: Geometry, psf, wavelengths=None, boundary: str = "reject") -> BlockH:
    return BlockH(geom, merge_psf(geom, psf, boundary), wavelengths)


def ratio(g: np.ndarray, q: np.ndarray) -> np.ndarray:
    """``u = g / q`` (Eq. 2), with ``u_i = 0`` where ``q_i = 0``."""
    g = np.asarray(g, dtype=np.float64).ravel()
    q = np.asarray(q, dtype=np.float64).ravel()
    u = np.zeros_like(q)
    nz = q != 0
    u[nz] = g[nz] / q[nz]
    return u


def em_update(f: np.ndarray, z: np.ndarray, h: np.ndarray) -> np.ndarray:
    """``f * z / h`` (Eq. 2), with ``f_j = 0`` where ``h_j = 0``."""
    f = np.asarray(f, dtype=np.float64).ravel()
    out = np.zeros_like(f)
    nz = h != 0
    out[nz] = f[nz] * z[nz] / h[nz]
    return out


def stats(q: np.ndarray, g: np.ndarray) -> dict:
    """Global sums of one forward pass, in float64, over the support of H f.

    Reading of Eq. 2's likelihood (Shepp-Vardi EM): the Poisson log-likelihood
    up to the constant ``-sum log g!`` is ``sum_i g_i log q_i - q_i``. Pixels with
    ``q_i = 0`` are left out of every sum here (they add ``-q_i = 0`` when
    ``g_i = 0``; a pixel with ``g_i > 0 = q_i`` would make the full likelihood
    ``-inf``, which no measurement generated by H can produce).

    ``resid2 = sum (g_i - q_i)^2`` over the same support is a diagnostic, not
    a term of Eq. 2: off the support ``q_i = 0`` for every iterate, so the
    residual there is the data's own ``sum g_i^2``, a constant that says
    nothing about f; the statistic keeps the part that depends on f. Pinned
    by a hand-worked example that has a ``g > 0`` pixel off the support.
    """
    q = np.asarray(q, dtype=np.float64).ravel()
    g = np.asarray(g, dtype=np.float64).ravel()
    pos = q > 0
    return {
        "flux_hf": float(q[pos].sum()),
        "flux_g_covered": float(g[pos].sum()),
        "loglik": float(np.sum(g[pos] * np.log(q[pos])) - np.sum(q[pos])),
        "resid2": float(np.sum((g[pos] - q[pos]) ** 2)),
    }


def mlem(H: BlockH, g: np.ndarray, k: int, f0: np.ndarray | None = None,
         init: str = "ones"):
    """k EM updates (Eq. 2), following the loop of Algorithm 1.

    Starts from ``f0`` if given, else all ones (``init='ones'``) or ``H^T g``
    (``init='htg'``). Returns ``(f, history)`` where ``history[t]`` holds
    :func:`stats` of ``H f^(t)`` for t = 0..k (the last one for the final f).
    """
    g64 = np.asarray(g, dtype=np.float64).ravel()
    if f0 is not None:
        f = np.asarray(f0, dtype=np.float64).ravel().copy()
    elif init == "ones":
        f = np.ones(H.geom.m)
    elif init == "htg":
        f = H.adjoint(g64)
    else:
        raise ValueError(init)
    h = H.h()
    history = []
    for _ in range(k):
        q = H.forward(f)
        history.append(stats(q, g64))
        z = H.adjoint(ratio(g64, q))
        f = em_update(f, z, h)
    history.append(stats(H.forward(f), g64))
    return f, history


def em_step(H: BlockH, g: np.ndarray, f: np.ndarray) -> np.ndarray:
    """One EM update of Eq. 2 from the given iterate."""
    g64 = np.asarray(g, dtype=np.float64).ravel()
    q = H.forward(f)
    return em_update(f, H.adjoint(ratio(g64, q)), H.h())


# --- other solvers on the same projector pair (Sec. 2 names ART and MART) -------
#
# The paper lists ART and MART among the usual CTIS solvers and calls its
# projector scheme solver agnostic, without defining them. The oracle takes
# their simultaneous (whole-image) forms from the literature the paper cites
# for them: SART (Andersen and Kak's simultaneous algebraic reconstruction
# technique) and SMART (Byrne's simultaneous multiplicative ART). Both use
# the row sums ``r = H 1`` and column sums ``h = H^T 1`` and a relaxation
# ``lam``. Readings: a pixel with ``r_i = 0`` (no footprint) adds nothing;
# under SMART a pixel with ``g_i = 0`` or ``(H f)_i = 0`` has no logarithm
# and adds nothing; a voxel with ``h_j = 0`` (seen by no pixel) keeps its
# value; SART's iterate is clipped at 0 after every update (f stays a
# radiance).

def row_sums(H: BlockH) -> np.ndarray:
    """``r_i = sum_j H_ij``."""
    return H.forward(np.ones(H.geom.m))


def sart_step(H: BlockH, g: np.ndarray, f: np.ndarray, lam: float = 1.0) -> np.ndarray:
    """``f + lam * (H^T ((g - H f) / r)) / h``, then clipped at 0."""
    g = np.asarray(g, dtype=np.float64).ravel()
    f = np.asarray(f, dtype=np.float64).ravel()
    r, h = row_sums(H), H.h()
    q = H.forward(f)
    u = np.zeros_like(q)
    on = r > 0
    u[on] = (g[on] - q[on]) / r[on]
    z = H.adjoint(u)
    step = np.zeros_like(f)
    seen = h > 0
    step[seen] = z[seen] / h[seen]
    return np.maximum(f + lam * step, 0.0)


def smart_step(H: BlockH, g: np.ndarray, f: np.ndarray, lam: float = 1.0) -> np.ndarray:
    """``f * exp(lam * (H^T log(g / H f)) / h)``."""
    g = np.asarray(g, dtype=np.float64).ravel()
    f = np.asarray(f, dtype=np.float64).ravel()
    h = H.h()
    q = H.forward(f)
    u = np.zeros_like(q)
    on = (g > 0) & (q > 0)
    u[on] = np.log(g[on] / q[on])
    z = H.adjoint(u)
    step = np.zeros_like(f)
    seen = h > 0
    step[seen] = z[seen] / h[seen]
    return f * np.exp(lam * step)


def solve(H: BlockH, g: np.ndarray, k: int, solver: str = "em", lam: float = 1.0,
          f0: np.ndarray | None = None):
    """k updates of ``solver`` ('em', 'sart' or 'smart') from ``f0`` or ones;
    returns ``(f, history)`` with :func:`stats` of ``H f^(t)``, t = 0..k."""
    step = {"em": lambda f: em_step(H, g, f), "sart": lambda f: sart_step(H, g, f, lam),
            "smart": lambda f: smart_step(H, g, f, lam)}[solver]
    g64 = np.asarray(g, dtype=np.float64).ravel()
    f = np.ones(H.geom.m) if f0 is None else np.asarray(f0, dtype=np.float64).ravel().copy()
    history = []
    for _ in range(k):
        history.append(stats(H.forward(f), g64))
        f = step(f)
    history.append(stats(H.forward(f), g64))
    return f, history


# --- pointwise evaluation for full-size parity on sampled outputs -------------

def forward_at(geom: Geometry, taps: Taps, f: np.ndarray, xs, ys) -> np.ndarray:
    """``(H f)`` at FPA pixels (xs, ys): sum over every tap of every wavelength of
    the datacube value that lands there (zero where the field-stop index is out
    of range)."""
    f = np.asarray(f, dtype=np.float64).reshape(geom.w, geom.alpha, geom.a)
    xs = np.asarray(xs, dtype=np.int64)
    ys = np.asarray(ys, dtype=np.int64)
    out = np.zeros(xs.size)
    for s in range(geom.w):
        tx, ty, tv = taps.of(s)
        if taps.wrap:   # the one offset d = p + gamma r with i = tap + d (mod n)
            d = (xs[:, None] + geom.gamma * ys[:, None] - tx[None, :] - geom.gamma * ty[None, :]) % geom.n
            p, r = d % geom.gamma, d // geom.gamma
        else:
            p = xs[:, None] - tx[None, :]
            r = ys[:, None] - ty[None, :]
        ok = (p >= 0) & (p < geom.a) & (r >= 0) & (r < geom.alpha)
        vals = np.where(ok, f[s][np.clip(r, 0, geom.alpha - 1), np.clip(p, 0, geom.a - 1)], 0.0)
        out += vals @ tv
    return out


def adjoint_at(geom: Geometry, taps: Taps, u: np.ndarray, s_idx, ps, rs) -> np.ndarray:
    """``(H^T u)`` at voxels (p, r, s): the calibration image of wavelength s
    shifted by (p, r), dotted with u."""
    u = np.asarray(u, dtype=np.float64).reshape(geom.xi, geom.gamma)
    out = np.zeros(len(s_idx))
    for t, (s, p, r) in enumerate(zip(s_idx, ps, rs)):
        tx, ty, tv = taps.of(int(s))
        x, y = tx + p, ty + r
        if taps.wrap:
            out[t] = np.dot(u.ravel()[(x + geom.gamma * y) % geom.n], tv)
            continue
        on = (x >= 0) & (x < geom.gamma) & (y >= 0) & (y < geom.xi)   # off the FPA: dropped
        out[t] = np.dot(u[y[on], x[on]], tv[on])
    return out


# --- whole projections as shifted sums (for problems too large for BlockH) ---

def _paste(geom: Geometry, x: int, y: int):
    """FPA rows/columns that the field stop shifted by tap (x, y) covers, and
    the matching field-stop rows/columns (the parts off the FPA dropped, as
    the clip reading does; under the reject reading nothing is dropped)."""
    x0, x1 = max(x, 0), min(x + geom.a, geom.gamma)
    y0, y1 = max(y, 0), min(y + geom.alpha, geom.xi)
    if x0 >= x1 or y0 >= y1:   # the shifted field stop misses the FPA
        return None
    return (slice(y0, y1), slice(x0, x1)), (slice(y0 - y, y1 - y), slice(x0 - x, x1 - x))


def forward_shifts(geom: Geometry, taps: Taps, f: np.ndarray) -> np.ndarray:
    """``H f`` (Eq. 1) straight from Sec. 2's columns: every tap (x, y, v) of
    wavelength s adds v times the field-stop image f_s pasted at (x, y). The
    same operator as :class:`BlockH` without building the matrix (memory O(m
    + n)), for the large workloads; the wrap reading is not supported."""
    if taps.wrap:
        raise ValueError("forward_shifts: the wrap reading needs BlockH")
    f = np.asarray(f, dtype=np.float64).reshape(geom.w, geom.alpha, geom.a)
    out = np.zeros((geom.xi, geom.gamma))
    for s in range(geom.w):
        for x, y, v in zip(*taps.of(s)):
            cut = _paste(geom, int(x), int(y))
            if cut is not None:
                (fy, fx), (sy, sx) = cut
                out[fy, fx] += v * f[s, sy, sx]
    return out.ravel()


def adjoint_shifts(geom: Geometry, taps: Taps, u: np.ndarray) -> np.ndarray:
    """``H^T u`` as the transpose of :func:`forward_shifts`: voxel (p, r, s)
    collects, for every tap (x, y, v) of s, v times u at (x + p, y + r)."""
    if taps.wrap:
        raise ValueError("adjoint_shifts: the wrap reading needs BlockH")
    u = np.asarray(u, dtype=np.float64).reshape(geom.xi, geom.gamma)
    out = np.zeros((geom.w, geom.alpha, geom.a))
    for s in range(geom.w):
        for x, y, v in zip(*taps.of(s)):
            cut = _paste(geom, int(x), int(y))
            if cut is not None:
                (fy, fx), (sy, sx) = cut
                out[s, sy, sx] += v * u[fy, fx]
    return out.ravel()


def h_shifts(geom: Geometry, taps: Taps) -> np.ndarray:
    """``h = H^T 1`` (Eq. 2) through :func:`adjoint_shifts`."""
    return adjoint_shifts(geom, taps, np.ones(geom.n))


def mlem_shifts(geom: Geometry, taps: Taps, g: np.ndarray, k: int,
                f0: np.ndarray | None = None):
    """:func:`mlem` (Eq. 2, Algorithm 1's loop) with the shifted-sum
    projectors. Returns ``(f, history)`` like :func:`mlem`."""
    g64 = np.asarray(g, dtype=np.float64).ravel()
    f = np.ones(geom.m) if f0 is None else np.asarray(f0, dtype=np.float64).ravel().copy()
    h = h_shifts(geom, taps)
    history = []
    for _ in range(k):
        q = forward_shifts(geom, taps, f)
        history.append(stats(q, g64))
        f = em_update(f, adjoint_shifts(geom, taps, ratio(g64, q)), h)
    history.append(stats(forward_shifts(geom, taps, f), g64))
    return f, history


# --- the paper's own formulations, used as independent cross-checks ------------

def dense_H(geom: Geometry, psf) -> np.ndarray:
    """H assembled literally from Eqs. 5-7: ``H_i = C_i E`` (tiny sizes only).

    ``Q = [I_a; 0]`` (gamma x a), ``E = [I_alpha kron Q; 0]`` (n x a alpha) and
    ``C_i`` the n x n circulant whose first column is the vectorised calibration
    image of wavelength i (the response to field-stop pixel (0, 0)).
    """
    a, al, ga, n = geom.a, geom.alpha, geom.gamma, geom.n
    Q = np.vstack([np.eye(a), np.zeros((ga - a, a))])
    top = np.kron(np.eye(al), Q)
    E = np.vstack([top, np.zeros((n - top.shape[0], a * al))])
    ptr, x, y, v = psf
    blocks = []
    for s in range(geom.w):
        c = np.zeros(n)
        lo, hi = int(ptr[s]), int(ptr[s + 1])
        for k in range(lo, hi):
            c[int(x[k]) + ga * int(y[k])] += float(v[k])
        # circulant: column t is c rolled down by t
        C = np.empty((n, n))
        for t in range(n):
            C[:, t] = np.roll(c, t)
        blocks.append(C @ E)
    return np.hstack(blocks)


def _calibration_column(geom: Geometry, taps: Taps, s: int) -> np.ndarray:
    c = np.zeros(geom.n)
    xs, ys, vs = taps.of(s)
    np.add.at(c, xs + geom.gamma * ys, vs)
    return c


def fft_forward(geom: Geometry, psf, f: np.ndarray, boundary: str = "reject") -> np.ndarray:
    """Eq. 13: ``g = F^-1 sum_i d_i * (F v_i)`` with ``d_i = F c_i`` and
    ``v_i = E f_i`` placed by the Sec. 3 index map (real FFT of length n).
    The transform's product is circular, so this is the wrap reading; under
    the reject rule the wrap never happens."""
    if boundary == "clip":
        raise ValueError("the FFT form has no clip reading")
    taps = merge_psf(geom, psf, boundary)
    f = np.asarray(f, dtype=np.float64).ravel()
    imap = index_map(geom)
    v = np.zeros(geom.n * geom.w)
    v[imap] = f
    acc = np.zeros(geom.n // 2 + 1, dtype=np.complex128)
    for s in range(geom.w):
        d = np.fft.rfft(_calibration_column(geom, taps, s))
        acc += d * np.fft.rfft(v[s * geom.n:(s + 1) * geom.n])
    return np.fft.irfft(acc, n=geom.n)


def fft_adjoint(geom: Geometry, psf, u: np.ndarray, boundary: str = "reject") -> np.ndarray:
    """Eqs. 14, 17: ``C_i^T u = F^-1(conj(d_i) * F u)``, then the transposed index
    map ``zeta = (I_w kron E)^T z`` gathers voxel values (Sec. 3)."""
    if boundary == "clip":
        raise ValueError("the FFT form has no clip reading")
    taps = merge_psf(geom, psf, boundary)
    U = np.fft.rfft(np.asarray(u, dtype=np.float64).ravel())
    z = np.zeros(geom.n * geom.w)
    for s in range(geom.w):
        d = np.fft.rfft(_calibration_column(geom, taps, s))
        z[s * geom.n:(s + 1) * geom.n] = np.fft.irfft(np.conj(d) * U, n=geom.n)
    return z[index_map(geom)]


# --- bfloat16 storage form ------------------------------------------------------

def round_bf16(x) -> np.ndarray:
    """Rounds float32 values to the nearest bfloat16 (ties to even), returned as
    float32: bfloat16 keeps the sign, the 8-bit exponent and the top 7 mantissa
    bits of a float32, so rounding adds half of the dropped 16-bit field (plus
    one when the kept last bit is odd, which breaks ties to even) and clears it.
    Finite inputs only (the PSF values and datacubes it is used on)."""
    bits = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32)


def em_step_stored(H: BlockH, g: np.ndarray, f: np.ndarray, store) -> np.ndarray:
    """One EM update (Eq. 2) computed in float64 from the stored iterate ``f``,
    whose result is then stored through ``store`` (e.g. rounding to float32
    then bfloat16, as a reduced-precision datacube keeps it)."""
    return np.asarray(store(em_step(H, g, f)), dtype=np.float64)


# --- gradients (for the differentiable projector) ------------------------------

def psf_value_grad(geom: Geometry, taps: Taps, f: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """``d <gy, H f> / d v_{s,k} = sum_{p,r} f_s(p, r) gy(x_k + p, y_k + r)``.

    H is linear in each merged tap value, and tap (s, k) contributes
    ``v_{s,k} f_s(p, r)`` to pixel ``(x_k + p, y_k + r)``. One value per merged
    tap, in the order of ``taps``.
    """
    f = np.asarray(f, dtype=np.float64).reshape(geom.w, geom.alpha, geom.a)
    gy = np.asarray(gy, dtype=np.float64).reshape(geom.xi, geom.gamma)
    out = np.zeros(taps.v.size)
    if taps.wrap:
        P, R = np.meshgrid(np.arange(geom.a), np.arange(geom.alpha))   # [alpha][a]
        flat = gy.ravel()
        for t in range(taps.v.size):
            s, x, y = int(taps.s[t]), int(taps.x[t]), int(taps.y[t])
            out[t] = np.sum(f[s] * flat[(x + P + geom.gamma * (y + R)) % geom.n])
        return out
    for t in range(taps.v.size):
        s, x, y = int(taps.s[t]), int(taps.x[t]), int(taps.y[t])
        # the part of the shifted field stop on the FPA (all of it unless clipped)
        p0, p1 = max(0, -x), min(geom.a, geom.gamma - x)
        r0, r1 = max(0, -y), min(geom.alpha, geom.xi - y)
        if p0 < p1 and r0 < r1:
            out[t] = np.sum(f[s, r0:r1, p0:p1] * gy[y + r0:y + r1, x + p0:x + p1])
    return out


def poisson_nll(q: np.ndarray, g: np.ndarray) -> float:
    """``sum_i q_i - g_i log q_i`` (negative Poisson log-likelihood, no constant)."""
    return -stats(q, g)["loglik"]


def with_values(taps: Taps, v: np.ndarray) -> Taps:
    return Taps(taps.s, taps.x, taps.y, np.asarray(v, dtype=np.float64), taps.ptr, taps.wrap)


def unrolled_nll_shifts(geom: Geometry, taps: Taps, g: np.ndarray, f0: np.ndarray, k: int) -> float:
    """:func:`unrolled_nll` with the shifted-sum projectors (no matrix: for the
    full-size workloads)."""
    _, hist = mlem_shifts(geom, taps, g, k, f0)
    return -hist[k]["loglik"]


def unrolled_nll(geom: Geometry, taps: Taps, g: np.ndarray, f0: np.ndarray, k: int) -> float:
    """Poisson NLL of g under ``H f^(k)`` after k EM updates from ``f0``, with H
    (and hence h) built from the tap values in ``taps``."""
    H = BlockH(geom, taps)
    f = np.asarray(f0, dtype=np.float64).ravel()
    for _ in range(k):
        f = em_step(H, g, f)
    return poisson_nll(H.forward(f), g)
