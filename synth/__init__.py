"""Seeded synthetic CTIS workloads: calibration PSFs, scenes and Poisson noise.

This module only draws random numbers and lays out arrays. It holds none of the
reconstruction arithmetic: the mean FPA image ``H f`` that the noise model needs
is computed by the caller (the FP64 oracle in tests, the GPU forward projector in
the benchmark) and passed in.

Geometry (White, Bell, Haygood, Sec. 2): a field stop of ``a x alpha`` pixels seen
at ``w`` wavelengths is imaged onto a ``gamma x xi`` focal-plane array (FPA). One
calibration image per wavelength is recorded with a point source at field-stop
pixel (0, 0); under shift-invariance every other column of H is a shift of it.

Layouts used throughout the project:
  * datacube ``f[s][r][p]`` (wavelength, field-stop row, field-stop column),
    flat index ``j = s*a*alpha + r*a + p`` (the zero-based ``j`` of Sec. 3);
  * FPA image ``g[y][x]``, flat index ``i = x + gamma*y``;
  * PSF of wavelength s: CSR over wavelengths, ``psf_ptr[w+1]`` and per nonzero
    ``psf_x, psf_y`` (int32 FPA coordinates of the response to pixel (0,0)) and
    ``psf_val`` (float32, >= 0).

The synthetic PSF follows a grating CTIS: an N x N grid of diffraction orders,
the zeroth order undispersed, the others displaced along their radial direction
by ``disp`` pixels per wavelength step, centred on the middle wavelength. Each
spot is a truncated S x S Gaussian.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic CTIS instrument + scene recipe."""

    name: str
    a: int
    alpha: int
    w: int
    gamma: int
    xi: int
    orders: int          # N: N x N grid of diffraction orders
    pitch: float         # pixels between adjacent orders
    disp: float          # pixels per wavelength step (non-zero orders)
    spot: int            # S: S x S support of each spot
    sigma: float         # Gaussian width of a spot, pixels
    scene: str           # "mask_spectra" or "segmentation"
    peak: float          # peak expected counts of the noiseless image
    k: int               # EM iterations of the workload
    seed: int = 0
    regions: int = 12

    @property
    def ell(self) -> int:
        return self.a * self.alpha

    @property
    def m(self) -> int:
        return self.a * self.alpha * self.w

    @property
    def n(self) -> int:
        return self.gamma * self.xi

    @property
    def nnz_per_image(self) -> int:
        return self.orders * self.orders * self.spot * self.spot

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# The five workloads the project measures and tests on.
TINY = Workload("tiny_16x16x8_fpa96", 16, 16, 8, 96, 96, 3, 28.0, 1.0, 3, 0.7,
                "mask_spectra", 1000.0, 20)
REALISTIC = Workload("realistic_128x128x64_fpa1024", 128, 128, 64, 1024, 1024, 5,
                     180.0, 1.5, 3, 0.8, "segmentation", 4000.0, 100)
LARGE = Workload("large_256x256x128_fpa2048", 256, 256, 128, 2048, 2048, 5, 360.0,
                 2.0, 5, 1.2, "segmentation", 10000.0, 50)
MODEL_A = Workload("model_a_64x64x32_fpa512", 64, 64, 32, 512, 512, 5, 90.0, 1.5, 3,
                   0.8, "segmentation", 4000.0, 100)
MODEL_B = REALISTIC.with_(name="model_b_128x128x64_fpa1024")
AUTOGRAD = REALISTIC.with_(name="autograd_128x128x64_fpa1024", k=10)

WORKLOADS = {wl.name: wl for wl in (TINY, REALISTIC, LARGE, MODEL_A, MODEL_B, AUTOGRAD)}


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Independent PCG64 streams per purpose so that, e.g., the PSF does not
    # change when the scene recipe does.
    return np.random.Generator(np.random.PCG64([seed, stream]))


def order_offsets(N: int):
    """Order indices (ox, oy) in [-N//2, N//2]^2, row-major over oy then ox."""
    h = N // 2
    return [(ox, oy) for oy in range(-h, h + 1) for ox in range(-h, h + 1)]


def make_psf(wl: Workload, seed: int | None = None):
    """Calibration PSFs for every wavelength, as CSR-over-wavelength COO arrays.

    Returns ``(psf_ptr int32[w+1], psf_x int32[nnz], psf_y int32[nnz],
    psf_val float32[nnz])``. Values are rounded to float32 here, once, so that
    every consumer sees the identical numbers.
    """
    seed = wl.seed if seed is None else seed
    rng = _rng(seed, 1)
    N, S = wl.orders, wl.spot
    orders = order_offsets(N)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=len(orders))
    c0x = (wl.gamma - wl.a) // 2
    c0y = (wl.xi - wl.alpha) // 2
    half = S // 2
    ptr = [0]
    xs, ys, vs = [], [], []
    for s in range(wl.w):
        t = s - (wl.w - 1) / 2.0
        for oi, (ox, oy) in enumerate(orders):
            norm = math.hypot(ox, oy)
            cx = c0x + wl.pitch * ox
            cy = c0y + wl.pitch * oy
            if norm > 0:
                cx += t * wl.disp * ox / norm
                cy += t * wl.disp * oy / norm
            bx = math.floor(cx + 0.5) - half
            by = math.floor(cy + 0.5) - half
            px = np.arange(bx, bx + S)
            py = np.arange(by, by + S)
            gx = np.exp(-((px - cx) ** 2) / (2 * wl.sigma ** 2))
            gy = np.exp(-((py - cy) ** 2) / (2 * wl.sigma ** 2))
            spot = gy[:, None] * gx[None, :]
            spot /= spot.sum()
            eff = (1.0 + 0.3 * math.sin(2 * math.pi * s / wl.w + phases[oi])) / (N * N)
            spot *= eff
            yy, xx = np.meshgrid(py, px, indexing="ij")
            xs.append(xx.ravel())
            ys.append(yy.ravel())
            vs.append(spot.ravel())
        ptr.append(ptr[-1] + len(orders) * S * S)
    return (np.asarray(ptr, dtype=np.int32),
            np.concatenate(xs).astype(np.int32),
            np.concatenate(ys).astype(np.int32),
            np.concatenate(vs).astype(np.float32))


def _spectra(rng: np.random.Generator, count: int, w: int) -> np.ndarray:
    """``count`` smooth random spectra of length w: 3 Gaussian bumps each."""
    s = np.arange(w, dtype=np.float64)
    centres = rng.uniform(0.0, w - 1, size=(count, 3))
    widths = rng.uniform(w / 16.0, w / 4.0, size=(count, 3))
    amps = rng.uniform(0.2, 1.0, size=(count, 3))
    out = np.zeros((count, w))
    for b in range(3):
        out += amps[:, b:b + 1] * np.exp(
            -((s[None, :] - centres[:, b:b + 1]) ** 2) / (2 * widths[:, b:b + 1] ** 2))
    return out


def make_scene(wl: Workload, seed: int | None = None) -> np.ndarray:
    """Nonnegative datacube ``f[s][r][p]`` (float32) of the workload's scene kind."""
    seed = wl.seed if seed is None else seed
    rng = _rng(seed, 2)
    a, al, w = wl.a, wl.alpha, wl.w
    if wl.scene == "mask_spectra":
        mask = rng.uniform(0.0, 1.0, size=(al, a))
        spec = _spectra(rng, al * a, w).reshape(al, a, w)
        f = mask[:, :, None] * spec
    elif wl.scene == "segmentation":
        R = wl.regions
        seeds = rng.uniform(0.0, 1.0, size=(R, 2)) * np.array([a, al])
        level = rng.uniform(0.2, 1.0, size=R)
        spec = _spectra(rng, R, w)
        pp, rr = np.meshgrid(np.arange(a) + 0.5, np.arange(al) + 0.5)
        d2 = (pp[:, :, None] - seeds[None, None, :, 0]) ** 2 + \
             (rr[:, :, None] - seeds[None, None, :, 1]) ** 2
        region = np.argmin(d2, axis=2)                     # [alpha][a]
        f = level[region][:, :, None] * spec[region]       # [alpha][a][w]
    else:
        raise ValueError(f"unknown scene kind {wl.scene!r}")
    return np.ascontiguousarray(np.transpose(f, (2, 0, 1))).astype(np.float32)


def make_measurement(mean_image: np.ndarray, peak: float, seed: int):
    """Poisson counts for a noiseless image scaled to ``max == peak``.

    ``mean_image`` is ``H f_true`` computed by the caller. Returns
    ``(g float32, scale)``: the counts and the factor applied to the mean image,
    so the caller can scale ``f_true`` by the same factor.
    """
    q = np.asarray(mean_image, dtype=np.float64)
    mx = float(q.max())
    scale = peak / mx if mx > 0 else 1.0
    rng = _rng(seed, 3)
    g = rng.poisson(q * scale).astype(np.float32)
    return g, scale


def random_positive(shape, seed: int, lo: float = 0.05, hi: float = 1.0) -> np.ndarray:
    """Uniform float32 values in [lo, hi) (projector inputs for parity tests)."""
    return _rng(seed, 4).uniform(lo, hi, size=shape).astype(np.float32)


def random_sparse_psf(w: int, nnz: int, xmax: int, ymax: int, seed: int,
                      duplicates: int = 0):
    """Unstructured PSF: ``nnz`` random positions per wavelength in
    ``[0, xmax] x [0, ymax]``, plus ``duplicates`` repeated positions per
    wavelength (to exercise merging). Same CSR layout as :func:`make_psf`."""
    rng = _rng(seed, 5)
    ptr = [0]
    xs, ys, vs = [], [], []
    for _ in range(w):
        x = rng.integers(0, xmax + 1, size=nnz)
        y = rng.integers(0, ymax + 1, size=nnz)
        if duplicates:
            pick = rng.integers(0, nnz, size=duplicates)
            x = np.concatenate([x, x[pick]])
            y = np.concatenate([y, y[pick]])
        v = rng.uniform(0.01, 1.0, size=x.size)
        xs.append(x)
        ys.append(y)
        vs.append(v)
        ptr.append(ptr[-1] + x.size)
    return (np.asarray(ptr, dtype=np.int32), np.concatenate(xs).astype(np.int32),
            np.concatenate(ys).astype(np.int32), np.concatenate(vs).astype(np.float32))
