"""Shared test helpers: error metrics and workload setup (no method arithmetic)."""
import numpy as np

import oracle as O
import synth


def floored_rel(a, b, floor_frac=1e-6):
    """max_j |a_j - b_j| / max(|b_j|, floor_frac * max|b|)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    floor = floor_frac * max(np.abs(b).max(), 1e-300)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def avg_rel_pixel_err(a, b, floor_frac=1e-6):
    """The paper's reconstruction-quality figure (Sec. 4): the mean over
    voxels of |a_j - b_j| / b_j, here over the voxels with
    b_j > floor_frac * max b (the paper's sum divides by values that may be 0)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    on = b > floor_frac * max(b.max(), 1e-300)
    return float(np.mean(np.abs(a[on] - b[on]) / b[on]))


def geometry(wl):
    return O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)


def problem(wl, seed=None):
    """(geom, psf, H, f_true, g) with g ~ Poisson(H f_true) scaled to wl.peak."""
    geom = geometry(wl)
    psf = synth.make_psf(wl, seed)
    H = O.build_H(geom, psf)
    f_true = synth.make_scene(wl, seed).ravel()
    g, scale = synth.make_measurement(H.forward(f_true), wl.peak, wl.seed if seed is None else seed)
    return geom, psf, H, f_true * scale, g
