"""Randomised parity: seeded random geometries (field stops from 1 pixel to
several tiles with ragged tails, 1-6 wavelengths), random sparse PSFs with
duplicate entries and random spot blobs (so K = 1, 3 and 5 all occur), under
the reject, clip and wrap boundaries, over both forward tile shapes:
projectors and three EM updates against the FP64 oracle, with the parity
suite's bounds."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import Plan
from tests.helpers import floored_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _case(seed):
    rng = np.random.default_rng(seed)
    a, al = int(rng.integers(1, 71)), int(rng.integers(1, 71))
    w = int(rng.integers(1, 7))
    ga, xi = a + int(rng.integers(0, 121)), al + int(rng.integers(0, 121))
    mode = ("reject", "clip", "wrap")[int(rng.integers(0, 3))]
    clip = mode == "clip"
    blob = int(rng.integers(1, 6))           # side of the spot blobs: K = 1, 3 or 5 boxes
    ptr, xs, ys, vs = [0], [], [], []
    for _ in range(w):
        for _ in range(int(rng.integers(0, 5))):   # blobs (a wavelength may have none)
            if clip:
                x0 = int(rng.integers(-a - blob, ga + 1))
                y0 = int(rng.integers(-al - blob, xi + 1))
            elif mode == "wrap":                  # anywhere on the FPA
                x0 = int(rng.integers(0, max(1, ga - blob + 1)))
                y0 = int(rng.integers(0, max(1, xi - blob + 1)))
            else:
                x0 = int(rng.integers(0, ga - a + 2 - blob)) if ga - a + 2 - blob > 0 else 0
                y0 = int(rng.integers(0, xi - al + 2 - blob)) if xi - al + 2 - blob > 0 else 0
            for dy in range(blob):
                for dx in range(blob):
                    x, y = x0 + dx, y0 + dy
                    if mode == "reject" and (x + a - 1 >= ga or y + al - 1 >= xi):
                        continue
                    if mode == "wrap" and (x >= ga or y >= xi):
                        continue
                    xs.append(x)
                    ys.append(y)
                    vs.append(float(rng.uniform(0.01, 1.0)))
                    if rng.random() < 0.1:           # a duplicate entry
                        xs.append(x)
                        ys.append(y)
                        vs.append(float(rng.uniform(0.01, 1.0)))
        ptr.append(len(xs))
    psf = (np.array(ptr, np.int32), np.array(xs, np.int32), np.array(ys, np.int32),
           np.array(vs, np.float32))
    return O.Geometry(a, al, w, ga, xi), psf, mode


@pytest.mark.parametrize("seed", range(24))
def test_random_geometry_projectors_and_em(seed):
    geom, psf, boundary = _case(1000 + seed)
    H = O.build_H(geom, psf, boundary=boundary)
    f = synth.random_positive((geom.w, geom.alpha, geom.a), 2000 + seed)
    r = synth.random_positive((geom.xi, geom.gamma), 3000 + seed)
    g = (synth.random_positive(geom.n, 4000 + seed) * 50).astype(np.float32)
    tile = ("32x32", "32x16")[seed % 2]   # both forward tile shapes
    with Plan(geom.a, geom.alpha, geom.w, geom.gamma, geom.xi, psf, boundary=boundary,
              forward_tile=tile) as plan:
        hf = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy().ravel()
        ht = plan.adjoint(torch.from_numpy(r).cuda()).cpu().numpy().ravel()
        out, _ = plan.reconstruct(torch.from_numpy(g.reshape(geom.xi, geom.gamma)).cuda(), 3,
                                  init="ones")
        plan.check()
        out = out.cpu().numpy().ravel()
    ref_f, ref_t = H.forward(f.ravel()), H.adjoint(r.ravel())
    for got, ref in ((hf, ref_f), (ht, ref_t)):
        if np.any(ref):
            assert floored_rel(got, ref) <= 1e-5
        else:
            assert not np.any(got)
    ref, _ = O.mlem(H, g, 3)
    if np.any(ref):
        assert floored_rel(out, ref) <= 3e-5
    else:
        assert not np.any(out)
