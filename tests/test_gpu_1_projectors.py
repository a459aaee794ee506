"""GPU parity of the projector pair and of the plan tables against the FP64 oracle.

Integer tables are compared bit-exactly; projector values within the float32
bound 1e-5 (max floored-relative error): each output is a sum of at most a few
hundred nonnegative float32 products, whose worst-case rounding error is
below 6e-8 * terms relative to the sum."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle as O
import synth
from paper_2006_01573_gb300 import CtisError, Plan
from tests.helpers import floored_rel, geometry

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _cases():
    wl5 = synth.Workload("k5", 20, 24, 6, 120, 110, 3, 36.0, 1.2, 5, 1.2, "segmentation", 100.0, 3)
    deep = synth.Workload("deep", 24, 20, 40, 140, 130, 3, 40.0, 0.5, 3, 0.8, "segmentation", 100.0, 3)
    ragged = synth.Workload("ragged", 13, 11, 3, 49, 43, 3, 14.0, 1.0, 3, 0.7, "mask_spectra", 100.0, 3)
    return {
        "tiny": (synth.TINY, synth.make_psf(synth.TINY)),
        "k5": (wl5, synth.make_psf(wl5)),
        "deep_multichunk": (deep, synth.make_psf(deep)),
        "ragged": (ragged, synth.make_psf(ragged)),
        "sparse_dups": (synth.TINY, synth.random_sparse_psf(8, 30, 96 - 16, 96 - 16, 3, duplicates=5)),
    }


CASES = _cases()


def _blob_case():
    """One wavelength with an 8x7 blob (split into 5x5 boxes) and a lone tap."""
    wl = synth.Workload("blob", 12, 10, 2, 40, 36, 1, 0.0, 0.0, 1, 1.0, "mask_spectra", 1.0, 1)
    xs, ys, vs, ptr = [], [], [], [0]
    rng = np.random.default_rng(5)
    for s in range(2):
        for y in range(7):
            for x in range(8):
                xs.append(3 + x + s)
                ys.append(4 + y)
                vs.append(rng.uniform(0.1, 1.0))
        xs.append(25)
        ys.append(20)
        vs.append(0.5)
        ptr.append(len(xs))
    return wl, (np.array(ptr, np.int32), np.array(xs, np.int32), np.array(ys, np.int32),
                np.array(vs, np.float32))


CASES["blob_split"] = _blob_case()


def _plan(wl, psf, dtype="f32", forward_tile="32x32"):
    return Plan(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi, psf, dtype=dtype, forward_tile=forward_tile)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tables_bit_exact(name):
    wl, psf = CASES[name]
    geom = geometry(wl)
    taps = O.merge_psf(geom, psf)
    with _plan(wl, psf) as plan:
        s, x, y, v, h = plan.export_taps()
    assert np.array_equal(s, taps.s) and np.array_equal(x, taps.x) and np.array_equal(y, taps.y)
    assert np.array_equal(v, taps.v.astype(np.float32))
    H = O.BlockH(geom, taps)
    h_ref = H.h().reshape(geom.w, -1)
    assert np.all(h_ref == h_ref[:, :1])          # in-bounds PSF: h constant per wavelength
    np.testing.assert_allclose(h, h_ref[:, 0], rtol=1.2e-7, atol=0)


@pytest.mark.parametrize("name", ["tiny", "ragged"])
def test_index_map_bit_exact(name):
    wl, psf = CASES[name]
    with _plan(wl, psf) as plan:
        got = plan.index_map().cpu().numpy()
    assert np.array_equal(got, O.index_map(geometry(wl)))


def test_delta_psf_forward_is_exact_paste():
    geom = O.Geometry(13, 9, 3, 50, 40)
    x0, y0 = [0, 20, 37], [0, 31, 5]
    psf = (np.arange(4, dtype=np.int32), np.array(x0, np.int32), np.array(y0, np.int32),
           np.ones(3, np.float32))
    f = synth.random_positive((3, 9, 13), 3)
    with Plan(13, 9, 3, 50, 40, psf) as plan:
        hf = plan.forward(torch.from_numpy(f).cuda()).cpu().numpy()
    expect = np.zeros((40, 50), np.float32)
    for s in range(3):
        expect[y0[s]:y0[s] + 9, x0[s]:x0[s] + 13] += f[s]
    assert np.array_equal(hf, expect)


@pytest.mark.parametrize("tile", ["32x32", "32x16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_forward_parity(name, tile):
    wl, psf = CASES[name]
    geom = geometry(wl)
    H = O.build_H(geom, psf)
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 11)
    with _plan(wl, psf, forward_tile=tile) as plan:
        assert plan.forward_tile() == tile
        hf = plan.forward(torch.from_numpy(f).cuda())
        plan.check()
        hf = hf.cpu().numpy()
    ref = H.forward(f.ravel())
    assert floored_rel(hf, ref) <= TOL
    assert np.all(hf.ravel()[ref == 0] == 0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_parity(name):
    wl, psf = CASES[name]
    geom = geometry(wl)
    H = O.build_H(geom, psf)
    r = synth.random_positive((wl.xi, wl.gamma), 12)
    with _plan(wl, psf) as plan:
        out = plan.adjoint(torch.from_numpy(r).cuda())
        plan.check()
        out = out.cpu().numpy()
    assert floored_rel(out, H.adjoint(r.ravel())) <= TOL


def test_adjoint_identity_on_gpu():
    wl, psf = CASES["tiny"]
    f = synth.random_positive((wl.w, wl.alpha, wl.a), 21)
    r = synth.random_positive((wl.xi, wl.gamma), 22)
    with _plan(wl, psf) as plan:
        hf = plan.forward(torch.from_numpy(f).cuda()).double().cpu().numpy()
        htr = plan.adjoint(torch.from_numpy(r).cuda()).double().cpu().numpy()
    lhs = np.sum(hf * r)
    rhs = np.sum(f * htr)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_projectors_are_deterministic_and_stream_ordered():
    wl, psf = CASES["deep_multichunk"]
    f = torch.from_numpy(synth.random_positive((wl.w, wl.alpha, wl.a), 31)).cuda()
    s = torch.cuda.Stream()
    with _plan(wl, psf) as plan, torch.cuda.stream(s):
        a = plan.forward(f).clone()
        b = plan.forward(f).clone()
        ra = plan.adjoint(a).clone()
        rb = plan.adjoint(a).clone()
        plan.check()
    assert torch.equal(a, b) and torch.equal(ra, rb)


@pytest.mark.parametrize("wl", [synth.REALISTIC, synth.LARGE], ids=lambda w: w.name)
def test_full_size_sampled_outputs(wl):
    """Full-size projectors in the benchmark's launch configuration, checked on
    sampled outputs that the oracle evaluates one by one."""
    geom = geometry(wl)
    psf = synth.make_psf(wl)
    taps = O.merge_psf(geom, psf)
    f = synth.make_scene(wl)
    rng = np.random.default_rng(0)
    with _plan(wl, psf) as plan:
        hf = plan.forward(torch.from_numpy(f).cuda())
        r = torch.from_numpy(synth.random_positive((wl.xi, wl.gamma), 7)).cuda()
        z = plan.adjoint(r)
        plan.check()
        hf, z, r = hf.cpu().numpy(), z.cpu().numpy(), r.cpu().numpy()
    # forward: sample covered pixels (weighted toward the orders) plus random ones
    cov = np.argwhere(hf > 0)
    pick = cov[rng.choice(len(cov), 300, replace=False)]
    xs = np.concatenate([pick[:, 1], rng.integers(0, wl.gamma, 100)])
    ys = np.concatenate([pick[:, 0], rng.integers(0, wl.xi, 100)])
    ref = O.forward_at(geom, taps, f.ravel(), xs, ys)
    assert floored_rel(hf[ys, xs], ref) <= TOL
    ss = rng.integers(0, wl.w, 200)
    ps = rng.integers(0, wl.a, 200)
    rs = rng.integers(0, wl.alpha, 200)
    ref = O.adjoint_at(geom, taps, r.ravel(), ss, ps, rs)
    assert floored_rel(z[ss, rs, ps], ref) <= TOL


def test_out_of_bounds_psf_is_rejected():
    psf = (np.array([0, 1], np.int32), np.array([40], np.int32), np.array([3], np.int32),
           np.ones(1, np.float32))
    with pytest.raises(CtisError) as e:
        Plan(16, 16, 1, 50, 50, psf)
    assert e.value.code == -2
