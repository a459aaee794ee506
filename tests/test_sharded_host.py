"""The wavelength-sharded EM reconstruction on the CPU (no GPU): two gloo
ranks on 127.0.0.1 each own a contiguous slice of the wavelengths
(shard_wavelengths), build the FP64 oracle's H from their slice's
calibration images alone (slice_psf), and run EM exchanging only the
partial image H_r f_r (an all-reduce of n floats per iteration, Eq. 8's sum
over wavelength blocks split by rank). The gathered slices must equal the
oracle's single-process EM, and every rank must see the same statistics.
This checks the host side of ctis_reconstruct_sharded: the partition, the
slicing of the PSF, and that the exchange is exactly the sum of the slices'
images."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_wavelengths_partitions_contiguously():
    sys.path.insert(0, ROOT)
    from paper_2006_01573_gb300 import shard_wavelengths
    for w in (1, 2, 3, 7, 8, 64, 65):
        for world in range(1, min(w, 6) + 1):
            parts = [shard_wavelengths(w, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == w
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard_wavelengths(3, 4, 0)


def test_slice_psf_gives_the_slice_blocks_of_H():
    sys.path.insert(0, ROOT)
    import oracle as O
    import synth
    from paper_2006_01573_gb300 import slice_psf
    wl = synth.TINY
    psf = synth.make_psf(wl)
    geom = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    H = O.build_H(geom, psf)
    s0, s1 = 3, 6
    sub = O.Geometry(wl.a, wl.alpha, s1 - s0, wl.gamma, wl.xi)
    Hs = O.build_H(sub, slice_psf(psf, s0, s1))
    for j in range(s1 - s0):
        assert (Hs.blocks[j] != H.blocks[s0 + j]).nnz == 0


def _rank(rank, world, port, k, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import oracle as O
    import synth
    from paper_2006_01573_gb300 import shard_wavelengths, slice_psf
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = synth.TINY
        psf = synth.make_psf(wl)
        full = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
        g, _ = synth.make_measurement(O.build_H(full, psf).forward(synth.make_scene(wl).ravel()),
                                      wl.peak, wl.seed)
        s0, s1 = shard_wavelengths(wl.w, world, rank)
        geom = O.Geometry(wl.a, wl.alpha, s1 - s0, wl.gamma, wl.xi)
        H = O.build_H(geom, slice_psf(psf, s0, s1))
        h = H.h()
        f = np.ones(geom.m)
        g64 = np.asarray(g, dtype=np.float64)
        stats = []
        for it in range(k + 1):
            qv = torch.from_numpy(H.forward(f))
            dist.all_reduce(qv)                      # sum of the slices' images
            qv = qv.numpy()
            stats.append(O.stats(qv, g64))
            if it == k:
                break
            f = O.em_update(f, H.adjoint(O.ratio(g64, qv)), h)
        q.put((rank, (s0, s1), f, stats))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reconstruct_like_one_process():
    sys.path.insert(0, ROOT)
    import oracle as O
    import synth
    k, world = 6, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, k, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        rank, sl, f, st = q.get(timeout=180)
        res[rank] = (sl, f, st)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = synth.TINY
    geom = O.Geometry(wl.a, wl.alpha, wl.w, wl.gamma, wl.xi)
    H = O.build_H(geom, synth.make_psf(wl))
    g, _ = synth.make_measurement(H.forward(synth.make_scene(wl).ravel()), wl.peak, wl.seed)
    f_ref, hist = O.mlem(H, g, k)
    got = np.concatenate([res[r][1] for r in range(world)])
    assert [res[r][0] for r in range(world)] == [(0, 4), (4, 8)]
    np.testing.assert_allclose(got, f_ref, rtol=1e-12, atol=1e-14 * np.abs(f_ref).max())
    for it in range(k + 1):
        assert res[0][2][it] == res[1][2][it]           # every rank holds the same sums
        for key, v in hist[it].items():
            assert res[0][2][it][key] == pytest.approx(v, rel=1e-12)
