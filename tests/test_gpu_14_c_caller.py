"""The C ABI from plain C on the GPU: tests/c/abi_gpu_reconstruct.c, built
with gcc against include/ctis.h, libctis.so and the CUDA runtime (no Python
or PyTorch in that process), reconstructs the tiny workload; its iterate and
statistics match the FP64 oracle within the EM suite's bounds."""
import os
import subprocess

import numpy as np
import pytest

import __graft_entry__
import oracle as O
import synth
import paper_2006_01573_gb300 as ctis
from tests.helpers import floored_rel, problem

pytestmark = pytest.mark.gpu


def test_plain_c_caller_reconstructs(tmp_path):
    __graft_entry__.build()
    root = os.path.dirname(os.path.dirname(__file__))
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.dirname(ctis.LIB_PATH)
    exe = str(tmp_path / "abi_gpu_reconstruct")
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror",
                    "-I", os.path.join(root, "include"), "-I", os.path.join(cuda, "include"),
                    os.path.join(root, "tests", "c", "abi_gpu_reconstruct.c"), "-o", exe,
                    "-L", libdir, "-lctis", "-Wl,-rpath," + libdir,
                    "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, "lib64")],
                   check=True)
    wl = synth.TINY
    geom, psf, H, _, g = problem(wl)
    k = 5
    ptr, x, y, v = psf
    lines = [f"{wl.a} {wl.alpha} {wl.w} {wl.gamma} {wl.xi} {k} {len(v)}",
             " ".join(str(int(p)) for p in ptr)]
    lines += [f"{int(a)} {int(b)} {float(c):.9g}" for a, b, c in zip(x, y, v)]
    lines.append(" ".join(f"{float(t):.9g}" for t in np.asarray(g, np.float32)))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    vals = np.array(out.stdout.split(), dtype=np.float64)
    f, st = vals[:geom.m], vals[geom.m:].reshape(k + 1, 4)
    ref, hist = O.mlem(H, g, k)
    assert floored_rel(f, ref) <= k * 1e-5
    for t in range(k + 1):
        assert abs(st[t, 2] - hist[t]["loglik"]) <= 1e-5 * abs(hist[t]["loglik"])
