"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/ctis.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__
import paper_2006_01573_gb300 as ctis
from paper_2006_01573_gb300 import _native

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ctis.h")


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return ctis.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(ctis_\w+)\s*\(", text, re.M)))


def test_header_declares_expected_entry_points():
    assert set(declared_functions()) == set(_native.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", ctis.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (ctis_\w+)$", out, re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_status_strings(lib):
    assert lib.ctis_status_string(0) == b"CTIS_OK"
    assert lib.ctis_status_string(-2) == b"CTIS_ERR_OUT_OF_BOUNDS"
    assert lib.ctis_status_string(-5) == b"CTIS_ERR_TIMEOUT"


def _create(lib, a, al, w, ga, xi, ptr, x, y, v, dtype=0):
    h = ctypes.c_void_p()
    i32 = lambda arr: np.ascontiguousarray(arr, np.int32).ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    f32 = np.ascontiguousarray(v, np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    keep = [np.ascontiguousarray(t, np.int32) for t in (ptr, x, y)]
    rc = lib.ctis_plan_create(ctypes.byref(h), a, al, w, ga, xi, *[k.ctypes.data_as(
        ctypes.POINTER(ctypes.c_int32)) for k in keep], f32, dtype)
    return rc, h


@pytest.mark.parametrize("case,expect", [
    (dict(a=0), -1),                                   # bad size
    (dict(dtype=7), -1),                               # bad dtype
    (dict(ptr=[1, 1]), -1),                            # psf_ptr[0] != 0
    (dict(v=[-1.0]), -1),                              # negative value
    (dict(v=[np.nan]), -1),                            # non-finite value
    (dict(x=[7]), -2),                                 # shifted copy leaves the FPA (x)
    (dict(y=[-1]), -2),                                # negative y
    (dict(a=12), -2),                                  # field stop wider than the FPA
])
def test_host_side_argument_errors(lib, case, expect):
    args = dict(a=4, al=4, w=1, ga=10, xi=10, ptr=[0, 1], x=[6], y=[6], v=[1.0], dtype=0)
    args.update(case)
    rc, h = _create(lib, args["a"], args["al"], args["w"], args["ga"], args["xi"], args["ptr"],
                    args["x"], args["y"], args["v"], args["dtype"])
    assert rc == expect, lib.ctis_last_error()
    assert not h.value
    assert lib.ctis_last_error()


def test_destroy_null_is_ok(lib):
    assert lib.ctis_plan_destroy(None) == 0


def test_header_compiles_as_c_and_a_c_caller_links(lib, tmp_path):
    """include/ctis.h is plain C: a C99 program built with gcc against it and
    libctis.so runs the host-only entry points (no GPU needed)."""
    root = os.path.dirname(os.path.dirname(__file__))
    exe = str(tmp_path / "abi_host_only")
    libdir = os.path.dirname(ctis.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "c", "abi_host_only.c"), "-o", exe,
                    "-L", libdir, "-lctis", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "reject CTIS_ERR_OUT_OF_BOUNDS" in out.stdout
    first = out.stdout.splitlines()[0].split()
    # each wavelength's two nonzeros are 8-connected: one 3 x 3 cluster each;
    # a 6 x 5 footprint on a 10 x 9 FPA meets at least one 32 x 32 tile
    assert first[:4] == ["clusters", "2", "k", "3"] and int(first[5]) >= 1 and int(first[7]) >= 2


def test_header_constants_match_the_binding():
    """The enum values the header declares are the ones the binding passes."""
    text = open(HEADER).read()
    consts = {name: int(val) for name, val in re.findall(r"\b(CTIS_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    for name in ("CTIS_F32", "CTIS_BF16", "CTIS_BOUNDARY_REJECT", "CTIS_BOUNDARY_CLIP",
                 "CTIS_BOUNDARY_WRAP", "CTIS_SOLVER_EM", "CTIS_SOLVER_SART", "CTIS_SOLVER_SMART",
                 "CTIS_INIT_ONES", "CTIS_INIT_HTG", "CTIS_TILE_32X32", "CTIS_TILE_32X16"):
        assert consts[name] == getattr(_native, name), name
    assert consts["CTIS_NSTATS"] == _native.NSTATS
    assert consts["CTIS_DEBUG_DROP_COPIES"] == 1
    assert consts["CTIS_DEBUG_SERIAL_LAUNCH"] == 2
    assert consts["CTIS_ERR_TIMEOUT"] == -5 and consts["CTIS_ERR_UNSUPPORTED"] == -6
