"""ctypes binding of libctis.so (argument marshalling only).

Every computation happens in the library's CUDA kernels; this module checks
tensor shapes, dtypes and devices, passes raw pointers and the current CUDA
stream, and turns status codes into exceptions. There is no CPU fallback: if
the library is missing, importing a Plan fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libctis.so")

CTIS_F32, CTIS_BF16 = 0, 1
CTIS_BOUNDARY_REJECT, CTIS_BOUNDARY_CLIP, CTIS_BOUNDARY_WRAP = 0, 1, 2
CTIS_SOLVER_EM, CTIS_SOLVER_SART, CTIS_SOLVER_SMART = 0, 1, 2
_SOLVER = {"em": CTIS_SOLVER_EM, "sart": CTIS_SOLVER_SART, "smart": CTIS_SOLVER_SMART}
_BOUNDARY = {"reject": CTIS_BOUNDARY_REJECT, "clip": CTIS_BOUNDARY_CLIP,
             "wrap": CTIS_BOUNDARY_WRAP}
CTIS_INIT_ONES, CTIS_INIT_HTG = 1, 2
CTIS_TILE_32X32, CTIS_TILE_32X16 = 0, 1
_TILE = {"32x32": CTIS_TILE_32X32, "32x16": CTIS_TILE_32X16}
NSTATS = 4
STAT_NAMES = ("flux_hf", "flux_g", "loglik", "resid2")

_lib = None

# int reduce(float* q_dev, int64_t n, void* ctx, void* stream) (ctis_reduce_fn)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_void_p)

# Every symbol include/ctis.h declares, for the ABI export test.
EXPORTED = (
    "ctis_plan_create", "ctis_plan_create_ex", "ctis_plan_destroy", "ctis_plan_get_info", "ctis_plan_export_taps",
    "ctis_index_map", "ctis_forward", "ctis_adjoint", "ctis_reconstruct", "ctis_plan_check",
    "ctis_plan_set_profiling", "ctis_plan_kernel_times", "ctis_forward_static_scratch",
    "ctis_plan_set_values", "ctis_psf_grad", "ctis_unrolled_nll_grad", "ctis_reconstruct_batched",
    "ctis_plan_autotune", "ctis_plan_set_schedule", "ctis_tables_inspect",
    "ctis_fft_forward", "ctis_fft_adjoint", "ctis_fft_reconstruct", "ctis_reconstruct_solver",
    "ctis_plan_set_debug", "ctis_reconstruct_batched_solver", "ctis_plan_time_launches",
    "ctis_reconstruct_sharded",
    "ctis_fma_peak", "ctis_status_string", "ctis_last_error",
)


class CtisError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{message} [{code}]")
        self.code = code


class PlanInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "a", "alpha", "w", "gamma", "xi", "m", "n", "nnz", "clusters", "cluster_k",
        "fwd_tiles", "fwd_tasks", "fwd_items", "adj_tiles", "adj_tasks", "adj_items",
        "scratch_bytes", "dtype", "fwd_warps", "adj_warps", "fwd_chunk", "adj_chunk",
        "fwd_load_milli", "adj_load_milli", "fwd_split_q", "adj_split_q", "fwd_skew_pm",
        "adj_skew_pm", "boundary", "fwd_tile_w", "fwd_tile_h")]


class TablesInfo(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int)] + [(name, ctypes.c_int64) for name in (
        "clusters", "cluster_k", "tiles", "tasks", "witems", "warps", "warps_per_cta", "tile_w",
        "tile_h", "chunk", "split_q", "skew_pm", "load_milli")]


class PlanOptions(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int), ("tasks_per_item", ctypes.c_int),
                ("item_overhead_q", ctypes.c_int), ("cta_skew_permille", ctypes.c_int),
                ("boundary", ctypes.c_int), ("forward_tile", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


def load(path: str = LIB_PATH):
    """Load libctis.so and declare its C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "or python -m paper_2006_01573_gb300.build")
    lib = ctypes.CDLL(path)
    P, I, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
    i32p = ctypes.POINTER(ctypes.c_int32)
    f32p = ctypes.POINTER(ctypes.c_float)
    sig = {
        "ctis_plan_create": (I, [ctypes.POINTER(P), I, I, I, I, I, i32p, i32p, i32p, f32p, I]),
        "ctis_plan_create_ex": (I, [ctypes.POINTER(P), I, I, I, I, I, i32p, i32p, i32p, f32p, I,
                                    ctypes.POINTER(PlanOptions)]),
        "ctis_plan_destroy": (I, [P]),
        "ctis_plan_get_info": (I, [P, ctypes.POINTER(PlanInfo)]),
        "ctis_plan_export_taps": (I, [P, i32p, i32p, i32p, f32p, f32p]),
        "ctis_index_map": (I, [P, VP, VP]),
        "ctis_forward": (I, [P, VP, VP, VP]),
        "ctis_adjoint": (I, [P, VP, VP, VP]),
        "ctis_reconstruct": (I, [P, VP, VP, I, I, VP, VP]),
        "ctis_reconstruct_solver": (I, [P, VP, VP, I, I, I, ctypes.c_float, VP, VP]),
        "ctis_plan_check": (I, [P, VP]),
        "ctis_forward_static_scratch": (I, [P, VP, VP, VP]),
        "ctis_plan_set_profiling": (I, [P, I]),
        "ctis_plan_set_debug": (I, [P, I]),
        "ctis_plan_kernel_times": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)]),
        "ctis_plan_set_values": (I, [P, f32p]),
        "ctis_plan_autotune": (I, [P, VP, VP]),
        "ctis_plan_set_schedule": (I, [P, I, I, I, I]),
        "ctis_fft_forward": (I, [P, VP, VP, VP]),
        "ctis_fft_adjoint": (I, [P, VP, VP, VP]),
        "ctis_fft_reconstruct": (I, [P, VP, VP, I, I, VP]),
        "ctis_reconstruct_batched": (I, [ctypes.POINTER(P), I, I, ctypes.POINTER(I),
                                         ctypes.POINTER(VP), ctypes.POINTER(VP), I, I, VP, VP]),
        "ctis_reconstruct_batched_solver": (I, [ctypes.POINTER(P), I, I, ctypes.POINTER(I),
                                                ctypes.POINTER(VP), ctypes.POINTER(VP), I, I, I,
                                                ctypes.c_float, VP, VP]),
        "ctis_psf_grad": (I, [P, VP, VP, VP, VP]),
        "ctis_unrolled_nll_grad": (I, [P, VP, VP, I, VP, VP, VP, VP]),
        "ctis_tables_inspect": (I, [I, I, I, I, I, i32p, i32p, i32p, f32p, I,
                                    ctypes.POINTER(PlanOptions), I, I, i32p,
                                    ctypes.POINTER(TablesInfo)] + [i32p] * 8),
        "ctis_plan_time_launches": (I, [P, VP, I, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), VP]),
        "ctis_fma_peak": (I, [I, I, I, I, VP, VP]),
        "ctis_reconstruct_sharded": (I, [P, VP, VP, I, I, VP, REDUCE_FN, VP, VP]),
        "ctis_status_string": (ctypes.c_char_p, [I]),
        "ctis_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        lib = load()
        raise CtisError(rc, f"{lib.ctis_status_string(rc).decode()}: "
                            f"{lib.ctis_last_error().decode()}")


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def tables_inspect(a, alpha, w, gamma, xi, psf, forward: bool, n_ctas: int, dtype: str = "f32",
                   block_sm=None, tasks_per_item: int = 0, item_overhead_q: int = 0,
                   cta_skew_permille: int = 0, boundary: str = "reject",
                   forward_tile: str = "32x32") -> dict:
    """Host-only view of one projector's work lists and schedule
    (ctis_tables_inspect; no device needed). Returns the info fields and the
    arrays as numpy int32 arrays."""
    lib = load()
    ptr, _ = _arr(psf[0], np.int32)
    x, _ = _arr(psf[1], np.int32)
    y, _ = _arr(psf[2], np.int32)
    v, _ = _arr(psf[3], np.float32)
    i32 = lambda arr: None if arr is None else arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    opt = PlanOptions(ctypes.sizeof(PlanOptions), int(tasks_per_item), int(item_overhead_q),
                      int(cta_skew_permille), _BOUNDARY[boundary], _TILE[forward_tile])
    bsm = None if block_sm is None else np.ascontiguousarray(block_sm, dtype=np.int32)
    dt = {"f32": CTIS_F32, "bf16": CTIS_BF16}[dtype]
    info = TablesInfo(ctypes.sizeof(TablesInfo))
    args = [a, alpha, w, gamma, xi, i32(ptr), i32(x), i32(y),
            v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), dt, ctypes.byref(opt),
            1 if forward else 0, int(n_ctas), i32(bsm), ctypes.byref(info)]
    _check(lib.ctis_tables_inspect(*args, *([None] * 8)))
    n = {f: int(getattr(info, f)) for f, _ in TablesInfo._fields_[1:]}
    out = {
        "cluster_sxy": np.zeros((n["clusters"], 3), np.int32),
        "tile_xyp": np.zeros((n["tiles"], 3), np.int32),
        "tile_task_ptr": np.zeros(n["tiles"] + 1, np.int32),
        "task_cluster": np.zeros(n["tasks"], np.int32),
        "warp_begin": np.zeros(n["warps"] + 1, np.int32),
        "item_tile": np.zeros(n["witems"], np.int32),
        "item_chunk": np.zeros((n["witems"], 2), np.int32),
        "item_range": np.zeros((n["witems"], 2), np.int32),
    }
    _check(lib.ctis_tables_inspect(*args, *(i32(out[k]) for k in (
        "cluster_sxy", "tile_xyp", "tile_task_ptr", "task_cluster", "warp_begin", "item_tile",
        "item_chunk", "item_range"))))
    out.update(n)
    return out


class Plan:
    """A CTIS reconstruction plan on the current CUDA device.

    ``psf`` is ``(psf_ptr[w+1], psf_x, psf_y, psf_val)`` in host memory; see
    include/ctis.h for layouts. Datacubes are torch tensors shaped
    ``(w, alpha, a)`` (float32, or bfloat16 for ``dtype='bf16'``), FPA images
    ``(xi, gamma)`` float32, all on the plan's device.
    """

    def __init__(self, a, alpha, w, gamma, xi, psf, dtype: str = "f32", tasks_per_item: int = 0,
                 item_overhead_q: int = 0, cta_skew_permille: int = 0, boundary: str = "reject",
                 forward_tile: str = "32x32"):
        lib = load()
        ptr, _ = _arr(psf[0], np.int32)
        x, _ = _arr(psf[1], np.int32)
        y, _ = _arr(psf[2], np.int32)
        v, _ = _arr(psf[3], np.float32)
        if ptr.size != w + 1:
            raise ValueError("psf_ptr must have w+1 entries")
        self.dtype = {"f32": CTIS_F32, "bf16": CTIS_BF16}[dtype]
        handle = ctypes.c_void_p()
        i32 = lambda arr: arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        opt = PlanOptions(ctypes.sizeof(PlanOptions), int(tasks_per_item), int(item_overhead_q),
                          int(cta_skew_permille), _BOUNDARY[boundary], _TILE[forward_tile])
        _check(lib.ctis_plan_create_ex(ctypes.byref(handle), a, alpha, w, gamma, xi, i32(ptr),
                                       i32(x), i32(y),
                                       v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       self.dtype, ctypes.byref(opt)))
        self._h = handle
        self.a, self.alpha, self.w, self.gamma, self.xi = a, alpha, w, gamma, xi
        # bumped by every set_values: tells a pending autograd backward whether
        # the plan still holds the tap values its forward projected with
        self.values_version = 0

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().ctis_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- metadata ---------------------------------------------------------------
    def info(self) -> dict:
        inf = PlanInfo()
        _check(load().ctis_plan_get_info(self._h, ctypes.byref(inf)))
        return {name: getattr(inf, name) for name, _ in PlanInfo._fields_}

    def export_taps(self):
        """Merged PSF table ``(s, x, y, val)`` sorted by (s, y, x), and ``h[w]``."""
        nnz = self.info()["nnz"]
        s = np.zeros(nnz, np.int32)
        x = np.zeros(nnz, np.int32)
        y = np.zeros(nnz, np.int32)
        v = np.zeros(nnz, np.float32)
        h = np.zeros(self.w, np.float32)
        i32 = lambda arr: arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        f32 = lambda arr: arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        _check(load().ctis_plan_export_taps(self._h, i32(s), i32(x), i32(y), f32(v), f32(h)))
        return s, x, y, v, h

    # -- helpers ------------------------------------------------------------------
    def _f_dtype(self):
        import torch
        return torch.bfloat16 if self.dtype == CTIS_BF16 else torch.float32

    def _check_cube(self, f, dtype=None):
        import torch
        dtype = dtype or self._f_dtype()
        if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == dtype and
                f.is_contiguous() and f.numel() == self.w * self.alpha * self.a):
            raise ValueError(f"datacube must be a contiguous CUDA {dtype} tensor of "
                             f"{self.w}x{self.alpha}x{self.a} elements")

    def _check_fpa(self, g):
        import torch
        if not (isinstance(g, torch.Tensor) and g.is_cuda and g.dtype == torch.float32 and
                g.is_contiguous() and g.numel() == self.xi * self.gamma):
            raise ValueError(f"FPA image must be a contiguous CUDA float32 tensor of "
                             f"{self.xi}x{self.gamma} elements")

    # -- operations -----------------------------------------------------------------
    def forward(self, f, out=None, stream=None):
        """``H f`` as an ``(xi, gamma)`` float32 tensor."""
        import torch
        self._check_cube(f)
        if out is None:
            out = torch.empty((self.xi, self.gamma), device=f.device, dtype=torch.float32)
        self._check_fpa(out)
        _check(load().ctis_forward(self._h, ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def adjoint(self, r, out=None, stream=None):
        """``H^T r`` as a ``(w, alpha, a)`` float32 tensor."""
        import torch
        self._check_fpa(r)
        if out is None:
            out = torch.empty((self.w, self.alpha, self.a), device=r.device, dtype=torch.float32)
        self._check_cube(out, torch.float32)
        _check(load().ctis_adjoint(self._h, ctypes.c_void_p(r.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def reconstruct(self, g, k: int, f=None, init: str | None = "ones", stats=False,
                    stream=None, solver: str = "em", relax: float = 1.0):
        """k EM updates (Eq. 2), or of ``solver`` 'sart' / 'smart' with
        relaxation ``relax`` (ctis_reconstruct_solver). Returns ``(f, stats)``.
        ``stats`` may be False, True (allocate) or a float64 CUDA tensor of
        ``(k+1, 4)`` to fill: rows 0..k-1 describe ``H f^(t+1)`` of each
        iteration, row k the returned f. Reusing the same f, g and stats
        tensors replays the plan's cached graph."""
        import torch
        self._check_fpa(g)
        if f is None:
            if init is None:
                raise ValueError("init=None needs an initial f")
            f = torch.empty((self.w, self.alpha, self.a), device=g.device, dtype=self._f_dtype())
        self._check_cube(f)
        flags = {"ones": CTIS_INIT_ONES, "htg": CTIS_INIT_HTG, None: 0}[init]
        st = None
        if isinstance(stats, torch.Tensor):
            st = stats
            if not (st.is_cuda and st.dtype == torch.float64 and st.is_contiguous() and
                    st.numel() >= (k + 1) * NSTATS):
                raise ValueError("stats must be a contiguous CUDA float64 tensor of (k+1)*4")
        elif stats:
            st = torch.empty((k + 1, NSTATS), device=g.device, dtype=torch.float64)
        _check(load().ctis_reconstruct_solver(
            self._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(f.data_ptr()), k, flags,
            _SOLVER[solver], float(relax),
            ctypes.c_void_p(st.data_ptr() if st is not None else 0), _stream(stream)))
        return f, st

    def index_map(self, stream=None):
        import torch
        out = torch.empty(self.w * self.alpha * self.a, device="cuda", dtype=torch.int64)
        _check(load().ctis_index_map(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def set_debug(self, drop_copies: bool = False, serial_launch: bool = False):
        """Test and measurement hooks (ctis_plan_set_debug): with
        ``drop_copies`` every bounded wait in the gather kernels runs out and
        ``check()`` raises CTIS_ERR_TIMEOUT; with ``serial_launch`` the
        projectors are plain launches instead of programmatic dependent
        launches."""
        _check(load().ctis_plan_set_debug(self._h, (1 if drop_copies else 0) |
                                          (2 if serial_launch else 0)))

    def set_profiling(self, enable: bool):
        _check(load().ctis_plan_set_profiling(self._h, int(bool(enable))))

    def kernel_times(self):
        """``{'forward': (ms_total, launches), 'adjoint': (ms_total, launches)}`` of
        the last reconstruct call made with profiling enabled (waits for it)."""
        fm, am = ctypes.c_double(), ctypes.c_double()
        fn, an = ctypes.c_int(), ctypes.c_int()
        _check(load().ctis_plan_kernel_times(self._h, ctypes.byref(fm), ctypes.byref(fn),
                                             ctypes.byref(am), ctypes.byref(an)))
        return {"forward": (fm.value, fn.value), "adjoint": (am.value, an.value)}

    def reconstruct_sharded(self, g, k: int, f=None, init: str = "ones", stats: bool = False,
                            reduce=None, stream=None):
        """k EM updates of this plan's wavelength slice (ctis_reconstruct_sharded):
        ``reduce(q)`` gets the slice's partial image q (a CUDA float32 tensor
        of the FPA's shape, a view of the plan's buffer) each iteration and
        must leave the sum over the ranks in it, on the current stream; None:
        the slice is the whole problem. Returns ``(f, stats or None)``."""
        import torch
        self._check_fpa(g)
        if f is None:
            f = torch.empty((self.w, self.alpha, self.a), device=g.device, dtype=self._f_dtype())
        self._check_cube(f)
        flags = {"ones": CTIS_INIT_ONES, "htg": CTIS_INIT_HTG, "given": 0}[init]
        st = torch.empty((k + 1, NSTATS), device=g.device, dtype=torch.float64) if stats else None
        cb = None
        if reduce is not None:
            shape = (self.xi, self.gamma)

            def _cb(q_ptr, n, ctx, strm):
                try:
                    q = _wrap_device_floats(q_ptr, int(n), g.device).view(shape)
                    reduce(q)
                    return 0
                except Exception:   # reported to the library as a failed reduction
                    return 1
            cb = REDUCE_FN(_cb)
        _check(load().ctis_reconstruct_sharded(
            self._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(f.data_ptr()), int(k), flags,
            ctypes.c_void_p(st.data_ptr() if st is not None else 0),
            cb if cb is not None else REDUCE_FN(), None, _stream(stream)))
        return f, st

    def time_launches(self, g, reps: int = 20, stream=None):
        """Average milliseconds per EM launch ``(forward, adjoint)`` over
        ``reps`` back-to-back launches of each (ctis_plan_time_launches; no
        event between the launches). Overwrites the plan's internal copies."""
        self._check_fpa(g)
        fm, am = ctypes.c_double(), ctypes.c_double()
        _check(load().ctis_plan_time_launches(self._h, ctypes.c_void_p(g.data_ptr()), int(reps),
                                              ctypes.byref(fm), ctypes.byref(am), _stream(stream)))
        return fm.value, am.value

    def check(self, stream=None):
        """Synchronise the stream and raise if a kernel reported a device-side failure."""
        _check(load().ctis_plan_check(self._h, _stream(stream)))

    def autotune(self, g, stream=None):
        """Time the EM launches over candidate work schedules (and, for the
        forward, both tile shapes) with ``g`` as the measurement and keep the
        fastest (synchronous). Returns the chosen schedules ``(forward,
        adjoint)`` (see ``schedules``; ``forward_tile`` gives the shape)."""
        self._check_fpa(g)
        _check(load().ctis_plan_autotune(self._h, ctypes.c_void_p(g.data_ptr()), _stream(stream)))
        return self.schedules()

    # -- the paper's FFT form (comparison path) ------------------------------------
    def fft_forward(self, f, out=None, stream=None):
        """``H f`` by the paper's FFT form (Eqs. 11, 13); float32 plans."""
        import torch
        self._check_cube(f, torch.float32)
        out = out if out is not None else torch.empty((self.xi, self.gamma), device=f.device)
        _check(load().ctis_fft_forward(self._h, ctypes.c_void_p(f.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def fft_adjoint(self, r, out=None, stream=None):
        """``H^T r`` by the paper's FFT form (Eqs. 14, 17); float32 plans."""
        import torch
        self._check_fpa(r)
        out = out if out is not None else torch.empty((self.w, self.alpha, self.a), device=r.device)
        _check(load().ctis_fft_adjoint(self._h, ctypes.c_void_p(r.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def fft_reconstruct(self, g, k: int, f=None, stream=None):
        """k EM updates with the FFT-form projectors (Algorithm 1), from ones
        or from ``f`` (float32, updated in place); returns f."""
        import torch
        self._check_fpa(g)
        flags = 0
        if f is None:
            f = torch.empty((self.w, self.alpha, self.a), device=g.device)
            flags = CTIS_INIT_ONES
        else:
            self._check_cube(f, torch.float32)
        _check(load().ctis_fft_reconstruct(self._h, ctypes.c_void_p(g.data_ptr()),
                                           ctypes.c_void_p(f.data_ptr()), int(k), flags,
                                           _stream(stream)))
        return f

    def set_schedule(self, forward: bool, sched):
        """Reschedule one projector: ``sched`` is ``(kind, value, skew)`` as
        ``schedules()`` reports it (kind "chunk" or "split"; value 0 with
        kind "chunk": the model's choice)."""
        kind, value, skew = sched
        if kind not in ("chunk", "split"):
            raise ValueError(f"schedule kind must be 'chunk' or 'split', got {kind!r}")
        chunk, split = (int(value), 0) if kind == "chunk" else (0, int(value))
        _check(load().ctis_plan_set_schedule(self._h, 1 if forward else 0, chunk, split, int(skew)))

    def forward_tile(self) -> str:
        """The forward's output tile shape, ``"32x32"`` or ``"32x16"`` (the
        plan's option until ``autotune`` picks the faster one)."""
        i = self.info()
        return f"{int(i['fwd_tile_w'])}x{int(i['fwd_tile_h'])}"

    def schedules(self):
        """The projectors' work schedules ``(forward, adjoint)``, each
        ``("chunk", tasks_per_item, skew)`` or ``("split", item_overhead_q,
        skew)``, skew the CTA priority skew in permille."""
        info = self.info()
        out = []
        for side in ("fwd", "adj"):
            q = int(info[side + "_split_q"])
            kind, v = ("split", q) if q > 0 else ("chunk", int(info[side + "_chunk"]))
            out.append((kind, v, int(info[side + "_skew_pm"])))
        return tuple(out)

    # -- gradients ---------------------------------------------------------------
    @property
    def nnz(self) -> int:
        return int(self.info()["nnz"])

    def set_values(self, vals):
        """Replace the stored tap values (``export_taps`` order; host array or
        tensor of nnz float32, finite and >= 0) and recompute h."""
        if hasattr(vals, "detach"):
            import torch
            vals = vals.detach().to("cpu", dtype=torch.float32).numpy()
        v = np.ascontiguousarray(vals, dtype=np.float32).ravel()
        if v.size != self.nnz:
            raise ValueError(f"expected {self.nnz} tap values, got {v.size}")
        keep, ptr = _arr(v, np.float32)
        _check(load().ctis_plan_set_values(self._h, ptr))
        self.values_version += 1

    def psf_grad(self, f, r, out=None, stream=None):
        """``d <r, H f> / d v_t`` for every stored tap t (float32, nnz)."""
        import torch
        self._check_cube(f)
        self._check_fpa(r)
        if out is None:
            out = torch.empty(self.nnz, device=r.device, dtype=torch.float32)
        if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and
                out.numel() == self.nnz):
            raise ValueError("out must be a contiguous CUDA float32 tensor of nnz elements")
        _check(load().ctis_psf_grad(self._h, ctypes.c_void_p(f.data_ptr()),
                                    ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    _stream(stream)))
        return out

    def unrolled_nll_grad(self, g, k: int, f0=None, want_df0: bool = False, stream=None):
        """Poisson NLL after k EM updates from f0 (or ones) and its gradients:
        ``(nll float64 scalar tensor, dL/dv (nnz), dL/df0 or None)``."""
        import torch
        self._check_fpa(g)
        if f0 is not None:
            self._check_cube(f0, torch.float32)
        nll = torch.empty(1, device=g.device, dtype=torch.float64)
        dval = torch.empty(self.nnz, device=g.device, dtype=torch.float32)
        df0 = (torch.empty((self.w, self.alpha, self.a), device=g.device, dtype=torch.float32)
               if want_df0 else None)
        _check(load().ctis_unrolled_nll_grad(
            self._h, ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(f0.data_ptr() if f0 is not None else 0), int(k),
            ctypes.c_void_p(nll.data_ptr()), ctypes.c_void_p(dval.data_ptr()),
            ctypes.c_void_p(df0.data_ptr() if df0 is not None else 0), _stream(stream)))
        return nll[0], dval, df0


def reconstruct_batched(plans, plan_idx, gs, k: int, fs=None, init: str | None = "ones",
                        stats=False, stream=None, solver: str = "em", relax: float = 1.0):
    """k EM updates on every frame i: plan ``plans[plan_idx[i]]``, counts
    ``gs[i]``, result in ``fs[i]`` (allocated when ``fs`` is None; read as the
    initial guess when ``init`` is None). One CUDA graph for the whole batch.
    ``solver`` / ``relax`` as in ``Plan.reconstruct`` ('em', 'sart', 'smart').
    Returns ``(fs, stats)`` with stats a ``(nframes, k+1, 4)`` float64 tensor
    when requested."""
    import torch
    nframes = len(plan_idx)
    if len(gs) != nframes:
        raise ValueError("one g per frame")
    if any(not 0 <= i < len(plans) for i in plan_idx):
        raise ValueError("plan_idx out of range")
    if fs is None:
        if init is None:
            raise ValueError("init=None needs initial fs")
        fs = [torch.empty((plans[i].w, plans[i].alpha, plans[i].a), device=gs[n].device,
                          dtype=plans[i]._f_dtype()) for n, i in enumerate(plan_idx)]
    for n, i in enumerate(plan_idx):
        plans[i]._check_fpa(gs[n])
        plans[i]._check_cube(fs[n])
    flags = {"ones": CTIS_INIT_ONES, "htg": CTIS_INIT_HTG, None: 0}[init]
    st = None
    if isinstance(stats, torch.Tensor):
        st = stats
    elif stats:
        st = torch.empty((nframes, k + 1, NSTATS), device=gs[0].device, dtype=torch.float64)
    hp = (ctypes.c_void_p * len(plans))(*[p._h for p in plans])
    idx = (ctypes.c_int * nframes)(*plan_idx)
    gp = (ctypes.c_void_p * nframes)(*[g.data_ptr() for g in gs])
    fp = (ctypes.c_void_p * nframes)(*[f.data_ptr() for f in fs])
    _check(load().ctis_reconstruct_batched_solver(
        hp, len(plans), nframes, idx, gp, fp, int(k), flags, _SOLVER[solver], float(relax),
        ctypes.c_void_p(st.data_ptr() if st is not None else 0), _stream(stream)))
    return fs, st


def fma_peak(packed: bool = False, blocks_per_sm: int = 8, threads: int = 256, iters: int = 4096,
             sms: int | None = None, reps: int = 5):
    """FP32 FMA rate of this GPU (ctis_fma_peak): TFLOP/s of the best of
    ``reps`` timed launches of ``blocks_per_sm`` CTAs of ``threads`` threads
    per SM, with the FLOP count the header states."""
    import torch
    dev = torch.cuda.current_device()
    if sms is None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * blocks_per_sm
    out = torch.empty(blocks * threads, device="cuda", dtype=torch.float32)
    st = torch.cuda.current_stream()
    lib = load()
    run = lambda: _check(lib.ctis_fma_peak(1 if packed else 0, blocks, threads, iters,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(st.cuda_stream)))
    run()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        run()
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    flops = 2.0 * blocks * threads * iters * 32 * (2 if packed else 1)
    return flops / (best * 1e-3) / 1e12


def _wrap_device_floats(ptr: int, n: int, device):
    """A torch float32 tensor viewing n floats of device memory the library
    owns (no copy); valid only during the callback that received it."""
    import torch

    class _Cuda:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (int(ptr), False),
                                    "version": 3}
    return torch.as_tensor(_Cuda(), device=device)


def shard_wavelengths(w: int, world: int, rank: int):
    """Contiguous wavelength slice [s0, s1) of rank `rank` among `world`
    ranks: sizes differ by at most one, lower ranks get the larger ones."""
    if not (0 <= rank < world) or w < world:
        raise ValueError(f"{world} ranks cannot each own wavelengths of w = {w}")
    base, extra = divmod(w, world)
    s0 = rank * base + min(rank, extra)
    return s0, s0 + base + (1 if rank < extra else 0)


def slice_psf(psf, s0: int, s1: int):
    """The calibration images of wavelengths [s0, s1) as a PSF of its own
    (psf_ptr rebased to 0): the input of a slice's plan."""
    ptr = np.asarray(psf[0], dtype=np.int64)
    lo, hi = int(ptr[s0]), int(ptr[s1])
    return ((ptr[s0:s1 + 1] - lo).astype(np.int32), np.asarray(psf[1])[lo:hi],
            np.asarray(psf[2])[lo:hi], np.asarray(psf[3])[lo:hi])
