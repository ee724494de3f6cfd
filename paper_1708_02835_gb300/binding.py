"""ctypes binding of libegs.so with the same names as the C ABI.

Tensors are torch CUDA tensors (device pointers are passed as-is) or, where
the C ABI accepts host memory, NumPy arrays / CPU tensors.  The stream is
torch's current CUDA stream unless one is given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

EGS_OK, EGS_ERR_ARG, EGS_ERR_NOT_PD, EGS_ERR_OOM, EGS_ERR_CUDA, EGS_ERR_TIMEOUT, EGS_ERR_BUSY, \
    EGS_ERR_UNIMPLEMENTED, EGS_ERR_INACCURATE = range(9)
EGS_FP64, EGS_MIX_FP32, EGS_MIX_TF32, EGS_MIX_BF16 = range(4)
PRECISIONS = {"fp64": EGS_FP64, "fp32": EGS_MIX_FP32, "tf32": EGS_MIX_TF32, "bf16": EGS_MIX_BF16}

_STATUS_NAMES = {0: "EGS_OK", 1: "EGS_ERR_ARG", 2: "EGS_ERR_NOT_PD", 3: "EGS_ERR_OOM", 4: "EGS_ERR_CUDA",
                 5: "EGS_ERR_TIMEOUT", 6: "EGS_ERR_BUSY", 7: "EGS_ERR_UNIMPLEMENTED", 8: "EGS_ERR_INACCURATE"}


class EgsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class NotPositiveDefinite(EgsError):
    pass


class MixedInaccurate(EgsError):
    """The mixed-precision factor was too inexact for Sigma(theta)."""


class egs_info(ctypes.Structure):
    _fields_ = [("loglik", ctypes.c_double), ("logdet", ctypes.c_double), ("quad", ctypes.c_double),
                ("fail_index", ctypes.c_int64), ("fail_tile", ctypes.c_int64), ("tile", ctypes.c_int32),
                ("band", ctypes.c_int32), ("launches", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("quad_unrefined", ctypes.c_double), ("ms_generate", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_solve", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_potrf", ctypes.c_double),
                ("ms_trsm", ctypes.c_double), ("ms_update", ctypes.c_double), ("ms_trsv", ctypes.c_double),
                ("ms_update_f64", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class egs_opts(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("band", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("distance", ctypes.c_int32), ("xband", ctypes.c_int32)]


class egs_trace_rec(ctypes.Structure):
    _fields_ = [("kclass", ctypes.c_int32), ("step", ctypes.c_int32), ("stream", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double)]


TRACE_CLASSES = ("generate", "potrf", "trsm", "update", "solve", "other", "update_f64")


class egs_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("band", ctypes.c_int32), ("fallback_fp64", ctypes.c_int32), ("xband", ctypes.c_int32)]


class egs_serve_stats(ctypes.Structure):
    _fields_ = [("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("evals_per_s", ctypes.c_double), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("inflight_peak", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t), ("fallbacks", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# egs_set_allocator's hook types: alloc(bytes, stream, ctx) -> device pointer,
# free(ptr, bytes, stream, ctx)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
# Every pair of ctypes callbacks ever installed stays alive for the life of
# the process: a server or batch keeps calling the hooks it was created with
# after the allocator has been replaced.
_hooks_alive = []


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libegs.so (building it first if asked).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libegs.so is not built (%s); run paper_1708_02835_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    c = ctypes
    vp, i64, i32, pd = c.c_void_p, c.c_int64, c.c_int32, c.POINTER(c.c_double)
    sig = {
        "egs_last_error": (c.c_char_p, []),
        "egs_version": (c.c_char_p, []),
        "egs_default_tile": (i32, [i64, c.c_int]),
        "egs_tiles_bytes": (c.c_size_t, [i64, i32, c.c_int, i32]),
        "egs_loglik_workspace_bytes": (c.c_size_t, [i64, i32, c.c_int, i32]),
        "egs_matern_tiles": (c.c_int, [vp, i64, pd, i32, c.c_int, i32, vp, vp]),
        "egs_potrf_tiles": (c.c_int, [vp, i64, i32, c.POINTER(i64), vp]),
        "egs_trsv_tiles": (c.c_int, [vp, i64, i32, vp, vp, pd, pd, vp]),
        "egs_trsv_tiles_noalloc": (c.c_int, [vp, i64, i32, vp, vp, pd, pd, vp]),
        "egs_simulate": (c.c_int, [vp, vp, pd, i64, i32, vp, vp]),
        "egs_loglik": (c.c_int, [vp, vp, pd, i64, c.c_int, pd, c.POINTER(egs_info), vp]),
        "egs_loglik_ex": (c.c_int, [vp, vp, pd, i64, c.c_int, c.POINTER(egs_opts), pd, c.POINTER(egs_info), vp]),
        "egs_tc_gemm_test": (c.c_int, [vp, vp, i32, i32, i32, c.c_int, vp, vp]),
        "egs_tc_gemm_test_withhold": (c.c_int, [vp, vp, i32, i32, i32, c.c_int, vp, i64, vp]),
        "egs_ozaki_gemm_test": (c.c_int, [vp, vp, i32, i32, i32, vp, vp]),
        "egs_batch_create": (c.c_int, [i32, c.POINTER(i64), i32, c.c_int, c.POINTER(vp)]),
        "egs_batch_run": (c.c_int, [vp, c.POINTER(vp), c.POINTER(vp), pd, pd, c.POINTER(c.c_int), vp]),
        "egs_batch_destroy": (c.c_int, [vp]),
        "egs_batch_launches": (i32, [vp]),
        "egs_batch_tile": (i32, [vp]),
        "egs_batch_workspace_bytes": (c.c_size_t, [vp]),
        "egs_loglik_batched": (c.c_int, [i32, c.POINTER(i64), c.POINTER(vp), c.POINTER(vp), pd, c.c_int, pd,
                                         c.POINTER(c.c_int), vp]),
        "egs_loglik_ind": (c.c_int, [vp, vp, pd, i64, i32, i32, pd, c.POINTER(egs_info), vp]),
        "egs_batch_autotune": (c.c_int, [i32, c.POINTER(i64), c.POINTER(vp), c.POINTER(vp), pd, c.c_int,
                                         c.POINTER(i32), pd, vp]),
        "egs_batch_tuned_tile": (i32, [i64, c.c_int]),
        "egs_batch_tasks": (i64, [vp]),
        "egs_batch_set_wait_limit": (c.c_int, [vp, i64, i64]),
        "egs_predict": (c.c_int, [vp, vp, i64, vp, i64, pd, c.c_int, c.POINTER(egs_opts), vp, c.POINTER(egs_info),
                                  vp]),
        "egs_trace_last": (c.c_int, [c.POINTER(egs_trace_rec), i64, c.POINTER(i64)]),
        "egs_serve_create": (c.c_int, [c.POINTER(egs_serve_config), c.POINTER(vp)]),
        "egs_serve_add_field": (c.c_int, [vp, vp, vp, i64, c.POINTER(i64)]),
        "egs_serve_submit": (c.c_int, [vp, i64, pd, c.c_int, c.POINTER(i64)]),
        "egs_serve_wait": (c.c_int, [vp, i64, i32, pd, c.POINTER(egs_info)]),
        "egs_serve_stats": (c.c_int, [vp, c.POINTER(egs_serve_stats)]),
        "egs_serve_destroy": (c.c_int, [vp]),
        "egs_set_allocator": (c.c_int, [_ALLOC_FN, _FREE_FN, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != EGS_OK:
        msg = load_library().egs_last_error().decode()
        if status == EGS_ERR_NOT_PD:
            raise NotPositiveDefinite(status, msg)
        if status == EGS_ERR_INACCURATE:
            raise MixedInaccurate(status, msg)
        raise EgsError(status, msg)


def _ptr(t):
    """Device or host address of a torch tensor or NumPy array (contiguous)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _theta(theta):
    th = (ctypes.c_double * 3)(*[float(v) for v in theta])
    return ctypes.cast(th, ctypes.POINTER(ctypes.c_double)), th


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def egs_last_error() -> str:
    return load_library().egs_last_error().decode()


def egs_set_allocator(alloc=None, free=None):
    """Route the library's device allocations through the caller's functions:
    alloc(nbytes, stream) returns a device pointer (an int; 0 when it cannot),
    usable in stream order on stream (a cudaStream_t as an int, 0 = legacy);
    free(ptr, nbytes, stream) returns it.  Both None restores the library's
    own cudaMallocAsync.  The library may call them from its serving thread,
    and servers and batches keep the hooks they were created with (the
    callbacks are therefore never released)."""
    lib = load_library()
    if alloc is None and free is None:
        _check(lib.egs_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        return
    if alloc is None or free is None:
        _check(lib.egs_set_allocator(_ALLOC_FN(lambda n, st, c: None) if alloc else _ALLOC_FN(),
                                     _FREE_FN(lambda p, n, st, c: None) if free else _FREE_FN(), None))
        return

    def a(nbytes, stream, ctx):
        return alloc(int(nbytes), int(stream or 0)) or None

    def f(ptr, nbytes, stream, ctx):
        free(int(ptr), int(nbytes), int(stream or 0))

    hooks = (_ALLOC_FN(a), _FREE_FN(f))
    _hooks_alive.append(hooks)
    _check(lib.egs_set_allocator(hooks[0], hooks[1], None))


def use_torch_allocator():
    """egs_set_allocator with PyTorch's caching allocator on the current device."""
    import torch

    dev = torch.cuda.current_device()

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, dev, stream)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    egs_set_allocator(alloc, free)


def egs_trace_last() -> list:
    """Per-launch trace of this thread's last egs_loglik_ex(timing=3) call:
    a list of (class name, step, stream, start_ms, end_ms) in enqueue order."""
    lib = load_library()
    cnt = ctypes.c_int64(0)
    _check(lib.egs_trace_last(None, 0, ctypes.byref(cnt)))
    buf = (egs_trace_rec * max(cnt.value, 1))()
    _check(lib.egs_trace_last(buf, cnt.value, ctypes.byref(cnt)))
    return [(TRACE_CLASSES[r.kclass], r.step, r.stream, r.start_ms, r.end_ms) for r in buf[:cnt.value]]


def egs_version() -> str:
    return load_library().egs_version().decode()


def egs_default_tile(n: int, precision="fp64") -> int:
    return load_library().egs_default_tile(n, _prec(precision))


def egs_tiles_bytes(n: int, tile: int, precision="fp64", band: int = 2) -> int:
    return load_library().egs_tiles_bytes(n, tile, _prec(precision), band)


def egs_loglik_workspace_bytes(n: int, tile: int = 0, precision="fp64", band: int = 2) -> int:
    return load_library().egs_loglik_workspace_bytes(n, tile, _prec(precision), band)


def egs_matern_tiles(locs, n: int, theta, tile: int, tiles, precision="fp64", band: int = 2, stream=None):
    """Sigma(theta) (Eq. 2) into the lower-tile layout (asynchronous)."""
    tp, _keep = _theta(theta)
    _check(load_library().egs_matern_tiles(_ptr(locs), n, tp, tile, _prec(precision), band, _ptr(tiles),
                                           _stream(stream)))


def egs_potrf_tiles(tiles, n: int, tile: int, stream=None) -> int:
    """Tile Cholesky in place; returns -1 or raises NotPositiveDefinite."""
    fi = ctypes.c_int64(-1)
    _check(load_library().egs_potrf_tiles(_ptr(tiles), n, tile, ctypes.byref(fi), _stream(stream)))
    return fi.value


def egs_trsv_tiles(tiles, n: int, tile: int, z, y, stream=None) -> tuple:
    """Forward solve L y = z; returns (logdet, quad)."""
    ld, q = ctypes.c_double(), ctypes.c_double()
    _check(load_library().egs_trsv_tiles(_ptr(tiles), n, tile, _ptr(z), _ptr(y), ctypes.byref(ld), ctypes.byref(q),
                                         _stream(stream)))
    return ld.value, q.value


def egs_trsv_tiles_noalloc(tiles, n: int, tile: int, z, y, stream=None) -> tuple:
    """egs_trsv_tiles with its scratch in the library's fixed device array
    (no allocation); returns (logdet, quad)."""
    ld, q = ctypes.c_double(), ctypes.c_double()
    _check(load_library().egs_trsv_tiles_noalloc(_ptr(tiles), n, tile, _ptr(z), _ptr(y), ctypes.byref(ld),
                                                 ctypes.byref(q), _stream(stream)))
    return ld.value, q.value


DISTANCES = {"euclidean": 0, "great_circle": 1}


def egs_loglik_ex(locs, z, theta, n: int, precision="fp64", tile: int = 0, band: int = 0, refine: int = 0,
                  timing: int = 0, workspace=None, stream=None, distance="euclidean", xband: int = 0) -> tuple:
    """One evaluation of Eq. 1; returns (loglik, info dict).  distance
    "great_circle": locations are (longitude, latitude) in degrees.  xband
    (FP32 mode): FP64-accurate updates for tiles with i - j < xband."""
    tp, _keep = _theta(theta)
    opts = egs_opts(tile=tile, band=band, refine=refine, timing=int(timing),
                    workspace=_ptr(workspace) if workspace is not None else None,
                    workspace_bytes=(workspace.numel() * workspace.element_size()) if workspace is not None else 0,
                    distance=DISTANCES[distance], xband=int(xband))
    out = ctypes.c_double()
    info = egs_info()
    st = load_library().egs_loglik_ex(_ptr(locs), _ptr(z), tp, n, _prec(precision), ctypes.byref(opts),
                                      ctypes.byref(out), ctypes.byref(info), _stream(stream))
    _check(st)
    return out.value, info.as_dict()


def egs_simulate(locs, e, theta, n: int, z, tile: int = 0, stream=None):
    """Algorithm 1 on the GPU: z = L e with Sigma(theta) = L L^T (FP64)."""
    tp, _keep = _theta(theta)
    _check(load_library().egs_simulate(_ptr(locs), _ptr(e), tp, n, tile, _ptr(z), _stream(stream)))


def egs_loglik(locs, z, theta, n: int, precision="fp64", stream=None) -> float:
    """One evaluation of Eq. 1 with default options; returns l(theta)."""
    tp, _keep = _theta(theta)
    out = ctypes.c_double()
    info = egs_info()
    _check(load_library().egs_loglik(_ptr(locs), _ptr(z), tp, n, _prec(precision), ctypes.byref(out),
                                     ctypes.byref(info), _stream(stream)))
    return out.value


def egs_tc_gemm_test(A, B, C, precision="tf32", stream=None):
    """C = A B^T on the tcgen05 pipeline (A: M x K, B: N x K, C: M x N FP32)."""
    M, K = A.shape
    N = B.shape[0]
    _check(load_library().egs_tc_gemm_test(_ptr(A), _ptr(B), M, N, K, _prec(precision), _ptr(C), _stream(stream)))


def egs_tc_gemm_test_withhold(A, B, C, precision="tf32", withhold_stage=0, stream=None):
    """egs_tc_gemm_test with one ring stage's loads never issued: raises
    EgsError(EGS_ERR_TIMEOUT) once the bounded wait for it runs out."""
    M, K = A.shape
    N = B.shape[0]
    _check(load_library().egs_tc_gemm_test_withhold(_ptr(A), _ptr(B), M, N, K, _prec(precision), _ptr(C),
                                                    int(withhold_stage), _stream(stream)))


def egs_ozaki_gemm_test(A, B, C, stream=None):
    """C = A B^T (FP64) by exact BF16 slicing on tcgen05 (A: M x K, B: N x K)."""
    M, K = A.shape
    N = B.shape[0]
    _check(load_library().egs_ozaki_gemm_test(_ptr(A), _ptr(B), M, N, K, _ptr(C), _stream(stream)))


def egs_predict(locs_obs, z_obs, n: int, locs_new, m: int, theta, z_new, precision="fp64", tile: int = 0,
                band: int = 0, refine: int = 0, stream=None, distance="euclidean") -> dict:
    """Kriging prediction Z_1 = Sigma_12 Sigma_22^-1 Z_2 (Eq. 5, Algorithm 3) into z_new; returns the info dict."""
    tp, _keep = _theta(theta)
    opts = egs_opts(tile=tile, band=band, refine=refine, distance=DISTANCES[distance])
    info = egs_info()
    _check(load_library().egs_predict(_ptr(locs_obs), _ptr(z_obs), n, _ptr(locs_new), m, tp, _prec(precision),
                                      ctypes.byref(opts), _ptr(z_new), ctypes.byref(info), _stream(stream)))
    return info.as_dict()


def egs_loglik_ind(locs, z, theta, n: int, tile: int = 0, super_tiles: int = 1, stream=None):
    """IND approximation (Section 6.8): l summed over diagonal super tiles; returns (l, info)."""
    tp, _keep = _theta(theta)
    out = ctypes.c_double()
    info = egs_info()
    _check(load_library().egs_loglik_ind(_ptr(locs), _ptr(z), tp, n, tile, super_tiles, ctypes.byref(out),
                                         ctypes.byref(info), _stream(stream)))
    return out.value, info.as_dict()


class egs_batch:
    """A planned batch of independent problems (sizes fixed at creation)."""

    def __init__(self, ns, tile: int = 0, precision="fp64"):
        lib = load_library()
        self.ns = [int(v) for v in ns]
        arr = (ctypes.c_int64 * len(self.ns))(*self.ns)
        h = ctypes.c_void_p()
        _check(lib.egs_batch_create(len(self.ns), arr, int(tile), _prec(precision), ctypes.byref(h)))
        self._h = h

    @property
    def launches(self) -> int:
        return load_library().egs_batch_launches(self._h)

    @property
    def tile(self) -> int:
        return load_library().egs_batch_tile(self._h)

    @property
    def workspace_bytes(self) -> int:
        return load_library().egs_batch_workspace_bytes(self._h)

    @property
    def tasks(self) -> int:
        """Tasks of the persistent launch (0 for a step-synchronous batch)."""
        return load_library().egs_batch_tasks(self._h)

    def set_wait_limit(self, limit_ns: int, withhold_task: int = -1):
        """Bound of every dependency wait of the persistent launch; a task
        whose completion is withheld (failure tests), or -1."""
        _check(load_library().egs_batch_set_wait_limit(self._h, int(limit_ns), int(withhold_task)))

    def run(self, locs, z, thetas, stream=None, raise_on_not_pd=False):
        """locs[i], z[i]: per-problem arrays (device tensors or host arrays);
        thetas: nprob x 3.  Returns (loglik array, status array)."""
        lib = load_library()
        npb = len(self.ns)
        lp = (ctypes.c_void_p * npb)(*[_ptr(a) for a in locs])
        zp = (ctypes.c_void_p * npb)(*[_ptr(a) for a in z])
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(npb, 3))
        out = np.empty(npb)
        stat = (ctypes.c_int * npb)()
        st = lib.egs_batch_run(self._h, lp, zp, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stat, _stream(stream))
        # per-problem failures (not positive definite, mixed factor too
        # inexact) are reported in the status array unless asked to raise
        if st != EGS_OK and (st not in (EGS_ERR_NOT_PD, EGS_ERR_INACCURATE) or raise_on_not_pd):
            _check(st)
        return out, np.array(list(stat))

    def close(self):
        if self._h:
            load_library().egs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_inputs(locs, z, thetas):
    npb = len(locs)
    lp = (ctypes.c_void_p * npb)(*[_ptr(a) for a in locs])
    zp = (ctypes.c_void_p * npb)(*[_ptr(a) for a in z])
    th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(npb, 3))
    return lp, zp, th


def egs_batch_autotune(ns, locs, z, thetas, precision="fp64", stream=None) -> tuple:
    """Time tiles 64 / 128 / 256 on these inputs; the library keeps the best
    for egs_batch(tile=0).  Returns (best tile, {tile: ms})."""
    lib = load_library()
    npb = len(ns)
    arr = (ctypes.c_int64 * npb)(*[int(v) for v in ns])
    lp, zp, th = _batch_inputs(locs, z, thetas)
    best = ctypes.c_int32(0)
    ms = (ctypes.c_double * 3)()
    _check(lib.egs_batch_autotune(npb, arr, lp, zp, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  _prec(precision), ctypes.byref(best), ms, _stream(stream)))
    return best.value, {64: ms[0], 128: ms[1], 256: ms[2]}


def egs_batch_tuned_tile(nmax: int, precision="fp64") -> int:
    return load_library().egs_batch_tuned_tile(int(nmax), _prec(precision))


def egs_loglik_batched(locs, z, thetas, ns, precision="fp64", stream=None):
    """One-shot batched evaluation; returns (loglik array, status array)."""
    b = egs_batch(ns, 0, precision)
    try:
        return b.run(locs, z, thetas, stream)
    finally:
        b.close()


class egs_server:
    """Serving loop (C ABI egs_serve_*): resident fields, budgeted admission."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 4, tile: int = 0, band: int = 0,
                 fallback_fp64: bool = False, xband: int = 0):
        cfg = egs_serve_config(hbm_budget_bytes=int(hbm_budget_bytes), max_inflight=int(max_inflight),
                               tile=int(tile), band=int(band), fallback_fp64=int(bool(fallback_fp64)),
                               xband=int(xband))
        h = ctypes.c_void_p()
        _check(load_library().egs_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def add_field(self, locs, z, n: int) -> int:
        fid = ctypes.c_int64()
        _check(load_library().egs_serve_add_field(self._h, _ptr(locs), _ptr(z), int(n), ctypes.byref(fid)))
        return fid.value

    def submit(self, field_id: int, theta, precision="fp64") -> int:
        tp, _keep = _theta(theta)
        t = ctypes.c_int64()
        _check(load_library().egs_serve_submit(self._h, int(field_id), tp, _prec(precision), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        out = ctypes.c_double()
        info = egs_info()
        st = load_library().egs_serve_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(out), ctypes.byref(info))
        _check(st)
        return out.value, info.as_dict()

    def stats(self) -> dict:
        s = egs_serve_stats()
        _check(load_library().egs_serve_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self._h:
            load_library().egs_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
