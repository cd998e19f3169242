"""Python binding of the GB300 TV/L2 reconstruction library (``libtvcs.so``).

Thin ctypes marshalling over the C ABI declared in ``include/tvcs.h``: every
function here has the name of the C entry point it calls, converts torch
tensors or numpy arrays to raw pointers and turns negative status codes into
``TvcsError``.  All solver arithmetic runs in the library's CUDA kernels;
there is no Python or CPU fallback, and importing this module fails loudly
when the library has not been built (``python paper_1001_1774_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtvcs.so")

TVCS_OK = 0
TVCS_NOT_CONVERGED = 1
TVCS_ERR_INVALID_ARG = -1
TVCS_ERR_OOM = -2
TVCS_ERR_CUDA = -3
TVCS_ERR_TIMEOUT = -4
TVCS_ERR_DIVERGED = -5
TVCS_ERR_UNSUPPORTED = -6

TVCS_ALGO_IADM, TVCS_ALGO_FTVCS = 0, 1
TVCS_PREC_FP32, TVCS_PREC_BF16X2, TVCS_PREC_FP8_BF16 = 0, 1, 2
TVCS_INIT_ATF, TVCS_INIT_ZERO, TVCS_INIT_GIVEN = 0, 1, 2
TVCS_A_STORED, TVCS_A_REGENERATE = 0, 1
(TVCS_STATE_U, TVCS_STATE_W, TVCS_STATE_LAMBDA, TVCS_STATE_G, TVCS_STATE_R, TVCS_STATE_RHS,
 TVCS_STATE_F) = range(7)

EXPORTED = ["tvcs_default_options", "tvcs_create", "tvcs_create_partial_dct", "tvcs_solve",
            "tvcs_solve_batched",
            "tvcs_solve_continuation",
            "tvcs_destroy", "tvcs_last_error", "tvcs_get_tau", "tvcs_get_state",
            "tvcs_set_state", "tvcs_iterate", "tvcs_run_stage", "tvcs_time_stage", "tvcs_apply",
            "tvcs_apply_noalloc", "tvcs_apply_batched", "tvcs_test_hold_grid_barrier",
            "tvcs_test_gemm_shape"]


class tvcs_options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("tau", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("init", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("power_iters", ctypes.c_int), ("timeout_cycles", ctypes.c_longlong),
                ("host_loop", ctypes.c_int), ("a_mode", ctypes.c_int),
                ("batch_compact", ctypes.c_int), ("autotune", ctypes.c_int)]


class tvcs_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("stopped_by_tol", ctypes.c_int), ("rel_change", ctypes.c_double),
                ("tv", ctypes.c_double), ("resid2", ctypes.c_double),
                ("objective", ctypes.c_double), ("kkt_primal", ctypes.c_double),
                ("kkt_dual", ctypes.c_double), ("lambda_max_norm", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TvcsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("tvcs status %d: %s" % (status, message))
        self.status = status
        self.results = None   # per-problem summaries of a batched call that failed


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtvcs.so is not built (%s); run `python paper_1001_1774_gb300/build.py`"
                          % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
    H = ctypes.c_void_p
    sig = {
        "tvcs_default_options": ([ctypes.POINTER(tvcs_options)], None),
        "tvcs_create": ([ctypes.POINTER(H), vp, u64, i, i, d, d, d, ctypes.POINTER(tvcs_options)], i),
        "tvcs_create_partial_dct": ([ctypes.POINTER(H), vp, i, i, d, d, d,
                                     ctypes.POINTER(tvcs_options)], i),
        "tvcs_solve": ([H, vp, vp, ctypes.POINTER(tvcs_result)], i),
        "tvcs_solve_batched": ([vp, i, vp, vp, vp, vp], i),
        "tvcs_solve_continuation": ([H, vp, vp, vp, i, vp], i),
        "tvcs_destroy": ([H], i),
        "tvcs_last_error": ([], ctypes.c_char_p),
        "tvcs_get_tau": ([H, ctypes.POINTER(d)], i),
        "tvcs_get_state": ([H, i, vp], i),
        "tvcs_set_state": ([H, i, vp], i),
        "tvcs_iterate": ([H, i, ctypes.POINTER(tvcs_result)], i),
        "tvcs_run_stage": ([H, i], i),
        "tvcs_time_stage": ([H, i, i, ctypes.POINTER(d)], i),
        "tvcs_apply": ([H, vp, vp, vp, vp], i),
        "tvcs_apply_noalloc": ([vp, i, i, vp, vp, vp, vp, vp], i),
        "tvcs_apply_batched": ([H, i, vp, vp, vp, vp], i),
        "tvcs_test_hold_grid_barrier": ([H, i], i),
        "tvcs_test_gemm_shape": ([H, i, i, i, i], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def _check(status: int) -> int:
    if status < 0:
        raise TvcsError(status, _lib.tvcs_last_error().decode(errors="replace"))
    return status


def _ptr(x, count: int | None = None, writable: bool = False):
    """Raw pointer of a contiguous float32 torch tensor or numpy array (host or device)."""
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float32 or not x.is_contiguous():
                raise TypeError("expected a contiguous float32 tensor")
            if count is not None and x.numel() != count:
                raise ValueError("expected %d elements, got %d" % (count, x.numel()))
            return ctypes.c_void_p(x.data_ptr())
    except ImportError:
        pass
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags.c_contiguous:
            raise TypeError("expected a C-contiguous float32 array")
        if writable and not x.flags.writeable:
            raise TypeError("output array is read-only")
        if count is not None and x.size != count:
            raise ValueError("expected %d elements, got %d" % (count, x.size))
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError("unsupported array type %r" % type(x))


def _ready(*arrays) -> None:
    """The library orders its device work on the handle's stream, which does not
    wait for other streams.  Before a call that reads or writes torch CUDA tensors,
    finish the work queued on torch's current stream of each device involved (the
    tensors' producers, and pending readers of output buffers): once per device."""
    try:
        import torch
    except ImportError:
        return
    devs = set()
    for a in arrays:
        for x in (a if isinstance(a, (list, tuple)) else (a,)):
            if isinstance(x, torch.Tensor) and x.is_cuda:
                devs.add(x.device)
    for d in devs:
        torch.cuda.current_stream(d).synchronize()


def tvcs_default_options() -> tvcs_options:
    o = tvcs_options()
    _lib.tvcs_default_options(ctypes.byref(o))
    return o


class Handle:
    """Owns a tvcs_handle; also records the sizes for argument checks."""

    def __init__(self, ptr: int, m: int, n: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.m = m
        self.n = n
        self.N = n * n
        self._keep = []

    def __del__(self):
        try:
            if self.ptr and self.ptr.value:
                _lib.tvcs_destroy(self.ptr)
                self.ptr = ctypes.c_void_p(None)
        except Exception:
            pass


def tvcs_create(A, seed: int, m: int, n: int, mu: float, beta: float, tol: float,
                opt: tvcs_options | None = None) -> Handle:
    h = ctypes.c_void_p()
    _ready(A)
    pa = _ptr(A, m * n * n) if A is not None else None
    _check(_lib.tvcs_create(ctypes.byref(h), pa, int(seed) & (2**64 - 1), int(m), int(n),
                            float(mu), float(beta), float(tol),
                            ctypes.byref(opt) if opt is not None else None))
    return Handle(h.value, m, n)


def tvcs_create_partial_dct(rows, n: int, mu: float, beta: float, tol: float,
                            opt: tvcs_options | None = None) -> Handle:
    """Partial-DCT encoder: the coefficients `rows` (indices k1 n + k2) of the
    orthonormal 2D DCT of the n x n image."""
    r = np.ascontiguousarray(rows, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.tvcs_create_partial_dct(ctypes.byref(h), r.ctypes.data, int(r.size), int(n),
                                        float(mu), float(beta), float(tol),
                                        ctypes.byref(opt) if opt is not None else None))
    return Handle(h.value, int(r.size), n)


def tvcs_destroy(h: Handle) -> None:
    if h.ptr and h.ptr.value:
        _check(_lib.tvcs_destroy(h.ptr))
        h.ptr = ctypes.c_void_p(None)


def tvcs_solve(h: Handle, f, u) -> tvcs_result:
    res = tvcs_result()
    _ready(f, u)
    _check(_lib.tvcs_solve(h.ptr, _ptr(f, h.m), _ptr(u, h.N, True), ctypes.byref(res)))
    return res


def tvcs_solve_batched(hs, f_list, u_list, mu=None) -> list:
    count = len(hs)
    assert len(f_list) == count and len(u_list) == count
    _ready(f_list, u_list)
    harr = (ctypes.c_void_p * count)(*[h.ptr.value for h in hs])
    farr = (ctypes.c_void_p * count)(*[_ptr(f, h.m).value for f, h in zip(f_list, hs)])
    uarr = (ctypes.c_void_p * count)(*[_ptr(u, h.N, True).value for u, h in zip(u_list, hs)])
    muarr = (ctypes.c_double * count)(*mu) if mu is not None else None
    res = (tvcs_result * count)()
    try:
        _check(_lib.tvcs_solve_batched(harr, count, farr, uarr, muarr, res))
    except TvcsError as e:
        e.results = list(res)
        raise
    return list(res)


def tvcs_solve_continuation(h: Handle, f, u, betas) -> list:
    """Continuation in beta; returns one tvcs_result per stage."""
    n = len(betas)
    barr = (ctypes.c_double * n)(*[float(b) for b in betas])
    res = (tvcs_result * n)()
    _ready(f, u)
    _check(_lib.tvcs_solve_continuation(h.ptr, _ptr(f, h.m), _ptr(u, h.N, True), barr, n, res))
    return list(res)


def tvcs_get_tau(h: Handle) -> float:
    t = ctypes.c_double()
    _check(_lib.tvcs_get_tau(h.ptr, ctypes.byref(t)))
    return t.value


_STATE_SIZE = {TVCS_STATE_U: lambda h: h.N, TVCS_STATE_W: lambda h: 2 * h.N,
               TVCS_STATE_LAMBDA: lambda h: 2 * h.N, TVCS_STATE_G: lambda h: h.N,
               TVCS_STATE_R: lambda h: h.m, TVCS_STATE_RHS: lambda h: h.N,
               TVCS_STATE_F: lambda h: h.m}


def tvcs_get_state(h: Handle, which: int, dst) -> None:
    _ready(dst)
    _check(_lib.tvcs_get_state(h.ptr, which, _ptr(dst, _STATE_SIZE[which](h), True)))


def tvcs_set_state(h: Handle, which: int, src) -> None:
    _ready(src)
    _check(_lib.tvcs_set_state(h.ptr, which, _ptr(src, _STATE_SIZE[which](h))))


def tvcs_iterate(h: Handle, iters: int) -> tvcs_result:
    res = tvcs_result()
    _check(_lib.tvcs_iterate(h.ptr, int(iters), ctypes.byref(res)))
    return res


def tvcs_run_stage(h: Handle, stage: int) -> None:
    _check(_lib.tvcs_run_stage(h.ptr, int(stage)))


def tvcs_time_stage(h: Handle, stage: int, reps: int) -> float:
    ms = ctypes.c_double()
    _check(_lib.tvcs_time_stage(h.ptr, int(stage), int(reps), ctypes.byref(ms)))
    return ms.value


def tvcs_apply(h: Handle, x, y, r, g) -> None:
    _ready(x, y, r, g)
    _check(_lib.tvcs_apply(h.ptr, _ptr(x, h.N), _ptr(y, h.m) if y is not None else None,
                           _ptr(r, h.m, True), _ptr(g, h.N, True)))


def tvcs_apply_noalloc(A, m: int, n: int, x, y, r, g, stream: int | None = None) -> None:
    """r = A x - y and g = A^T r from device tensors, allocating no device memory
    (see include/tvcs.h for who needs this and its limits).  stream: a raw
    cudaStream_t; None runs on torch's current stream of the current device, so
    the call is ordered after the work that produced the inputs there."""
    N = n * n
    if stream is None:
        import torch
        stream = int(torch.cuda.current_stream().cuda_stream)
    _check(_lib.tvcs_apply_noalloc(_ptr(A, m * N), int(m), int(n), _ptr(x, N),
                                   _ptr(y, m) if y is not None else None, _ptr(r, m, True),
                                   _ptr(g, N, True), ctypes.c_void_p(stream or 0)))


def tvcs_apply_batched(h: Handle, count: int, X, Y, R, G) -> None:
    """R = A X - Y and G = A^T R for `count` images (rows of X, Y, R, G)."""
    _ready(X, Y, R, G)
    _check(_lib.tvcs_apply_batched(h.ptr, int(count), _ptr(X, count * h.N),
                                   _ptr(Y, count * h.m) if Y is not None else None,
                                   _ptr(R, count * h.m, True), _ptr(G, count * h.N, True)))


def tvcs_test_hold_grid_barrier(h: Handle, extra: int) -> None:
    """Timeout test hook: the product kernel's grid barrier waits for `extra`
    arrivals that never come (0 restores normal operation)."""
    _check(_lib.tvcs_test_hold_grid_barrier(h.ptr, int(extra)))


def tvcs_test_gemm_shape(h: Handle, grid1: int, pair1: int, grid2: int, pair2: int) -> None:
    """Test hook: launch shape of the two batched GEMMs (blocks, and 1 for CTA
    pairs); grid1 = grid2 = 0 returns the choice to the tuner."""
    _check(_lib.tvcs_test_gemm_shape(h.ptr, int(grid1), int(pair1), int(grid2), int(pair2)))


def tvcs_last_error() -> str:
    return _lib.tvcs_last_error().decode(errors="replace")


def get_state(h: Handle, which: int) -> np.ndarray:
    """Convenience: a host numpy copy of one state array."""
    out = np.empty(_STATE_SIZE[which](h), dtype=np.float32)
    tvcs_get_state(h, which, out)
    return out
