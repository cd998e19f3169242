"""FP64 CPU oracle for TV/L2 reconstruction from random projections.

TEST INFRASTRUCTURE ONLY: a plain binary64 restatement of Xiao & Yang's
Algorithm 1 (FTVCS) and Algorithm 2 (IADM) in C (``tvcs_oracle.c``), loaded
through ctypes.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this package; the GPU library never does, and the two
share no code.  Functions whose result has no independent pin would say
"parity unpinned" here; every function below is pinned by a test in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvcs_oracle.c")
_HDR = os.path.join(_HERE, "tvcs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

IADM, FTVCS = 0, 1
INIT_ATF, INIT_ZERO, INIT_GIVEN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, binary64, OpenMP, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("mu", ctypes.c_double),
                ("beta", ctypes.c_double), ("tau", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("algo", ctypes.c_int), ("w_sign", ctypes.c_int),
                ("init", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("stopped_by_tol", ctypes.c_int),
                ("rel_change", ctypes.c_double), ("tv", ctypes.c_double),
                ("resid2", ctypes.c_double), ("objective", ctypes.c_double),
                ("atv", ctypes.c_double), ("kkt_primal", ctypes.c_double),
                ("kkt_dual", ctypes.c_double), ("lambda_max_norm", ctypes.c_double),
                ("lambda_align", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            sig = {
                "oracle_D": ([i, vp, vp, vp], None),
                "oracle_Dt": ([i, vp, vp, vp], None),
                "oracle_shrink": ([i, d, vp, vp, vp, vp], None),
                "oracle_dtd_eigs": ([i, vp], None),
                "oracle_dft2": ([i, i, vp, vp], None),
                "oracle_usolve": ([i, d, vp, vp], None),
                "oracle_Au": ([i, i64, vp, vp, vp, vp], None),
                "oracle_At": ([i, i64, vp, vp, vp], None),
                "oracle_lambda_max": ([i, i64, vp, i], d),
                "oracle_tv": ([i, vp], d),
                "oracle_solve": ([ctypes.POINTER(_Params), vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                  ctypes.POINTER(_Info)], i),
                "oracle_kkt": ([ctypes.POINTER(_Params), vp, vp, vp, vp, vp,
                                ctypes.POINTER(_Info)], None),
                "oracle_num_threads": ([], i),
                "oracle_set_num_threads": ([i], None),
                "oracle_dct2": ([i, i, vp, vp], None),
                "oracle_dct_Au": ([i, i, vp, vp, vp, vp], None),
                "oracle_dct_At": ([i, i, vp, vp, vp], None),
                "oracle_solve_dct": ([ctypes.POINTER(_Params), vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      ctypes.POINTER(_Info)], i),
                "oracle_kkt_dct": ([ctypes.POINTER(_Params), vp, vp, vp, vp, vp,
                                    ctypes.POINTER(_Info)], None),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _f64(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(k: int) -> None:
    """Threads of the oracle's parallel loops from now on (results do not depend on it)."""
    _load().oracle_set_num_threads(int(k))


def D(u: np.ndarray):
    """Forward differences (D1 u, D2 u) with periodic boundary, each (n, n)."""
    u = _f64(u)
    n = u.shape[0]
    d1 = np.empty((n, n)); d2 = np.empty((n, n))
    _load().oracle_D(n, u.ctypes.data, d1.ctypes.data, d2.ctypes.data)
    return d1, d2


def Dt(y1: np.ndarray, y2: np.ndarray) -> np.ndarray:
    y1 = _f64(y1); y2 = _f64(y2)
    n = y1.shape[0]
    out = np.empty((n, n))
    _load().oracle_Dt(n, y1.ctypes.data, y2.ctypes.data, out.ctypes.data)
    return out


def shrink(z1, z2, t: float):
    z1 = _f64(z1).ravel(); z2 = _f64(z2).ravel()
    w1 = np.empty_like(z1); w2 = np.empty_like(z2)
    _load().oracle_shrink(z1.size, t, z1.ctypes.data, z2.ctypes.data, w1.ctypes.data,
                          w2.ctypes.data)
    return w1, w2


def dtd_eigs(n: int) -> np.ndarray:
    lam = np.empty((n, n))
    _load().oracle_dtd_eigs(n, lam.ctypes.data)
    return lam


def dft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    x = np.asarray(x)
    n = x.shape[0]
    re = np.ascontiguousarray(x.real, dtype=np.float64).copy()
    im = np.ascontiguousarray(x.imag if np.iscomplexobj(x) else np.zeros_like(re),
                              dtype=np.float64).copy()
    _load().oracle_dft2(n, int(inverse), re.ctypes.data, im.ctypes.data)
    return re + 1j * im


def usolve(b: np.ndarray, c: float) -> np.ndarray:
    """Solve (D^T D + c I) u = b (eqs. (eqnorm)/(eqnorm11))."""
    b = _f64(b)
    n = b.shape[0]
    u = np.empty((n, n))
    _load().oracle_usolve(n, c, b.ctypes.data, u.ctypes.data)
    return u


def Au(A: np.ndarray, u: np.ndarray, f: np.ndarray | None = None) -> np.ndarray:
    A = _f32(A)
    m, N = A.shape
    u = _f64(u).ravel()
    r = np.empty(m)
    fk = _f32(f) if f is not None else None
    _load().oracle_Au(m, N, A.ctypes.data, u.ctypes.data,
                      fk.ctypes.data if fk is not None else None, r.ctypes.data)
    return r


def At(A: np.ndarray, r: np.ndarray) -> np.ndarray:
    A = _f32(A)
    m, N = A.shape
    r = _f64(r).ravel()
    g = np.empty(N)
    _load().oracle_At(m, N, A.ctypes.data, r.ctypes.data, g.ctypes.data)
    return g


def lambda_max(A: np.ndarray, iters: int = 100) -> float:
    A = _f32(A)
    m, N = A.shape
    return float(_load().oracle_lambda_max(m, N, A.ctypes.data, iters))


def default_tau(A: np.ndarray, iters: int = 100) -> float:
    """tau = 1/(1.01 lambda_max(A^T A)) (App. B: (1/tau) I - A^T A >= 0)."""
    return 1.0 / (1.01 * lambda_max(A, iters))


def tv(u: np.ndarray) -> float:
    u = _f64(u)
    return float(_load().oracle_tv(u.shape[0], u.ctypes.data))


@dataclass
class Result:
    u: np.ndarray          # (n, n)
    w: np.ndarray          # (2, n, n)
    lam: np.ndarray        # (2, n, n)
    info: dict
    hist: np.ndarray | None     # (iters, 4): objective, atv, rel change, ||Au-f||^2
    u_hist: np.ndarray | None   # (iters+1, n, n)


def _params(n, m, mu, beta, tau, tol, max_iter, algo, w_sign, init):
    return _Params(n, m, mu, beta, tau, tol, max_iter, algo, w_sign, init)


def solve(A: np.ndarray, f: np.ndarray, n: int, mu: float, beta: float, tau: float,
          tol: float = 0.0, max_iter: int = 100, algo: int = IADM, w_sign: int = 1,
          init: int = INIT_ATF, u0: np.ndarray | None = None, lam0: np.ndarray | None = None,
          record: bool = False, record_u: bool = False) -> Result:
    """Run Algorithm 2 (IADM, default) or Algorithm 1 (FTVCS)."""
    A = _f32(A)
    f = _f32(f)
    m, N = A.shape
    assert N == n * n and f.size == m
    if u0 is not None:
        init = INIT_GIVEN
    p = _params(n, m, mu, beta, tau, tol, max_iter, algo, w_sign, init)
    u = np.empty((n, n)); w = np.empty((2, n, n)); lam = np.empty((2, n, n))
    hist = np.zeros((max(max_iter, 1), 4)) if record else None
    uh = np.zeros((max_iter + 1, n, n)) if record_u else None
    u0a = _f64(u0).reshape(n, n) if u0 is not None else None
    l0a = _f64(lam0).reshape(2, n, n) if lam0 is not None else None
    info = _Info()
    rc = _load().oracle_solve(ctypes.byref(p), A.ctypes.data, f.ctypes.data,
                              u0a.ctypes.data if u0a is not None else None,
                              l0a.ctypes.data if l0a is not None else None,
                              u.ctypes.data, w.ctypes.data, lam.ctypes.data,
                              hist.ctypes.data if hist is not None else None,
                              uh.ctypes.data if uh is not None else None,
                              ctypes.byref(info))
    if rc != 0:
        raise ValueError("oracle_solve failed with code %d" % rc)
    d = {k: getattr(info, k) for k, _ in _Info._fields_}
    k = d["iters"]
    return Result(u, w, lam, d, hist[:k] if hist is not None else None,
                  uh[:k + 1] if uh is not None else None)


# ---- partial-DCT encoder (Sec. 3.2, reading C18) ----

def _rows(rows) -> np.ndarray:
    return np.ascontiguousarray(rows, dtype=np.int32)


def dct2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Orthonormal 2D DCT-II C x C^T of an n x n image (inverse: C^T x C)."""
    x = _f64(x)
    n = x.shape[0]
    out = np.empty((n, n))
    _load().oracle_dct2(n, 1 if inverse else 0, x.ctypes.data, out.ctypes.data)
    return out


def dct_Au(n: int, rows, u: np.ndarray, f: np.ndarray | None = None) -> np.ndarray:
    """r = (C u C^T)[rows] - f."""
    rows = _rows(rows)
    u = _f64(u)
    r = np.empty(rows.size)
    fp = _f32(f) if f is not None else None
    _load().oracle_dct_Au(n, rows.size, rows.ctypes.data, u.ctypes.data,
                          fp.ctypes.data if fp is not None else None, r.ctypes.data)
    return r


def dct_At(n: int, rows, r: np.ndarray) -> np.ndarray:
    """g = A^T r = C^T S C, S zero except S[rows] = r."""
    rows = _rows(rows)
    r = _f64(r)
    g = np.empty(n * n)
    _load().oracle_dct_At(n, rows.size, rows.ctypes.data, r.ctypes.data, g.ctypes.data)
    return g


def solve_dct(rows, f: np.ndarray, n: int, mu: float, beta: float, tau: float,
              tol: float = 0.0, max_iter: int = 100, algo: int = IADM, init: int = INIT_ATF,
              u0: np.ndarray | None = None, lam0: np.ndarray | None = None,
              record: bool = False) -> Result:
    """solve() with the partial-DCT encoder A = (rows of the orthonormal 2D DCT)."""
    rows = _rows(rows)
    f = _f32(f)
    m = rows.size
    assert f.size == m
    if u0 is not None:
        init = INIT_GIVEN
    p = _params(n, m, mu, beta, tau, tol, max_iter, algo, 1, init)
    u = np.empty((n, n)); w = np.empty((2, n, n)); lam = np.empty((2, n, n))
    hist = np.zeros((max(max_iter, 1), 4)) if record else None
    u0a = _f64(u0).reshape(n, n) if u0 is not None else None
    l0a = _f64(lam0).reshape(2, n, n) if lam0 is not None else None
    info = _Info()
    rc = _load().oracle_solve_dct(ctypes.byref(p), rows.ctypes.data, f.ctypes.data,
                                  u0a.ctypes.data if u0a is not None else None,
                                  l0a.ctypes.data if l0a is not None else None,
                                  u.ctypes.data, w.ctypes.data, lam.ctypes.data,
                                  hist.ctypes.data if hist is not None else None, None,
                                  ctypes.byref(info))
    if rc != 0:
        raise ValueError("oracle_solve_dct failed with code %d" % rc)
    d = {k: getattr(info, k) for k, _ in _Info._fields_}
    k = d["iters"]
    return Result(u, w, lam, d, hist[:k] if hist is not None else None, None)


def kkt(A, f, n, mu, beta, u, w, lam) -> dict:
    A = _f32(A); f = _f32(f)
    m, N = A.shape
    p = _params(n, m, mu, beta, 1.0, 0.0, 0, IADM, 1, INIT_ATF)
    u = _f64(u); w = _f64(w); lam = _f64(lam)
    info = _Info()
    _load().oracle_kkt(ctypes.byref(p), A.ctypes.data, f.ctypes.data, u.ctypes.data,
                       w.ctypes.data, lam.ctypes.data, ctypes.byref(info))
    return {k: getattr(info, k) for k, _ in _Info._fields_}
