"""Seeded synthetic inputs for TV/L2 reconstruction from random projections.

Xiao & Yang reconstruct an n x n image ubar from f = N(A ubar) (Sec. 1,
eq. (obser)) with A an m x n^2 i.i.d. Gaussian encoding matrix and additive
Gaussian noise (Sec. 3.1).  Their test images (Shepp-Logan, Sec. 3.1-3.2, and
the natural images of Table 2) are not available here; seeded piecewise-
constant phantoms of random ellipses (and, for the 128 x 128 workload, a random
rectangle grid) stand in for them, at the paper's sizes, sampling ratios and
noise levels.

This module generates inputs only and holds none of the solver's arithmetic.
The CPU oracle's tests, the GPU tests and the benchmark all draw from it.
The counter-based Gaussian generator lives in ``synth.c`` (compiled on first
use); its recipe is stated at the top of that file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` with gcc (IEEE binary32, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.synth_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.synth_philox4x32_10.restype = None
            lib.synth_ln.argtypes = [ctypes.c_float]
            lib.synth_ln.restype = ctypes.c_float
            lib.synth_cossin_turns.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_float)]
            lib.synth_cossin_turns.restype = None
            lib.synth_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                          ctypes.c_int64, ctypes.c_void_p]
            lib.synth_normals.restype = None
            lib.synth_gauss_scale.argtypes = [ctypes.c_int]
            lib.synth_gauss_scale.restype = ctypes.c_float
            lib.synth_gaussian_rows.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
            lib.synth_gaussian_rows.restype = None
            lib.synth_measure.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64,
                                          ctypes.c_void_p]
            lib.synth_measure.restype = ctypes.c_double
            lib.synth_measure_seeded.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_double,
                                                 ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_measure_seeded.restype = ctypes.c_double
            lib.synth_ln_array.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_ln_array.restype = None
            lib.synth_cossin_array.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]
            lib.synth_cossin_array.restype = None
            _lib = lib
    return _lib


# ----------------------------------------------------------------------------
# Generator primitives (thin wrappers over synth.c)
# ----------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 counter words and 2 key words -> 4 uint32."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def ln32(x: float) -> float:
    return float(_load().synth_ln(ctypes.c_float(x)))


def cossin_turns(xb: int):
    c = ctypes.c_float()
    s = ctypes.c_float()
    _load().synth_cossin_turns(ctypes.c_uint32(xb), ctypes.byref(c), ctypes.byref(s))
    return float(c.value), float(s.value)


def ln32_array(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty_like(x)
    _load().synth_ln_array(x.size, x.ctypes.data, out.ctypes.data)
    return out


def cossin_turns_array(xb: np.ndarray):
    xb = np.ascontiguousarray(xb, dtype=np.uint32)
    c = np.empty(xb.shape, dtype=np.float32)
    s = np.empty(xb.shape, dtype=np.float32)
    _load().synth_cossin_array(xb.size, xb.ctypes.data, c.ctypes.data, s.ctypes.data)
    return c, s


def normals(seed: int, stream: int, e0: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    _load().synth_normals(seed, stream, e0, count, out.ctypes.data)
    return out


def gauss_scale(m: int) -> np.float32:
    return np.float32(_load().synth_gauss_scale(m))


def gaussian_matrix(seed: int, m: int, N: int, row0: int = 0, nrows: int | None = None,
                    out: np.ndarray | None = None) -> np.ndarray:
    """Rows [row0, row0+nrows) of the m x N encoding matrix with i.i.d. N(0, 1/m)
    entries (Sec. 3.1), float32, row-major."""
    if nrows is None:
        nrows = m - row0
    if out is None:
        out = np.empty((nrows, N), dtype=np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.shape == (nrows, N)
    _load().synth_gaussian_rows(seed, m, N, row0, nrows, out.ctypes.data)
    return out


def measure(A: np.ndarray, ubar: np.ndarray, c: float, noise_seed: int):
    """f = A ubar + sigma*eps with sigma = c * RMS(A ubar) (Sec. 3.1 noise model).
    Returns (f float32[m], sigma)."""
    m, N = A.shape
    assert A.dtype == np.float32 and A.flags.c_contiguous
    ub = np.ascontiguousarray(ubar, dtype=np.float32).reshape(-1)
    assert ub.size == N
    f = np.empty(m, dtype=np.float32)
    sigma = _load().synth_measure(A.ctypes.data, m, N, ub.ctypes.data, c, noise_seed,
                                  f.ctypes.data)
    if sigma < 0:
        raise MemoryError("synth_measure: allocation failed")
    return f, float(sigma)


def measure_seeded(seed: int, m: int, N: int, ubar: np.ndarray, c: float, noise_seed: int):
    """measure(gaussian_matrix(seed, m, N), ubar, c, noise_seed), bit for bit, with
    each row of A generated while it is used (no m x N array)."""
    ub = np.ascontiguousarray(ubar, dtype=np.float32).reshape(-1)
    assert ub.size == N
    f = np.empty(m, dtype=np.float32)
    sigma = _load().synth_measure_seeded(seed, m, N, ub.ctypes.data, c, noise_seed, f.ctypes.data)
    if sigma < 0:
        raise MemoryError("synth_measure_seeded: allocation failed")
    return f, float(sigma)


# ----------------------------------------------------------------------------
# Phantoms (stand-ins for the paper's Shepp-Logan and natural test images)
# ----------------------------------------------------------------------------

def phantom(n: int, n_ellipses: int, seed: int, rect_grid: bool = False) -> np.ndarray:
    """Piecewise-constant n x n phantom, float32, values in [0, 1].

    Pixel centres x = (2c+1)/n - 1, y = (2r+1)/n - 1.  An optional k x k grid
    (k in 4..8) of axis-aligned cells over a random sub-square is painted
    first, each cell set to U[0,1] with probability 1/2.  Then each ellipse
    (centre U[-0.7,0.7]^2, semi-axes U[0.05,0.5], angle U[0,pi), intensity
    U[0,1]) is painted in order, later shapes overwriting earlier ones."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x7E11]))
    coords = (2.0 * np.arange(n) + 1.0) / n - 1.0
    X, Y = np.meshgrid(coords, coords)  # X varies along columns, Y along rows
    img = np.zeros((n, n), dtype=np.float64)
    if rect_grid:
        k = int(rng.integers(4, 9))
        side = rng.uniform(0.5, 1.6)
        x0 = rng.uniform(-1.0, 1.0 - side)
        y0 = rng.uniform(-1.0, 1.0 - side)
        cell = side / k
        for a in range(k):
            for b in range(k):
                on = rng.uniform() < 0.5
                val = rng.uniform()
                if on:
                    mask = ((X >= x0 + b * cell) & (X < x0 + (b + 1) * cell) &
                            (Y >= y0 + a * cell) & (Y < y0 + (a + 1) * cell))
                    img[mask] = val
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.7, 0.7, size=2)
        ax, ay = rng.uniform(0.05, 0.5, size=2)
        th = rng.uniform(0.0, np.pi)
        val = rng.uniform()
        ct, st = np.cos(th), np.sin(th)
        xr = (X - cx) * ct + (Y - cy) * st
        yr = -(X - cx) * st + (Y - cy) * ct
        img[(xr / ax) ** 2 + (yr / ay) ** 2 <= 1.0] = val
    return img.astype(np.float32)


# ----------------------------------------------------------------------------
# Named workloads (shapes, ratios and noise levels of the paper's experiments)
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    name: str
    n: int
    m: int
    seed: int              # seed of A
    mu: float
    beta: float
    tol: float
    max_iter: int
    noise_c: float
    ubar: np.ndarray       # (n, n) float32
    A: np.ndarray | None   # (m, n*n) float32, or None when not materialised on the host
    f: np.ndarray | None   # (m,) float32
    sigma: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n * self.n


def sampled_m(n: int, ratio: float) -> int:
    """m = floor(ratio * n^2) measurements for a sampling ratio (Sec. 3.1)."""
    return int(np.floor(ratio * n * n + 1e-9))


def make_problem(n: int, ratio: float, seed: int, n_ellipses: int, mu: float,
                 beta: float = 10.0, tol: float = 1e-4, max_iter: int = 500,
                 noise_c: float = 1e-3, rect_grid: bool = False, name: str = "custom",
                 m: int | None = None, phantom_seed: int | None = None,
                 noise_seed: int | None = None, materialise: bool = True) -> Problem:
    """One problem: phantom, A from `seed`, f = A ubar + noise.  With
    materialise=False, A is not kept (Problem.A is None) and f comes from
    measure_seeded, identical to the materialised f."""
    if m is None:
        m = sampled_m(n, ratio)
    ps = seed if phantom_seed is None else phantom_seed
    ns = seed + 1_000_003 if noise_seed is None else noise_seed
    ubar = phantom(n, n_ellipses, ps, rect_grid=rect_grid)
    if materialise:
        A = gaussian_matrix(seed, m, n * n)
        f, sigma = measure(A, ubar, noise_c, ns)
    else:
        A = None
        f, sigma = measure_seeded(seed, m, n * n, ubar, noise_c, ns)
    return Problem(name, n, m, seed, mu, beta, tol, max_iter, noise_c, ubar, A, f, sigma)


def workload_n32() -> Problem:
    """Single 32 x 32 image, m = 307 (ratio 0.3), A from seed 0, 6 ellipses,
    noise 1e-3 * RMS, mu = 1e3, beta = 10, relative-change tol 1e-4, <= 500 its."""
    return make_problem(32, 0.3, 0, 6, 1e3, 10.0, 1e-4, 500, 1e-3, name="n32_m307")


def workload_n256() -> Problem:
    """Single 256 x 256 image, m = 13107 (ratio 0.2), 20 ellipses, noise 5e-3 * RMS,
    mu = 5e2, beta = 10 (the reduced-precision storage workload; A is 3.4 GB in binary32)."""
    return make_problem(256, 0.2, 2, 20, 5e2, 10.0, 0.0, 300, 5e-3, name="n256_m13107")


def workload_shared_batch(count: int = 256, n: int = 128, ratio: float = 0.3, seed: int = 1,
                          n_ellipses: int = 12):
    """`count` images sharing one Gaussian A (m = ratio n^2): image b is a seeded
    ellipse phantom, its noise level is U[1e-3, 1e-2] RMS, and mu cycles over
    {2e2, 5e2, 1e3, 2e3}.  Returns (A, [ubar_b], F (count x m), [mu_b], [sigma_b])."""
    m = sampled_m(n, ratio)
    A = gaussian_matrix(seed, m, n * n)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7C]))
    mus = [2e2, 5e2, 1e3, 2e3]
    ubars, F, mu, sig = [], np.empty((count, m), np.float32), [], []
    for b in range(count):
        ub = phantom(n, n_ellipses, 1000 + 7 * b + seed)
        c = float(rng.uniform(1e-3, 1e-2))
        f, s = measure(A, ub, c, 500_000 + b)
        ubars.append(ub)
        F[b] = f
        mu.append(mus[b % 4])
        sig.append(s)
    return A, ubars, F, mu, sig


def workload_n128() -> Problem:
    """Single 128 x 128 image, m = 4915 (ratio 0.3), 12 ellipses plus a random
    rectangle grid, noise 1e-3 * RMS, mu = 1e3, beta = 10, 300 iterations."""
    return make_problem(128, 0.3, 1, 12, 1e3, 10.0, 0.0, 300, 1e-3, rect_grid=True,
                        name="n128_m4915")


UNEVEN_SIDES = (64, 96, 128, 192)
UNEVEN_RATIOS = (0.1, 0.2, 0.3, 0.5)


def uneven_shape(seed: int):
    """(n, ratio) of problem `seed` of the uneven batch: each drawn uniformly
    from UNEVEN_SIDES and UNEVEN_RATIOS by a generator seeded with `seed`."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x0E7E]))
    return UNEVEN_SIDES[int(rng.integers(4))], UNEVEN_RATIOS[int(rng.integers(4))]


def workload_uneven(count: int = 64, first_seed: int = 1, materialise: bool = False,
                    sides=None) -> list:
    """`count` independent problems with seeds first_seed, first_seed+1, ...:
    n and m/n^2 from uneven_shape (or n restricted to `sides`, redrawn in turn),
    A ~ N(0, 1/m) from the problem's seed, a 10-ellipse phantom, noise
    1e-3 * RMS, mu = 1e3, beta = 10, tol 1e-4, <= 500 iterations."""
    out = []
    for s in range(first_seed, first_seed + count):
        n, ratio = uneven_shape(s)
        if sides is not None:
            n = tuple(sides)[(s - first_seed) % len(sides)]
        out.append(make_problem(n, ratio, s, 10, 1e3, 10.0, 1e-4, 500, 1e-3,
                                name="uneven_%d" % s, materialise=materialise))
    return out


# ----------------------------------------------------------------------------
# Partial-DCT encoder inputs (Sec. 3.2): A = m rows of the orthonormal 2D DCT
# ----------------------------------------------------------------------------

def dct_rows(seed: int, n: int, m: int) -> np.ndarray:
    """m distinct coefficient indices k1*n + k2 of the n x n DCT, chosen uniformly
    at random (seeded), in increasing order; int32."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xDC7]))
    return np.sort(rng.choice(n * n, size=m, replace=False)).astype(np.int32)


def measure_dct(rows: np.ndarray, ubar: np.ndarray, sigma: float, noise_seed: int) -> np.ndarray:
    """f = (orthonormal 2D DCT of ubar)[rows] + sigma * eps (Sec. 3.2: Gaussian noise
    of standard deviation sigma, absolute), eps from stream 1 of noise_seed; float32."""
    import scipy.fft
    X = scipy.fft.dctn(np.asarray(ubar, dtype=np.float64), norm="ortho").ravel()
    eps = normals(noise_seed, 1, 0, rows.size).astype(np.float64)
    return (X[rows] + sigma * eps).astype(np.float32)


def make_dct_problem(n: int, ratio: float, seed: int, n_ellipses: int, mu: float,
                     beta: float = 2.0 ** 6, tol: float = 5e-5, max_iter: int = 1000,
                     sigma: float = 1e-3, name: str = "dct") -> Problem:
    """One partial-DCT problem: a seeded phantom, m = floor(ratio n^2) DCT rows, f with
    absolute noise sigma.  Problem.A is None; the rows are in Problem.extra['rows']."""
    m = sampled_m(n, ratio)
    rows = dct_rows(seed, n, m)
    ubar = phantom(n, n_ellipses, seed)
    f = measure_dct(rows, ubar, sigma, seed + 1_000_003)
    return Problem(name, n, m, seed, mu, beta, tol, max_iter, sigma, ubar, None, f, sigma,
                   extra={"rows": rows})


def workload_dct128() -> Problem:
    """Sec. 3.2's partial-DCT experiment: a 128 x 128 phantom (stand-in for the
    Shepp-Logan image, 10 ellipses), 30% of the DCT coefficients (m = 4915),
    noise of standard deviation 0.001, mu = 500 (a row of Table 1), beta = 2^6,
    tol 5e-5 (the step tau = 1.9 of the same section is passed by the caller),
    at most 5000 iterations (the FP64 oracle stops after 2403)."""
    return make_dct_problem(128, 0.3, 3, 10, 500.0, 2.0 ** 6, 5e-5, 5000, 1e-3,
                            name="dct128_m4915")
