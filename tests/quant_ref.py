"""numpy emulation of the reduced-precision storages of A (test side).

BF16X2:   A = hi + lo, hi = bf16(A), lo = bf16(A - hi), round to nearest even.
FP8_BF16: A = s q + c, s = max_j |A_ij| / 448 per row (binary32 division),
          q = e4m3(A / s) (round to nearest even, saturating at +-448),
          c = bf16(binary32(A - s q)); decoded as binary32(s q + c).
The e4m3 value set is enumerated from its bit layout (sign, 4 exponent bits,
bias 7, 3 mantissa bits; exponent field 0 holds the subnormals m 2^-9; the
code S.1111.111 is NaN), so the rounding here depends on no GPU code.
"""
import numpy as np


def bf16_rne(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def split_bf16x2(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float32)
    hi = bf16_rne(A)
    lo = bf16_rne((A - hi).astype(np.float32))   # A - hi is exact in binary32
    return hi, lo


def _e4m3_table():
    vals, codes = [], []
    for code in range(128):
        e = (code >> 3) & 0xF
        mbits = code & 0x7
        if e == 0xF and mbits == 0x7:
            continue   # NaN
        v = (mbits / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + mbits / 8.0) * 2.0 ** (e - 7)
        vals.append(v)
        codes.append(code)
    order = np.argsort(vals)
    return np.array(vals)[order], np.array(codes)[order]


_E4M3_VALS, _E4M3_CODES = _e4m3_table()
E4M3_MAX = float(_E4M3_VALS[-1])   # 448


def e4m3_rne(x: np.ndarray) -> np.ndarray:
    """Nearest e4m3 value, ties to the even mantissa, saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    idx = np.searchsorted(_E4M3_VALS, a)          # first value >= a
    idx = np.clip(idx, 1, len(_E4M3_VALS) - 1)
    lo_v, hi_v = _E4M3_VALS[idx - 1], _E4M3_VALS[idx]
    lo_c, hi_c = _E4M3_CODES[idx - 1], _E4M3_CODES[idx]
    d_lo, d_hi = a - lo_v, hi_v - a
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & ((hi_c & 1) == 0))
    v = np.where(pick_hi, hi_v, lo_v)
    v = np.where(a == 0.0, 0.0, v)
    return np.copysign(v, x)


def quant_fp8(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float32)
    mx = np.max(np.abs(A), axis=1)
    s = np.where(mx > 0, (mx / np.float32(448.0)).astype(np.float32), np.float32(1.0))
    s = s.astype(np.float32)
    q = e4m3_rne((A / s[:, None]).astype(np.float32))
    # one rounding of A - s q (s q is exact in binary64: 24 x 4 significant bits)
    c = bf16_rne((A.astype(np.float64) - s[:, None].astype(np.float64) * q).astype(np.float32))
    return s, q.astype(np.float32), c


def effective_A(A: np.ndarray, prec: int) -> np.ndarray:
    """The binary32 matrix the GPU multiplies with for storage `prec`."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    if prec == 0:
        return A
    if prec == 1:
        hi, lo = split_bf16x2(A)
        return (hi + lo).astype(np.float32)
    s, q, c = quant_fp8(A)
    return (s[:, None].astype(np.float64) * q + c).astype(np.float32)
