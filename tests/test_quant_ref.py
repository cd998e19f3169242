"""Pins for the test-side emulation of the reduced-precision storages of A."""
import numpy as np
import torch

import quant_ref as q
import synth


def test_bf16_rounding_matches_torch():
    A = synth.gaussian_matrix(3, 64, 1024)
    t = torch.from_numpy(A.ravel()).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(t, q.bf16_rne(A).ravel())


def test_e4m3_rounding_matches_torch_in_range():
    x = (np.random.default_rng(0).standard_normal(200000) * 100).astype(np.float32)
    x = x[np.abs(x) <= 448.0]
    tq = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(tq, q.e4m3_rne(x).astype(np.float32))
    # saturation (the GPU conversion is the saturating one)
    assert q.e4m3_rne(np.array([1e6, -500.0]))[0] == 448.0
    assert q.e4m3_rne(np.array([-500.0]))[0] == -448.0
    assert len(q._E4M3_VALS) == 127 and q.E4M3_MAX == 448.0


def test_bf16x2_split_is_exact_sum_within_2_pow_minus_16():
    A = synth.gaussian_matrix(5, 200, 4096)
    hi, lo = q.split_bf16x2(A)
    s = (hi + lo).astype(np.float32)
    assert np.array_equal(s.astype(np.float64), hi.astype(np.float64) + lo.astype(np.float64))
    rel = np.abs(s.astype(np.float64) - A) / np.abs(A)
    assert rel.max() <= 2.0 ** -16


def test_fp8_bf16_storage_error():
    A = synth.gaussian_matrix(6, 200, 4096)
    Ae = q.effective_A(A, 2).astype(np.float64)
    err = np.abs(Ae - A)
    s, _, _ = q.quant_fp8(A)
    # |A - s q| <= half an e4m3 step (2^-4 relative, or 2^-10 s below the normal range);
    # the bf16 correction (8 significant bits, unit round-off 2^-8) leaves 2^-8 of that,
    # and decoding s q + c in binary32 adds one rounding
    bound = 2.0 ** -8 * np.maximum(2.0 ** -4 * np.abs(A), 2.0 ** -10 * s[:, None])
    assert np.all(err <= bound + 2.0 ** -23 * np.abs(A))
    assert np.sqrt(np.mean((err / np.abs(A)) ** 2)) < 2e-4
