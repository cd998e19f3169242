"""Pins of the oracle's partial-DCT encoder (Sec. 3.2, reading C18: rows of the
orthonormal 2D DCT-II).  Each checks the oracle against something other than
itself: a library DCT, closed forms, orthonormality, the dense-matrix solver."""
import numpy as np
import pytest
import scipy.fft

import oracle
import synth


@pytest.mark.parametrize("n", [4, 7, 16])
def test_dct2_matches_library_orthonormal_dct(n):
    x = np.random.default_rng(n).standard_normal((n, n))
    assert np.allclose(oracle.dct2(x), scipy.fft.dctn(x, norm="ortho"), atol=1e-13)
    assert np.allclose(oracle.dct2(x, inverse=True), scipy.fft.idctn(x, norm="ortho"), atol=1e-13)


def test_dct2_closed_forms():
    n = 8
    # a constant image has only the (0, 0) coefficient, equal to n times the constant
    X = oracle.dct2(np.full((n, n), 0.5))
    assert abs(X[0, 0] - 0.5 * n) < 1e-13 and np.max(np.abs(X.ravel()[1:])) < 1e-13
    # a separable cosine basis image maps to one coefficient
    k1, k2 = 3, 5
    j = np.arange(n)
    b = lambda k: np.sqrt(2.0 / n) * np.cos(np.pi * (2 * j + 1) * k / (2 * n))
    X = oracle.dct2(np.outer(b(k1), b(k2)))
    E = np.zeros((n, n)); E[k1, k2] = 1.0
    assert np.max(np.abs(X - E)) < 1e-13


def test_partial_dct_rows_are_orthonormal_and_adjoint():
    n, m = 16, 77
    rows = synth.dct_rows(4, n, m)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(n * n)
    r = rng.standard_normal(m)
    Au = oracle.dct_Au(n, rows, u)
    Atr = oracle.dct_At(n, rows, r)
    assert abs(Au @ r - u @ Atr) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(r)
    assert np.allclose(oracle.dct_Au(n, rows, Atr), r, atol=1e-13)      # A A^T = I
    assert abs(np.linalg.norm(Atr) - np.linalg.norm(r)) < 1e-12          # A^T isometric


def test_dct_rows_and_measurements():
    rows = synth.dct_rows(7, 32, 307)
    assert rows.dtype == np.int32 and rows.size == 307
    assert np.all(np.diff(rows) > 0) and rows[0] >= 0 and rows[-1] < 1024
    assert np.array_equal(rows, synth.dct_rows(7, 32, 307))
    P = synth.make_dct_problem(32, 0.3, 7, 5, 500.0, sigma=0.0)
    assert np.allclose(P.f, oracle.dct_Au(32, P.extra["rows"], P.ubar.ravel()), atol=1e-6)


def test_solve_dct_matches_dense_matrix_solver():
    # the operator path of the solver against the dense path on the explicit matrix
    n, m = 8, 24
    P = synth.make_dct_problem(n, 0.0, 9, 3, 200.0, beta=16.0, sigma=1e-3)
    rows = synth.dct_rows(9, n, m)
    f = synth.measure_dct(rows, P.ubar, 1e-3, 5)
    C = scipy.fft.dct(np.eye(n), norm="ortho", axis=0)          # C[k][j]
    A = np.kron(C, C)[rows]                                       # rows of C x C^T, vectorised
    ref = oracle.solve(A.astype(np.float32), f, n, 200.0, 16.0, 0.9, max_iter=60)
    got = oracle.solve_dct(rows, f, n, 200.0, 16.0, 0.9, max_iter=60)
    # the dense path rounds A's entries to binary32 (~6e-8 relative)
    assert np.linalg.norm(got.u - ref.u) <= 1e-5 * np.linalg.norm(ref.u)


def test_solve_dct_reaches_kkt_point():
    n = 8
    P = synth.make_dct_problem(n, 0.4, 11, 3, 100.0, beta=32.0, sigma=1e-3)
    res = oracle.solve_dct(P.extra["rows"], P.f, n, 100.0, 32.0, 1.9, tol=1e-13, max_iter=20000)
    assert res.info["kkt_primal"] < 1e-6 * (1 + res.info["tv"])
    assert res.info["kkt_dual"] < 1e-5 * 100.0 * (1 + np.sqrt(res.info["resid2"]))
    assert res.info["lambda_max_norm"] <= 1 + 1e-6
