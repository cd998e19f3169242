"""Pins for the oracle's building blocks, each against something other than
the oracle itself: explicit dense matrices built from the index definitions,
closed forms, numpy/LAPACK routines, and the shrinkage lemma."""
import os

import numpy as np
import pytest

import oracle
import synth
from indep_solvers import diff_matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [2, 3, 4, 8, 13])
def test_D_and_Dt_match_explicit_matrix(n):
    rng = np.random.default_rng(n)
    Dm = diff_matrix(n)
    u = rng.standard_normal((n, n))
    d1, d2 = oracle.D(u)
    ref = Dm @ u.ravel()
    N = n * n
    assert np.allclose(d1.ravel(), ref[:N], atol=1e-14)
    assert np.allclose(d2.ravel(), ref[N:], atol=1e-14)
    y1, y2 = rng.standard_normal((2, n, n))
    out = oracle.Dt(y1, y2)
    assert np.allclose(out.ravel(), Dm.T @ np.concatenate([y1.ravel(), y2.ravel()]), atol=1e-13)
    # adjointness <D u, y> = <u, D^T y>
    assert np.dot(d1.ravel(), y1.ravel()) + np.dot(d2.ravel(), y2.ravel()) == pytest.approx(
        np.dot(u.ravel(), out.ravel()), rel=1e-12)


def test_D_annihilates_constants():
    # N(D) = constants (used by Assumption 1).
    d1, d2 = oracle.D(np.full((7, 7), 3.25))
    assert np.all(d1 == 0) and np.all(d2 == 0)


def _load_shrink_golden():
    rows = []
    with open(os.path.join(GOLDEN, "shrink_cases.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_shrink_golden_cases():
    g = _load_shrink_golden()
    for beta, z1, z2, w1, w2 in g:
        a, b = oracle.shrink([z1], [z2], 1.0 / beta)
        assert a[0] == pytest.approx(w1, abs=1e-15)
        assert b[0] == pytest.approx(w2, abs=1e-15)


def test_shrink_is_identity_minus_disc_projection_and_minimiser():
    # eq. (sop): s(a) = a - P_B(a), B the disc of radius 1/beta; and it is the
    # unique minimiser of ||w|| + (beta/2)||w - z||^2 (eq. (fixu)).
    rng = np.random.default_rng(2)
    beta = 3.0
    z = rng.standard_normal((2, 4000)) * rng.choice([0.01, 0.3, 1.0, 5.0], size=4000)
    w1, w2 = oracle.shrink(z[0], z[1], 1.0 / beta)
    nz = np.hypot(z[0], z[1])
    scale = np.minimum(1.0, (1.0 / beta) / np.maximum(nz, 1e-300))
    p1, p2 = z[0] * scale, z[1] * scale
    assert np.allclose(w1, z[0] - p1, atol=1e-14) and np.allclose(w2, z[1] - p2, atol=1e-14)

    def obj(a, b, zz1, zz2):
        return np.hypot(a, b) + 0.5 * beta * ((a - zz1) ** 2 + (b - zz2) ** 2)

    base = obj(w1, w2, z[0], z[1])
    for _ in range(20):
        d = rng.standard_normal((2, z.shape[1])) * 1e-3
        assert np.all(obj(w1 + d[0], w2 + d[1], z[0], z[1]) >= base - 1e-15)


def test_shrink_nonexpansive_lemma():
    # Lemma (App. A): ||s(a)-s(b)||^2 <= ||a-b||^2 - ||P_B(a)-P_B(b)||^2.
    rng = np.random.default_rng(3)
    beta = 2.0
    a = rng.standard_normal((2, 5000)) * 0.7
    b = rng.standard_normal((2, 5000)) * 0.7
    sa = np.array(oracle.shrink(a[0], a[1], 1 / beta))
    sb = np.array(oracle.shrink(b[0], b[1], 1 / beta))
    pa, pb = a - sa, b - sb
    lhs = np.sum((sa - sb) ** 2, axis=0)
    rhs = np.sum((a - b) ** 2, axis=0) - np.sum((pa - pb) ** 2, axis=0)
    assert np.all(lhs <= rhs + 1e-12)


@pytest.mark.parametrize("n", [4, 8, 16, 32, 96])
def test_dtd_eigs_closed_form(n):
    lam = oracle.dtd_eigs(n)
    s = 4.0 * np.sin(np.pi * np.arange(n) / n) ** 2
    assert np.allclose(lam, s[:, None] + s[None, :], atol=1e-12)


def test_dtd_eigs_golden_n4():
    ref = np.loadtxt(os.path.join(GOLDEN, "dtd_eigs_n4.txt"))
    assert np.allclose(oracle.dtd_eigs(4), ref, atol=1e-13)


@pytest.mark.parametrize("n", [4, 8])
def test_dtd_eigs_match_dense_eigensolve(n):
    Dm = diff_matrix(n)
    ev = np.sort(np.linalg.eigvalsh(Dm.T @ Dm))
    assert np.allclose(np.sort(oracle.dtd_eigs(n).ravel()), ev, atol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 6, 8, 12])
def test_dft2_matches_numpy_fft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    assert np.allclose(oracle.dft2(x), np.fft.fft2(x), atol=1e-11)
    assert np.allclose(oracle.dft2(x, inverse=True), np.fft.ifft2(x), atol=1e-13)


@pytest.mark.parametrize("n,c", [(4, 0.5), (8, 3.0), (12, 0.01), (16, 7.5)])
def test_usolve_matches_dense_solve(n, c):
    rng = np.random.default_rng(n)
    Dm = diff_matrix(n)
    H = Dm.T @ Dm + c * np.eye(n * n)
    b = rng.standard_normal((n, n))
    ref = np.linalg.solve(H, b.ravel()).reshape(n, n)
    assert np.allclose(oracle.usolve(b, c), ref, atol=1e-12)


def test_products_match_numpy():
    rng = np.random.default_rng(4)
    m, n = 53, 9
    A = rng.standard_normal((m, n * n)).astype(np.float32)
    u = rng.standard_normal(n * n)
    f = rng.standard_normal(m).astype(np.float32)
    A64 = A.astype(np.float64)
    assert np.allclose(oracle.Au(A, u, f), A64 @ u - f.astype(np.float64), atol=1e-12)
    assert np.allclose(oracle.Au(A, u), A64 @ u, atol=1e-12)
    r = rng.standard_normal(m)
    assert np.allclose(oracle.At(A, r), A64.T @ r, atol=1e-12)


def test_lambda_max_power_iteration():
    A = synth.gaussian_matrix(0, 307, 1024)
    ev = np.linalg.eigvalsh(A.astype(np.float64).T @ A.astype(np.float64))[-1]
    lm = oracle.lambda_max(A, 100)
    assert lm <= ev * (1 + 1e-12)
    assert lm >= 0.97 * ev
    # Marchenko-Pastur edge (1 + sqrt(N/m))^2 for N(0, 1/m) entries
    assert lm == pytest.approx((1 + np.sqrt(1024 / 307)) ** 2, rel=0.08)


def test_tv_value():
    rng = np.random.default_rng(6)
    u = rng.standard_normal((10, 10))
    d = diff_matrix(10) @ u.ravel()
    assert oracle.tv(u) == pytest.approx(np.sum(np.hypot(d[:100], d[100:])), rel=1e-13)
