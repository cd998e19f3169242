"""Products and solves with A stored as bf16 hi+lo or fp8 e4m3 + bf16
correction, and the binary32 path for 192 x 192 and 256 x 256 images (rows
split over a thread-block cluster), against the FP64 oracle.

Two comparisons per case: against the oracle run on the matrix the GPU
actually multiplies with (the storage decoded by the test-side emulation in
quant_ref.py), which checks the kernel arithmetic at the binary32 tolerances;
and against the oracle on the exact binary32 A, which measures the storage
error itself (reported per result).
"""
import numpy as np
import pytest
import torch

import oracle
import quant_ref
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    return tv


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def handle(tv, A, m, n, mu, beta, prec, tau, max_iter=500):
    opt = tv.tvcs_default_options()
    opt.precision = prec
    opt.tau = tau
    opt.max_iter = max_iter
    return tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, n, mu, beta, 0.0, opt)


@pytest.mark.parametrize("prec,n,m", [(1, 32, 307), (2, 32, 307), (1, 64, 1229), (2, 64, 1229),
                                      (1, 128, 4915), (2, 128, 4915), (0, 192, 1000),
                                      (1, 192, 777), (2, 192, 500), (0, 256, 700), (1, 256, 301),
                                      (2, 256, 153)])
def test_precision_products(tv, prec, n, m):
    N = n * n
    A = synth.gaussian_matrix(40 + n + prec, m, N)
    Ae = quant_ref.effective_A(A, prec)
    rng = np.random.default_rng(n + m + prec)
    x = rng.standard_normal(N).astype(np.float32)
    y = rng.standard_normal(m).astype(np.float32)
    h = handle(tv, A, m, n, 1.0, 1.0, prec, 0.1)
    r = np.empty(m, np.float32)
    g = np.empty(N, np.float32)
    tv.tvcs_apply(h, x, y, r, g)
    r64, g64 = r.astype(np.float64), g.astype(np.float64)
    absA = np.abs(Ae.astype(np.float64))
    rr = oracle.Au(Ae, x, y)
    assert np.all(np.abs(r64 - rr) <= 1e-5 * (absA @ np.abs(x.astype(np.float64))) + 1e-30)
    gr = oracle.At(Ae, r64)
    assert np.all(np.abs(g64 - gr) <= 1e-5 * (absA.T @ np.abs(r64)) + 1e-30)
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cluster_products_repeat_bitwise(tv, prec):
    """The 256 x 256 products (rows split over a 4-block cluster) sum each row's
    block parts in a fixed order after an exchange whose stores complete on the
    receiving block's barrier: a part read before it landed would change r (and g)
    from one launch to the next.  Five launches on the same inputs, 2000 rows (55-56
    per cluster, each exchange slot reused 14 times), must agree bit for bit."""
    n, m = 256, 2000
    N = n * n
    opt = tv.tvcs_default_options()
    opt.precision = prec
    opt.tau = 0.1
    h = tv.tvcs_create(None, 11 + prec, m, n, 1.0, 1.0, 0.0, opt)
    rng = np.random.default_rng(5 + prec)
    x = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.standard_normal(m).astype(np.float32)).cuda()
    runs = []
    for _ in range(5):
        r = torch.empty(m, device="cuda")
        g = torch.empty(N, device="cuda")
        tv.tvcs_apply(h, x, y, r, g)
        runs.append((r.cpu().numpy(), g.cpu().numpy()))
    tv.tvcs_destroy(h)
    r0, g0 = runs[0]
    assert np.all(np.isfinite(r0)) and np.all(np.isfinite(g0)) and np.any(r0 != 0)
    for r1, g1 in runs[1:]:
        assert np.array_equal(r0, r1) and np.array_equal(g0, g1)


@pytest.mark.parametrize("prec", [1, 2])
def test_precision_fixed_50_iterations(tv, prec):
    P = synth.make_problem(64, 0.3, 9, 6, 1e3, 10.0, noise_c=1e-3)
    tau = oracle.default_tau(P.A)
    Ae = quant_ref.effective_A(P.A, prec)
    h = handle(tv, P.A, P.m, P.n, P.mu, P.beta, prec, tau, max_iter=50)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve(h, P.f, u)
    assert res.iters == 50
    same = oracle.solve(Ae, P.f, P.n, P.mu, P.beta, tau, max_iter=50)
    exact = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=50)
    assert rel(u, same.u) <= 1e-5          # kernel arithmetic
    err = rel(u, exact.u)                  # storage error of A, stated per result
    print("precision %d: rel image error vs FP64 oracle on exact A = %.3e" % (prec, err))
    assert err <= (1e-4 if prec == 1 else 1e-3)
    tv.tvcs_destroy(h)


def test_workload_n256_storages(tv):
    # n = 256, m = 13107 (ratio 0.2), 20 ellipses, noise 5e-3 RMS, mu = 5e2: binary32,
    # bf16 hi+lo and fp8 + bf16 storage, 30 iterations each, vs the FP64 oracle on the
    # exact binary32 A.
    P = synth.workload_n256()
    iters = 30
    tau = oracle.default_tau(P.A, 20)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=iters)
    errs = {}
    for prec in (0, 1, 2):
        h = handle(tv, P.A, P.m, P.n, P.mu, P.beta, prec, tau, max_iter=iters)
        u = torch.empty(P.N, dtype=torch.float32, device="cuda")
        res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
        assert res.iters == iters
        errs[prec] = rel(u.cpu().numpy(), ref.u)
        tv.tvcs_destroy(h)
    print("n=256 rel image errors vs FP64 oracle after %d iterations: fp32 %.2e, bf16x2 %.2e, "
          "fp8+bf16 %.2e" % (iters, errs[0], errs[1], errs[2]))
    assert errs[0] <= 1e-5
    assert errs[1] <= 1e-4
    assert errs[2] <= 1e-3
