"""The partial-DCT encoder (Sec. 3.2, reading C18) on the GPU against the FP64
oracle through the C ABI: products per entry within 1e-5 of the |C| |x|
bound, solves at fixed iteration counts within 1e-5 relative image error, the
Sec. 3.2 workload to its tolerance within 1e-4."""
import numpy as np
import pytest
import torch

import oracle
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


def dct_handle(tv, rows, n, mu=500.0, beta=64.0, tau=1.9, max_iter=50, tol=0.0, algo=0):
    opt = tv.tvcs_default_options()
    opt.tau = tau
    opt.max_iter = max_iter
    opt.algo = algo
    return tv.tvcs_create_partial_dct(rows, n, mu, beta, tol, opt)


@pytest.mark.parametrize("n,ratio", [(16, 0.3), (32, 0.3), (48, 0.2), (64, 0.5), (96, 0.1),
                                     (128, 0.3)])
def test_dct_products_parity(tv, n, ratio):
    m = synth.sampled_m(n, ratio)
    rows = synth.dct_rows(n + 1, n, m)
    rng = np.random.default_rng(n)
    perm = rng.permutation(m)            # the caller's order need not be increasing
    rows_c = rows[perm]
    x = rng.standard_normal(n * n).astype(np.float32)
    y = rng.standard_normal(m).astype(np.float32)
    h = dct_handle(tv, rows_c, n)
    r = np.empty(m, np.float32)
    g = np.empty(n * n, np.float32)
    tv.tvcs_apply(h, x, y, r, g)
    rr = oracle.dct_Au(n, rows_c, x, y)
    # |C| has entries <= sqrt(2/n): |(C X C^T)_k| <= (2/n) sum |x| bounds each term's scale
    scale_r = (2.0 / n) * np.sum(np.abs(x)) + np.abs(y)
    assert np.all(np.abs(r - rr) <= 1e-5 * scale_r)
    gr = oracle.dct_At(n, rows_c, r.astype(np.float64))
    scale_g = (2.0 / n) * np.sum(np.abs(r))
    assert np.all(np.abs(g - gr) <= 1e-5 * scale_g)
    assert tv.tvcs_get_tau(h) == pytest.approx(1.9)
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("case", ["all", "one", "one_row"])
def test_dct_products_edge_sets(tv, case):
    # every coefficient (A is the whole orthonormal 2D DCT, so A^T A = I and
    # g = x - A^T y), a single coefficient, and all samples in one coefficient row
    # (every block but one of the cluster has no sampled entry)
    n = 32
    if case == "all":
        rows = np.random.default_rng(1).permutation(n * n).astype(np.int32)
    elif case == "one":
        rows = np.array([n * n - 1], np.int32)
    else:
        rows = np.arange(5 * n, 6 * n, dtype=np.int32)[::-1].copy()
    m = len(rows)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n * n).astype(np.float32)
    y = rng.standard_normal(m).astype(np.float32)
    h = dct_handle(tv, rows, n)
    r = np.empty(m, np.float32)
    g = np.empty(n * n, np.float32)
    tv.tvcs_apply(h, x, y, r, g)
    rr = oracle.dct_Au(n, rows, x, y)
    scale_r = (2.0 / n) * np.sum(np.abs(x)) + np.abs(y)
    assert np.all(np.abs(r - rr) <= 1e-5 * scale_r)
    gr = oracle.dct_At(n, rows, r.astype(np.float64))
    assert np.all(np.abs(g - gr) <= 1e-5 * max((2.0 / n) * np.sum(np.abs(r)), 1e-30))
    if case == "all":   # A^T A = I: g = x - A^T y, checked against the oracle's A^T alone
        aty = oracle.dct_At(n, rows, y.astype(np.float64))
        assert np.allclose(g, x - aty, rtol=0, atol=1e-5 * np.abs(x).max() * 4)
    else:
        assert np.isfinite(g).all()
    tv.tvcs_destroy(h)


def test_dct_power_iteration_gives_unit_lambda_max(tv):
    n, m = 32, 300
    rows = synth.dct_rows(3, n, m)
    opt = tv.tvcs_default_options()
    h = tv.tvcs_create_partial_dct(rows, n, 500.0, 64.0, 0.0, opt)
    assert tv.tvcs_get_tau(h) == pytest.approx(1.0 / 1.01, rel=1e-5)   # A A^T = I
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("algo", [0, 1])
def test_dct_solve_fixed_iterations(tv, algo):
    P = synth.make_dct_problem(32, 0.3, 13, 6, 500.0)
    rows = P.extra["rows"]
    h = dct_handle(tv, rows, 32, mu=P.mu, beta=P.beta, tau=1.9, max_iter=60, algo=algo)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve(h, P.f, u)
    ref = oracle.solve_dct(rows, P.f, 32, P.mu, P.beta, 1.9, max_iter=60, algo=algo)
    assert res.iters == 60
    assert rel(u, ref.u) <= 1e-5
    assert abs(res.objective - ref.info["objective"]) <= 1e-5 * ref.info["objective"]
    tv.tvcs_destroy(h)


def test_dct_rejects_bad_rows(tv):
    opt = tv.tvcs_default_options()
    with pytest.raises(tv.TvcsError):
        tv.tvcs_create_partial_dct(np.array([3, 5, 3], np.int32), 16, 1.0, 1.0, 0.0, opt)
    with pytest.raises(tv.TvcsError):
        tv.tvcs_create_partial_dct(np.array([0, 256], np.int32), 16, 1.0, 1.0, 0.0, opt)
    with pytest.raises(tv.TvcsError):
        tv.tvcs_create_partial_dct(np.array([0, 1], np.int32), 192, 1.0, 1.0, 0.0, opt)


def test_dct_workload_128_to_tolerance(tv):
    # Sec. 3.2: 128 x 128, 30% of the DCT coefficients, sigma 0.001, tau 1.9, beta 2^6,
    # stop at 5e-5; mu = 500 (a row of Table 1)
    P = synth.workload_dct128()
    rows = P.extra["rows"]
    h = dct_handle(tv, rows, 128, mu=P.mu, beta=P.beta, tau=1.9, max_iter=P.max_iter, tol=P.tol)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    assert res.status == tv.TVCS_OK and res.stopped_by_tol == 1
    full = oracle.solve_dct(rows, P.f, 128, P.mu, P.beta, 1.9, tol=P.tol, max_iter=P.max_iter)
    assert abs(res.iters - full.info["iters"]) <= max(2, full.info["iters"] // 50)
    same = oracle.solve_dct(rows, P.f, 128, P.mu, P.beta, 1.9, max_iter=res.iters)
    assert rel(u.cpu().numpy(), same.u) <= 1e-4
    assert abs(res.objective - same.info["objective"]) <= 1e-6 * same.info["objective"]
    # the reconstruction error against the phantom is small at 30% sampling
    assert rel(u.cpu().numpy(), P.ubar) < 0.2
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("algo", [0, 1])
def test_dct_beta_continuation_matches_oracle_stages(tv, algo):
    # Sec. 3.1's continuation in beta (2^4 .. 2^7) with the partial-DCT encoder: each stage
    # warm-started from the last stage's u (and lambda for IADM), w restarted at 0
    P = synth.make_dct_problem(32, 0.3, 5, 6, 200.0)
    rows = P.extra["rows"]
    betas = [16.0, 32.0, 64.0, 128.0]
    h = dct_handle(tv, rows, 32, mu=P.mu, beta=64.0, tau=1.9, max_iter=30, algo=algo)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve_continuation(h, P.f, u, betas)
    assert len(res) == 4 and all(r.iters == 30 for r in res)
    u0 = lam0 = None
    for b in betas:
        ref = oracle.solve_dct(rows, P.f, 32, P.mu, b, 1.9, max_iter=30, algo=algo, u0=u0,
                               lam0=lam0 if algo == 0 else None)
        u0, lam0 = ref.u, ref.lam
    assert rel(u, ref.u) <= 1e-5
    tv.tvcs_destroy(h)


def test_dct_handles_in_a_batched_call_equal_single_solves(tv):
    # several partial-DCT problems (different rows, data and mu) through
    # tvcs_solve_batched: the same results as one solve per handle
    probs = [synth.make_dct_problem(32, ratio, seed, 6, mu)
             for ratio, seed, mu in ((0.3, 11, 100.0), (0.2, 12, 300.0), (0.5, 13, 50.0))]
    hs = [dct_handle(tv, P.extra["rows"], 32, mu=P.mu, beta=64.0, tau=1.9, max_iter=40) for P in probs]
    us = [np.empty(P.N, np.float32) for P in probs]
    res = tv.tvcs_solve_batched(hs, [P.f for P in probs], us, [P.mu for P in probs])
    for h, P, u, r in zip(hs, probs, us, res):
        u1 = np.empty(P.N, np.float32)
        r1 = tv.tvcs_solve(h, P.f, u1)
        assert r.iters == r1.iters == 40
        assert np.array_equal(u, u1)
    for h in hs:
        tv.tvcs_destroy(h)

