"""Failure statuses of the solver, exercised in forms that fault no GPU.

TVCS_ERR_DIVERGED: a non-finite measurement makes the iterate non-finite; the
u-step's stop test (eq. (stop)) records it, the run ends, and the call returns
the status while the handle stays usable (the next finite solve matches the
FP64 oracle).  In batches only the affected image or problem reports it.

TVCS_ERR_TIMEOUT: the product kernel's grid barrier is made to wait for one
arrival that never comes (a test hook); its bounded spin runs out after
timeout_cycles, every block records the timeout, lets its own copies land and
returns; the call reports the status and the next call on the handle succeeds.
"""
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


def _single(tv, P, tau, iters, timeout_cycles=0):
    opt = tv.tvcs_default_options()
    opt.tau = tau
    opt.max_iter = iters
    opt.timeout_cycles = timeout_cycles
    return tv.tvcs_create(torch.from_numpy(P.A).cuda(), 0, P.m, P.n, P.mu, P.beta, 0.0, opt)


def test_nan_measurement_single_solve_diverges_then_handle_is_usable(tv):
    P = synth.make_problem(32, 0.3, 0, 6, 1e3, 10.0, name="nan_single")
    tau = oracle.default_tau(P.A)
    h = _single(tv, P, tau, 40)
    f_bad = P.f.copy()
    f_bad[17] = np.nan
    u = np.empty(P.N, np.float32)
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_solve(h, f_bad, u)
    assert ei.value.status == tv.TVCS_ERR_DIVERGED
    res = tv.tvcs_solve(h, P.f, u)
    assert res.iters == 40 and res.status == tv.TVCS_OK
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=40)
    assert rel(u, ref.u) <= 1e-5
    tv.tvcs_destroy(h)


def test_nan_measurement_in_shared_batch_only_that_image_fails(tv):
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=5, n=32, ratio=0.3, seed=9, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    opt = tv.tvcs_default_options()
    opt.precision = tv.TVCS_PREC_BF16X2
    opt.tau = tau
    opt.max_iter = 30
    h = tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, 32, 1e3, 10.0, 0.0, opt)
    Fs = [F[b].copy() for b in range(5)]
    Fs[3][0] = np.inf
    us = [np.empty(N, np.float32) for _ in range(5)]
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_solve_batched([h] * 5, Fs, us, mus)
    assert ei.value.status == tv.TVCS_ERR_DIVERGED
    res = ei.value.results
    assert res[3].status == tv.TVCS_ERR_DIVERGED
    for b in (0, 1, 2, 4):
        assert res[b].status >= 0 and res[b].iters == 30
        ref = oracle.solve(A, F[b], 32, mus[b], 10.0, tau, max_iter=30)
        assert rel(us[b], ref.u) <= 1e-4, b
    # the handle still solves a finite batch
    res2 = tv.tvcs_solve_batched([h] * 5, [F[b] for b in range(5)], us, mus)
    assert all(r.iters == 30 for r in res2)
    ref = oracle.solve(A, F[3], 32, mus[3], 10.0, tau, max_iter=30)
    assert rel(us[3], ref.u) <= 1e-4
    tv.tvcs_destroy(h)


def test_nan_measurement_in_uneven_batch_only_that_problem_fails(tv):
    probs = [synth.make_problem(n, r, 91 + k, 4, 1e3, 10.0, noise_c=1e-3)
             for k, (n, r) in enumerate([(32, 0.3), (16, 0.5), (48, 0.2)])]
    hs = []
    for P in probs:
        opt = tv.tvcs_default_options()
        opt.tau = 0.1
        opt.max_iter = 20
        opt.a_mode = tv.TVCS_A_REGENERATE
        hs.append(tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, 0.0, opt))
    fs = [P.f.copy() for P in probs]
    fs[1][2] = np.nan
    us = [np.empty(P.N, np.float32) for P in probs]
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_solve_batched(hs, fs, us)
    assert ei.value.status == tv.TVCS_ERR_DIVERGED
    res = ei.value.results
    assert res[1].status == tv.TVCS_ERR_DIVERGED
    for k in (0, 2):
        P = probs[k]
        assert res[k].status >= 0 and res[k].iters == 20
        ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, 0.1, max_iter=20)
        assert rel(us[k], ref.u) <= 1e-5
    for h in hs:
        tv.tvcs_destroy(h)


@pytest.mark.parametrize("n,m", [(32, 307), (128, 4915)])
def test_grid_barrier_timeout_is_reported_and_handle_recovers(tv, n, m):
    # 2^22 SM cycles (about 2 ms at 2 GHz): far above any wait of a normal launch
    # (one product launch takes 10-60 us), so only the held barrier runs out.
    N = n * n
    P = synth.make_problem(n, m / N, 3, 6, 1e3, 10.0, name="timeout")
    tau = oracle.default_tau(P.A, 30)
    h = _single(tv, P, tau, 20, timeout_cycles=1 << 22)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(N).astype(np.float32)
    r_ok = np.empty(m, np.float32)
    g_ok = np.empty(N, np.float32)
    tv.tvcs_apply(h, x, P.f, r_ok, g_ok)
    tv.tvcs_test_hold_grid_barrier(h, 1)
    r = np.empty(m, np.float32)
    g = np.empty(N, np.float32)
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_apply(h, x, P.f, r, g)
    assert ei.value.status == tv.TVCS_ERR_TIMEOUT
    u = np.empty(N, np.float32)
    with pytest.raises(tv.TvcsError) as ei:
        tv.tvcs_solve(h, P.f, u)
    assert ei.value.status == tv.TVCS_ERR_TIMEOUT
    # released: the same handle gives the same products and a correct solve
    tv.tvcs_test_hold_grid_barrier(h, 0)
    tv.tvcs_apply(h, x, P.f, r, g)
    assert np.array_equal(r, r_ok) and np.array_equal(g, g_ok)
    res = tv.tvcs_solve(h, P.f, u)
    assert res.iters == 20
    ref = oracle.solve(P.A, P.f, n, P.mu, P.beta, tau, max_iter=20)
    assert rel(u, ref.u) <= 1e-5
    tv.tvcs_destroy(h)
