"""Products with A regenerated inside the kernel and the uneven batch (row a9),
against the FP64 oracle through the C ABI.

Tolerances are those of test_gpu_parity: products per entry 1e-5 of |A||x|
(and of |A|^T |r| for g); fixed-iteration runs 1e-5 relative image error; runs
to eq. (stop) 1e-4 relative image error at the GPU's iteration count.  The
regenerated entries themselves are checked bit for bit against the input
generator: with x = e_j the product returns column j exactly, and with
x = 0, y = -e_i, g = A^T e_i returns row i exactly (sums of one entry and
exact zeros).
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


def regen_handle(tv, seed, m, n, mu=1.0, beta=10.0, tau=0.1, max_iter=50, tol=0.0, init=0):
    opt = tv.tvcs_default_options()
    opt.tau = tau
    opt.max_iter = max_iter
    opt.init = init
    opt.a_mode = tv.TVCS_A_REGENERATE
    return tv.tvcs_create(None, seed, m, n, mu, beta, tol, opt)


# ----------------------------------------------------------------------------- entries, products

@pytest.mark.parametrize("n,m,seed", [(16, 77, 5), (64, 409, 6), (192, 2000, 7)])
def test_regenerated_entries_bit_exact(tv, n, m, seed):
    N = n * n
    h = regen_handle(tv, seed, m, n)
    rng = np.random.default_rng(1)
    r = np.empty(m, np.float32)
    g = np.empty(N, np.float32)
    A = synth.gaussian_matrix(seed, m, N)
    for j in [0, 3, N - 1] + list(rng.integers(0, N, 2)):
        x = np.zeros(N, np.float32)
        x[j] = 1.0
        tv.tvcs_apply(h, x, None, r, g)
        assert np.array_equal(r, A[:, j])
    for i in [0, m - 1, int(rng.integers(0, m))]:
        y = np.zeros(m, np.float32)
        y[i] = -1.0
        tv.tvcs_apply(h, np.zeros(N, np.float32), y, r, g)
        assert np.array_equal(g, synth.gaussian_matrix(seed, m, N, row0=i, nrows=1)[0])
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("n,m", [(16, 1), (16, 77), (32, 307), (48, 500), (64, 409), (96, 1843),
                                 (128, 4915), (128, 151), (192, 3686)])
def test_regen_products_parity(tv, n, m):
    N = n * n
    seed = 31 + n + m
    A = synth.gaussian_matrix(seed, m, N)
    rng = np.random.default_rng(n + m)
    x = rng.standard_normal(N).astype(np.float32)
    y = rng.standard_normal(m).astype(np.float32)
    h = regen_handle(tv, seed, m, n)
    r = torch.empty(m, dtype=torch.float32, device="cuda")
    g = torch.empty(N, dtype=torch.float32, device="cuda")
    tv.tvcs_apply(h, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), r, g)
    r = r.cpu().numpy().astype(np.float64)
    g = g.cpu().numpy().astype(np.float64)
    A64 = np.abs(A.astype(np.float64))
    assert np.all(np.abs(r - oracle.Au(A, x, y)) <= 1e-5 * (A64 @ np.abs(x.astype(np.float64))) + 1e-30)
    assert np.all(np.abs(g - oracle.At(A, r)) <= 1e-5 * (A64.T @ np.abs(r)) + 1e-30)
    tv.tvcs_destroy(h)


def test_regen_agrees_with_stored_generated_A(tv):
    n, m, seed = 96, 2764, 12
    N = n * n
    opt = tv.tvcs_default_options()
    opt.tau = 0.1
    hs = tv.tvcs_create(None, seed, m, n, 1.0, 10.0, 0.0, opt)      # A generated into memory
    hr = regen_handle(tv, seed, m, n)                                # A regenerated per product
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N).astype(np.float32)
    r1, r2 = np.empty(m, np.float32), np.empty(m, np.float32)
    g1, g2 = np.empty(N, np.float32), np.empty(N, np.float32)
    tv.tvcs_apply(hs, x, None, r1, g1)
    tv.tvcs_apply(hr, x, None, r2, g2)
    assert rel(r2, r1) <= 1e-6 and rel(g2, g1) <= 1e-6
    tv.tvcs_destroy(hs)
    tv.tvcs_destroy(hr)


def test_regen_auto_tau_matches_oracle(tv):
    P = synth.workload_n32()
    opt = tv.tvcs_default_options()
    opt.a_mode = tv.TVCS_A_REGENERATE
    h = tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, 0.0, opt)
    assert tv.tvcs_get_tau(h) == pytest.approx(oracle.default_tau(P.A), rel=1e-4)
    tv.tvcs_destroy(h)


def test_regen_rejects_stored_A_and_other_precisions(tv):
    opt = tv.tvcs_default_options()
    opt.a_mode = tv.TVCS_A_REGENERATE
    A = np.zeros((10, 256), np.float32)
    with pytest.raises(tv.TvcsError):
        tv.tvcs_create(A, 0, 10, 16, 1.0, 1.0, 0.0, opt)
    opt.precision = tv.TVCS_PREC_BF16X2
    with pytest.raises(tv.TvcsError):
        tv.tvcs_create(None, 0, 10, 16, 1.0, 1.0, 0.0, opt)


# ----------------------------------------------------------------------------- single solves

def test_regen_solve_fixed_50_iterations_n32(tv):
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    h = regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, tau, max_iter=50)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve(h, P.f, u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=50)
    assert res.iters == 50
    assert rel(u, ref.u) <= 1e-5
    assert abs(res.objective - ref.info["objective"]) <= 1e-6 * ref.info["objective"]
    tv.tvcs_destroy(h)


def test_regen_solve_to_tolerance(tv):
    P = synth.make_problem(32, 0.3, 0, 6, 50.0, 20.0, noise_c=1e-3)
    tau = oracle.default_tau(P.A)
    h = regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, tau, max_iter=3000, tol=1e-4)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve(h, P.f, u)
    assert res.status == tv.TVCS_OK and res.stopped_by_tol == 1
    same = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=res.iters)
    assert rel(u, same.u) <= 1e-4
    assert abs(res.objective - same.info["objective"]) <= 1e-6 * same.info["objective"]
    tv.tvcs_destroy(h)


# ----------------------------------------------------------------------------- uneven batch

def uneven_problems(shapes, first_seed=41, mus=None):
    out = []
    for k, (n, ratio) in enumerate(shapes):
        mu = mus[k] if mus else 1e3
        out.append(synth.make_problem(n, ratio, first_seed + k, 4, mu, 10.0, noise_c=1e-3))
    return out


SHAPES = [(16, 0.3), (32, 0.2), (48, 0.1), (64, 0.3), (32, 0.5), (16, 0.5), (64, 0.1)]


def test_uneven_batch_fixed_iterations(tv):
    mus = [2e2, 5e2, 1e3, 2e3, 1e3, 5e2, 1e3]
    probs = uneven_problems(SHAPES, mus=mus)
    taus = [oracle.default_tau(P.A) for P in probs]
    hs = [regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, t, max_iter=40)
          for P, t in zip(probs, taus)]
    us = [np.empty(P.N, np.float32) for P in probs]
    res = tv.tvcs_solve_batched(hs, [P.f for P in probs], us)
    for P, t, u, r in zip(probs, taus, us, res):
        ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, t, max_iter=40)
        assert r.iters == 40
        assert rel(u, ref.u) <= 1e-5, (P.n, P.m)
        assert abs(r.objective - ref.info["objective"]) <= 1e-5 * ref.info["objective"]
    # the same problem set again reuses the batch state and gives the same result
    us2 = [np.empty(P.N, np.float32) for P in probs]
    tv.tvcs_solve_batched(hs, [P.f for P in probs], us2)
    for a, b in zip(us, us2):
        assert np.array_equal(a, b)
    for h in hs:
        tv.tvcs_destroy(h)


def test_uneven_batch_with_mu_overrides(tv):
    probs = uneven_problems(SHAPES[:4], first_seed=61)
    hs = [regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, 0.1, max_iter=30) for P in probs]
    us = [np.empty(P.N, np.float32) for P in probs]
    mus = [300.0, 600.0, 900.0, 1200.0]
    tv.tvcs_solve_batched(hs, [P.f for P in probs], us, mus)
    for P, h, u, mu in zip(probs, hs, us, mus):
        ref = oracle.solve(P.A, P.f, P.n, mu, P.beta, 0.1, max_iter=30)
        assert rel(u, ref.u) <= 1e-5
    for h in hs:
        tv.tvcs_destroy(h)


def test_uneven_batch_per_problem_stop(tv):
    # Different mu and sizes converge at different iterations: every problem
    # stops on its own eq. (stop) and leaves the product launch's work list.
    mus = [50.0, 100.0, 50.0, 200.0]
    probs = [synth.make_problem(n, r, 71 + k, 6, mus[k], 20.0, noise_c=1e-3)
             for k, (n, r) in enumerate([(32, 0.3), (16, 0.5), (48, 0.2), (32, 0.5)])]
    taus = [oracle.default_tau(P.A) for P in probs]
    hs = [regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, t, max_iter=3000, tol=1e-4)
          for P, t in zip(probs, taus)]
    us = [np.empty(P.N, np.float32) for P in probs]
    res = tv.tvcs_solve_batched(hs, [P.f for P in probs], us)
    iters = [r.iters for r in res]
    assert len(set(iters)) > 1
    for P, t, u, r in zip(probs, taus, us, res):
        assert r.status == tv.TVCS_OK and r.stopped_by_tol == 1
        full = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, t, tol=1e-4, max_iter=3000)
        assert abs(r.iters - full.info["iters"]) <= 1
        same = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, t, max_iter=r.iters)
        assert rel(u, same.u) <= 1e-4
        assert abs(r.objective - same.info["objective"]) <= 1e-6 * same.info["objective"]
    for h in hs:
        tv.tvcs_destroy(h)


def test_uneven_batch_single_problem_and_single_measurement(tv):
    # count = 1, and a problem with m = 1 next to a regular one
    P = synth.make_problem(16, 0.0, 81, 3, 1e3, 10.0, m=1, noise_c=0.0)
    Q = synth.make_problem(32, 0.3, 82, 3, 1e3, 10.0, noise_c=1e-3)
    taup = oracle.default_tau(P.A)
    hp = regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, taup, max_iter=20)
    hq = regen_handle(tv, Q.seed, Q.m, Q.n, Q.mu, Q.beta, 0.1, max_iter=20)
    u1 = np.empty(Q.N, np.float32)
    tv.tvcs_solve_batched([hq], [Q.f], [u1])
    assert rel(u1, oracle.solve(Q.A, Q.f, Q.n, Q.mu, Q.beta, 0.1, max_iter=20).u) <= 1e-5
    up, uq = np.empty(P.N, np.float32), np.empty(Q.N, np.float32)
    tv.tvcs_solve_batched([hp, hq], [P.f, Q.f], [up, uq])
    # m = 1 cancels the residual (see test_single_measurement_degenerate_case): 1e-4
    refp = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, taup, max_iter=20)
    assert rel(up, refp.u) <= 1e-4
    assert rel(uq, u1) <= 1e-5
    tv.tvcs_destroy(hp)
    tv.tvcs_destroy(hq)


def test_uneven_workload_64_problems_sampled(tv):
    # The 64-problem batch at full size (n in {64, 96, 128, 192}, m/n^2 in
    # {0.1, 0.2, 0.3, 0.5}, A regenerated in the kernel, to tol 1e-4).  The
    # oracle checks the problems it finishes in seconds (every n = 64 one with
    # m <= 1229); the others must converge with finite results.
    probs = synth.workload_uneven(64, materialise=False)
    hs, taus = [], []
    for P in probs:
        h = regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, 0.0, max_iter=P.max_iter, tol=P.tol)
        hs.append(h)
        taus.append(tv.tvcs_get_tau(h))
    us = [np.empty(P.N, np.float32) for P in probs]
    res = tv.tvcs_solve_batched(hs, [P.f for P in probs], us)
    for r in res:
        assert r.status in (tv.TVCS_OK, tv.TVCS_NOT_CONVERGED)
        assert np.isfinite(r.objective)
    checked = 0
    for P, t, u, r in zip(probs, taus, us, res):
        if P.n != 64 or P.m > 1229:
            continue
        A = synth.gaussian_matrix(P.seed, P.m, P.N)
        same = oracle.solve(A, P.f, P.n, P.mu, P.beta, t, max_iter=r.iters)
        assert rel(u, same.u) <= 1e-4, (P.seed, P.n, P.m)
        checked += 1
    assert checked >= 3
    for h in hs:
        tv.tvcs_destroy(h)


def test_uneven_workload_64_problems_every_side_fixed_iterations(tv):
    # The whole 64-problem batch (A regenerated in the kernel) for a fixed 20
    # iterations; a seeded sample covering every image side (64, 96, 128, 192) and
    # every sampling ratio of the larger sides is compared with the FP64 oracle at
    # 1e-5 (the oracle regenerates each sampled A on the host).
    probs = synth.workload_uneven(64, materialise=False)
    iters = 20
    hs, taus = [], []
    for P in probs:
        h = regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, 0.0, max_iter=iters, tol=0.0)
        hs.append(h)
        taus.append(tv.tvcs_get_tau(h))
    us = [np.empty(P.N, np.float32) for P in probs]
    res = tv.tvcs_solve_batched(hs, [P.f for P in probs], us)
    assert all(r.iters == iters for r in res)
    sample = {3: (64, 0.5), 28: (96, 0.1), 6: (96, 0.3), 18: (96, 0.5), 15: (128, 0.1),
              22: (128, 0.2), 12: (128, 0.5), 5: (192, 0.1), 58: (192, 0.3), 23: (192, 0.5)}
    seen = set()
    for k, P in enumerate(probs):
        if P.seed not in sample:
            continue
        assert (P.n, round(P.m / P.N, 1)) == sample[P.seed]
        A = synth.gaussian_matrix(P.seed, P.m, P.N)
        ref = oracle.solve(A, P.f, P.n, P.mu, P.beta, taus[k], max_iter=iters)
        del A
        err = rel(us[k], ref.u)
        print("seed %d n %d m %d: rel image err %.2e" % (P.seed, P.n, P.m, err))
        assert err <= 1e-5, (P.seed, P.n, P.m, err)
        assert abs(res[k].objective - ref.info["objective"]) <= 1e-5 * ref.info["objective"]
        seen.add(P.n)
    assert seen == {64, 96, 128, 192}
    for h in hs:
        tv.tvcs_destroy(h)


def test_uneven_results_do_not_depend_on_the_batch_or_the_tuned_plan(tv):
    # The regenerating products add every sum in an order fixed by the problem
    # alone (row segments, chunk slots), whatever launch shape the tuner picks for
    # a problem set.  A problem solved in three different batches (each tuned on
    # its own: different widest rows, tile heights and chunk-to-cluster
    # assignments) gives bit-identical images and summaries.
    probs = uneven_problems(SHAPES, first_seed=101)
    extra = uneven_problems([(96, 0.2), (128, 0.1)], first_seed=151)
    hs = [regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, 0.1, max_iter=25) for P in probs]
    hx = [regen_handle(tv, P.seed, P.m, P.n, P.mu, P.beta, 0.1, max_iter=25) for P in extra]
    u_all = [np.empty(P.N, np.float32) for P in probs]
    r_all = tv.tvcs_solve_batched(hs, [P.f for P in probs], u_all)
    # the first three problems next to two larger ones (wider rows: other tiles)
    sub = [0, 1, 2]
    u_sub = [np.empty(probs[k].N, np.float32) for k in sub] + [np.empty(P.N, np.float32) for P in extra]
    r_sub = tv.tvcs_solve_batched([hs[k] for k in sub] + hx, [probs[k].f for k in sub] + [P.f for P in extra],
                                  u_sub)
    for j, k in enumerate(sub):
        assert np.array_equal(u_sub[j], u_all[k]), k
        assert r_sub[j].objective == r_all[k].objective and r_sub[j].resid2 == r_all[k].resid2
    # one problem alone
    for k in (3, 6):
        u1 = np.empty(probs[k].N, np.float32)
        r1 = tv.tvcs_solve_batched([hs[k]], [probs[k].f], [u1])
        assert np.array_equal(u1, u_all[k]), k
        assert r1[0].objective == r_all[k].objective
    # and the batch against the oracle, so that the equal results are also right
    for k in (0, 6):
        P = probs[k]
        ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, 0.1, max_iter=25)
        assert rel(u_all[k], ref.u) <= 1e-5
    for h in hs + hx:
        tv.tvcs_destroy(h)


def test_regen_autotune_off_gives_the_same_results(tv):
    # With autotune off the first candidate shape runs untimed; the regenerating
    # products add in a fixed order, so single solves and an uneven batch give
    # bit-identical results either way.
    probs = uneven_problems(SHAPES[:4], first_seed=171)
    res = {}
    for tune in (1, 0):
        hs = []
        for P in probs:
            opt = tv.tvcs_default_options()
            opt.tau = 0.1
            opt.max_iter = 15
            opt.a_mode = tv.TVCS_A_REGENERATE
            opt.autotune = tune
            hs.append(tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, 0.0, opt))
        us = [np.empty(P.N, np.float32) for P in probs]
        tv.tvcs_solve_batched(hs, [P.f for P in probs], us)
        u0 = np.empty(probs[0].N, np.float32)
        tv.tvcs_solve(hs[0], probs[0].f, u0)
        res[tune] = (us, u0)
        for h in hs:
            tv.tvcs_destroy(h)
    for a, b in zip(res[1][0], res[0][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[1][1], res[0][1])
