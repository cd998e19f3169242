"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (binary32 iterates, binary64 oracle):
  * products r = A x - y, g = A^T r: per entry |err| <= 1e-5 * (|A| |x|)_i (and
    the same for g with |A|^T |r|) -- a binary32 dot of N <= 16384 terms summed
    by fixed-order partials carries at most ~log2(N) * 2^-24 relative to the
    absolute sum, ~1e-6, with margin;
  * one iteration: 1e-5 relative (norm-wise) on u, w, lambda;
  * fixed 50 iterations: <= 1e-5 relative image error (the required bar);
  * convergence runs: <= 1e-4 relative image error, <= 1e-6 relative objective gap.
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


def make_handle(tv, P, tau, algo=0, init=0, max_iter=500, on_device=True, tol=0.0, seed_only=False):
    opt = tv.tvcs_default_options()
    opt.tau = tau
    opt.algo = algo
    opt.init = init
    opt.max_iter = max_iter
    if seed_only:
        return tv.tvcs_create(None, P.seed, P.m, P.n, P.mu, P.beta, tol, opt)
    A = torch.from_numpy(P.A).cuda() if on_device else P.A
    return tv.tvcs_create(A, 0, P.m, P.n, P.mu, P.beta, tol, opt)


def small_problem(n, m, seed=3, mu=1e3, beta=10.0):
    return synth.make_problem(n, 0.0, seed, 4, mu, beta, m=m, noise_c=1e-3)


# ----------------------------------------------------------------------------- generator (a9 recipe)

@pytest.mark.parametrize("n,m,seed", [(32, 307, 0), (128, 4915, 1)])
def test_device_generator_bit_exact(tv, n, m, seed):
    N = n * n
    opt = tv.tvcs_default_options()
    opt.tau = 0.1
    h = tv.tvcs_create(None, seed, m, n, 1.0, 1.0, 0.0, opt)
    rng = np.random.default_rng(0)
    r = np.empty(m, np.float32)
    g = np.empty(N, np.float32)
    for j in [0, 1, 2, 3, N - 1] + list(rng.integers(0, N, 3)):
        x = np.zeros(N, np.float32)
        x[j] = 1.0
        tv.tvcs_apply(h, x, None, r, g)         # r = A e_j = column j, exactly
        col = np.array([synth.gaussian_matrix(seed, m, N, row0=i, nrows=1)[0, j]
                        for i in range(0, m, max(1, m // 64))], np.float32)
        assert np.array_equal(r[::max(1, m // 64)], col)
    for i in [0, m - 1, int(rng.integers(0, m))]:
        y = np.zeros(m, np.float32)
        y[i] = -1.0
        tv.tvcs_apply(h, np.zeros(N, np.float32), y, r, g)   # g = A^T e_i = row i, exactly
        assert np.array_equal(g, synth.gaussian_matrix(seed, m, N, row0=i, nrows=1)[0])
    tv.tvcs_destroy(h)


# ----------------------------------------------------------------------------- rows a6, a7

@pytest.mark.parametrize("n,m", [(16, 1), (16, 77), (32, 307), (48, 500), (64, 1229),
                                 (96, 2764), (128, 4915), (128, 151), (128, 153)])
def test_products_parity(tv, n, m):
    N = n * n
    A = synth.gaussian_matrix(11 + n, m, N)
    rng = np.random.default_rng(n + m)
    x = rng.standard_normal(N).astype(np.float32)
    y = rng.standard_normal(m).astype(np.float32)
    opt = tv.tvcs_default_options()
    opt.tau = 0.1
    h = tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, n, 1.0, 1.0, 0.0, opt)
    r = torch.empty(m, dtype=torch.float32, device="cuda")
    g = torch.empty(N, dtype=torch.float32, device="cuda")
    tv.tvcs_apply(h, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), r, g)
    r = r.cpu().numpy().astype(np.float64)
    g = g.cpu().numpy().astype(np.float64)
    rr = oracle.Au(A, x, y)
    scale_r = np.abs(A.astype(np.float64)) @ np.abs(x.astype(np.float64))
    assert np.all(np.abs(r - rr) <= 1e-5 * scale_r + 1e-30)
    # g is compared with the oracle's A^T applied to the GPU's own r (the input of that product)
    gr = oracle.At(A, r)
    scale_g = np.abs(A.astype(np.float64)).T @ np.abs(r)
    assert np.all(np.abs(g - gr) <= 1e-5 * scale_g + 1e-30)
    tv.tvcs_destroy(h)


# ----------------------------------------------------------------------------- rows a1-a3, a4-a5

@pytest.mark.parametrize("n,m", [(32, 307), (96, 2764), (128, 4915)])
def test_stage_parity(tv, n, m):
    P = small_problem(n, m)
    N = P.N
    tau = 0.11
    rng = np.random.default_rng(5)
    u0 = (P.ubar + 0.1 * rng.standard_normal((n, n))).astype(np.float32)
    lam0 = (0.3 * rng.standard_normal((2, n, n))).astype(np.float32)
    h = make_handle(tv, P, tau)
    tv.tvcs_set_state(h, tv.TVCS_STATE_F, P.f)
    tv.tvcs_set_state(h, tv.TVCS_STATE_U, u0.ravel())
    tv.tvcs_set_state(h, tv.TVCS_STATE_LAMBDA, lam0.ravel())
    # stage 1 (rows a1-a5): w-step, right-hand side, FFT u-solve
    tv.tvcs_run_stage(h, 1)
    w = tv.get_state(h, tv.TVCS_STATE_W).reshape(2, n, n)
    lam = tv.get_state(h, tv.TVCS_STATE_LAMBDA).reshape(2, n, n)
    rhs = tv.get_state(h, tv.TVCS_STATE_RHS).reshape(n, n)
    u64 = u0.astype(np.float64)
    d1, d2 = oracle.D(u64)
    z1 = d1 + lam0[0] / P.beta
    z2 = d2 + lam0[1] / P.beta
    w1, w2 = oracle.shrink(z1, z2, 1.0 / P.beta)
    w_ref = np.stack([w1.reshape(n, n), w2.reshape(n, n)])
    assert np.array_equal(lam, lam0)
    assert rel(w, w_ref) <= 1e-5
    g = oracle.At(P.A, oracle.Au(P.A, u64, P.f))
    # increment form of eq. (eqnorm11) times beta: D^T (beta (w - D u) - lambda) - mu g
    y = P.beta * (w_ref - np.stack([d1, d2])) - lam0
    rhs_ref = oracle.Dt(y[0], y[1]) - P.mu * g.reshape(n, n)
    assert rel(rhs, rhs_ref) <= 1e-5
    # the printed right-hand side of eq. (eqnorm11) and the oracle's u-solve of it
    yp = w_ref - lam0 / P.beta
    b_paper = oracle.Dt(yp[0], yp[1]) + (P.mu / (P.beta * tau)) * (u64 - tau * g.reshape(n, n))
    u_paper = oracle.usolve(b_paper, P.mu / (P.beta * tau))
    # the FFT solve for the increment, u^{k+1} = u^k + d
    u1 = tv.get_state(h, tv.TVCS_STATE_U).reshape(n, n)
    u_ref = u64 + oracle.usolve(rhs.astype(np.float64) / P.beta, P.mu / (P.beta * tau))
    assert rel(u1, u_ref) <= 1e-6
    assert rel(u1, u_paper) <= 1e-5
    # stage 2 (products) then stage 1 again applies the deferred multiplier update (eq. (udlamb))
    tv.tvcs_run_stage(h, 2)
    tv.tvcs_run_stage(h, 1)
    lam2 = tv.get_state(h, tv.TVCS_STATE_LAMBDA).reshape(2, n, n)
    e1, e2 = oracle.D(u1.astype(np.float64))
    lam_ref = lam0 - P.beta * (w.astype(np.float64) - np.stack([e1, e2]))
    assert rel(lam2, lam_ref) <= 1e-5
    tv.tvcs_destroy(h)


# ----------------------------------------------------------------------------- whole iterations

@pytest.mark.parametrize("algo", [0, 1])
def test_one_iteration_from_random_state(tv, algo):
    P = small_problem(64, 1229)
    n = P.n
    tau = oracle.default_tau(P.A)
    rng = np.random.default_rng(9)
    u0 = (P.ubar + 0.05 * rng.standard_normal((n, n))).astype(np.float32)
    lam0 = (0.5 * rng.standard_normal((2, n, n))).astype(np.float32) if algo == 0 else \
        np.zeros((2, n, n), np.float32)
    h = make_handle(tv, P, tau, algo=algo)
    tv.tvcs_set_state(h, tv.TVCS_STATE_F, P.f)
    tv.tvcs_set_state(h, tv.TVCS_STATE_U, u0.ravel())
    tv.tvcs_set_state(h, tv.TVCS_STATE_LAMBDA, lam0.ravel())
    res = tv.tvcs_iterate(h, 1)
    assert res.iters == 1
    ref = oracle.solve(P.A, P.f, n, P.mu, P.beta, tau, max_iter=1, algo=algo,
                       u0=u0, lam0=lam0 if algo == 0 else None)
    assert rel(tv.get_state(h, tv.TVCS_STATE_U), ref.u) <= 1e-5
    assert rel(tv.get_state(h, tv.TVCS_STATE_W), ref.w) <= 1e-5
    if algo == 0:
        assert rel(tv.get_state(h, tv.TVCS_STATE_LAMBDA), ref.lam) <= 1e-5
    tv.tvcs_destroy(h)


def test_fixed_50_iterations_n32(tv):
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=50)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=50)
    assert res.iters == 50
    assert rel(u.cpu().numpy(), ref.u) <= 1e-5
    assert abs(res.objective - ref.info["objective"]) <= 1e-6 * ref.info["objective"]
    tv.tvcs_destroy(h)


def test_convergence_parity_fast_setting(tv):
    # A setting that converges in a few hundred iterations (mu=50, beta=20 at
    # n=32): eq. (stop) must fire at (nearly) the same iteration, and the
    # results must agree at the tolerances of a converged run.
    P = synth.make_problem(32, 0.3, 0, 6, 50.0, 20.0, noise_c=1e-3)
    tau = oracle.default_tau(P.A)
    tol = 1e-4
    h = make_handle(tv, P, tau, max_iter=3000, tol=tol)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve(h, P.f, u)          # host pointers
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, tol=tol, max_iter=3000)
    assert res.status == tv.TVCS_OK and res.stopped_by_tol == 1
    assert abs(res.iters - ref.info["iters"]) <= 1
    same = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=res.iters)
    assert rel(u, same.u) <= 1e-4
    assert abs(res.objective - same.info["objective"]) <= 1e-6 * same.info["objective"]
    tv.tvcs_destroy(h)


def objective_exact(A, f, u, mu):
    """Phi(u) of eq. (tv) for a binary32 image, evaluated in binary64 (the oracle's TV)."""
    u = np.asarray(u, dtype=np.float64)
    n = int(round(np.sqrt(u.size)))
    r = A.astype(np.float64) @ u.ravel() - f.astype(np.float64)
    return oracle.tv(u.reshape(n, n)) + 0.5 * mu * float(r @ r)


def test_workload_n32_converges_to_tol(tv):
    # The n=32, m=307 workload (mu=1e3, beta=10, tol 1e-4) with an iteration cap large
    # enough for eq. (stop) to end the run (the oracle needs about 4.4K iterations):
    # the stop iteration within one of the oracle's, the image within 1e-4 and the
    # objective within 1e-6 of the oracle's converged run (Thm 4: the iterates
    # converge to a KKT point, so the two runs meet at the same solution).
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    cap = 20000
    h = make_handle(tv, P, tau, max_iter=cap, tol=P.tol)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve(h, P.f, u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, tol=P.tol, max_iter=cap)
    assert res.status == tv.TVCS_OK and res.stopped_by_tol == 1
    assert ref.info["iters"] < cap
    assert abs(res.iters - ref.info["iters"]) <= 1
    same = ref if res.iters == ref.info["iters"] else oracle.solve(
        P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=res.iters)
    assert rel(u, same.u) <= 1e-4 and rel(u, ref.u) <= 1e-4
    obj = same.info["objective"]
    assert abs(res.objective - obj) <= 1e-6 * obj                      # reported by the GPU
    assert abs(objective_exact(P.A, P.f, u, P.mu) - obj) <= 1e-6 * obj  # of the GPU's image
    print("n32 to tol: %d iterations, image %.2e, objective %.2e" %
          (res.iters, rel(u, same.u), abs(res.objective - obj) / obj))
    tv.tvcs_destroy(h)


def test_workload_n32_to_500_iterations(tv):
    # n=32, m=307, mu=1e3, beta=10, tol 1e-4, <= 500 iterations.
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=P.max_iter, tol=P.tol)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, tol=P.tol, max_iter=P.max_iter)
    assert abs(res.iters - ref.info["iters"]) <= 1
    same = ref if res.iters == ref.info["iters"] else oracle.solve(
        P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=res.iters)
    ug = u.cpu().numpy().astype(np.float64)
    assert rel(ug, same.u) <= 1e-4
    # This run ends at the iteration cap, away from the optimum, where the
    # objective is first-order in the iterate: |Phi(u) - Phi(v)| <= L ||u - v|| with
    # L = sqrt(8N) (TV: ||D|| <= sqrt(8), N terms) + mu ||A u - f|| ||A|| (fidelity).
    # (The 1e-6 gap of converged runs is checked in test_convergence_parity_fast_setting.)
    lip = np.sqrt(8 * P.N) + P.mu * np.sqrt(same.info["resid2"]) * np.sqrt(oracle.lambda_max(P.A))
    gap = abs(res.objective - same.info["objective"])
    assert gap <= 2.0 * lip * np.linalg.norm(ug - same.u.ravel()) + 1e-9 * same.info["objective"]
    assert gap <= 1e-5 * same.info["objective"]
    assert res.kkt_dual == pytest.approx(same.info["kkt_dual"], rel=1e-3)
    assert res.lambda_max_norm == pytest.approx(same.info["lambda_max_norm"], rel=1e-4)
    tv.tvcs_destroy(h)


def test_ftvcs_mode_50_iterations(tv):
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, algo=1, max_iter=50)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=50, algo=oracle.FTVCS)
    assert rel(u.cpu().numpy(), ref.u) <= 1e-5
    assert np.all(tv.get_state(h, tv.TVCS_STATE_LAMBDA) == 0)
    tv.tvcs_destroy(h)


def test_single_measurement_degenerate_case(tv):
    # m = 1: the fit of one measurement becomes nearly exact, so r = a.u - f cancels:
    # kappa = sum_j |a_j u_j| / |r| reaches ~3e3 within a few iterations, and a binary32
    # dot then leaves r with a relative error up to ~sqrt(N) 2^-24 kappa ~ 1e-3.  The
    # GPU's r must stay within that dot-product bound of the exact residual of its own
    # iterate, and the image within 1e-4 of the oracle's (vs 1e-5 when m is not tiny).
    n, m, iters = 16, 1, 20
    P = small_problem(n, m)
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=iters)
    u = np.empty(P.N, np.float32)
    tv.tvcs_solve(h, P.f, u)
    ref = oracle.solve(P.A, P.f, n, P.mu, P.beta, tau, max_iter=iters)
    assert rel(u, ref.u) <= 1e-4
    r = tv.get_state(h, tv.TVCS_STATE_R).astype(np.float64)
    a = P.A.astype(np.float64)[0]
    r_exact = a @ u.astype(np.float64) - float(P.f[0])
    bound = 2 * np.sqrt(P.N) * 2.0**-24 * (np.sum(np.abs(a * u)) + abs(float(P.f[0])))
    assert abs(r[0] - r_exact) <= bound
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("n,m,iters", [(16, 76, 30), (48, 77, 30), (96, 921, 30), (64, 409, 30),
                                       (16, 33, 20)])
def test_ragged_and_small_sizes(tv, n, m, iters):
    P = small_problem(n, m)
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=iters)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, n, P.mu, P.beta, tau, max_iter=iters)
    assert res.iters == iters
    # binary32 bound: each u-step's FFT round trip adds ~(2 log2 n + 4) 2^-24 of the step,
    # and w, lambda, g carry one rounding each; 1e-5 holds with margin for these iteration
    # counts (the increment form keeps the round-off proportional to the step).
    assert rel(u.cpu().numpy(), ref.u) <= 1e-5
    tv.tvcs_destroy(h)


def test_init_modes_and_zero_iterations(tv):
    P = small_problem(32, 307)
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=1)
    u = np.empty(P.N, np.float32)
    # u^0 = A^T f (reading C3): zero iterations via tvcs_iterate after set_state of f
    hz = make_handle(tv, P, tau, init=tv.TVCS_INIT_ZERO, max_iter=20)
    tv.tvcs_solve(hz, P.f, u)
    ref = oracle.solve(P.A, P.f, 32, P.mu, P.beta, tau, max_iter=20, init=oracle.INIT_ZERO)
    assert rel(u, ref.u) <= 1e-5
    tv.tvcs_solve(h, P.f, u)
    ref1 = oracle.solve(P.A, P.f, 32, P.mu, P.beta, tau, max_iter=1)
    assert rel(u, ref1.u) <= 1e-5
    tv.tvcs_destroy(h)
    tv.tvcs_destroy(hz)


def test_auto_tau_matches_oracle_power_iteration(tv):
    P = synth.workload_n32()
    opt = tv.tvcs_default_options()
    h = tv.tvcs_create(torch.from_numpy(P.A).cuda(), 0, P.m, P.n, P.mu, P.beta, 0.0, opt)
    assert tv.tvcs_get_tau(h) == pytest.approx(oracle.default_tau(P.A), rel=1e-4)
    tv.tvcs_destroy(h)


def test_seed_generated_A_solve(tv):
    P = small_problem(64, 1229, seed=21)
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=30, seed_only=True)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, 64, P.mu, P.beta, tau, max_iter=30)
    assert rel(u.cpu().numpy(), ref.u) <= 1e-5
    tv.tvcs_destroy(h)


def test_batched_entry_point_matches_single_solves(tv):
    probs = [small_problem(32, 307, seed=s) for s in (1, 2, 3)]
    hs, fs, us = [], [], []
    for P in probs:
        hs.append(make_handle(tv, P, 0.12, max_iter=25))
        fs.append(P.f)
        us.append(np.empty(P.N, np.float32))
    mus = [200.0, 500.0, 1000.0]
    res = tv.tvcs_solve_batched(hs, fs, us, mus)
    for P, u, r, mu in zip(probs, us, res, mus):
        ref = oracle.solve(P.A, P.f, 32, mu, P.beta, 0.12, max_iter=25)
        assert r.iters == 25
        assert rel(u, ref.u) <= 1e-5
    for h in hs:
        tv.tvcs_destroy(h)


def test_workload_n128_300_iterations(tv):
    # The benchmark workload at full size, in the launch configuration bench.py times.
    P = synth.workload_n128()
    tau = oracle.default_tau(P.A, 100)
    h = make_handle(tv, P, tau, max_iter=300)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=300)
    assert res.iters == 300
    assert rel(u.cpu().numpy(), ref.u) <= 1e-4
    assert abs(res.objective - ref.info["objective"]) <= 1e-5 * ref.info["objective"]
    tv.tvcs_destroy(h)


def test_workload_n128_is_positively_homogeneous(tv):
    # At the full benchmark size, where the oracle is compared above: the problem
    # (4 f, mu / 4, beta / 4) has the minimisers 4 u*, and every step of the iteration
    # commutes with that scaling (the shrink threshold 1/beta, the divisor
    # beta Lambda_pq + mu/tau, the terms beta w and mu g).  With a power of two every
    # binary32 operation of the kernels commutes with it too, so the runs agree bit for bit.
    P = synth.workload_n128()
    tau = oracle.default_tau(P.A, 100)
    A = torch.from_numpy(P.A).cuda()
    us, objs = [], []
    for c in (1.0, 4.0):
        opt = tv.tvcs_default_options()
        opt.tau = tau
        opt.max_iter = 300
        h = tv.tvcs_create(A, 0, P.m, P.n, P.mu / c, P.beta / c, 0.0, opt)
        u = torch.empty(P.N, dtype=torch.float32, device="cuda")
        res = tv.tvcs_solve(h, torch.from_numpy(c * P.f).cuda(), u)
        assert res.iters == 300
        us.append(u.cpu().numpy())
        objs.append(res.objective)
        tv.tvcs_destroy(h)
    assert np.any(us[0])
    assert np.array_equal(us[1], 4.0 * us[0])
    assert objs[1] == pytest.approx(4.0 * objs[0], rel=1e-12)


def test_binding_waits_for_the_torch_stream_that_wrote_f(tv):
    # the handle's stream does not wait for torch's streams; the binding finishes the
    # work queued on the current torch stream before the call, so an f whose copy sits
    # behind a ~50 ms device delay on that stream is read complete
    P = small_problem(32, 307)
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, max_iter=20)
    u_ref = np.empty(P.N, np.float32)
    tv.tvcs_solve(h, P.f, u_ref)
    side = torch.cuda.Stream()
    f_host = torch.from_numpy(P.f).pin_memory()
    with torch.cuda.stream(side):
        f = torch.zeros(P.m, dtype=torch.float32, device="cuda")
        u = torch.full((P.N,), float("nan"), device="cuda")
        torch.cuda._sleep(100_000_000)
        f.copy_(f_host, non_blocking=True)
        res = tv.tvcs_solve(h, f, u)
    assert res.iters == 20
    assert np.array_equal(u.cpu().numpy(), u_ref)
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("algo", [0, 1])
def test_zero_measurements_give_the_zero_image(tv, algo):
    # f = 0: u = 0 is the minimiser, u^0 = A^T f = 0, and eq. (stop) with reading C5
    # (||u^k|| = 0: stop once ||u^{k+1}|| = 0) ends the solve after one iteration, as in
    # the oracle.
    P = small_problem(32, 307)
    tau = oracle.default_tau(P.A)
    h = make_handle(tv, P, tau, algo=algo, max_iter=50, tol=1e-4)
    f0 = np.zeros(P.m, np.float32)
    u = np.full(P.N, np.nan, np.float32)
    res = tv.tvcs_solve(h, f0, u)
    ref = oracle.solve(P.A, f0, P.n, P.mu, P.beta, tau, tol=1e-4, max_iter=50, algo=algo)
    assert ref.info["iters"] == 1
    assert res.iters == 1 and res.stopped_by_tol == 1 and res.status == tv.TVCS_OK
    assert not np.any(u) and res.objective == 0.0
    tv.tvcs_destroy(h)


def test_workload_n128_300_iterations_ftvcs(tv):
    # Algorithm 1 (FTVCS, lambda = 0) on the benchmark workload at full size.
    P = synth.workload_n128()
    tau = oracle.default_tau(P.A, 100)
    h = make_handle(tv, P, tau, algo=1, max_iter=300)
    u = torch.empty(P.N, dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve(h, torch.from_numpy(P.f).cuda(), u)
    ref = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=300, algo=oracle.FTVCS)
    assert res.iters == 300
    assert rel(u.cpu().numpy(), ref.u) <= 1e-4
    assert abs(res.objective - ref.info["objective"]) <= 1e-5 * ref.info["objective"]
    assert np.all(tv.get_state(h, tv.TVCS_STATE_LAMBDA) == 0)
    tv.tvcs_destroy(h)


@pytest.mark.parametrize("algo", [1, 0])
def test_beta_continuation_matches_oracle_stages(tv, algo):
    # Sec. 3.1's practice: beta = 2^4 .. 2^7, each stage warm-started from the last.
    P = synth.make_problem(32, 0.3, 5, 6, 1e3, 10.0, noise_c=1e-3)
    tau = oracle.default_tau(P.A)
    betas = [2.0 ** 4, 2.0 ** 5, 2.0 ** 6, 2.0 ** 7]
    h = make_handle(tv, P, tau, algo=algo, max_iter=40)
    u = np.empty(P.N, np.float32)
    res = tv.tvcs_solve_continuation(h, P.f, u, betas)
    assert len(res) == 4 and all(r.iters == 40 for r in res)
    u0 = lam0 = None
    for b in betas:   # the oracle, stage after stage from the previous stage's u and lambda
        ref = oracle.solve(P.A, P.f, P.n, P.mu, b, tau, max_iter=40,
                           algo=oracle.FTVCS if algo == 1 else oracle.IADM, u0=u0,
                           lam0=lam0 if algo == 0 else None)
        u0, lam0 = ref.u, ref.lam
    assert rel(u, ref.u) <= 1e-5
    # the handle's own beta is in force again: a plain solve equals a fresh handle's
    u1 = np.empty(P.N, np.float32)
    tv.tvcs_solve(h, P.f, u1)
    h2 = make_handle(tv, P, tau, algo=algo, max_iter=40)
    u2 = np.empty(P.N, np.float32)
    tv.tvcs_solve(h2, P.f, u2)
    assert np.array_equal(u1, u2)
    tv.tvcs_destroy(h)
    tv.tvcs_destroy(h2)


# ----------------------------------------------------------------------------- reduction accuracy

@pytest.mark.parametrize("n,m,precision", [(128, 4915, 0), (128, 4915, 1), (32, 307, 0)])
def test_resid2_is_the_binary64_sum_of_the_stored_residual(tv, n, m, precision):
    # ||r||^2 of eq. (stop) and of the objective is summed on the device in double-single
    # binary32 pairs (exact squares, renormalised additions: about 44 bits), not in
    # binary64.  Against the binary64 sum of the squares of the same stored binary32
    # residual it agrees to 1e-9 of the sum (m <= 4915 additions of at most 2^-44
    # each bound it by 3e-10); a plain binary32 sum misses by 1e-7 to 1e-5.
    P = small_problem(n, m, seed=21)
    opt = tv.tvcs_default_options()
    opt.tau = oracle.default_tau(P.A)
    opt.precision = precision
    opt.max_iter = 30
    h = tv.tvcs_create(torch.from_numpy(P.A).cuda(), 0, P.m, P.n, P.mu, P.beta, 0.0, opt)
    u = np.empty(P.N, np.float32)
    tv.tvcs_solve(h, P.f, u)
    for k in (1, 7):
        res = tv.tvcs_iterate(h, k)
        r = np.empty(P.m, np.float32)
        tv.tvcs_get_state(h, tv.TVCS_STATE_R, r)
        exact = float(np.sum(r.astype(np.float64) ** 2))
        naive = float(np.sum(r * r, dtype=np.float32))
        print("n %d prec %d: resid2 rel err %.2e (binary32 sum %.2e)"
              % (n, precision, abs(res.resid2 - exact) / exact, abs(naive - exact) / exact))
        assert abs(res.resid2 - exact) <= 1e-9 * exact
    tv.tvcs_destroy(h)
