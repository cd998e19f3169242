"""Pins for the oracle's Algorithms 1 (FTVCS) and 2 (IADM)."""
import numpy as np
import pytest

import oracle
import synth
from indep_solvers import chambolle_pock, diff_matrix, dual_projected_gradient


def _problem(n, m, mu, beta, seed=7, noise_c=1e-2):
    return synth.make_problem(n, 0.0, seed, 3, mu, beta, m=m, noise_c=noise_c)


def _dense_step(P, tau, u, lam, iadm=True):
    """One iteration written with explicit dense matrices (eqs. (iadmw) with the
    augmented-Lagrangian sign, (eqnorm11), (udlamb)); FTVCS when iadm=False."""
    n, N = P.n, P.N
    A = P.A.astype(np.float64)
    f = P.f.astype(np.float64)
    Dm = diff_matrix(n)
    beta, mu = P.beta, P.mu
    u = u.ravel()
    lam = lam.ravel() if iadm else np.zeros(2 * N)
    g = A.T @ (A @ u - f)
    z = Dm @ u + lam / beta
    nz = np.hypot(z[:N], z[N:])
    fac = np.where(nz > 1 / beta, (nz - 1 / beta) / np.where(nz > 0, nz, 1), 0.0)
    w = z * np.concatenate([fac, fac])
    c = mu / (beta * tau)
    H = Dm.T @ Dm + c * np.eye(N)
    rhs = Dm.T @ (w - lam / beta) + c * (u - tau * g)
    un = np.linalg.solve(H, rhs)
    lam_n = lam - beta * (w - Dm @ un) if iadm else lam
    return un.reshape(n, n), w.reshape(2, n, n), lam_n.reshape(2, n, n)


@pytest.mark.parametrize("iadm", [True, False])
def test_one_step_matches_dense_equations(iadm):
    P = _problem(8, 40, 30.0, 5.0)
    tau = oracle.default_tau(P.A)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal((8, 8))
    lam0 = rng.standard_normal((2, 8, 8)) * 0.5
    R = oracle.solve(P.A, P.f, 8, P.mu, P.beta, tau, max_iter=1,
                     algo=oracle.IADM if iadm else oracle.FTVCS, u0=u0, lam0=lam0)
    un, w, lam = _dense_step(P, tau, u0, lam0, iadm)
    assert np.allclose(R.u, un, atol=1e-12)
    assert np.allclose(R.w, w, atol=1e-12)
    if iadm:
        assert np.allclose(R.lam, lam, atol=1e-12)


def test_default_initial_point_is_backprojection():
    # Reading C3: u^0 = A^T f.
    P = _problem(8, 30, 10.0, 10.0)
    R = oracle.solve(P.A, P.f, 8, P.mu, P.beta, 0.1, max_iter=0)
    ref = P.A.astype(np.float64).T @ P.f.astype(np.float64)
    assert np.allclose(R.u.ravel(), ref, atol=1e-13)


def test_ftvcs_penalty_objective_monotone():
    # Thm 1's setting with tau <= 1/lambda_max: each FTVCS step minimises a
    # majoriser of eq. (atv), so the penalty objective never increases.
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, P.n, 50.0, 20.0, tau, max_iter=300, algo=oracle.FTVCS,
                     record=True)
    atv = R.hist[:, 1]
    assert np.all(np.diff(atv) <= 1e-10 * np.abs(atv[1:]))


def test_ftvcs_finite_support_and_qlinear_rate():
    # Thm 2: w_i^k = 0 for i in L = {i: ||D_i u*|| <= 1/beta} after finitely many
    # iterations.  Thm 3: ||u^k - u*|| decays q-linearly.
    P = _problem(8, 40, 30.0, 5.0)
    tau = oracle.default_tau(P.A)
    star = oracle.solve(P.A, P.f, 8, P.mu, P.beta, tau, max_iter=20000, algo=oracle.FTVCS)
    R = oracle.solve(P.A, P.f, 8, P.mu, P.beta, tau, max_iter=600, algo=oracle.FTVCS,
                     record_u=True)
    d1, d2 = oracle.D(star.u)
    L = np.hypot(d1, d2).ravel() < 1.0 / P.beta - 1e-6
    assert L.sum() > 0
    late = []
    for k in range(400, 600):
        a1, a2 = oracle.D(R.u_hist[k])
        w1, w2 = oracle.shrink(a1, a2, 1.0 / P.beta)
        late.append(np.max(np.hypot(w1, w2)[L]))
    assert max(late) == 0.0
    err = np.array([np.linalg.norm(R.u_hist[k] - star.u) for k in range(100, 400)])
    ratios = err[1:] / err[:-1]
    assert np.all(ratios < 1.0)
    assert np.max(ratios[-100:]) < 0.999


@pytest.mark.parametrize("n,m,mu,beta,iters", [(8, 96, 20.0, 20.0, 3000), (8, 19, 20.0, 20.0, 20000),
                                                (16, 77, 5.0, 50.0, 20000)])
def test_iadm_reaches_kkt_point(n, m, mu, beta, iters):
    # Thm 4 (via App. B): IADM converges to a solution of eq. (eqftvdcs), whose
    # optimality system is w = D u, D^T lambda + mu A^T (A u - f) = 0 and
    # lambda_i in the subdifferential of ||.|| at w_i.
    P = _problem(n, m, mu, beta)
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, n, mu, beta, tau, max_iter=iters)
    i = R.info
    scale = max(1.0, np.linalg.norm(R.u))
    assert i["kkt_primal"] <= 1e-6 * scale
    assert i["kkt_dual"] <= 1e-6 * scale * mu
    assert i["lambda_max_norm"] <= 1.0 + 1e-8
    assert i["lambda_align"] <= 1e-6


def test_printed_w_sign_does_not_reach_kkt_point():
    # Reading C1: with D_i u - lambda_i/beta (as printed in eq. (iadmw)) the
    # iteration does not reach the optimality system above; with "+" it does.
    P = _problem(8, 96, 20.0, 20.0)
    tau = oracle.default_tau(P.A)
    good = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=3000)
    bad = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=3000, w_sign=-1)
    assert good.info["kkt_dual"] < 1e-8
    kd = bad.info["kkt_dual"]
    assert not np.isfinite(kd) or kd > 1e-2 or bad.info["lambda_align"] > 1e-2


def test_kkt_report_matches_dense_definitions():
    # The summary the oracle reports for a state (u, w, lambda), recomputed from the
    # definitions with the explicit matrices D = (D1; D2) and A: TV = sum_i ||D_i u||,
    # ||A u - f||^2, the objective of eq. (tv), the penalty objective of eq. (atv),
    # ||w - D u||, ||D^T lambda + mu A^T (A u - f)||, max_i ||lambda_i|| and the
    # largest ||lambda_i - w_i / ||w_i|||.
    n, m, mu, beta = 6, 20, 3.0, 7.0
    rng = np.random.default_rng(11)
    A = (rng.standard_normal((m, n * n)) / np.sqrt(m)).astype(np.float32)
    f = rng.standard_normal(m).astype(np.float32)
    u = rng.standard_normal(n * n)
    w = rng.standard_normal(2 * n * n)
    w[5] = w[5 + n * n] = 0.0   # one w_i = 0 (no alignment term there)
    lam = rng.standard_normal(2 * n * n)
    D = diff_matrix(n)
    N = n * n
    A64 = A.astype(np.float64)
    d = D @ u
    r = A64 @ u - f.astype(np.float64)
    e = w - d
    got = oracle.kkt(A, f, n, mu, beta, u, w, lam)
    tv = np.sum(np.hypot(d[:N], d[N:]))
    assert got["tv"] == pytest.approx(tv, rel=1e-13)
    assert got["resid2"] == pytest.approx(r @ r, rel=1e-13)
    assert got["objective"] == pytest.approx(tv + 0.5 * mu * (r @ r), rel=1e-13)
    atv = np.sum(np.hypot(w[:N], w[N:])) + 0.5 * beta * (e @ e) + 0.5 * mu * (r @ r)
    assert got["atv"] == pytest.approx(atv, rel=1e-13)
    assert got["kkt_primal"] == pytest.approx(np.linalg.norm(e), rel=1e-13)
    dual = D.T @ lam + mu * (A64.T @ r)
    assert got["kkt_dual"] == pytest.approx(np.linalg.norm(dual), rel=1e-12)
    assert got["lambda_max_norm"] == pytest.approx(np.max(np.hypot(lam[:N], lam[N:])), rel=1e-14)
    wn = np.hypot(w[:N], w[N:])
    nz = wn > 0
    al = np.hypot(lam[:N][nz] - w[:N][nz] / wn[nz], lam[N:][nz] - w[N:][nz] / wn[nz])
    assert got["lambda_align"] == pytest.approx(np.max(al), rel=1e-13)


def test_warm_start_at_a_kkt_point_stays_there():
    # The warm start of the beta-continuation (Sec. 3.1; u^0 and lambda^0 given, w^0 = 0):
    # at a KKT point (u*, lambda*) of eq. (eqftvdcs) the first w-step returns w* = D u*
    # (lambda* lies in the subdifferential at D u*), the u-step's right-hand side
    # D^T (beta (w* - D u*) - lambda*) - mu A^T (A u* - f) vanishes by dual feasibility,
    # and the multiplier update leaves lambda* unchanged: the iteration stays put.
    P = _problem(8, 96, 20.0, 20.0)
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=20000, tol=1e-15)
    assert R.info["kkt_dual"] <= 1e-12
    W = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=5, u0=R.u, lam0=R.lam)
    assert np.max(np.abs(W.u - R.u)) <= 1e-12 * max(1.0, np.abs(R.u).max())
    assert np.max(np.abs(W.lam - R.lam)) <= 1e-10
    # and a warm start away from it does move
    M = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=5, u0=R.u + 1e-3, lam0=R.lam)
    assert np.max(np.abs(M.u - R.u)) > 1e-5


def test_matches_independent_dual_solver_n8():
    # Full column rank (m = 96 >= N = 64): unique minimiser.
    P = _problem(8, 96, 20.0, 20.0)
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=20000, tol=1e-15)
    u_dual, _ = dual_projected_gradient(P.A, P.f, 8, 20.0)
    assert np.max(np.abs(R.u - u_dual)) <= 1e-8 * max(1.0, np.max(np.abs(u_dual)))


def test_objective_matches_chambolle_pock_underdetermined():
    # m = 19 < N = 64 (ratio 0.3): compare the optimal value only (reading C11).
    P = synth.make_problem(8, 0.3, 7, 3, 20.0, 20.0, noise_c=1e-2)
    assert P.m == 19
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, 8, 20.0, 20.0, tau, max_iter=50000)
    _, obj = chambolle_pock(P.A, P.f, 8, 20.0, iters=200000)
    assert R.info["objective"] == pytest.approx(obj, rel=1e-6)


def test_stop_rule_first_crossing():
    # Eq. (stop) with reading C5: the loop ends at the first k with
    # ||u^k - u^{k-1}|| <= tol ||u^{k-1}||.
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, P.n, 50.0, 20.0, tau, tol=2e-3, max_iter=500, record=True)
    rc = R.hist[:, 2]
    assert R.info["stopped_by_tol"] == 1
    assert rc[-1] <= 2e-3 and np.all(rc[:-1] > 2e-3)


@pytest.mark.parametrize("algo", [oracle.IADM, oracle.FTVCS])
def test_zero_measurements_stop_at_the_zero_image(algo):
    # With f = 0 the objective sum_i ||D_i u|| + (mu/2)||Au||^2 is >= 0 and vanishes at
    # u = 0, a minimiser.  The back-projection A^T f is 0 and every step keeps u, w and
    # lambda at 0, so eq. (stop) with reading C5 (||u^k|| = 0: stop once ||u^{k+1}|| = 0)
    # ends the run after the first iteration.
    P = _problem(16, 77, 1e3, 10.0)
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, np.zeros(P.m, np.float32), P.n, P.mu, P.beta, tau, tol=1e-4,
                     max_iter=50, algo=algo)
    assert R.info["iters"] == 1 and R.info["stopped_by_tol"] == 1
    assert not np.any(R.u) and not np.any(R.w) and not np.any(R.lam)
    assert R.info["objective"] == 0.0


@pytest.mark.parametrize("algo", [oracle.IADM, oracle.FTVCS])
def test_iteration_is_positively_homogeneous(algo):
    # TV is positively homogeneous, so for c > 0 the problem (c f, mu / c, beta / c) has the
    # minimisers c u* of (f, mu, beta), and each step of Algorithms 1-2 maps the iterates
    # (u, w, lambda) of the first run to (c u, c w, lambda) of the second: the shrink
    # threshold 1/beta, the u-step divisor beta Lambda_pq + mu/tau and the terms beta w and
    # mu g of the right-hand side each scale so that the step commutes with c.  A term with
    # the wrong power of beta or mu breaks that.  For c a power of two every binary64
    # operation commutes with the scaling, so the two runs agree bit for bit.
    P = _problem(16, 77, 1e3, 10.0)
    tau = oracle.default_tau(P.A)
    c = 4.0
    R1 = oracle.solve(P.A, P.f, P.n, P.mu, P.beta, tau, max_iter=40, algo=algo)
    R2 = oracle.solve(P.A, c * P.f, P.n, P.mu / c, P.beta / c, tau, max_iter=40, algo=algo)
    assert np.any(R1.u)
    assert np.array_equal(R2.u, c * R1.u)
    assert np.array_equal(R2.w, c * R1.w)
    assert np.array_equal(R2.lam, R1.lam)
    assert R2.info["objective"] == c * R1.info["objective"]


def test_iadm_objective_decreases_to_optimum_on_32x32():
    # Fig. 2 shows decreasing objective values; for IADM we check that the
    # objective approaches the optimal value (reading C13), and that IADM beats
    # FTVCS at the same beta (the comparison of Fig. 1).
    P = synth.workload_n32()
    tau = oracle.default_tau(P.A)
    R = oracle.solve(P.A, P.f, P.n, 50.0, 20.0, tau, max_iter=3000, record=True)
    obj = R.hist[:, 0]
    best = obj[-1]
    assert obj[100] > best and obj[1000] - best < 0.1 * (obj[100] - best)
    Rf = oracle.solve(P.A, P.f, P.n, 50.0, 20.0, tau, max_iter=3000, algo=oracle.FTVCS)
    ubar = P.ubar.astype(np.float64)
    re_i = np.linalg.norm(R.u - ubar) / np.linalg.norm(ubar)
    re_f = np.linalg.norm(Rf.u - ubar) / np.linalg.norm(ubar)
    assert re_i < re_f
