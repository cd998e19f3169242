"""Independent TV/L2 solvers used only to pin the oracle.

Both solve min_u sum_i ||D_i u||_2 + (mu/2) ||A u - f||^2 (eq. (tv)) by
methods other than the paper's: they build the difference operator as an
explicit dense matrix from its index definition and share no code with
``oracle/``.
"""
import numpy as np


def diff_matrix(n: int) -> np.ndarray:
    """Explicit 2N x N matrix D = (D1; D2), periodic boundary:
    (D1 u)[r,c] = u[r,c+1] - u[r,c], (D2 u)[r,c] = u[r+1,c] - u[r,c]."""
    N = n * n
    D = np.zeros((2 * N, N))
    for r in range(n):
        for c in range(n):
            i = r * n + c
            D[i, r * n + (c + 1) % n] += 1.0
            D[i, i] -= 1.0
            D[N + i, ((r + 1) % n) * n + c] += 1.0
            D[N + i, i] -= 1.0
    return D


def tv_value(D: np.ndarray, u: np.ndarray) -> float:
    N = D.shape[1]
    d = D @ u.ravel()
    return float(np.sum(np.hypot(d[:N], d[N:])))


def _project_balls(p: np.ndarray, N: int) -> np.ndarray:
    nrm = np.maximum(1.0, np.hypot(p[:N], p[N:]))
    return np.concatenate([p[:N] / nrm, p[N:] / nrm])


def dual_projected_gradient(A, f, n, mu, iters=200000, tol=1e-15):
    """Maximise the dual q(p) = min_u <D u, p> + (mu/2)||A u - f||^2 over
    ||p_i|| <= 1 by accelerated projected gradient (FISTA with adaptive
    restart).  Needs A^T A nonsingular (m >= N): then
    u(p) = (A^T A)^{-1} (A^T f - D^T p / mu) and grad q = D u(p)."""
    A = np.asarray(A, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    N = n * n
    D = diff_matrix(n)
    AtA = A.T @ A
    L_chol = np.linalg.cholesky(AtA)

    def solve_AtA(b):
        return np.linalg.solve(L_chol.T, np.linalg.solve(L_chol, b))

    Atf = A.T @ f
    Minv = solve_AtA(np.eye(N))
    H = D @ Minv @ D.T / mu                      # -Hessian of q
    Lip = np.linalg.eigvalsh(H)[-1]
    base = D @ (Minv @ Atf)
    p = np.zeros(2 * N)
    y = p.copy()
    t = 1.0
    u_prev = None
    for k in range(iters):
        grad = base - H @ y
        p_new = _project_balls(y + grad / Lip, N)
        if np.dot(p_new - p, y - p_new) > 0:      # adaptive restart (O'Donoghue-Candes)
            t = 1.0
            y = p.copy()
            continue
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        y = p_new + ((t - 1.0) / t_new) * (p_new - p)
        p, t = p_new, t_new
        if k % 200 == 0:
            u = solve_AtA(Atf - D.T @ p / mu)
            if u_prev is not None and np.linalg.norm(u - u_prev) <= tol * np.linalg.norm(u):
                break
            u_prev = u
    u = solve_AtA(Atf - D.T @ p / mu)
    return u.reshape(n, n), p


def chambolle_pock(A, f, n, mu, iters=400000):
    """Primal-dual hybrid gradient (Chambolle & Pock 2011, Algorithm 1 with
    theta = 1) on min_u F(K u) with K = [D; A], F(y1, y2) =
    sum_i ||y1_i|| + (mu/2)||y2 - f||^2 and G = 0."""
    A = np.asarray(A, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    N = n * n
    D = diff_matrix(n)
    K = np.vstack([D, A])
    Lk = np.linalg.norm(K, 2)
    sig = tau = 0.99 / Lk
    u = np.zeros(N)
    ubar = u.copy()
    y = np.zeros(K.shape[0])
    for _ in range(iters):
        v = y + sig * (K @ ubar)
        y1 = _project_balls(v[:2 * N], N)
        y2 = (v[2 * N:] - sig * f) / (1.0 + sig / mu)
        y = np.concatenate([y1, y2])
        u_new = u - tau * (K.T @ y)
        ubar = 2.0 * u_new - u
        u = u_new
    obj = tv_value(D, u) + 0.5 * mu * float(np.sum((A @ u - f) ** 2))
    return u.reshape(n, n), obj
