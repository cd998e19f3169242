"""Batched path: many images sharing one A, products as tcgen05 BF16x3 GEMMs.

The GEMM computes D = X_hi Y_hi + X_hi Y_lo + X_lo Y_hi with bf16 hi/lo
splits; the reference below forms exactly that sum in binary64 from the
test-side emulation of the splits (quant_ref.py), so the comparison checks
the tensor-core arithmetic at binary32 accumulation tolerance (1e-5 of the
absolute sums).  Whole solves are compared with the FP64 oracle on the exact
binary32 A (the split's representation error is part of that difference).
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


def bf16x3(Xh, Xl, Yh, Yl):
    """X (rows x K) times Y^T (cols x K) as the three-term split product, binary64."""
    Xh, Xl, Yh, Yl = (np.asarray(t, dtype=np.float64) for t in (Xh, Xl, Yh, Yl))
    return Xh @ Yh.T + Xh @ Yl.T + Xl @ Yh.T


def objective_exact(A, f, u, mu):
    """Phi(u) of eq. (tv) for a binary32 image, evaluated in binary64 (the oracle's TV)."""
    u = np.asarray(u, dtype=np.float64)
    n = int(round(np.sqrt(u.size)))
    r = A.astype(np.float64) @ u.ravel() - f.astype(np.float64)
    return oracle.tv(u.reshape(n, n)) + 0.5 * mu * float(r @ r)


def check_converged(A, f, n, mu, beta, tau, tol, cap, u, r):
    """A batched image run to its own eq. (stop) against the FP64 oracle on the exact
    binary32 A (Thm 4: both runs converge to the same KKT point): the stop iteration
    within one of the oracle's, the image within 1e-4 and the objective within 1e-6,
    both the value the GPU reports and that of the GPU's image evaluated exactly."""
    ref = oracle.solve(A, f, n, mu, beta, tau, tol=tol, max_iter=cap)
    assert r.stopped_by_tol == 1 and ref.info["iters"] < cap
    assert abs(r.iters - ref.info["iters"]) <= 1, (r.iters, ref.info["iters"])
    same = ref if r.iters == ref.info["iters"] else oracle.solve(A, f, n, mu, beta, tau,
                                                                 max_iter=r.iters)
    err = rel(u, same.u)
    obj = same.info["objective"]
    gap_rep = abs(r.objective - obj) / obj
    gap_img = abs(objective_exact(A, f, u, mu) - obj) / obj
    print("mu %g: %d iterations, image %.2e, objective reported %.2e, of the image %.2e"
          % (mu, r.iters, err, gap_rep, gap_img))
    assert err <= 1e-4 and rel(u, ref.u) <= 1e-4
    assert gap_img <= 1e-6
    assert gap_rep <= 1e-6


def bf16_handle(tv, A, m, n, mu=1.0, beta=10.0, tau=0.1, max_iter=50, tol=0.0):
    opt = tv.tvcs_default_options()
    opt.precision = tv.TVCS_PREC_BF16X2
    opt.tau = tau
    opt.max_iter = max_iter
    return tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, n, mu, beta, tol, opt)


def check_batched_products(A, X, Y, R, G, rng):
    """R = A X - Y and G = A^T R against the split products formed in binary64."""
    count, N = X.shape
    m = A.shape[0]
    Ah, Al = quant_ref.split_bf16x2(A)
    Xh, Xl = quant_ref.split_bf16x2(X)
    # rows of A checked: all for small m, a seeded sample for the full-size case
    rows = np.arange(m) if m * N <= 2_000_000 else np.sort(rng.choice(m, 400, replace=False))
    Rref = bf16x3(Ah[rows], Al[rows], Xh, Xl).T - Y[:, rows].astype(np.float64)
    scale = (np.abs(Ah[rows].astype(np.float64)) + np.abs(Al[rows])) @ np.abs(X.astype(np.float64)).T
    assert np.all(np.abs(R[:, rows].astype(np.float64) - Rref) <= 1e-5 * scale.T + 1e-30)
    # G = A^T R with the GPU's own R (its bf16 split) as input
    Rh, Rl = quant_ref.split_bf16x2(R)
    Aeff = (Ah + Al).astype(np.float32)
    Th, Tl = quant_ref.split_bf16x2(np.ascontiguousarray(Aeff.T))
    cols = np.arange(N) if m * N <= 2_000_000 else np.sort(rng.choice(N, 400, replace=False))
    Gref = bf16x3(Th[cols], Tl[cols], Rh, Rl).T
    gscale = np.abs(Aeff.T[cols].astype(np.float64)) @ np.abs(R.astype(np.float64)).T
    assert np.all(np.abs(G[:, cols].astype(np.float64) - Gref) <= 1e-5 * gscale.T + 1e-30)


@pytest.mark.parametrize("n,m,count", [(32, 307, 1), (32, 307, 7), (32, 300, 256), (64, 1229, 40),
                                       (128, 4915, 64)])
def test_batched_products(tv, n, m, count):
    N = n * n
    A = synth.gaussian_matrix(70 + n, m, N)
    rng = np.random.default_rng(count + n)
    X = rng.standard_normal((count, N)).astype(np.float32)
    Y = rng.standard_normal((count, m)).astype(np.float32)
    h = bf16_handle(tv, A, m, n)
    R = np.empty((count, m), np.float32)
    G = np.empty((count, N), np.float32)
    tv.tvcs_apply_batched(h, count, X, Y, R, G)
    check_batched_products(A, X, Y, R, G, rng)
    tv.tvcs_destroy(h)


def set_pair_shape(tv, h, pairs):
    """Both GEMMs on CTA pairs: the first of `pairs` (pairs of blocks) that fits."""
    for p in pairs:
        try:
            tv.tvcs_test_gemm_shape(h, 2 * p, 1, 2 * p, 1)
            return p
        except tv.TvcsError as e:
            assert e.status == tv.TVCS_ERR_UNSUPPORTED
    pytest.fail("no pair shape fits")


# M = m rows in 256-row pair tiles: m = 307 leaves the odd block of the last
# tile wholly past the matrix; 40 and 200 images give each block of a pair
# 32 and 112 of the running columns (a 64-row box that reaches into the other
# block's half or past the images); one to three pairs walk several tiles each,
# so both accumulators are reused; n = 128 is the full-size operand.
@pytest.mark.parametrize("n,m,count,pairs", [(32, 307, 7, (76, 72, 64)), (32, 307, 7, (1,)),
                                             (64, 1229, 40, (76, 72, 64)), (64, 1229, 200, (3,)),
                                             (128, 4915, 256, (76, 72, 64)), (32, 307, 300, (76, 72, 64)),
                                             (32, 307, 290, (1,)), (64, 1229, 512, (76, 72, 64))])
def test_gemm_on_cta_pairs(tv, n, m, count, pairs):
    # The GEMMs on clusters of two blocks that share each 256-row tile
    # (tcgen05 cta_group::2): the same checks as the single-block kernel against
    # the split products in binary64 (1e-5 of the absolute sums), and agreement with
    # the single-block shape within the same bound: a different stream-K split
    # regroups binary32 sums of up to K = m or n^2 terms (whole-K tiles against
    # tiles split over several blocks), which is not bitwise.  Above 256 images the
    # pair kernel runs two N tiles per X tile; the single-block shape then runs as
    # two calls (the first 256 images, the rest).
    N = n * n
    A = synth.gaussian_matrix(90 + n, m, N)
    rng = np.random.default_rng(count + 3 * n)
    X = rng.standard_normal((count, N)).astype(np.float32)
    Y = rng.standard_normal((count, m)).astype(np.float32)
    out = []
    for pair in (1, 0):
        h = bf16_handle(tv, A, m, n)
        if pair:
            p = set_pair_shape(tv, h, pairs)
            print("pairs", p)
        else:
            tv.tvcs_test_gemm_shape(h, 152 if n > 32 else 64, 0, 152 if n > 32 else 64, 0)
        R = np.empty((count, m), np.float32)
        G = np.empty((count, N), np.float32)
        for lo, hi in ([(0, count)] if pair or count <= 256 else [(0, 256), (256, count)]):
            Rp = np.empty((hi - lo, m), np.float32)
            Gp = np.empty((hi - lo, N), np.float32)
            tv.tvcs_apply_batched(h, hi - lo, np.ascontiguousarray(X[lo:hi]), np.ascontiguousarray(Y[lo:hi]),
                                  Rp, Gp)
            R[lo:hi], G[lo:hi] = Rp, Gp
        out.append((R, G))
        tv.tvcs_destroy(h)
    (R1, G1), (R0, G0) = out
    check_batched_products(A, X, Y, R1, G1, rng)
    A64 = np.abs(A.astype(np.float64))
    dr = np.max(np.abs(R1.astype(np.float64) - R0) / (np.abs(X.astype(np.float64)) @ A64.T + 1e-30))
    dg = np.max(np.abs(G1.astype(np.float64) - G0) / (np.abs(R0.astype(np.float64)) @ A64 + 1e-30))
    print("pair vs single shape, of the absolute sums: R %.2e, G %.2e" % (dr, dg))
    assert dr <= 1e-5 and dg <= 1e-5


def test_gemm_pair_shape_solves_and_rejects_bad_shapes(tv):
    # 20-iteration batched solves with both GEMMs on CTA pairs agree with the
    # single-block shape to the parity tolerance 1e-5; malformed shapes are refused.
    n, m, count = 64, 1229, 48
    N = n * n
    A = synth.gaussian_matrix(78, m, N)
    rng = np.random.default_rng(9)
    F = rng.standard_normal((count, m)).astype(np.float32)
    res = []
    for pair in (1, 0):
        h = bf16_handle(tv, A, m, n, mu=1e3, max_iter=20)
        if pair:
            set_pair_shape(tv, h, (76, 72, 64))
        else:
            tv.tvcs_test_gemm_shape(h, 152, 0, 152, 0)
        us = [np.empty(N, np.float32) for _ in range(count)]
        tv.tvcs_solve_batched([h] * count, [np.ascontiguousarray(F[b]) for b in range(count)], us)
        res.append(us)
        if pair:
            for bad in ((3, 1, 4, 1), (4, 2, 4, 1), (-1, 0, 4, 0), (4, 0, 0, 0), (100000, 0, 4, 0)):
                with pytest.raises(tv.TvcsError) as ei:
                    tv.tvcs_test_gemm_shape(h, *bad)
                assert ei.value.status == tv.TVCS_ERR_INVALID_ARG, bad
            with pytest.raises(tv.TvcsError) as ei:
                tv.tvcs_test_gemm_shape(h, 2 * 100000, 1, 4, 0)
            assert ei.value.status in (tv.TVCS_ERR_UNSUPPORTED, tv.TVCS_ERR_INVALID_ARG)
        tv.tvcs_destroy(h)
    for b in range(count):
        assert rel(res[0][b], res[1][b]) <= 1e-5, b


def test_batched_solve_matches_oracle_and_single_image(tv):
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=8, n=32, ratio=0.3, seed=3, n_ellipses=6)
    m, N = A.shape
    n = 32
    tau = oracle.default_tau(A)
    iters = 40
    h = bf16_handle(tv, A, m, n, mu=1e3, tau=tau, max_iter=iters)
    us = [np.empty(N, np.float32) for _ in range(8)]
    res = tv.tvcs_solve_batched([h] * 8, [F[b] for b in range(8)], us, mus)
    for b in range(8):
        assert res[b].iters == iters
        ref = oracle.solve(A, F[b], n, mus[b], 10.0, tau, max_iter=iters)
        err = rel(us[b], ref.u)
        assert err <= 1e-4, (b, err)
        assert res[b].objective == pytest.approx(ref.info["objective"], rel=1e-4)
    # one image through the single-image bf16x2 path (binary32 u, same storage of A)
    h1 = bf16_handle(tv, A, m, n, mu=mus[5], tau=tau, max_iter=iters)
    u1 = np.empty(N, np.float32)
    tv.tvcs_solve(h1, F[5], u1)
    assert rel(us[5], u1) <= 1e-4
    tv.tvcs_destroy(h)
    tv.tvcs_destroy(h1)


@pytest.mark.parametrize("n,count,ratio", [(64, 5, 0.2), (192, 3, 0.1), (256, 3, 0.05)])
def test_batched_solve_other_sizes(tv, n, count, ratio):
    # the bf16 hi+lo sides not covered above (32, 128 are): 64 with the one-block-per-image
    # u-solve; 192 and 256 with the cluster u-solve per image and pair GEMMs of 144 and 256
    # tiles over K = n^2 columns of A
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=count, n=n, ratio=ratio, seed=7 + n, n_ellipses=5)
    m, N = A.shape
    tau = oracle.default_tau(A)
    iters = 25 if n <= 64 else 15
    h = bf16_handle(tv, A, m, n, mu=1e3, tau=tau, max_iter=iters)
    us = [np.empty(N, np.float32) for _ in range(count)]
    res = tv.tvcs_solve_batched([h] * count, [F[b] for b in range(count)], us, mus)
    for b in range(count):
        assert res[b].iters == iters
        ref = oracle.solve(A, F[b], n, mus[b], 10.0, tau, max_iter=iters)
        err = rel(us[b], ref.u)
        print("n %d image %d: %.2e" % (n, b, err))
        assert err <= 1e-4, (n, b)
    tv.tvcs_destroy(h)


def test_batched_per_image_stop(tv):
    # images stop on their own eq. (stop): a run to tol gives per-image iteration counts
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=4, n=32, ratio=0.3, seed=4, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    mus = [20.0, 50.0, 100.0, 200.0]
    h = bf16_handle(tv, A, m, 32, mu=1e3, beta=20.0, tau=tau, max_iter=3000, tol=1e-4)
    us = [np.empty(N, np.float32) for _ in range(4)]
    res = tv.tvcs_solve_batched([h] * 4, [F[b] for b in range(4)], us, mus)
    for b in range(4):
        check_converged(A, F[b], 32, mus[b], 20.0, tau, 1e-4, 3000, us[b], res[b])
    assert len({r.iters for r in res}) > 1
    tv.tvcs_destroy(h)


def test_batched_zero_measurements_leave_after_one_iteration(tv):
    # an image with f = 0 stops after its first iteration with u = 0 exactly (reading C5)
    # and leaves the GEMMs; the other images run on and still match the oracle
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=5, n=32, ratio=0.3, seed=8, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    F = [F[b] for b in range(5)]
    F[2] = np.zeros(m, np.float32)
    h = bf16_handle(tv, A, m, 32, mu=1e3, beta=20.0, tau=tau, max_iter=3000, tol=1e-4)
    us = [np.full(N, np.nan, np.float32) for _ in range(5)]
    res = tv.tvcs_solve_batched([h] * 5, F, us, [50.0] * 5)
    assert res[2].iters == 1 and res[2].stopped_by_tol == 1
    assert not np.any(us[2]) and res[2].objective == 0.0
    for b in (0, 1, 3, 4):
        assert res[b].iters > 1
        check_converged(A, F[b], 32, 50.0, 20.0, tau, 1e-4, 3000, us[b], res[b])
    tv.tvcs_destroy(h)


def test_batched_iteration_count_not_a_multiple_of_the_loop_body(tv):
    # the loop graph holds 4 iterations per body: a run of 7 ends inside a body, and
    # the GEMMs and fix-ups of the rest of the body must not change any image
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=5, n=32, ratio=0.3, seed=6, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    h = bf16_handle(tv, A, m, 32, mu=1e3, tau=tau, max_iter=7)
    us = [np.empty(N, np.float32) for _ in range(5)]
    res = tv.tvcs_solve_batched([h] * 5, [F[b] for b in range(5)], us, mus)
    for b in range(5):
        assert res[b].iters == 7
        ref = oracle.solve(A, F[b], 32, mus[b], 10.0, tau, max_iter=7)
        assert rel(us[b], ref.u) <= 1e-4, b
        assert res[b].objective == pytest.approx(ref.info["objective"], rel=1e-4)
    tv.tvcs_destroy(h)


def test_batched_compaction_is_exact(tv):
    # images stop at different iterations; with compaction the running images are packed
    # into the GEMMs' leading columns and the GEMMs shrink (40 columns -> 64-wide MMAs ->
    # 32-wide).  Every column is still a dot product over the same K in the same order,
    # so the results are identical to the run that keeps every column.
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=40, n=32, ratio=0.3, seed=5, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    mus = [20.0 * 1.3 ** (b % 12) for b in range(40)]
    out = {}
    for compact in (1, 0):
        opt = tv.tvcs_default_options()
        opt.precision = tv.TVCS_PREC_BF16X2
        opt.tau = tau
        opt.max_iter = 3000
        opt.batch_compact = compact
        h = tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, 32, 1e3, 20.0, 1e-4, opt)
        us = [np.empty(N, np.float32) for _ in range(40)]
        res = tv.tvcs_solve_batched([h] * 40, [F[b] for b in range(40)], us, mus)
        out[compact] = (us, res)
        tv.tvcs_destroy(h)
    (uc, rc), (uf, rf) = out[1], out[0]
    iters = [r.iters for r in rc]
    assert len(set(iters)) >= 6 and all(r.stopped_by_tol == 1 for r in rc)
    assert iters == [r.iters for r in rf]
    for b in range(40):
        assert np.array_equal(uc[b], uf[b]), b
        assert rc[b].objective == rf[b].objective
    # and two of them against the oracle at convergence
    for b in (7, 11):
        check_converged(A, F[b], 32, mus[b], 20.0, tau, 1e-4, 3000, uc[b], rc[b])


def test_batched_compaction_is_exact_n128(tv):
    # 128 x 128 images: the u-solve adds the partial tiles of G = A^T R itself (no second
    # fix-up inside the loop), each image reading its column of the iteration that just
    # ended, and G is formed once at the end of the run.  Images stop at different
    # iterations; the compacted run (columns move as images leave) equals the run that
    # keeps every column bit for bit, and an image matches the oracle at convergence.
    count = 24
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=count, n=128, ratio=0.3, seed=6, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    mus = [100.0 * 1.35 ** (b % 8) for b in range(count)]
    out = {}
    for compact in (1, 0):
        opt = tv.tvcs_default_options()
        opt.precision = tv.TVCS_PREC_BF16X2
        opt.tau = tau
        opt.max_iter = 4000
        opt.batch_compact = compact
        h = tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, 128, 1e3, 10.0, 1e-4, opt)
        us = [np.empty(N, np.float32) for _ in range(count)]
        res = tv.tvcs_solve_batched([h] * count, [F[b] for b in range(count)], us, mus)
        out[compact] = (us, res)
        tv.tvcs_destroy(h)
    (uc, rc), (uf, rf) = out[1], out[0]
    iters = [r.iters for r in rc]
    print("stop iterations", sorted(set(iters)))
    assert len(set(iters)) >= 4 and all(r.stopped_by_tol == 1 for r in rc)
    assert iters == [r.iters for r in rf]
    for b in range(count):
        assert np.array_equal(uc[b], uf[b]), b
        assert rc[b].objective == rf[b].objective
        assert rc[b].kkt_dual == rf[b].kkt_dual   # the end-of-run G
    b = int(np.argmin(iters))
    check_converged(A, F[b], 128, mus[b], 10.0, tau, 1e-4, 4000, uc[b], rc[b])


@pytest.mark.parametrize("n,count,mu0", [(32, 400, 20.0), (128, 300, 100.0)])
def test_batched_compaction_above_256_images_is_exact(tv, n, count, mu0):
    # More than 256 images in one group: the pair GEMMs run two N tiles per tile of A,
    # and as images stop the running columns fall below 256, so the second N tile
    # empties; at n = 128 the u-solve also reads G's partial tiles by each image's
    # column of the iteration that just ended.  The compacted run equals the run that
    # keeps every column, bit for bit.
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=count, n=n, ratio=0.3, seed=8, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    mus = [mu0 * 1.35 ** (b % 8) for b in range(count)]
    beta = 20.0 if n == 32 else 10.0
    out = {}
    for compact in (1, 0):
        opt = tv.tvcs_default_options()
        opt.precision = tv.TVCS_PREC_BF16X2
        opt.tau = tau
        opt.max_iter = 4000
        opt.batch_compact = compact
        h = tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, n, 1e3, beta, 1e-4, opt)
        Fd = torch.from_numpy(F).cuda()
        U = torch.empty((count, N), dtype=torch.float32, device="cuda")
        res = tv.tvcs_solve_batched([h] * count, [Fd[b] for b in range(count)], [U[b] for b in range(count)], mus)
        out[compact] = (U.cpu().numpy(), res)
        tv.tvcs_destroy(h)
    (uc, rc), (uf, rf) = out[1], out[0]
    iters = [r.iters for r in rc]
    print("n %d, %d images: stop iterations %d .. %d (%d distinct)" % (n, count, min(iters), max(iters),
                                                                        len(set(iters))))
    # columns leave at many different iterations (a few images may reach the cap)
    assert len(set(iters)) >= 4 and sum(r.stopped_by_tol for r in rc) >= count // 2
    assert iters == [r.iters for r in rf]
    assert np.array_equal(uc, uf)
    for b in range(count):
        assert rc[b].objective == rf[b].objective and rc[b].kkt_dual == rf[b].kkt_dual, b


def test_batched_converges_with_the_shared_batch_parameters(tv):
    # The shared-A batch's parameters (mu cycling over 2e2, 5e2, 1e3, 2e3, beta = 10,
    # noise U[1e-3, 1e-2] RMS, tol 1e-4) at n = 32, m = 307 (ratio 0.3), where the FP64
    # oracle finishes every image's run to eq. (stop) in seconds: each image stops by
    # tol (up to about 5K iterations) and matches the oracle at convergence.
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=4, n=32, ratio=0.3, seed=21, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    cap = 30000
    h = bf16_handle(tv, A, m, 32, mu=1e3, beta=10.0, tau=tau, max_iter=cap, tol=1e-4)
    us = [np.empty(N, np.float32) for _ in range(4)]
    res = tv.tvcs_solve_batched([h] * 4, [F[b] for b in range(4)], us, mus)
    assert sorted(mus) == [2e2, 5e2, 1e3, 2e3]
    for b in range(4):
        check_converged(A, F[b], 32, mus[b], 10.0, tau, 1e-4, cap, us[b], res[b])
    tv.tvcs_destroy(h)


def test_batched_workload_256_images_n128(tv):
    # 256 images of 128 x 128 sharing one 4915 x 16384 A (bf16 hi/lo), mu cycling over
    # {2e2, 5e2, 1e3, 2e3}, noise U[1e-3, 1e-2] RMS; a fixed 30 iterations, a sample
    # of 8 images (2 per mu) compared with the FP64 oracle.
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=256, n=128, ratio=0.3, seed=1)
    m, N = A.shape
    tau = oracle.default_tau(A, 30)
    iters = 30
    h = bf16_handle(tv, A, m, 128, mu=1e3, tau=tau, max_iter=iters)
    U = torch.empty((256, N), dtype=torch.float32, device="cuda")
    Fd = torch.from_numpy(F).cuda()
    res = tv.tvcs_solve_batched([h] * 256, [Fd[b] for b in range(256)], [U[b] for b in range(256)], mus)
    Uh = U.cpu().numpy()
    for b in [0, 1, 2, 3, 128, 129, 130, 255]:
        assert res[b].iters == iters
        ref = oracle.solve(A, F[b], 128, mus[b], 10.0, tau, max_iter=iters)
        err = rel(Uh[b], ref.u)
        print("image %d mu %.0f rel err %.2e" % (b, mus[b], err))
        assert err <= 1e-4
    tv.tvcs_destroy(h)


def test_batched_more_than_512_images_run_in_groups(tv):
    # 600 images: two groups of 300 through the same tensor-core path (two N tiles of
    # 256 columns per X tile of A).  An image's column is independent of the other
    # columns and of how many run, so with one GEMM shape for every call each image
    # equals its result in a call that holds only its own group, and in a call of
    # 150 images (one N tile); a sample matches the FP64 oracle.
    count = 600
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=count, n=32, ratio=0.3, seed=12, n_ellipses=6)
    m, N = A.shape
    tau = oracle.default_tau(A)
    iters = 30
    h = bf16_handle(tv, A, m, 32, mu=1e3, tau=tau, max_iter=iters)
    set_pair_shape(tv, h, (76, 72, 64))
    Fd = torch.from_numpy(F).cuda()
    U = torch.empty((count, N), dtype=torch.float32, device="cuda")
    res = tv.tvcs_solve_batched([h] * count, [Fd[b] for b in range(count)], [U[b] for b in range(count)], mus)
    assert all(r.iters == iters for r in res)
    U2 = torch.empty((300, N), dtype=torch.float32, device="cuda")
    tv.tvcs_solve_batched([h] * 300, [Fd[300 + b] for b in range(300)], [U2[b] for b in range(300)],
                          mus[300:])
    U3 = torch.empty((150, N), dtype=torch.float32, device="cuda")
    tv.tvcs_solve_batched([h] * 150, [Fd[450 + b] for b in range(150)], [U3[b] for b in range(150)],
                          mus[450:])
    Uh, U2h, U3h = U.cpu().numpy(), U2.cpu().numpy(), U3.cpu().numpy()
    assert np.array_equal(Uh[300:], U2h)
    assert np.array_equal(Uh[450:], U3h)
    for b in (0, 299, 300, 599):
        ref = oracle.solve(A, F[b], 32, mus[b], 10.0, tau, max_iter=iters)
        assert rel(Uh[b], ref.u) <= 1e-4, b
    # the products entry point groups the same way
    X = np.ascontiguousarray(Uh[:520])
    R = np.empty((520, m), np.float32)
    G = np.empty((520, N), np.float32)
    tv.tvcs_apply_batched(h, 520, X, F[:520], R, G)
    R1 = np.empty((260, m), np.float32)
    G1 = np.empty((260, N), np.float32)
    tv.tvcs_apply_batched(h, 260, np.ascontiguousarray(X[260:]), np.ascontiguousarray(F[260:520]), R1, G1)
    assert np.array_equal(R[260:], R1) and np.array_equal(G[260:], G1)
    tv.tvcs_destroy(h)


def test_gemm_autotune_agrees_with_the_default_shape(tv):
    # The tuner picks each GEMM's number of persistent blocks by timing; a different
    # stream-K split regroups the K sums of a tile, so the products agree with the
    # default shape (one block per SM) to binary32 rounding of the sums, 1e-6 of the
    # absolute sums; 20-iteration solves agree to the parity tolerance 1e-5 (the
    # regrouped roundings carry through the iterations: about 1e-6 measured).
    n, m, count = 64, 1229, 48
    N = n * n
    A = synth.gaussian_matrix(77, m, N)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((count, N)).astype(np.float32)
    Y = rng.standard_normal((count, m)).astype(np.float32)
    out = {}
    for tune in (1, 0):
        opt = tv.tvcs_default_options()
        opt.precision = tv.TVCS_PREC_BF16X2
        opt.tau = 0.1
        opt.max_iter = 20
        opt.autotune = tune
        h = tv.tvcs_create(torch.from_numpy(A).cuda(), 0, m, n, 1e3, 10.0, 0.0, opt)
        R = np.empty((count, m), np.float32)
        G = np.empty((count, N), np.float32)
        tv.tvcs_apply_batched(h, count, X, Y, R, G)
        us = [np.empty(N, np.float32) for _ in range(count)]
        tv.tvcs_solve_batched([h] * count, [np.ascontiguousarray(Y[b]) for b in range(count)], us)
        out[tune] = (R, G, us)
        tv.tvcs_destroy(h)
    (R1, G1, u1), (R0, G0, u0) = out[1], out[0]
    A64 = np.abs(A.astype(np.float64))
    assert np.all(np.abs(R1.astype(np.float64) - R0) <= 1e-6 * (np.abs(X.astype(np.float64)) @ A64.T) + 1e-30)
    assert np.all(np.abs(G1.astype(np.float64) - G0) <= 1e-6 * (np.abs(R0.astype(np.float64)) @ A64) + 1e-30)
    for b in range(count):
        assert rel(u1[b], u0[b]) <= 1e-5, b


def test_batched_n128_u_solve_in_registers(tv):
    # 128 x 128 images take the u-solve whose 128-point transforms stay in the
    # registers of one warp: 6 images for 40 iterations against the FP64 oracle,
    # and image 2 against the single-image solve on the same bf16 hi+lo storage
    # (binary32 u-step on a thread-block cluster).
    A, ubars, F, mus, _ = synth.workload_shared_batch(count=6, n=128, ratio=0.3, seed=17, n_ellipses=8)
    m, N = A.shape
    tau = oracle.default_tau(A, 30)
    iters = 40
    h = bf16_handle(tv, A, m, 128, mu=1e3, tau=tau, max_iter=iters)
    us = [np.empty(N, np.float32) for _ in range(6)]
    res = tv.tvcs_solve_batched([h] * 6, [F[b] for b in range(6)], us, mus)
    for b in range(6):
        assert res[b].iters == iters
        ref = oracle.solve(A, F[b], 128, mus[b], 10.0, tau, max_iter=iters)
        err = rel(us[b], ref.u)
        print("n128 image %d: %.2e" % (b, err))
        assert err <= 1e-4, (b, err)
        assert res[b].objective == pytest.approx(ref.info["objective"], rel=1e-4)
    h1 = bf16_handle(tv, A, m, 128, mu=mus[2], tau=tau, max_iter=iters)
    u1 = np.empty(N, np.float32)
    tv.tvcs_solve(h1, F[2], u1)
    assert rel(us[2], u1) <= 1e-4
    tv.tvcs_destroy(h)
    tv.tvcs_destroy(h1)
