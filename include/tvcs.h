/*
 * tvcs.h -- C ABI of the GB300 (sm_103a) solver for TV/L2 image reconstruction
 * from random projections (Xiao & Yang, "A Fast Algorithm for Total Variation
 * Image Reconstruction from Random Projections").
 *
 * Problem (eq. (tv), Sec. 1):
 *     min_u  sum_i ||D_i u||_2 + (mu/2) ||A u - f||_2^2
 * u: n x n image (row-major, N = n*n pixels), A: m x N dense encoding matrix
 * (row-major), f: m measurements.  D_i u = (u[r][c+1]-u[r][c], u[r+1][c]-u[r][c])
 * with periodic boundary (Sec. 1.4, Sec. 2.1).
 *
 * Solver: Algorithm 2 (IADM, Sec. 2.2) or Algorithm 1 (FTVCS, Sec. 2.1).  Each
 * iteration is one isotropic shrinkage, the products A*u and A^T*(A u - f),
 * and one FFT pair (Sec. 3.1).  All arithmetic runs in this library's CUDA
 * kernels: binary32 for the iterates; the sums of squares of every iteration
 * (the norms of the stopping test, ||A u - f||^2) as binary32 double-single
 * pairs (exact squares, compensated sums: about 44 significant bits), compared
 * in binary64; binary64 for the objective and the optimality residuals at the
 * end of a run.
 *
 * Conventions for every entry point:
 *  - Pointers to arrays may be host (pageable or pinned) or device pointers;
 *    the library detects the kind with cudaPointerGetAttributes and copies
 *    through its own device buffers.  The caller keeps ownership of every
 *    array it passes; the library keeps no pointer to caller memory after a
 *    call returns.
 *  - All device work is ordered on the handle's stream (tvcs_options.stream).
 *    Every call is synchronous: it returns after its device work finished.
 *    The handle's stream does not wait for other streams: device arrays
 *    written (or still read) by work on another stream must be complete when
 *    the call is made, unless that stream is the handle's stream.
 *  - Errors: a negative tvcs_status, with a message for tvcs_last_error().
 *    No call aborts, throws or exits.  Arguments are validated before any
 *    device work, so invalid arguments never reach a kernel.
 *  - One handle must not be used by two host threads at the same time.
 */
#ifndef TVCS_H
#define TVCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tvcs_ctx* tvcs_handle;

typedef enum {
    TVCS_OK = 0,
    TVCS_NOT_CONVERGED = 1,      /* max_iter reached before eq. (stop) held (not an error) */
    TVCS_ERR_INVALID_ARG = -1,   /* null pointer, unsupported size, non-positive parameter */
    TVCS_ERR_OOM = -2,           /* device or host allocation failed */
    TVCS_ERR_CUDA = -3,          /* a CUDA runtime call failed (message names it) */
    TVCS_ERR_TIMEOUT = -4,       /* a bounded device wait gave up */
    TVCS_ERR_DIVERGED = -5,      /* non-finite iterate or objective */
    TVCS_ERR_UNSUPPORTED = -6    /* valid request this build does not implement */
} tvcs_status;

enum { TVCS_ALGO_IADM = 0, TVCS_ALGO_FTVCS = 1 };
/* Storage of A for the products: binary32; binary16-bfloat hi+lo split (the
 * entries are hi + lo with both rounded to nearest); FP8 E4M3 with a per-row
 * binary32 scale plus a bfloat16 correction. */
enum { TVCS_PREC_FP32 = 0, TVCS_PREC_BF16X2 = 1, TVCS_PREC_FP8_BF16 = 2 };
/* Initial point: A^T f (back-projection), zero, or caller-given (tvcs_set_state). */
enum { TVCS_INIT_ATF = 0, TVCS_INIT_ZERO = 1, TVCS_INIT_GIVEN = 2 };
/* Where the products get A from: device memory (stored once by tvcs_create), or
 * the counter-based generator inside the product kernel, so that A occupies no
 * memory and costs no memory traffic. */
enum { TVCS_A_STORED = 0, TVCS_A_REGENERATE = 1 };

typedef struct {
    int algo;            /* TVCS_ALGO_IADM (default) or TVCS_ALGO_FTVCS */
    double tau;          /* proximal step of eq. (line); <= 0: 1/(1.01*lambda_max(A^T A)),
                            lambda_max from power_iters rounds of power iteration */
    int max_iter;        /* iteration cap; <= 0: 500 */
    int precision;       /* TVCS_PREC_* */
    int init;            /* TVCS_INIT_* for tvcs_solve */
    void* stream;        /* cudaStream_t for all device work; NULL: a stream the handle owns */
    int power_iters;     /* <= 0: 100 */
    long long timeout_cycles; /* bound of every device spin-wait, in SM clock cycles; <= 0: 2^31 */
    int host_loop;       /* 0 (default): the iteration loop is one CUDA graph whose WHILE node
                            the kernels end; 1: the same kernels launched from the host per
                            iteration (for profilers that cannot look inside such graphs) */
    int a_mode;          /* TVCS_A_STORED (default) or TVCS_A_REGENERATE: every product
                            regenerates A's entries from the seed given to tvcs_create (A must
                            be NULL and precision TVCS_PREC_FP32; the entries are the binary32
                            values the generator would store, so both modes apply the same A) */
    int batch_compact;   /* 1 (default): in a shared-A batch (tvcs_solve_batched), an image that
                            met eq. (stop) leaves the tensor-core GEMMs after its last iteration:
                            the running images are packed into the leading columns and the GEMMs
                            shrink with them; 0: every image keeps its column to the end */
    int autotune;        /* 1 (default): launch shapes are picked by timing candidates on the
                            device and cached per device and problem size -- the shared-A batch's
                            two GEMMs (number of persistent blocks, hence the stream-K split) at
                            the first batched call, and the regenerating products (cluster size,
                            tile height, kernel variant) at tvcs_create; 0: the default shapes
                            (one GEMM block per SM; the first regenerating candidate).  A GEMM
                            shape changes the grouping of its K sums (results agree to binary32
                            rounding); a regenerating shape changes no result. */
} tvcs_options;

typedef struct {
    int iters;           /* completed iterations of this call */
    int status;          /* tvcs_status of the call */
    int stopped_by_tol;  /* 1 if eq. (stop) ended the loop */
    double rel_change;   /* ||u^k - u^{k-1}|| / ||u^{k-1}|| at the last iteration */
    double tv;           /* sum_i ||D_i u|| at the returned u */
    double resid2;       /* ||A u - f||^2 at the returned u */
    double objective;    /* tv + (mu/2) resid2 */
    double kkt_primal;   /* ||w - D u|| (after the final multiplier update) */
    double kkt_dual;     /* ||D^T lambda + mu A^T (A u - f)|| */
    double lambda_max_norm; /* max_i ||lambda_i|| */
    double ms;           /* device time of the iterations, milliseconds */
} tvcs_result;

/* Fills *opt with the defaults above.  Never fails for non-null opt. */
void tvcs_default_options(tvcs_options* opt);

/*
 * Creates a solver for one problem size and parameter set.
 *   A      m x n*n row-major binary32, host or device; NULL: generate A on the
 *          device from `seed` by the counter-based Gaussian recipe (Philox4x32-10
 *          and Box-Muller, entries N(0, 1/m); the recipe is stated at the top
 *          of the library's generator source, k_gen.cu).  A is copied (or generated) into device
 *          memory the handle owns, stored in opt->precision.
 *   m      number of measurements, 1 <= m <= 2^24
 *   n      image side: 16, 32, 48, 64, 96, 128, 192 or 256 with binary32 storage,
 *          32, 64, 128, 192 or 256 with the bf16 and fp8 storages (other sides
 *          return TVCS_ERR_INVALID_ARG)
 *   mu     > 0, beta > 0 (penalty of eq. (ALP)), tol >= 0 (eq. (stop); 0 disables)
 *   opt    nullable (defaults)
 * On success *out receives the handle (destroy with tvcs_destroy).
 */
tvcs_status tvcs_create(tvcs_handle* out, const float* A, uint64_t seed, int m, int n,
                        double mu, double beta, double tol, const tvcs_options* opt);

/*
 * Creates a solver whose encoder is the partial DCT of Sec. 3.2: A u =
 * (C U C^T)[rows], the m coefficients rows[0..m) (indices k1*n + k2, distinct,
 * any order; the measurements f follow that order) of the orthonormal 2D
 * DCT-II of the n x n image U, C[k][j] = a_k cos(pi (2j+1) k / (2n)),
 * a_0 = sqrt(1/n), a_k = sqrt(2/n).  No matrix is stored: each product is four
 * dense n x n transforms in one thread-block-cluster kernel.  rows is a host
 * array; n is 16, 32, 48, 64, 96 or 128; 1 <= m <= n*n.  opt (nullable) must
 * keep precision TVCS_PREC_FP32 and a_mode TVCS_A_STORED.  Every other entry
 * point works on the handle as on one with a stored A (tvcs_solve_batched
 * solves such handles one after another).
 */
tvcs_status tvcs_create_partial_dct(tvcs_handle* out, const int32_t* rows, int m, int n,
                                    double mu, double beta, double tol, const tvcs_options* opt);

/*
 * Solves from the handle's initial point (opt->init) with data f (m values,
 * host or device) and writes the n*n image to u (host or device).  Runs at
 * most max_iter iterations; res (nullable) receives the summary.
 * Returns TVCS_OK when eq. (stop) held, TVCS_NOT_CONVERGED when max_iter
 * ended the loop, or an error.
 */
tvcs_status tvcs_solve(tvcs_handle h, const float* f, float* u, tvcs_result* res);

/*
 * Solves `count` problems.  hs[i] are handles, f[i] (m_i values) and u[i]
 * (n_i*n_i values) host or device pointers; mu (nullable) overrides each
 * handle's mu (every mu[i] finite and > 0, else TVCS_ERR_INVALID_ARG before
 * any handle is used); res (nullable) receives count summaries.  When every hs[i] is
 * the same handle created with precision TVCS_PREC_BF16X2, the images iterate
 * together in groups of at most 256 (count > 256: ceil(count/256) groups of
 * nearly equal size, one after another): a group's u-steps run as one batched
 * launch and its products as tensor-core GEMMs (see tvcs_apply_batched); each
 * image stops on its own eq. (stop), and with opt->batch_compact (the default)
 * it then leaves the GEMMs, whose work shrinks with the images still running.
 * An image that fails (TVCS_ERR_DIVERGED, TVCS_ERR_TIMEOUT) reports it in its
 * result; the other images and groups still run, and the call returns that
 * status.  When every hs[i] was created with a_mode
 * TVCS_A_REGENERATE (count <= 1024, all on one device with equal algo, beta
 * and init, init TVCS_INIT_ATF or TVCS_INIT_ZERO; n, m, seed, mu, tau, tol and
 * max_iter may differ), all problems iterate together in one loop graph on
 * hs[0]'s stream: one batched u-step launch per image side n, then one
 * persistent product launch over all problems that regenerates every A in
 * the kernel; each problem stops on its own eq. (stop) and then leaves the
 * product launch's work.  hs[0] keeps that batch's device state until it is
 * destroyed or called with another problem set.  Otherwise the problems are
 * solved one after another, each on its handle's stream.
 */
tvcs_status tvcs_solve_batched(const tvcs_handle* hs, int count, const float* const* f,
                               float* const* u, const double* mu, tvcs_result* res);

/*
 * Continuation in beta (the practice of Sec. 3.1 for Algorithm 1): solves with
 * beta = betas[0] from the handle's initial point, then with betas[1], ...,
 * each stage warm-started from the previous stage's u and lambda (w restarted
 * at 0) and run to eq. (stop) or max_iter.  f (m values) and u (n*n values)
 * host or device; res (nullable) receives nbeta stage summaries.  The handle's
 * own beta is in force again when the call returns.  Returns the worst stage
 * status (TVCS_NOT_CONVERGED if a stage hit max_iter) or an error.
 */
tvcs_status tvcs_solve_continuation(tvcs_handle h, const float* f, float* u, const double* betas,
                                    int nbeta, tvcs_result* res);

/* Releases every resource of h (NULL is a no-op). */
tvcs_status tvcs_destroy(tvcs_handle h);

/* Message for the last non-OK status returned on the calling thread. */
const char* tvcs_last_error(void);

/* ---- Step-level access (for tests and tools; same conventions) ------------ */

/* tau used by the handle (auto or given). */
tvcs_status tvcs_get_tau(tvcs_handle h, double* tau);

enum { TVCS_STATE_U = 0,      /* n*n   current iterate u^k */
       TVCS_STATE_W = 1,      /* 2*n*n w^k (w1 plane, then w2 plane) */
       TVCS_STATE_LAMBDA = 2, /* 2*n*n lambda^k (lambda1 plane, then lambda2 plane) */
       TVCS_STATE_G = 3,      /* n*n   g^k = A^T (A u^k - f) */
       TVCS_STATE_R = 4,      /* m     r^k = A u^k - f */
       TVCS_STATE_RHS = 5,    /* n*n   right-hand side of the last u-step in increment form:
                                       D^T (beta (w - D u^k) - lambda) - mu g, i.e. eq.
                                       (eqnorm11) times beta minus (beta D^T D + mu/tau) u^k;
                                       the u-step solves for d = u^{k+1} - u^k */
       TVCS_STATE_F = 6 };    /* m     data f */

/* Copies one state array out (get) or in (set; only U, LAMBDA and F).  Setting U
 * or F recomputes r and g; setting LAMBDA clears any pending multiplier update. */
tvcs_status tvcs_get_state(tvcs_handle h, int which, float* dst);
tvcs_status tvcs_set_state(tvcs_handle h, int which, const float* src);

/* Runs exactly `iters` iterations from the current state (no stopping test),
 * then applies the pending multiplier update and fills res (nullable). */
tvcs_status tvcs_iterate(tvcs_handle h, int iters, tvcs_result* res);

/* Row-level entry points, the two launches of one iteration.  Stage 1: rows
 * a1-a5 (deferred multiplier update of eq. (udlamb), shrink of eq. (iadmw),
 * right-hand side, FFT u-solve of eq. (eqnorm11), stop norms of eq. (stop));
 * afterwards U, W, LAMBDA and RHS hold the new values.  Stage 2: rows a6-a7
 * (r = A u - f, g = A^T r, and the multiplier update becomes pending).  The
 * state moves as in one iteration of tvcs_iterate. */
tvcs_status tvcs_run_stage(tvcs_handle h, int stage);

/* Times `reps` back-to-back launches of one stage (1 or 2, as in
 * tvcs_run_stage, without its host-side bookkeeping) on the handle's stream
 * between two CUDA events; *ms receives the elapsed milliseconds.  Afterwards
 * the state is that of `reps` applications of the stage (stage 2 leaves it
 * unchanged).  Requires a state (tvcs_solve or tvcs_set_state first).
 * Stages 3-5 time the parts of a batched iteration on the state of the last
 * tvcs_solve_batched call: 3 the two GEMM kernels (R = A U, G = A^T R), 4 their
 * two epilogue kernels, 5 the batched u-solve.  Stages 6-7 time the parts of an
 * iteration of the last uneven batch whose first handle is h: 6 the
 * regenerating product launch over all problems with its reduction, 7 the
 * u-solve launches of all image sizes. */
tvcs_status tvcs_time_stage(tvcs_handle h, int stage, int reps, double* ms);

/* Products for `count` images that share the handle's A, the batched form of
 * tvcs_apply (the two matrix-vector products of eq. (line) for many images at
 * once): R = A X - Y and G = A^T R, computed as tensor-core GEMMs on bfloat16
 * hi+lo splits of A and of the operands (X_hi A_hi + X_lo A_hi + X_hi A_lo,
 * binary32 accumulation).  X: count x n*n, Y: count x m (nullable), R: count x m,
 * G: count x n*n, image after image, host or device.  Requires a handle created
 * with precision TVCS_PREC_BF16X2, n*n a multiple of 128 and count >= 1 (groups
 * as in tvcs_solve_batched: at most 512 images each, 256 where clusters of two
 * GEMM blocks cannot run). */
tvcs_status tvcs_apply_batched(tvcs_handle h, int count, const float* X, const float* Y,
                               float* R, float* G);

/* Products alone on caller data: r = A x - y (y nullable: r = A x) and
 * g = A^T r, with the handle's stored A.  x: N, y: m, r: m, g: N. */
tvcs_status tvcs_apply(tvcs_handle h, const float* x, const float* y, float* r, float* g);

/* Test hook for the failure status TVCS_ERR_TIMEOUT (the paper has no
 * counterpart).  With extra > 0, the grid barrier of the binary32 product kernel
 * (n <= 128) waits for `extra` arrivals that never come: its bounded spin runs
 * out after opt->timeout_cycles, every block records the timeout and returns,
 * and the call (tvcs_apply, tvcs_solve, ...) returns TVCS_ERR_TIMEOUT with the
 * handle still usable.  extra = 0 (the default) restores normal operation.
 * Other storages and encoders return TVCS_ERR_UNSUPPORTED. */
tvcs_status tvcs_test_hold_grid_barrier(tvcs_handle h, int extra);

/* Test hook for the launch shape of the two batched GEMMs (R = A U - F and
 * G = A^T R; the paper has no counterpart): grid1/grid2 persistent blocks, on
 * single blocks (pair 0, grid <= SM count) or on clusters of two blocks that
 * share each 256-row tile (pair 1, grid even, grid/2 <= the clusters that fit).
 * grid1 = grid2 = 0 returns the choice to the tuner (opt->autotune) or to one
 * block per SM.  Above 256 images a batch needs pair = 1 (two N tiles of 256
 * columns per tile of A), else the batched call returns TVCS_ERR_INVALID_ARG.
 * Takes effect at the next batched call, which re-plans the
 * stream-K split and rebuilds the batch buffers.  Results of different shapes
 * agree to binary32 rounding (a tile's K sums are grouped differently), not
 * bitwise.  TVCS_ERR_INVALID_ARG for a malformed shape, TVCS_ERR_UNSUPPORTED
 * for more pairs than fit. */
tvcs_status tvcs_test_gemm_shape(tvcs_handle h, int grid1, int pair1, int grid2, int pair2);

/* ---- Products without any device allocation -------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot call cudaMalloc when they need the products -- applications that
 * reserve all device memory in their own pool at start-up, that run under a
 * hard device-memory cap, or whose latency-critical loops cannot afford the
 * implicit synchronisation of an allocation.  It computes the same
 * r = A x - y (y nullable: r = A x) and g = A^T r as tvcs_apply, without a
 * handle and without allocating anything.
 *   A      m x n*n row-major binary32, device pointer; x: n*n, y: m (or NULL),
 *          r: m, g: n*n, all device memory of the current device (or managed
 *          memory), owned by the caller; host pointers and memory of another
 *          GPU return TVCS_ERR_INVALID_ARG
 *   n      16, 32, 48, 64, 96 or 128; 1 <= m <= 2^24
 *   stream cudaStream_t (NULL: the legacy default stream); the call returns
 *          after its device work finished.  It reads a status word back to the
 *          host and synchronises the stream, so it cannot be recorded by a
 *          stream capture: a capturing stream returns TVCS_ERR_INVALID_ARG
 *          before any work.
 * Work memory: one file-scope device array of 12 MiB (per-block partial sums
 * of A^T r and a control block), which every GPU that loads the library holds
 * until the process exits.  Sizes whose partial sums do not fit return
 * TVCS_ERR_INVALID_ARG with a message naming the limit.  The first call on a
 * device performs one-time set-up on that device (it looks up the array's
 * device address and sets the kernels' shared-memory limit).  Every call on a
 * device shares the same array and clears the parts that must start at zero,
 * so calls whose device work overlaps (other host threads, other streams)
 * race on it and must be serialised by the caller. */
tvcs_status tvcs_apply_noalloc(const float* A, int m, int n, const float* x, const float* y,
                               float* r, float* g, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TVCS_H */
