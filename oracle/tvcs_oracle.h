/*
 * FP64 CPU ORACLE for TV/L2 reconstruction from random projections
 * (Xiao & Yang, "A Fast Algorithm for Total Variation Image Reconstruction
 * from Random Projections").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of the paper's iterations in binary64.  It shares no code with
 * the GPU library; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  Nothing in the product path calls it.
 *
 * Conventions (n x n image, N = n^2, pixel (r, c) at index r*n + c):
 *   (D1 u)[r][c] = u[r][(c+1) mod n] - u[r][c]   horizontal difference
 *   (D2 u)[r][c] = u[(r+1) mod n][c] - u[r][c]   vertical difference
 *   periodic boundary (Sec. 2.1, the paragraph after eq. (foru));
 *   D_i u = ((D1 u)_i, (D2 u)_i) in R^2 (Sec. 1.4).
 *   Forward DFT is unnormalised with kernel exp(-2 pi i (p r + q c)/n); the
 *   inverse carries 1/n^2.
 *
 * Readings where the paper is silent or inconsistent (each is marked where it
 * is used below):
 *   C1  IADM w-step shrinks D_i u + lambda_i/beta (the minimiser of the
 *       augmented Lagrangian (ALP)); eq. (iadmw) prints "-".  w_sign = -1
 *       reproduces the printed sign for tests that show it fails.
 *   C3  u^0 = A^T f (Algorithms 1-2 print u^0 = f, which has the wrong length).
 *   C4  lambda^0 = 0, w^0 = 0.
 *   C5  stop after the u-update when ||u^{k+1}-u^k|| <= tol ||u^k|| (eq. (stop));
 *       when ||u^k|| = 0 stop only if ||u^{k+1}|| = 0.
 *   C6  shrink returns 0 when ||z|| <= 1/beta (covers z = 0, the 0*(0/0)=0 rule).
 *   C18 the partial-DCT encoder of Sec. 3.2 is a row subset of the orthonormal
 *       2D DCT-II applied to the n x n image (C u C^T).
 *
 * Parity pins: every function here is checked in tests/ against something
 * other than itself (closed forms, explicit dense matrices, an independent
 * dual solver, convergence theorems).  See the test files for each pin.
 */
#ifndef TVCS_ORACLE_H
#define TVCS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_IADM = 0, ORACLE_FTVCS = 1 };
enum { ORACLE_INIT_ATF = 0, ORACLE_INIT_ZERO = 1, ORACLE_INIT_GIVEN = 2 };

typedef struct {
    int n;           /* image side */
    int m;           /* number of measurements (rows of A) */
    double mu;       /* fidelity weight, eq. (tv) */
    double beta;     /* penalty parameter, eqs. (atv)/(ALP) */
    double tau;      /* proximal step, eq. (line); Thm 1 needs 0 < tau < 2/lambda_max(A^T A) */
    double tol;      /* relative-change tolerance, eq. (stop); 0 disables the test */
    int max_iter;    /* iteration cap */
    int algo;        /* ORACLE_IADM (Algorithm 2) or ORACLE_FTVCS (Algorithm 1) */
    int w_sign;      /* +1 (reading C1, default) or -1 (sign as printed in eq. (iadmw)) */
    int init;        /* ORACLE_INIT_ATF (C3), ORACLE_INIT_ZERO, ORACLE_INIT_GIVEN */
} oracle_params;

typedef struct {
    int iters;            /* completed iterations */
    int stopped_by_tol;   /* 1 if eq. (stop) ended the loop */
    double rel_change;    /* ||u^k - u^{k-1}|| / ||u^{k-1}|| at the last iteration */
    double tv;            /* sum_i ||D_i u|| at the returned u */
    double resid2;        /* ||A u - f||^2 at the returned u */
    double objective;     /* tv + (mu/2) resid2, eq. (tv) */
    double atv;           /* penalty objective eq. (atv) at (w, u) */
    double kkt_primal;    /* ||w - D u|| */
    double kkt_dual;      /* ||D^T lambda + mu A^T (A u - f)|| */
    double lambda_max_norm; /* max_i ||lambda_i|| (must be <= 1 at a solution) */
    double lambda_align;  /* max over i with w_i != 0 of ||lambda_i - w_i/||w_i|| || */
} oracle_info;

/* Sec. 1.4: forward differences with periodic boundary. */
void oracle_D(int n, const double* u, double* d1, double* d2);
/* Adjoint of oracle_D: out = D1^T y1 + D2^T y2. */
void oracle_Dt(int n, const double* y1, const double* y2, double* out);
/* Eq. (shrink) / eq. (sop): w = max(||z|| - t, 0) z/||z||, 0 when ||z|| <= t (C6). */
void oracle_shrink(int count, double t, const double* z1, const double* z2,
                   double* w1, double* w2);
/* Eigenvalues of D^T D (Sec. 2.1: block circulant, diagonalised by the 2D DFT):
 * the naive 2D DFT of D^T D applied to a unit impulse.  lam[p*n+q]. */
void oracle_dtd_eigs(int n, double* lam);
/* Naive separable 2D DFT in place (inverse: conjugate kernel and 1/n^2). */
void oracle_dft2(int n, int inverse, double* re, double* im);
/* Eq. (eqnorm)/(eqnorm11) solve: (D^T D + c I) u = b by DFT diagonalisation. */
void oracle_usolve(int n, double c, const double* b, double* u);
/* r = A u - f (f may be NULL -> r = A u).  A is m x N row-major binary32,
 * promoted exactly to binary64. */
void oracle_Au(int m, int64_t N, const float* A, const double* u, const float* f, double* r);
/* g = A^T r. */
void oracle_At(int m, int64_t N, const float* A, const double* r, double* g);
/* lambda_max(A^T A) by power iteration from v = 1/sqrt(N): iters rounds of
 * v <- A^T A v / ||A^T A v||, then the Rayleigh quotient ||A v||^2. */
double oracle_lambda_max(int m, int64_t N, const float* A, int iters);
/* sum_i ||D_i u||. */
double oracle_tv(int n, const double* u);

/* Algorithm 2 (IADM) or Algorithm 1 (FTVCS) from (u0, lambda0) (used only when
 * init == ORACLE_INIT_GIVEN; lambda0 may be NULL -> 0).
 * Outputs u[N], w[2N] (w1 then w2), lam[2N] (lambda1 then lambda2); any may
 * be NULL except u.  hist (nullable) receives, per iteration k = 1..iters, 4
 * doubles: objective (tv) at u^k, penalty objective (atv) at (w^k, u^k),
 * relative change, ||A u^k - f||^2.  u_hist (nullable) receives
 * u^0, u^1, ..., u^iters ((max_iter+1) x N).
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure. */
int oracle_solve(const oracle_params* p, const float* A, const float* f,
                 const double* u0, const double* lam0,
                 double* u, double* w, double* lam, double* hist, double* u_hist,
                 oracle_info* info);

/* Residuals of the IADM fixed point at a given (u, w, lambda) (Thm 4). */
void oracle_kkt(const oracle_params* p, const float* A, const float* f, const double* u,
                const double* w, const double* lam, oracle_info* info);

/* Partial-DCT encoder (Sec. 3.2; reading C18): the orthonormal 2D DCT-II
 * out = C x C^T of an n x n image (inverse: C^T x C), C[k][j] = a_k cos(pi (2j+1) k/(2n)),
 * and A = the rows `rows` (indices k1 n + k2) of that transform. */
void oracle_dct2(int n, int inverse, const double* x, double* out);
void oracle_dct_Au(int n, int m, const int32_t* rows, const double* u, const float* f, double* r);
void oracle_dct_At(int n, int m, const int32_t* rows, const double* r, double* g);
/* oracle_solve / oracle_kkt with the partial-DCT encoder instead of a dense A. */
int oracle_solve_dct(const oracle_params* p, const int32_t* rows, const float* f,
                     const double* u0, const double* lam0,
                     double* u, double* w, double* lam, double* hist, double* u_hist,
                     oracle_info* info);
void oracle_kkt_dct(const oracle_params* p, const int32_t* rows, const float* f, const double* u,
                    const double* w, const double* lam, oracle_info* info);

/* Number of OpenMP threads the oracle uses. */
int oracle_num_threads(void);
void oracle_set_num_threads(int k);

#ifdef __cplusplus
}
#endif
#endif
