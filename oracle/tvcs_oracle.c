/*
 * FP64 CPU ORACLE -- test infrastructure only (see tvcs_oracle.h).
 *
 * A plain restatement of Xiao & Yang's Algorithm 1 (FTVCS, Sec. 2.1) and
 * Algorithm 2 (IADM, Sec. 2.2) in binary64, in the paper's order and
 * notation.  Matrix products are plain loops over the binary32 entries of A
 * promoted to binary64; the u-subproblem is solved by a naive separable 2D DFT
 * whose divisor comes from the DFT of the D^T D stencil.  OpenMP splits loops
 * over independent outputs only, so results do not depend on the thread count.
 */
#include "tvcs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(r, c) ((int64_t)(r) * n + (c))

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (k >= 1); used to time the oracle
 * on one core beside all cores.  Results do not depend on it. */
void oracle_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k >= 1) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* Sec. 1.4 and eq. (tv): D_i in R^{2 x n^2} stacks row i of D^(1) and D^(2). */
void oracle_D(int n, const double* u, double* d1, double* d2)
{
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            d1[IDX(r, c)] = u[IDX(r, (c + 1) % n)] - u[IDX(r, c)];
            d2[IDX(r, c)] = u[IDX((r + 1) % n, c)] - u[IDX(r, c)];
        }
}

/* Transpose of oracle_D, written entry by entry from the definition of D:
 * pixel (r,c) appears with +1 in d1 at (r, c-1) and in d2 at (r-1, c), and
 * with -1 in both at (r, c). */
void oracle_Dt(int n, const double* y1, const double* y2, double* out)
{
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            int cm = (c + n - 1) % n, rm = (r + n - 1) % n;
            out[IDX(r, c)] = y1[IDX(r, cm)] - y1[IDX(r, c)] + y2[IDX(rm, c)] - y2[IDX(r, c)];
        }
}

/* Eq. (shrink), equivalently s(alpha) = alpha - P_B(alpha) of eq. (sop). */
void oracle_shrink(int count, double t, const double* z1, const double* z2,
                   double* w1, double* w2)
{
    for (int i = 0; i < count; ++i) {
        double nz = sqrt(z1[i] * z1[i] + z2[i] * z2[i]);
        if (nz <= t) {           /* C6: includes z = 0 (0 * (0/0) = 0) */
            w1[i] = 0.0;
            w2[i] = 0.0;
        } else {
            double s = (nz - t) / nz;
            w1[i] = s * z1[i];
            w2[i] = s * z2[i];
        }
    }
}

/* Naive 1D DFT of each of `count` rows of length n (stride `stride` between
 * elements, `dist` between rows), in place through a temporary.  Twiddles
 * cos/sin(2 pi t / n) with t = (j*k) mod n reduced exactly. */
static void dft_lines(int n, int inverse, double* re, double* im, int count,
                      int64_t stride, int64_t dist, const double* ct, const double* st)
{
    #pragma omp parallel
    {
        double* tr = (double*)malloc(sizeof(double) * (size_t)n);
        double* ti = (double*)malloc(sizeof(double) * (size_t)n);
        #pragma omp for schedule(static)
        for (int line = 0; line < count; ++line) {
            double* lr = re + (int64_t)line * dist;
            double* li = im + (int64_t)line * dist;
            for (int k = 0; k < n; ++k) {
                double sr = 0.0, si = 0.0;
                int t = 0;                      /* t = (j*k) mod n, advanced exactly */
                for (int j = 0; j < n; ++j, t = (t + k >= n) ? t + k - n : t + k) {
                    double c = ct[t];
                    double s = inverse ? st[t] : -st[t];
                    double xr = lr[(int64_t)j * stride], xi = li[(int64_t)j * stride];
                    sr += xr * c - xi * s;
                    si += xr * s + xi * c;
                }
                tr[k] = sr;
                ti[k] = si;
            }
            for (int k = 0; k < n; ++k) {
                lr[(int64_t)k * stride] = tr[k];
                li[(int64_t)k * stride] = ti[k];
            }
        }
        free(tr);
        free(ti);
    }
}

void oracle_dft2(int n, int inverse, double* re, double* im)
{
    double* ct = (double*)malloc(sizeof(double) * (size_t)n);
    double* st = (double*)malloc(sizeof(double) * (size_t)n);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < n; ++t) {
        ct[t] = cos(two_pi * (double)t / (double)n);
        st[t] = sin(two_pi * (double)t / (double)n);
    }
    dft_lines(n, inverse, re, im, n, 1, n, ct, st);   /* along c, every row */
    dft_lines(n, inverse, re, im, n, n, 1, ct, st);   /* along r, every column */
    if (inverse) {
        double s = 1.0 / ((double)n * (double)n);
        for (int64_t i = 0; i < (int64_t)n * n; ++i) { re[i] *= s; im[i] *= s; }
    }
    free(ct);
    free(st);
}

/* Sec. 2.1: under periodic boundary D^T D is block circulant, so it acts as a
 * circular convolution with its response k to a unit impulse at (0,0); the
 * 2D DFT of k gives its eigenvalues. */
void oracle_dtd_eigs(int n, double* lam)
{
    int64_t N = (int64_t)n * n;
    double* delta = (double*)calloc((size_t)N, sizeof(double));
    double* d1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)N);
    double* im = (double*)calloc((size_t)N, sizeof(double));
    delta[0] = 1.0;
    oracle_D(n, delta, d1, d2);
    oracle_Dt(n, d1, d2, lam);       /* k = D^T D e_0 */
    oracle_dft2(n, 0, lam, im);      /* eigenvalues are real: imaginary part ~ 0 */
    free(delta); free(d1); free(d2); free(im);
}

/* Eq. (eqnorm) / eq. (eqnorm11): (D^T D + c I) u = b, solved by two 2D DFTs. */
void oracle_usolve(int n, double c, const double* b, double* u)
{
    int64_t N = (int64_t)n * n;
    double* lam = (double*)malloc(sizeof(double) * (size_t)N);
    double* re = (double*)malloc(sizeof(double) * (size_t)N);
    double* im = (double*)calloc((size_t)N, sizeof(double));
    oracle_dtd_eigs(n, lam);
    memcpy(re, b, sizeof(double) * (size_t)N);
    oracle_dft2(n, 0, re, im);
    for (int64_t i = 0; i < N; ++i) {
        double d = lam[i] + c;
        re[i] /= d;
        im[i] /= d;
    }
    oracle_dft2(n, 1, re, im);
    memcpy(u, re, sizeof(double) * (size_t)N);
    free(lam); free(re); free(im);
}

/* g_k = A^T (A u^k - f) (eq. (line)) needs the two products below. */
void oracle_Au(int m, int64_t N, const float* A, const double* u, const float* f, double* r)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        const float* a = A + (int64_t)i * N;
        double acc = 0.0;
        for (int64_t j = 0; j < N; ++j) acc += (double)a[j] * u[j];
        r[i] = f ? acc - (double)f[i] : acc;
    }
}

void oracle_At(int m, int64_t N, const float* A, const double* r, double* g)
{
    const int64_t CB = 512;   /* column block per task */
    int64_t nblk = (N + CB - 1) / CB;
    #pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
        int64_t j0 = b * CB, j1 = j0 + CB < N ? j0 + CB : N;
        for (int64_t j = j0; j < j1; ++j) g[j] = 0.0;
        for (int i = 0; i < m; ++i) {
            const float* a = A + (int64_t)i * N;
            double ri = r[i];
            for (int64_t j = j0; j < j1; ++j) g[j] += (double)a[j] * ri;
        }
    }
}

/* ---- Partial-DCT encoder (Sec. 3.2): A = rows of the orthonormal 2D DCT ----
 * C[k][j] = a_k cos(pi (2j+1) k / (2n)), a_0 = sqrt(1/n), a_k = sqrt(2/n) (the
 * orthonormal DCT-II; reading C18: the 2D transform is C x C^T on the n x n
 * image).  The cosine is taken at the exactly reduced index (2j+1)k mod 4n. */
static double* dct_matrix(int n)
{
    double* C = (double*)malloc(sizeof(double) * (size_t)n * n);
    if (!C) return NULL;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        const double a = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
        for (int j = 0; j < n; ++j) {
            const long t = ((long)(2 * j + 1) * k) % (4L * n);
            C[(int64_t)k * n + j] = a * cos(2.0 * pi * (double)t / (4.0 * n));
        }
    }
    return C;
}

/* out = C x C^T (forward) or C^T x C (inverse), x and out n x n row-major. */
void oracle_dct2(int n, int inverse, const double* x, double* out)
{
    double* C = dct_matrix(n);
    double* t = (double*)malloc(sizeof(double) * (size_t)n * n);
    /* t = x C^T (forward: t[r][k] = sum_c x[r][c] C[k][c]) or x C (inverse) */
    #pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r)
        for (int k = 0; k < n; ++k) {
            double acc = 0.0;
            for (int c = 0; c < n; ++c)
                acc += x[(int64_t)r * n + c] * (inverse ? C[(int64_t)c * n + k] : C[(int64_t)k * n + c]);
            t[(int64_t)r * n + k] = acc;
        }
    /* out = C t (forward: out[k][q] = sum_r C[k][r] t[r][q]) or C^T t (inverse) */
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < n; ++k)
        for (int q = 0; q < n; ++q) {
            double acc = 0.0;
            for (int r = 0; r < n; ++r)
                acc += (inverse ? C[(int64_t)r * n + k] : C[(int64_t)k * n + r]) * t[(int64_t)r * n + q];
            out[(int64_t)k * n + q] = acc;
        }
    free(C);
    free(t);
}

/* r_i = (C u C^T)[rows_i] - f_i (f may be NULL). */
void oracle_dct_Au(int n, int m, const int32_t* rows, const double* u, const float* f, double* r)
{
    double* X = (double*)malloc(sizeof(double) * (size_t)n * n);
    oracle_dct2(n, 0, u, X);
    for (int i = 0; i < m; ++i) r[i] = f ? X[rows[i]] - (double)f[i] : X[rows[i]];
    free(X);
}

/* g = A^T r = C^T S C with S zero except S[rows_i] = r_i. */
void oracle_dct_At(int n, int m, const int32_t* rows, const double* r, double* g)
{
    double* S = (double*)calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < m; ++i) S[rows[i]] += r[i];
    oracle_dct2(n, 1, S, g);
    free(S);
}

/* The encoder as an operator: a dense binary32 matrix, or partial-DCT rows. */
typedef struct {
    int dct;                 /* 0: dense A, 1: partial DCT */
    int m;
    int64_t N;
    const float* A;          /* dense: m x N */
    int n;
    const int32_t* rows;     /* partial DCT: m coefficient indices */
} oracle_op;

static void op_Au(const oracle_op* op, const double* u, const float* f, double* r)
{
    if (op->dct)
        oracle_dct_Au(op->n, op->m, op->rows, u, f, r);
    else
        oracle_Au(op->m, op->N, op->A, u, f, r);
}

static void op_At(const oracle_op* op, const double* r, double* g)
{
    if (op->dct)
        oracle_dct_At(op->n, op->m, op->rows, r, g);
    else
        oracle_At(op->m, op->N, op->A, r, g);
}

static double dot(int64_t len, const double* x, const double* y)
{
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += x[i] * y[i];
    return s;
}

double oracle_lambda_max(int m, int64_t N, const float* A, int iters)
{
    double* v = (double*)malloc(sizeof(double) * (size_t)N);
    double* y = (double*)malloc(sizeof(double) * (size_t)m);
    double* z = (double*)malloc(sizeof(double) * (size_t)N);
    double v0 = 1.0 / sqrt((double)N);
    for (int64_t j = 0; j < N; ++j) v[j] = v0;
    for (int it = 0; it < iters; ++it) {
        oracle_Au(m, N, A, v, NULL, y);
        oracle_At(m, N, A, y, z);
        double nz = sqrt(dot(N, z, z));
        for (int64_t j = 0; j < N; ++j) v[j] = z[j] / nz;
    }
    oracle_Au(m, N, A, v, NULL, y);
    double lam = dot(m, y, y);
    free(v); free(y); free(z);
    return lam;
}

double oracle_tv(int n, const double* u)
{
    int64_t N = (int64_t)n * n;
    double* d1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)N);
    oracle_D(n, u, d1, d2);
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += sqrt(d1[i] * d1[i] + d2[i] * d2[i]);
    free(d1); free(d2);
    return s;
}

static void kkt_impl(const oracle_params* p, const oracle_op* op, const float* f, const double* u,
                     const double* w, const double* lam, oracle_info* info)
{
    int n = p->n, m = p->m;
    int64_t N = (int64_t)n * n;
    double* d1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)N);
    double* r = (double*)malloc(sizeof(double) * (size_t)m);
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    double* t = (double*)malloc(sizeof(double) * (size_t)N);
    oracle_D(n, u, d1, d2);
    double tv = 0.0, pr = 0.0, atv = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        tv += sqrt(d1[i] * d1[i] + d2[i] * d2[i]);
        double e1 = w[i] - d1[i], e2 = w[N + i] - d2[i];
        pr += e1 * e1 + e2 * e2;
        atv += sqrt(w[i] * w[i] + w[N + i] * w[N + i]) + 0.5 * p->beta * (e1 * e1 + e2 * e2);
    }
    op_Au(op, u, f, r);
    double r2 = dot(m, r, r);
    op_At(op, r, g);
    oracle_Dt(n, lam, lam + N, t);
    double du = 0.0, lmax = 0.0, align = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double e = t[i] + p->mu * g[i];
        du += e * e;
        double l1 = lam[i], l2 = lam[N + i];
        double ln = sqrt(l1 * l1 + l2 * l2);
        if (ln > lmax) lmax = ln;
        double wn = sqrt(w[i] * w[i] + w[N + i] * w[N + i]);
        if (wn > 0.0) {
            double a1 = l1 - w[i] / wn, a2 = l2 - w[N + i] / wn;
            double a = sqrt(a1 * a1 + a2 * a2);
            if (a > align) align = a;
        }
    }
    info->tv = tv;
    info->resid2 = r2;
    info->objective = tv + 0.5 * p->mu * r2;
    info->atv = atv + 0.5 * p->mu * r2;
    info->kkt_primal = sqrt(pr);
    info->kkt_dual = sqrt(du);
    info->lambda_max_norm = lmax;
    info->lambda_align = align;
    free(d1); free(d2); free(r); free(g); free(t);
}

void oracle_kkt(const oracle_params* p, const float* A, const float* f, const double* u,
                const double* w, const double* lam, oracle_info* info)
{
    oracle_op op = {0, p->m, (int64_t)p->n * p->n, A, p->n, NULL};
    kkt_impl(p, &op, f, u, w, lam, info);
}

void oracle_kkt_dct(const oracle_params* p, const int32_t* rows, const float* f, const double* u,
                    const double* w, const double* lam, oracle_info* info)
{
    oracle_op op = {1, p->m, (int64_t)p->n * p->n, NULL, p->n, rows};
    kkt_impl(p, &op, f, u, w, lam, info);
}

static int solve_impl(const oracle_params* p, const oracle_op* op, const float* f,
                      const double* u0, const double* lam0,
                      double* u_out, double* w_out, double* lam_out, double* hist, double* u_hist,
                      oracle_info* info)
{
    if (!p || !f || !u_out || !info) return -1;
    if (p->n < 2 || p->m < 1 || !(p->mu > 0) || !(p->beta > 0) || !(p->tau > 0) ||
        p->max_iter < 0 || (p->init == ORACLE_INIT_GIVEN && !u0))
        return -1;
    const int n = p->n, m = p->m;
    const int64_t N = (int64_t)n * n;
    const double beta = p->beta, mu = p->mu, tau = p->tau;
    const int iadm = p->algo == ORACLE_IADM;
    const double wsign = p->w_sign < 0 ? -1.0 : 1.0;

    double* u = (double*)malloc(sizeof(double) * (size_t)N);
    double* un = (double*)malloc(sizeof(double) * (size_t)N);
    double* w = (double*)calloc((size_t)(2 * N), sizeof(double));
    double* lam = (double*)calloc((size_t)(2 * N), sizeof(double));
    double* d1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* d2 = (double*)malloc(sizeof(double) * (size_t)N);
    double* z1 = (double*)malloc(sizeof(double) * (size_t)N);
    double* z2 = (double*)malloc(sizeof(double) * (size_t)N);
    double* b = (double*)malloc(sizeof(double) * (size_t)N);
    double* g = (double*)malloc(sizeof(double) * (size_t)N);
    double* r = (double*)malloc(sizeof(double) * (size_t)m);
    double* fd = (double*)malloc(sizeof(double) * (size_t)m);
    double* eig = (double*)malloc(sizeof(double) * (size_t)N);
    double* re = (double*)malloc(sizeof(double) * (size_t)N);
    double* im = (double*)malloc(sizeof(double) * (size_t)N);
    if (!u || !un || !w || !lam || !d1 || !d2 || !z1 || !z2 || !b || !g || !r || !fd ||
        !eig || !re || !im) {
        free(u); free(un); free(w); free(lam); free(d1); free(d2); free(z1); free(z2);
        free(b); free(g); free(r); free(fd); free(eig); free(re); free(im);
        return -2;
    }

    /* Initialisation (C3, C4). */
    if (p->init == ORACLE_INIT_GIVEN) {
        memcpy(u, u0, sizeof(double) * (size_t)N);
        if (lam0 && iadm) memcpy(lam, lam0, sizeof(double) * 2 * (size_t)N);
    } else if (p->init == ORACLE_INIT_ZERO) {
        memset(u, 0, sizeof(double) * (size_t)N);
    } else {
        for (int i = 0; i < m; ++i) fd[i] = (double)f[i];
        op_At(op, fd, u);
    }
    if (u_hist) memcpy(u_hist, u, sizeof(double) * (size_t)N);
    oracle_dtd_eigs(n, eig);

    /* g_0 = A^T (A u^0 - f), eq. (line). */
    op_Au(op, u, f, r);
    op_At(op, r, g);

    const double c = mu / (beta * tau);   /* mu/(beta tau) in eqs. (eqnorm)/(eqnorm11) */
    int k = 0, stopped = 0;
    double relchg = 0.0;
    while (k < p->max_iter) {
        /* Step 1: w^{k+1} by eq. (shrink) (FTVCS) or eq. (iadmw) with reading C1. */
        oracle_D(n, u, d1, d2);
        for (int64_t i = 0; i < N; ++i) {
            z1[i] = d1[i] + (iadm ? wsign * lam[i] / beta : 0.0);
            z2[i] = d2[i] + (iadm ? wsign * lam[N + i] / beta : 0.0);
        }
        oracle_shrink((int)N, 1.0 / beta, z1, z2, w, w + N);

        /* Step 2: u^{k+1} from eq. (eqnorm11) (eq. (eqnorm) when lambda = 0):
         * (D^T D + mu/(beta tau) I) u = D^T (w - lambda/beta) + mu/(beta tau) (u^k - tau g_k). */
        for (int64_t i = 0; i < N; ++i) {
            z1[i] = w[i] - (iadm ? lam[i] / beta : 0.0);
            z2[i] = w[N + i] - (iadm ? lam[N + i] / beta : 0.0);
        }
        oracle_Dt(n, z1, z2, b);
        for (int64_t i = 0; i < N; ++i) b[i] += c * (u[i] - tau * g[i]);
        memcpy(re, b, sizeof(double) * (size_t)N);
        memset(im, 0, sizeof(double) * (size_t)N);
        oracle_dft2(n, 0, re, im);
        for (int64_t i = 0; i < N; ++i) {
            double d = eig[i] + c;
            re[i] /= d;
            im[i] /= d;
        }
        oracle_dft2(n, 1, re, im);
        memcpy(un, re, sizeof(double) * (size_t)N);

        /* Step 3 (IADM): lambda^{k+1} = lambda^k - beta (w^{k+1} - D u^{k+1}), eq. (udlamb). */
        oracle_D(n, un, d1, d2);
        if (iadm)
            for (int64_t i = 0; i < N; ++i) {
                lam[i] -= beta * (w[i] - d1[i]);
                lam[N + i] -= beta * (w[N + i] - d2[i]);
            }

        /* Eq. (stop) with reading C5. */
        double dn = 0.0, on = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double e = un[i] - u[i];
            dn += e * e;
            on += u[i] * u[i];
        }
        dn = sqrt(dn);
        on = sqrt(on);
        relchg = on > 0.0 ? dn / on : (dn > 0.0 ? INFINITY : 0.0);
        memcpy(u, un, sizeof(double) * (size_t)N);
        ++k;

        /* g_{k+1} for the next linearisation, and the history record. */
        op_Au(op, u, f, r);
        op_At(op, r, g);
        if (hist) {
            double r2 = dot(m, r, r);
            double tv = 0.0, pen = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                tv += sqrt(d1[i] * d1[i] + d2[i] * d2[i]);
                double e1 = w[i] - d1[i], e2 = w[N + i] - d2[i];
                pen += sqrt(w[i] * w[i] + w[N + i] * w[N + i]) + 0.5 * beta * (e1 * e1 + e2 * e2);
            }
            double* h = hist + 4 * (int64_t)(k - 1);
            h[0] = tv + 0.5 * mu * r2;
            h[1] = pen + 0.5 * mu * r2;
            h[2] = relchg;
            h[3] = r2;
        }
        if (u_hist) memcpy(u_hist + (int64_t)k * N, u, sizeof(double) * (size_t)N);
        if (p->tol > 0.0 && (on > 0.0 ? dn <= p->tol * on : dn == 0.0)) {
            stopped = 1;
            break;
        }
    }

    memset(info, 0, sizeof(*info));
    kkt_impl(p, op, f, u, w, lam, info);
    info->iters = k;
    info->stopped_by_tol = stopped;
    info->rel_change = relchg;
    memcpy(u_out, u, sizeof(double) * (size_t)N);
    if (w_out) memcpy(w_out, w, sizeof(double) * 2 * (size_t)N);
    if (lam_out) memcpy(lam_out, lam, sizeof(double) * 2 * (size_t)N);

    free(u); free(un); free(w); free(lam); free(d1); free(d2); free(z1); free(z2);
    free(b); free(g); free(r); free(fd); free(eig); free(re); free(im);
    return 0;
}

int oracle_solve(const oracle_params* p, const float* A, const float* f,
                 const double* u0, const double* lam0,
                 double* u_out, double* w_out, double* lam_out, double* hist, double* u_hist,
                 oracle_info* info)
{
    if (!p || !A) return -1;
    oracle_op op = {0, p->m, (int64_t)p->n * p->n, A, p->n, NULL};
    return solve_impl(p, &op, f, u0, lam0, u_out, w_out, lam_out, hist, u_hist, info);
}

int oracle_solve_dct(const oracle_params* p, const int32_t* rows, const float* f,
                     const double* u0, const double* lam0,
                     double* u_out, double* w_out, double* lam_out, double* hist, double* u_hist,
                     oracle_info* info)
{
    if (!p || !rows) return -1;
    oracle_op op = {1, p->m, (int64_t)p->n * p->n, NULL, p->n, rows};
    return solve_impl(p, &op, f, u0, lam0, u_out, w_out, lam_out, hist, u_hist, info);
}
