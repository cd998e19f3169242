// Steps of rows a1-a5 on a band of image rows held in shared memory, shared
// by the two u-solve kernels (k_usolve.cu: one thread-block cluster per image,
// for latency; k_usolve_img.cu: one block per image streaming row stripes, for
// batches).  Every function is called by all threads of the block; the caller
// synchronises between steps.
//
// Band layout: rows r0 .. r0+R-1 are owned (R even).  su holds u rows
// r0-1 .. r0+R (R+2 rows, halo on both sides), swl the planes w1, w2, l1, l2 of
// rows r0-1 .. r0+R-1 (R+1 rows each, plane stride WL), sg the rows of g.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "fft.cuh"

namespace tvcs {

// a1-a3, first half: for rows r0-1 .. r0+R-1 (the halo row is recomputed, not
// stored), the deferred multiplier update (eq. (udlamb)), the shrink of
// D_i u + lambda_i / beta (eq. (iadmw) with reading C1, tie by reading C6) and
// y = beta (w - D u) - lambda.  Writes sy1 (rows r0 .., R rows), sy2 (rows r0-1
// .., R+1 rows) and the new w, lambda of the owned rows to wdst / ldst (planes
// N apart, image base pointers).
template <int NN>
__device__ __forceinline__ void step_wshrink(const float* su, const float* swl, int WL, int R,
                                             int r0, float beta, int pending, float* sy1,
                                             float* sy2, float* wdst, float* ldst, int tid,
                                             int nthr)
{
    constexpr int N = NN * NN;
    const float inv_beta = 1.0f / beta;
    for (int i = tid; i < (R + 1) * NN; i += nthr) {
        const int rr = i / NN, c = i - rr * NN;      // rr = 0 is the halo row r0-1
        const int row = (r0 - 1 + rr + NN) % NN;
        const int cp = (c + 1 == NN) ? 0 : c + 1;
        const float uc = su[rr * NN + c];
        const float d1 = su[rr * NN + cp] - uc;
        const float d2 = su[(rr + 1) * NN + c] - uc;
        const int gi = row * NN + c;
        float l1 = swl[2 * WL + i], l2 = swl[3 * WL + i];
        if (pending) {  // eq. (udlamb) for the previous iteration
            l1 -= beta * (swl[i] - d1);
            l2 -= beta * (swl[WL + i] - d2);
        }
        const float z1 = d1 + l1 * inv_beta, z2 = d2 + l2 * inv_beta;
        const float nz = sqrtf(z1 * z1 + z2 * z2);
        float w1 = 0.0f, w2 = 0.0f;
        if (nz > inv_beta) {
            const float s = (nz - inv_beta) / nz;
            w1 = s * z1;
            w2 = s * z2;
        }
        sy2[i] = beta * (w2 - d2) - l2;
        if (rr >= 1) {
            sy1[(rr - 1) * NN + c] = beta * (w1 - d1) - l1;
            wdst[gi] = w1;
            wdst[N + gi] = w2;
            ldst[gi] = l1;
            ldst[N + gi] = l2;
        }
    }
}

// a3, second half: rhs = D^T y - mu g of the owned rows (increment form of
// eq. (eqnorm11) times beta), two rows packed per complex value:
// wa[j NN + c] = (rhs[r0+2j][c], rhs[r0+2j+1][c]).  rhs_out (nullable, image
// base) receives the unpacked rows.
template <int NN>
__device__ __forceinline__ void step_rhs(const float* sy1, const float* sy2, const float* sg, int R,
                                         int r0, float mu, float2* wa, float* rhs_out, int tid,
                                         int nthr)
{
    for (int i = tid; i < (R / 2) * NN; i += nthr) {
        const int j = i / NN, c = i - j * NN;
        const int cm = (c == 0) ? NN - 1 : c - 1;
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lr = 2 * j + h;   // local owned row
            const float dty = sy1[lr * NN + cm] - sy1[lr * NN + c] + sy2[lr * NN + c] -
                              sy2[(lr + 1) * NN + c];
            v[h] = dty - mu * sg[lr * NN + c];
        }
        wa[i] = make_float2(v[0], v[1]);
        if (rhs_out) {
            rhs_out[(r0 + 2 * j) * NN + c] = v[0];
            rhs_out[(r0 + 2 * j + 1) * NN + c] = v[1];
        }
    }
}

// a3 in two parts, for a caller that has y before g: step_dty stores
// (D^T y)[r0+2j][c], (D^T y)[r0+2j+1][c] packed in wa[j NN + c]; step_sub_g then
// subtracts mu g, giving the packed rows of step_rhs.
template <int NN>
__device__ __forceinline__ void step_dty(const float* sy1, const float* sy2, int R, float2* wa,
                                         int tid, int nthr)
{
    for (int i = tid; i < (R / 2) * NN; i += nthr) {
        const int j = i / NN, c = i - j * NN;
        const int cm = (c == 0) ? NN - 1 : c - 1;
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lr = 2 * j + h;
            v[h] = sy1[lr * NN + cm] - sy1[lr * NN + c] + sy2[lr * NN + c] - sy2[(lr + 1) * NN + c];
        }
        wa[i] = make_float2(v[0], v[1]);
    }
}

template <int NN>
__device__ __forceinline__ void step_sub_g(const float* sg, int R, int r0, float mu, float2* wa,
                                           float* rhs_out, int tid, int nthr)
{
    for (int i = tid; i < (R / 2) * NN; i += nthr) {
        const int j = i / NN, c = i - j * NN;
        float2 v = wa[i];
        v.x = v.x - mu * sg[(2 * j) * NN + c];
        v.y = v.y - mu * sg[(2 * j + 1) * NN + c];
        wa[i] = v;
        if (rhs_out) {
            rhs_out[(r0 + 2 * j) * NN + c] = v.x;
            rhs_out[(r0 + 2 * j + 1) * NN + c] = v.y;
        }
    }
}

// a4: from the R/2 packed forward row transforms Z, the half spectra of the
// owned rows, X_q = (Z_q + conj Z_{n-q}) / 2 and Y_q = (Z_q - conj Z_{n-q}) / (2i),
// q = 0 .. n/2, stored at spec[lr * rs + q * qs] for local row lr.
template <int NN>
__device__ __forceinline__ void step_split(const float2* Z, int R, float2* spec, int rs, int qs,
                                           int tid, int nthr)
{
    constexpr int Q = NN / 2 + 1;
    for (int i = tid; i < (R / 2) * Q; i += nthr) {
        const int j = i / Q, q = i - j * Q;
        const float2 a = Z[j * NN + q];
        const float2 b = Z[j * NN + (NN - q) % NN];
        spec[(2 * j) * rs + q * qs] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        spec[(2 * j + 1) * rs + q * qs] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
    }
}

// a4: the divisor beta Lambda_pq + mu/tau for row frequency p, column frequency q.
__device__ __forceinline__ float solve_divisor(const float* s2, int p, int q, float beta,
                                               float mu_over_tau)
{
    return beta * (s2[p] + s2[q]) + mu_over_tau;
}

// a4: packs rows 2j, 2j+1 of the solved half spectra (local rows, layout as in
// step_split) into full-length inverse transforms wa[j NN + q] = X_q + i Y_q,
// using conjugate symmetry above n/2.
template <int NN>
__device__ __forceinline__ void step_pack_inverse(const float2* spec, int rs, int qs, int R,
                                                  float2* wa, int tid, int nthr)
{
    constexpr int Q = NN / 2 + 1;
    for (int i = tid; i < (R / 2) * NN; i += nthr) {
        const int j = i / NN, q = i - j * NN;
        const bool lo = q < Q;
        const int qq = lo ? q : NN - q;
        float2 Xv = spec[(2 * j) * rs + qq * qs];
        float2 Yv = spec[(2 * j + 1) * rs + qq * qs];
        if (qq == 0 || 2 * qq == NN) {  // exactly real bins
            Xv.y = 0.f;
            Yv.y = 0.f;
        }
        if (!lo) {
            Xv.y = -Xv.y;
            Yv.y = -Yv.y;
        }
        wa[i] = make_float2(Xv.x - Yv.y, Xv.y + Yv.x);
    }
}

// a4-a5: u <- u + d for the owned rows, d = z / n^2 from the packed inverse
// transforms z; uold points at row r0 of the old u (row stride NN).  Adds d^2
// and u_old^2 to the thread's double-single sums du2, u2.  When u_hi
// is set, the new u is also stored as bf16 hi/lo planes (round to nearest even
// of u, then of the exact remainder).
template <int NN>
__device__ __forceinline__ void step_update(const float2* z, const float* uold, int R, int r0,
                                            float* u, unsigned short* u_hi, unsigned short* u_lo,
                                            float2& du2, float2& u2, int tid, int nthr)
{
    const float sc = 1.0f / (float)(NN * NN);
    for (int i = tid; i < (R / 2) * NN; i += nthr) {
        const int j = i / NN, c = i - j * NN;
        const float2 v = z[i];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lr = 2 * j + h;
            const float d = (h == 0 ? v.x : v.y) * sc;
            const float o = uold[lr * NN + c];
            du2 = ds_add(du2, ds_sq(d));
            u2 = ds_add(u2, ds_sq(o));
            const float nw = o + d;
            u[(r0 + lr) * NN + c] = nw;
            if (u_hi) {
                const unsigned int bits = __float_as_uint(nw);
                const unsigned int hb = (bits + 0x7fffu + ((bits >> 16) & 1u)) & 0xffff0000u;
                const float rem = nw - __uint_as_float(hb);
                const unsigned int rb = __float_as_uint(rem);
                const unsigned int lb = (rb + 0x7fffu + ((rb >> 16) & 1u)) & 0xffff0000u;
                u_hi[(r0 + lr) * NN + c] = (unsigned short)(hb >> 16);
                u_lo[(r0 + lr) * NN + c] = (unsigned short)(lb >> 16);
            }
        }
    }
}

// a5: eq. (stop) and the loop bookkeeping of one image, from the sums
// ||u^{k+1} - u^k||^2 and ||u^k||^2 (one thread; the host derives the relative
// change from du2 and u2).
__device__ __forceinline__ void step_stop(Ctrl* ctrl, int par, int mode, double tdu, double tu)
{
    if (ctrl->algo == 0) ctrl->pending = 1;   // u moved: its multiplier update is due
    ctrl->wpar = par ^ 1;
    ctrl->du2 = tdu;
    ctrl->u2 = tu;
    if (mode == MODE_ITER) {
        const int it = ctrl->it + 1;
        ctrl->it = it;
        bool stop = false;
        if (!isfinite(tdu) || !isfinite(tu)) {
            set_error(ctrl, ERR_NONFINITE);
            stop = true;
        }
        const double tol = ctrl->tol;   // eq. (stop), reading C5
        if (tol > 0.0 && (tu > 0.0 ? tdu <= tol * tol * tu : tdu == 0.0)) {
            ctrl->stop_by_tol = 1;
            stop = true;
        }
        if (it >= ctrl->max_iter || ctrl->error != ERR_NONE) stop = true;
        if (stop) ctrl->done = 1;
    }
}

}  // namespace tvcs
