// Rows a1-a5 of one IADM/FTVCS iteration (Xiao & Yang, Sec. 2.1-2.2):
//   k_wstep_rowfft  multiplier update (eq. (udlamb), deferred from the last
//                   iteration), shrinkage (eq. (iadmw) with D_i u + lambda_i/beta,
//                   the minimiser of eq. (ALP)), u-step right-hand side
//                   (eq. (eqnorm11) times beta), forward row FFTs;
//   k_fft_cols      column FFT, divide by beta*Lambda_pq + mu/tau, inverse column FFT;
//   k_fft_rows_inv  inverse row FFTs -> u^{k+1}, binary64 norms of eq. (stop);
// and the end-of-run kernels (final multiplier update, objective, optimality
// residuals).
//
// Layout: u, g, rhs are n x n row-major binary32.  w and lambda are two
// planes each (D1 component, then D2 component) and are double-buffered
// (ctrl->wpar selects the current copy) because every block reads one halo
// row that its neighbour rewrites.  The half spectrum is n x (n/2+1) float2.
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace tvcs {

// ---------------------------------------------------------------------------
// w-step, right-hand side and forward row FFT.  One block per pair of rows
// (r0, r0+1), packed as one complex row z = x + i y.
// ---------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(256) k_wstep_rowfft(
    const float* __restrict__ u, float* __restrict__ wbuf, float* __restrict__ lbuf,
    const float* __restrict__ g,
    float* __restrict__ rhs_out, float2* __restrict__ spec, const float2* __restrict__ tw_g,
    float beta, float mu_over_tau, float mu, Ctrl* __restrict__ ctrl, int mode)
{
    constexpr int N = NN * NN;
    constexpr int Q = NN / 2 + 1;
    __shared__ float su[4][NN];            // u rows r0-1 .. r0+2
    __shared__ float sy1[3][NN], sy2[3][NN];  // beta*w^{k+1} - lambda^k, rows r0-1 .. r0+1
    __shared__ float sg[2][NN];
    __shared__ float2 ca[NN], cb[NN];
    __shared__ float2 tw[NN];

    const int tid = threadIdx.x;
    const int r0 = 2 * blockIdx.x;
    if (mode == MODE_ITER) {
        const int done = ctrl->done;
        if (blockIdx.x == 0 && tid == 0) ctrl->skip = done;
        if (done) return;
    }
    const int pending = ctrl->pending;
    const int par = ctrl->wpar;
    const float* wsrc = wbuf + (size_t)par * 2 * N;
    const float* lsrc = lbuf + (size_t)par * 2 * N;
    float* wdst = wbuf + (size_t)(par ^ 1) * 2 * N;
    float* ldst = lbuf + (size_t)(par ^ 1) * 2 * N;

    for (int i = tid; i < 4 * NN; i += blockDim.x) {
        const int rr = i / NN, c = i - rr * NN;
        const int row = (r0 - 1 + rr + NN) % NN;
        su[rr][c] = u[row * NN + c];
    }
    for (int i = tid; i < NN; i += blockDim.x) tw[i] = tw_g[i];
    __syncthreads();

    const float inv_beta = 1.0f / beta;
    for (int i = tid; i < 3 * NN; i += blockDim.x) {
        const int rr = i / NN, c = i - rr * NN;
        const int row = (r0 - 1 + rr + NN) % NN;
        const int cp = (c + 1 == NN) ? 0 : c + 1;
        const float uc = su[rr][c];
        const float d1 = su[rr][cp] - uc;
        const float d2 = su[rr + 1][c] - uc;
        const int gi = row * NN + c;
        float l1 = lsrc[gi], l2 = lsrc[N + gi];
        if (pending) {  // eq. (udlamb) for the previous iteration
            l1 -= beta * (wsrc[gi] - d1);
            l2 -= beta * (wsrc[N + gi] - d2);
        }
        // eq. (iadmw), reading C1: shrink D_i u + lambda_i / beta
        const float z1 = d1 + l1 * inv_beta, z2 = d2 + l2 * inv_beta;
        const float nz = sqrtf(z1 * z1 + z2 * z2);
        float w1 = 0.0f, w2 = 0.0f;
        if (nz > inv_beta) {  // reading C6: zero when ||z|| <= 1/beta
            const float s = (nz - inv_beta) / nz;
            w1 = s * z1;
            w2 = s * z2;
        }
        // y = beta (w^{k+1} - D u^k) - lambda^k: the increment form of eq. (eqnorm11)
        sy1[rr][c] = beta * (w1 - d1) - l1;
        sy2[rr][c] = beta * (w2 - d2) - l2;
        if (rr >= 1) {
            wdst[gi] = w1;
            wdst[N + gi] = w2;
            ldst[gi] = l1;
            ldst[N + gi] = l2;
        }
    }
    // g^k = A^T (A u^k - f) for the two owned rows.
    for (int i = tid; i < 2 * NN; i += blockDim.x) sg[i / NN][i % NN] = g[r0 * NN + i];
    __syncthreads();

    // eq. (eqnorm11) times beta, solved for the increment d = u^{k+1} - u^k:
    // (beta D^T D + (mu/tau) I) d = D^T (beta (w - D u^k) - lambda) - mu g.  Equal to the
    // printed form in exact arithmetic; the large (mu/tau) u^k term cancels analytically, so
    // the FFT round-off scales with the step, not with u.
    for (int c = tid; c < NN; c += blockDim.x) {
        const int cm = (c == 0) ? NN - 1 : c - 1;
        float v[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const float dty = sy1[rr + 1][cm] - sy1[rr + 1][c] + sy2[rr][c] - sy2[rr + 1][c];
            v[rr] = dty - mu * sg[rr][c];
        }
        ca[c] = make_float2(v[0], v[1]);
        if (rhs_out) {
            rhs_out[r0 * NN + c] = v[0];
            rhs_out[(r0 + 1) * NN + c] = v[1];
        }
    }
    __syncthreads();
    float2* Z = fft_block<NN, false>(ca, cb, tw, 1, NN);
    // Split the packed transform: X_q = (Z_q + conj Z_{n-q})/2, Y_q = (Z_q - conj Z_{n-q})/(2i)
    for (int q = tid; q < Q; q += blockDim.x) {
        const float2 a = Z[q];
        const float2 b = Z[(NN - q) % NN];
        float2 X = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
        float2 Y = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
        spec[r0 * Q + q] = X;
        spec[(r0 + 1) * Q + q] = Y;
    }
    // Flip the w/lambda buffer parity once every block has read it.
    if (tid == 0) {
        if (last_block_arrive(&ctrl->ticket_w)) ctrl->wpar = par ^ 1;
    }
}

// ---------------------------------------------------------------------------
// Column pass: CB columns of the half spectrum per block.
// ---------------------------------------------------------------------------
template <int NN, int CB>
__global__ void __launch_bounds__(128) k_fft_cols(float2* __restrict__ spec,
                                                  const float2* __restrict__ tw_g,
                                                  const float* __restrict__ s2_g, float beta,
                                                  float mu_over_tau, const Ctrl* __restrict__ ctrl,
                                                  int mode)
{
    constexpr int Q = NN / 2 + 1;
    __shared__ float2 a[CB * NN], b[CB * NN];
    __shared__ float2 tw[NN];
    __shared__ float s2[NN];
    if (mode == MODE_ITER && ctrl->skip) return;
    const int tid = threadIdx.x;
    const int q0 = blockIdx.x * CB;
    for (int i = tid; i < NN; i += blockDim.x) {
        tw[i] = tw_g[i];
        s2[i] = s2_g[i];
    }
    for (int i = tid; i < CB * NN; i += blockDim.x) {
        const int f = i % CB, p = i / CB;
        const int q = q0 + f;
        a[f * NN + p] = (q < Q) ? spec[p * Q + q] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* X = fft_block<NN, false>(a, b, tw, CB, NN);
    float2* other = (X == a) ? b : a;
    // divide by the eigenvalues of beta D^T D + (mu/tau) I (eq. (eqnorm11) times beta)
    for (int i = tid; i < CB * NN; i += blockDim.x) {
        const int f = i / NN, p = i - f * NN;
        const int q = min(q0 + f, Q - 1);
        const float d = beta * (s2[p] + s2[q]) + mu_over_tau;
        float2 v = X[i];
        v.x = v.x / d;
        v.y = v.y / d;
        X[i] = v;
    }
    __syncthreads();
    float2* Y = fft_block<NN, true>(X, other, tw, CB, NN);
    for (int i = tid; i < CB * NN; i += blockDim.x) {
        const int f = i % CB, p = i / CB;
        const int q = q0 + f;
        if (q < Q) spec[p * Q + q] = Y[f * NN + p];
    }
}

// ---------------------------------------------------------------------------
// Inverse row pass for rows (r0, r0+1), writes u^{k+1} and the stop norms.
// ---------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(128) k_fft_rows_inv(const float2* __restrict__ spec,
                                                      const float2* __restrict__ tw_g,
                                                      float* __restrict__ u,
                                                      double* __restrict__ part,
                                                      Ctrl* __restrict__ ctrl, int mode)
{
    constexpr int Q = NN / 2 + 1;
    __shared__ float2 a[NN], b[NN];
    __shared__ float2 tw[NN];
    __shared__ double red[32];
    if (mode == MODE_ITER && ctrl->skip) return;
    const int tid = threadIdx.x;
    const int r0 = 2 * blockIdx.x;
    for (int i = tid; i < NN; i += blockDim.x) tw[i] = tw_g[i];
    // Z = X + iY on the full circle from the two half spectra (Hermitian symmetry).
    for (int q = tid; q < NN; q += blockDim.x) {
        const bool lo = q < Q;
        const int qq = lo ? q : NN - q;
        float2 X = spec[r0 * Q + qq];
        float2 Y = spec[(r0 + 1) * Q + qq];
        if (qq == 0 || 2 * qq == NN) {  // exactly real bins
            X.y = 0.f;
            Y.y = 0.f;
        }
        if (!lo) {
            X.y = -X.y;
            Y.y = -Y.y;
        }
        a[q] = make_float2(X.x - Y.y, X.y + Y.x);
    }
    __syncthreads();
    float2* z = fft_block<NN, true>(a, b, tw, 1, NN);
    const float sc = 1.0f / (float)(NN * NN);
    double du2 = 0.0, u2 = 0.0;
    for (int c = tid; c < NN; c += blockDim.x) {
        const float2 v = z[c];
        const float d0 = v.x * sc, d1 = v.y * sc;   // the increment u^{k+1} - u^k
        const int i0 = r0 * NN + c, i1 = (r0 + 1) * NN + c;
        const float o0 = u[i0], o1 = u[i1];
        const float n0 = o0 + d0, n1 = o1 + d1;
        const double e0 = (double)n0 - (double)o0, e1 = (double)n1 - (double)o1;
        du2 += e0 * e0 + e1 * e1;
        u2 += (double)o0 * o0 + (double)o1 * o1;
        u[i0] = n0;
        u[i1] = n1;
    }
    const double s_du = block_sum(du2, red);
    const double s_u = block_sum(u2, red);
    if (tid == 0) {
        part[2 * blockIdx.x] = s_du;
        part[2 * blockIdx.x + 1] = s_u;
    }
    __shared__ int is_last;
    if (!last_block_all(&ctrl->ticket_fft, &is_last)) return;
    const double tdu = block_sum_array(part, gridDim.x, 2, red);
    const double tu = block_sum_array(part + 1, gridDim.x, 2, red);
    if (tid == 0) {
        {
            ctrl->du2 = tdu;
            ctrl->u2 = tu;
            ctrl->relchg = tu > 0.0 ? sqrt(tdu / tu) : (tdu > 0.0 ? INFINITY : 0.0);
            if (mode == MODE_ITER) {
                const int it = ctrl->it + 1;
                ctrl->it = it;
                bool stop = false;
                if (!isfinite(tdu) || !isfinite(tu)) {
                    set_error(ctrl, ERR_NONFINITE);
                    stop = true;
                }
                // eq. (stop), reading C5
                const double tol = ctrl->tol;
                if (tol > 0.0 && (tu > 0.0 ? tdu <= tol * tol * tu : tdu == 0.0)) {
                    ctrl->stop_by_tol = 1;
                    stop = true;
                }
                if (it >= ctrl->max_iter || ctrl->error != ERR_NONE) stop = true;
                if (stop) ctrl->done = 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// End of a run: apply the pending multiplier update in place, gather g,
// binary64 sums of TV and ||w - D u||^2.
// ---------------------------------------------------------------------------
template <int NN>
__global__ void __launch_bounds__(256) k_final1(const float* __restrict__ u, float* __restrict__ wbuf,
                                                float* __restrict__ lbuf, float beta,
                                                double* __restrict__ part, Ctrl* __restrict__ ctrl)
{
    constexpr int N = NN * NN;
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int par = ctrl->wpar;
    const int pending = ctrl->pending;
    float* w = wbuf + (size_t)par * 2 * N;
    float* lam = lbuf + (size_t)par * 2 * N;
    double tv = 0.0, kp = 0.0;
    if (i < N) {
        const int r = i / NN, c = i - r * NN;
        const float uc = u[i];
        const float d1 = u[r * NN + (c + 1) % NN] - uc;
        const float d2 = u[((r + 1) % NN) * NN + c] - uc;
        const float w1 = w[i], w2 = w[N + i];
        if (pending) {
            lam[i] -= beta * (w1 - d1);
            lam[N + i] -= beta * (w2 - d2);
        }
        tv = sqrt((double)d1 * d1 + (double)d2 * d2);
        const double e1 = (double)w1 - d1, e2 = (double)w2 - d2;
        kp = e1 * e1 + e2 * e2;
    }
    const double stv = block_sum(tv, red);
    const double skp = block_sum(kp, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = stv;
        part[2 * blockIdx.x + 1] = skp;
    }
    __shared__ int is_last;
    if (!last_block_all(&ctrl->ticket_fin, &is_last)) return;
    const double a = block_sum_array(part, gridDim.x, 2, red);
    const double b = block_sum_array(part + 1, gridDim.x, 2, red);
    if (threadIdx.x == 0) {
        ctrl->tv = a;
        ctrl->kkt_p2 = b;
        ctrl->pending = 0;
    }
}

// ||D^T lambda + mu g||^2 and max_i ||lambda_i|| (optimality system of eq. (eqftvdcs)).
template <int NN>
__global__ void __launch_bounds__(256) k_final2(const float* __restrict__ lbuf,
                                                const float* __restrict__ g, float mu,
                                                double* __restrict__ part, Ctrl* __restrict__ ctrl)
{
    constexpr int N = NN * NN;
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float* lam = lbuf + (size_t)ctrl->wpar * 2 * N;
    double kd = 0.0, lm = 0.0;
    if (i < N) {
        const int r = i / NN, c = i - r * NN;
        const int cm = (c + NN - 1) % NN, rm = (r + NN - 1) % NN;
        const double dty = (double)lam[r * NN + cm] - lam[i] + (double)lam[N + rm * NN + c] - lam[N + i];
        const double e = dty + (double)mu * g[i];
        kd = e * e;
        lm = sqrt((double)lam[i] * lam[i] + (double)lam[N + i] * lam[N + i]);
    }
    const double skd = block_sum(kd, red);
    const double slm = block_max(lm, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = skd;
        part[2 * blockIdx.x + 1] = slm;
    }
    __shared__ int is_last;
    if (!last_block_all(&ctrl->ticket_fin, &is_last)) return;
    const double a = block_sum_array(part, gridDim.x, 2, red);
    const double b = block_max_array(part + 1, gridDim.x, 2, red);
    if (threadIdx.x == 0) {
        ctrl->kkt_d2 = a;
        ctrl->lam_max = b;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <int NN>
static void launch_tv_set(const TvArgs& a, int which, cudaStream_t s)
{
    constexpr int N = NN * NN;
    constexpr int CB = 2;
    constexpr int Q = NN / 2 + 1;
    switch (which) {
        case 1:
            k_wstep_rowfft<NN><<<NN / 2, 256, 0, s>>>(a.u, a.w, a.lam, a.g,
                                                      a.rhs_out, a.spec, a.tw, a.beta,
                                                      a.mu_over_tau, a.mu, a.ctrl, a.mode);
            break;
        case 2:
            k_fft_cols<NN, CB><<<(Q + CB - 1) / CB, 128, 0, s>>>(a.spec, a.tw, a.s2, a.beta,
                                                                a.mu_over_tau, a.ctrl, a.mode);
            break;
        case 3:
            k_fft_rows_inv<NN><<<NN / 2, 128, 0, s>>>(a.spec, a.tw, a.u, a.part, a.ctrl, a.mode);
            break;
        case 4:
            k_final1<NN><<<(N + 255) / 256, 256, 0, s>>>(a.u, a.w, a.lam, a.beta, a.part, a.ctrl);
            break;
        case 5:
            k_final2<NN><<<(N + 255) / 256, 256, 0, s>>>(a.lam, a.g, a.mu, a.part, a.ctrl);
            break;
        default:
            break;
    }
}

bool tv_supported(int n)
{
    switch (n) {
        case 16: case 32: case 48: case 64: case 96: case 128: case 192: case 256:
            return true;
        default:
            return false;
    }
}

void launch_tv(int n, const TvArgs& a, int which, cudaStream_t s)
{
    switch (n) {
        case 16: launch_tv_set<16>(a, which, s); break;
        case 32: launch_tv_set<32>(a, which, s); break;
        case 48: launch_tv_set<48>(a, which, s); break;
        case 64: launch_tv_set<64>(a, which, s); break;
        case 96: launch_tv_set<96>(a, which, s); break;
        case 128: launch_tv_set<128>(a, which, s); break;
        case 192: launch_tv_set<192>(a, which, s); break;
        case 256: launch_tv_set<256>(a, which, s); break;
        default: break;
    }
}

}  // namespace tvcs
