// End-of-run kernels of the TV/L2 solver: the pending multiplier update of
// eq. (udlamb), the objective of eq. (tv) and the residuals of the optimality
// system of eq. (eqftvdcs) (Thm 4): ||w - D u||, ||D^T lambda + mu A^T (A u - f)||
// and max_i ||lambda_i||, all reduced in binary64.  (The per-iteration rows
// a1-a5 live in k_usolve.cu, rows a6-a7 in k_products.cu.)
//
// Layout: u, g are n x n row-major binary32; w and lambda are two planes each
// (D1 component, then D2 component), double-buffered, ctrl->wpar selecting
// the current copy.
#include "common.cuh"
#include "kernels.h"

namespace tvcs {

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
    {   // image blockIdx.y of a batch
        const int b = blockIdx.y;
        u += (size_t)b * N;
        wbuf += (size_t)b * 4 * N;
        lbuf += (size_t)b * 4 * N;
        part += (size_t)b * 2 * gridDim.x;
        ctrl += b;
    }
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
                                                double* __restrict__ part, Ctrl* __restrict__ ctrl,
                                                const float* __restrict__ mu_img)
{
    constexpr int N = NN * NN;
    __shared__ double red[32];
    {   // image blockIdx.y of a batch
        const int b = blockIdx.y;
        lbuf += (size_t)b * 4 * N;
        g += (size_t)b * N;
        part += (size_t)b * 2 * gridDim.x;
        ctrl += b;
        if (mu_img) mu = mu_img[b];
    }
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
    const dim3 grid((N + 255) / 256, a.nimg > 0 ? a.nimg : 1);
    if (which == 4)
        k_final1<NN><<<grid, 256, 0, s>>>(a.u, a.w, a.lam, a.beta, a.part, a.ctrl);
    else if (which == 5)
        k_final2<NN><<<grid, 256, 0, s>>>(a.lam, a.g, a.mu, a.part, a.ctrl, a.mu_img);
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
