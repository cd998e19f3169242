// Rows a1-a5 of one IADM/FTVCS iteration in ONE thread-block-cluster kernel
// (Xiao & Yang, Sec. 2.1-2.2):
//   a1  multiplier update lambda <- lambda - beta (w - D u)   (eq. (udlamb), deferred
//       from the previous iteration)
//   a2  w <- shrink(D u + lambda/beta, 1/beta)                 (eq. (iadmw), reading C1)
//   a3  right-hand side of the u-step in increment form
//   a4  FFT solve (beta D^T D + mu/tau I) d = rhs, u^{k+1} = u^k + d  (eq. (eqnorm11) x beta)
//   a5  binary64 norms of eq. (stop) and the stop decision
//
// A cluster of C blocks covers the n x n image; block k owns rows
// [k R, (k+1) R), R = n / C.  Phase A: w-step and right-hand side of the
// owned rows (plus one recomputed halo row), forward row FFTs (two real rows
// packed per complex transform), half spectrum kept in this block's shared
// memory.  Phase B: the n/2+1 spectrum columns are split over the blocks; the
// split at the end of phase A already stores each value into the shared memory
// of its column's block (remote stores, which do not stall the issuing
// thread), which transforms along the columns, divides by beta Lambda_pq +
// mu/tau, transforms back and scatters the columns home.  Phase C: inverse row FFTs,
// u update and norms.  Cluster barriers separate the phases, so the whole
// u-solve is one launch and the spectrum never leaves the chip.
//
// The solve is for the increment d = u^{k+1} - u^k:
//   (beta D^T D + (mu/tau) I) d = D^T (beta (w^{k+1} - D u^k) - lambda^k) - mu g^k,
// equal to eq. (eqnorm11) times beta in exact arithmetic; the large (mu/tau) u^k
// term cancels analytically, so binary32 round-off scales with the step.
#include <cooperative_groups.h>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"
#include "usolve_steps.cuh"

namespace cg = cooperative_groups;

namespace tvcs {

constexpr int US_THREADS = 256;

template <int NN, int C>
struct UsolveShape {
    static constexpr int R = NN / C;            // rows per block
    static constexpr int Q = NN / 2 + 1;        // half-spectrum columns
    // Phase B works on n/2 column slots: slot 0 carries the two real columns
    // q = 0 and q = n/2 as one complex column, slot q the column q (1 <= q < n/2).
    static constexpr int QC = (NN / 2) / C;     // column slots per block in phase B
    static constexpr int ROWFFT = (R / 2) * NN; // complex elements of the packed row transforms
    static constexpr int COLFFT = QC * NN;
    static constexpr int WORK = ROWFFT > COLFFT ? ROWFFT : COLFFT;
    // shared memory carve-up (bytes, each region 16-byte aligned)
    static constexpr size_t O_TW = 0;
    static constexpr size_t O_S2 = O_TW + NN * 8;
    static constexpr size_t O_U = O_S2 + ((NN * 4 + 15) / 16) * 16;
    static constexpr size_t O_G = O_U + (R + 2) * NN * 4;
    static constexpr size_t O_Y1 = O_G + R * NN * 4;
    static constexpr size_t O_Y2 = O_Y1 + R * NN * 4;
    static constexpr size_t O_SPEC = O_Y2 + (R + 1) * NN * 4;
    static constexpr size_t O_WA = O_SPEC + ((R * Q * 8 + 15) / 16) * 16;
    static constexpr size_t O_WB = O_WA + WORK * 8;
    static constexpr size_t O_WL = O_WB + WORK * 8;            // w1, w2, l1, l2 of rows r0-1 .. r0+R-1
    static constexpr size_t O_COL = O_WL + 4 * (R + 1) * NN * 4;   // QC columns, cluster-written
    // reciprocal divisors of this block's column slots (and of column n/2 for slot 0)
    static constexpr size_t O_RDIV = O_COL + (size_t)COLFFT * 8;
    static constexpr size_t O_RED = O_RDIV + (size_t)(QC + 1) * NN * 4;
    static constexpr size_t SMEM = O_RED + (64 + 2 * 16) * 8;
    static_assert(NN % C == 0 && R % 2 == 0, "each block owns an even number of rows");
    static_assert((NN / 2) % C == 0, "whole column slots per block");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Batches: image b = blockIdx.y uses u + b N, w/lambda + 4 b N, g + b N, its own
// control block ctrl + b and, when mu_img is set, mu = mu_img[b] (and tau =
// tau_img[b] when that is set too).  When u_hi is
// set, the new u is also written as bfloat16 hi/lo planes (operand of the
// batched products), at row img_slot[b] when img_slot is set (a compacted
// batch; -1: the image has stopped and writes no planes), else at row b.
// a4: the half spectra of the owned rows as in step_split (rows r0 + 2j and
// r0 + 2j + 1 from packed transform j), each column q stored into the column
// buffer of the block owning its slot: col[(slot mod QC) NN + row].  Columns
// 0 and n/2 are real along the rows (row transforms of real rows at frequency
// 0 and n/2) and share slot 0, as its real and imaginary parts.
template <int NN, int C>
__device__ __forceinline__ void split_to_columns(cg::cluster_group& cluster, const float2* Z,
                                                 int r0, float2* col, int tid, int nthr)
{
    using S = UsolveShape<NN, C>;
    constexpr int Q = S::Q, QC = S::QC, R = S::R;
    for (int i = tid; i < (R / 2) * Q; i += nthr) {
        const int j = i / Q, q = i - j * Q;
        const float2 a = Z[j * NN + q];
        const float2 b = Z[j * NN + (NN - q) % NN];
        const int slot = (2 * q == NN) ? 0 : q;
        const int owner = slot / QC, f = slot - owner * QC;
        float2* dst = cluster.map_shared_rank(col, owner) + f * NN + r0 + 2 * j;
        if (q == 0 || 2 * q == NN) {   // real values: the x (q = 0) or y (q = n/2) part
            float* d1 = reinterpret_cast<float*>(dst) + (q == 0 ? 0 : 1);
            d1[0] = 0.5f * (a.x + b.x);
            d1[2] = 0.5f * (a.y + b.y);
        } else {
            dst[0] = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            dst[1] = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
        }
    }
}

template <int NN, int C>
__global__ void __launch_bounds__(US_THREADS, 1) k_usolve_cluster(
    float* __restrict__ u, float* __restrict__ wbuf, float* __restrict__ lbuf,
    const float* __restrict__ g, float* __restrict__ rhs_out, const float2* __restrict__ tw_g,
    const float* __restrict__ s2_g, float beta, float mu_over_tau, float mu,
    Ctrl* __restrict__ ctrl, int mode, const float* __restrict__ mu_img,
    const float* __restrict__ tau_img, float tau, unsigned short* __restrict__ u_hi,
    unsigned short* __restrict__ u_lo, const int* __restrict__ img_slot)
{
    using S = UsolveShape<NN, C>;
    constexpr int R = S::R, Q = S::Q, QC = S::QC, N = NN * NN;
    {
        const int b = blockIdx.y;
        u += (size_t)b * N;
        wbuf += (size_t)b * 4 * N;
        lbuf += (size_t)b * 4 * N;
        g += (size_t)b * N;
        ctrl += b;
        if (u_hi) {
            const int row = img_slot ? img_slot[b] : b;
            if (row >= 0) {
                u_hi += (size_t)row * N;
                u_lo += (size_t)row * N;
            } else {
                u_hi = u_lo = nullptr;
            }
        }
        if (mu_img) {
            mu = mu_img[b];
            mu_over_tau = mu / (tau_img ? tau_img[b] : tau);
        }
    }
    extern __shared__ __align__(16) unsigned char smem[];
    float2* tw = reinterpret_cast<float2*>(smem + S::O_TW);
    float* s2 = reinterpret_cast<float*>(smem + S::O_S2);
    float* su = reinterpret_cast<float*>(smem + S::O_U);      // rows r0-1 .. r0+R
    float* sg = reinterpret_cast<float*>(smem + S::O_G);      // rows r0 .. r0+R-1
    float* sy1 = reinterpret_cast<float*>(smem + S::O_Y1);    // rows r0 .. r0+R-1
    float* sy2 = reinterpret_cast<float*>(smem + S::O_Y2);    // rows r0-1 .. r0+R-1
    float2* spec = reinterpret_cast<float2*>(smem + S::O_SPEC);  // R x Q, cluster-visible
    float2* wa = reinterpret_cast<float2*>(smem + S::O_WA);
    float2* wb = reinterpret_cast<float2*>(smem + S::O_WB);
    float* swl = reinterpret_cast<float*>(smem + S::O_WL);       // [4][(R+1) NN]
    float2* col = reinterpret_cast<float2*>(smem + S::O_COL);    // [QC][NN], cluster-written
    float* rdiv = reinterpret_cast<float*>(smem + S::O_RDIV);   // [QC + 1][NN]
    float2* red = reinterpret_cast<float2*>(smem + S::O_RED);    // [64] block reduction
    float2* cred = red + 64;                                     // [C][2] cluster partials

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int r0 = rank * R;
    // u, w, lambda, wpar and done were written by the previous u-solve, which
    // completed before the preceding product kernel passed its dependency wait;
    // only g and the products' control fields need this kernel's own wait.
    if (mode == MODE_ITER) {
        const int done = ctrl->done;   // stable during this kernel
        if (rank == 0 && tid == 0) ctrl->skip = done;
        if (done) {                    // uniform across the cluster: before any cluster barrier
            pdl_wait_then_release();   // completes only after the preceding grid
            return;
        }
    }
    // every block of the cluster has started before any distributed shared
    // memory access (the wait sits just before the first one, the column split)
    cluster_arrive();
    const int par = ctrl->wpar;
    const int pending = ctrl->pending;   // set by the previous u-solve (or the host)
    const float* wsrc = wbuf + (size_t)par * 2 * N;
    const float* lsrc = lbuf + (size_t)par * 2 * N;
    float* wdst = wbuf + (size_t)(par ^ 1) * 2 * N;
    float* ldst = lbuf + (size_t)(par ^ 1) * 2 * N;

    // ---------------- phase A ----------------
    // Inputs by asynchronous 16-byte copies: twiddles, 4 sin^2 table, u rows
    // r0-1 .. r0+R, and w, lambda rows r0-1 .. r0+R-1 before the dependency wait
    // (under a programmatic dependent launch they arrive while the products
    // finish), g rows r0 .. r0+R-1 after it.
    constexpr int CPR = NN / 4;       // 16-byte chunks per row
    constexpr int WL = (R + 1) * NN;
    for (int i = tid; i < NN / 2; i += nthr) cp_async16(tw + 2 * i, tw_g + 2 * i);
    for (int i = tid; i < CPR; i += nthr) cp_async16(s2 + 4 * i, s2_g + 4 * i);
    for (int i = tid; i < (R + 2) * CPR; i += nthr) {
        const int rr = i / CPR, c4 = i - rr * CPR;
        const int row = (r0 - 1 + rr + NN) % NN;
        cp_async16(su + rr * NN + 4 * c4, u + row * NN + 4 * c4);
    }
    for (int i = tid; i < (R + 1) * CPR; i += nthr) {
        const int rr = i / CPR, c4 = i - rr * CPR;
        const int gi = ((r0 - 1 + rr + NN) % NN) * NN + 4 * c4;
        const int li = rr * NN + 4 * c4;
        cp_async16(swl + li, wsrc + gi);
        cp_async16(swl + WL + li, wsrc + N + gi);
        cp_async16(swl + 2 * WL + li, lsrc + gi);
        cp_async16(swl + 3 * WL + li, lsrc + N + gi);
    }
    cp_async_wait_all();
    __syncthreads();
    // a1-a3 up to D^T y need no g: under a programmatic dependent launch they run
    // while the products finish.  So do the reciprocals 1 / (beta Lambda_pq + mu/tau)
    // of this block's column slots, which phase B only multiplies by: rdiv[f n + p]
    // for slot q0 + f (column 0 for slot 0), rdiv[QC n + p] for column n/2.
    {
        const int q0r = rank * QC;
        for (int i = tid; i < (QC + 1) * NN; i += nthr) {
            const int f = i / NN, p = i - f * NN;
            const int q = f < QC ? q0r + f : NN / 2;
            rdiv[i] = 1.0f / solve_divisor(s2, p, q, beta, mu_over_tau);
        }
    }
    step_wshrink<NN>(su, swl, WL, R, r0, beta, pending, sy1, sy2, wdst, ldst, tid, nthr);
    __syncthreads();
    step_dty<NN>(sy1, sy2, R, wa, tid, nthr);
    pdl_wait_then_release();   // g is complete
    for (int i = tid; i < R * CPR; i += nthr) cp_async16(sg + 4 * i, g + r0 * NN + 4 * i);
    cp_async_wait_all();
    __syncthreads();
    step_sub_g<NN>(sg, R, r0, mu, wa, rhs_out, tid, nthr);
    __syncthreads();
    float2* Zr = fft_block<NN, false>(wa, wb, tw, R / 2, NN);
    cluster_wait();
    split_to_columns<NN, C>(cluster, Zr, r0, col, tid, nthr);
    cluster.sync();   // every block's columns are complete

    // ---------------- phase B: columns ----------------
    const int q0 = rank * QC;   // first column slot of this block
    constexpr int ncol = QC;
    float2* X = fft_block<NN, false>(col, wb, tw, ncol, NN);
    float2* other = (X == col) ? wb : col;
    for (int i = tid; i < ncol * NN; i += nthr) {
        const int f = i / NN;
        if (q0 + f == 0) continue;   // slot 0: below
        const float rd = rdiv[i];
        float2 v = X[i];
        v.x *= rd;
        v.y *= rd;
        X[i] = v;
    }
    if (q0 == 0) {
        // Slot 0 holds z = c0 + i cN of the real columns c0 (q = 0) and cN (q = n/2):
        // C0_k = (Z_k + conj Z_{n-k}) / 2, CN_k = (Z_k - conj Z_{n-k}) / (2i), each divided
        // by its own divisor (symmetric in k), recombined as Z_k = C0_k + i CN_k (and
        // Z_{n-k} = conj C0_k + i conj CN_k), so that the inverse gives c0' + i cN'.
        for (int k = tid; 2 * k <= NN; k += nthr) {
            const int km = (NN - k) % NN;
            const float2 zk = X[k], zm = X[km];
            float2 c0 = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            float2 cn = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            const float r0 = rdiv[k];
            const float rn = rdiv[QC * NN + k];
            c0.x *= r0;
            c0.y *= r0;
            cn.x *= rn;
            cn.y *= rn;
            X[k] = make_float2(c0.x - cn.y, c0.y + cn.x);
            if (km != k) X[km] = make_float2(c0.x + cn.y, cn.x - c0.y);
        }
    }
    __syncthreads();
    float2* Y = fft_block<NN, true>(X, other, tw, ncol, NN);
    for (int i = tid; i < ncol * NN; i += nthr) {
        const int f = i % ncol, p = i / ncol;
        float2* own = cluster.map_shared_rank(spec, p / R) + (p % R) * Q;
        const float2 v = Y[f * NN + p];
        if (q0 + f == 0) {   // back to the real columns 0 and n/2
            own[0] = make_float2(v.x, 0.f);
            own[NN / 2] = make_float2(v.y, 0.f);
        } else {
            own[q0 + f] = v;
        }
    }
    cluster.sync();   // every column is home

    // ---------------- phase C: inverse rows, u update, norms ----------------
    step_pack_inverse<NN>(spec, Q, 1, R, wa, tid, nthr);
    __syncthreads();
    float2* z = fft_block<NN, true>(wa, wb, tw, R / 2, NN);
    // double-single sums of squares (fixed order per thread, warp and block)
    float2 du2 = make_float2(0.f, 0.f), u2 = make_float2(0.f, 0.f);
    step_update<NN>(z, su + NN, R, r0, u, u_hi, u_lo, du2, u2, tid, nthr);
    block_sum_ds2(du2, u2, red);
    if (tid == 0) {
        float2* dst = cluster.map_shared_rank(cred, 0);
        dst[2 * rank] = du2;
        dst[2 * rank + 1] = u2;
    }
    cluster.sync();   // partials delivered to block 0; every block has read wpar and done
    if (rank == 0 && tid == 0) {
        float2 tdu = cred[0], tu = cred[1];
        for (int k = 1; k < C; ++k) {
            tdu = ds_add(tdu, cred[2 * k]);
            tu = ds_add(tu, cred[2 * k + 1]);
        }
        step_stop(ctrl, par, mode, ds_value(tdu), ds_value(tu));
    }
}

// ---------------------------------------------------------------------------
// Host side: cluster size per n (16 where it fits and the device allows it, else 8).
// ---------------------------------------------------------------------------
template <int NN, int C>
static cudaError_t configure_usolve_t()
{
    using S = UsolveShape<NN, C>;
    cudaError_t e = cudaFuncSetAttribute(k_usolve_cluster<NN, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    if (C > 8)
        e = cudaFuncSetAttribute(k_usolve_cluster<NN, C>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int NN, int C>
static bool cluster_fits_t()
{
    using S = UsolveShape<NN, C>;
    if (configure_usolve_t<NN, C>() != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(US_THREADS, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_usolve_cluster<NN, C>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

template <int NN, int C>
static void launch_usolve_t(const TvArgs& a, cudaStream_t s)
{
    using S = UsolveShape<NN, C>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, a.nimg > 0 ? a.nimg : 1, 1);
    cfg.blockDim = dim3(US_THREADS, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k_usolve_cluster<NN, C>, a.u, a.w, a.lam, a.g, a.rhs_out, a.tw, a.s2,
                       a.beta, a.mu_over_tau, a.mu, a.ctrl, a.mode, a.mu_img, a.tau_img,
                       a.tau, a.u_hi, a.u_lo, a.img_slot);
}

// Cluster sizes available per n: {16, 8} where both give an even row count and
// the shared memory fits (n = 192 needs 16).
#define TVCS_USOLVE_TABLE(X) \
    X(16, 8)                 \
    X(32, 16) X(32, 8)       \
    X(48, 8)                 \
    X(64, 16) X(64, 8)       \
    X(96, 16) X(96, 8)       \
    X(128, 16) X(128, 8)     \
    X(192, 16)               \
    X(256, 16)

bool usolve_cluster_fits(int n, int c)
{
#define X(NN, C) \
    if (n == NN && c == C) return cluster_fits_t<NN, C>();
    TVCS_USOLVE_TABLE(X)
#undef X
    return false;
}

int usolve_choose_cluster(int n)
{
#define X(NN, C) \
    if (n == NN && cluster_fits_t<NN, C>()) return C;
    TVCS_USOLVE_TABLE(X)
#undef X
    return 0;
}

void launch_usolve(int n, int cluster, const TvArgs& a, cudaStream_t s)
{
#define X(NN, C)                           \
    if (n == NN && cluster == C) {         \
        launch_usolve_t<NN, C>(a, s);      \
        return;                            \
    }
    TVCS_USOLVE_TABLE(X)
#undef X
}

}  // namespace tvcs
