// Products with the partial-DCT encoder (Sec. 3.2; reading C18): A is a set of
// m rows of the orthonormal 2D DCT-II, A u = (C U C^T)[rows], C[k][j] =
// a_k cos(pi (2j+1) k / (2n)).  Then
//   r = A u - f,  g = A^T r = C^T S C,  S zero except S[rows_i] = r_i,
// with no matrix of size m x n^2 anywhere: four dense n x n transforms of the
// image (the two matrix-vector products of eq. (line) for this encoder).
//
// One thread-block cluster of CL blocks; block q owns image rows (and
// coefficient rows) [q R, (q+1) R), R = n / CL.  Per block:
//   1  Y = U C^T for its rows of u                       (row transform)
//   2  Z = C Y_all for its coefficient rows, Y_all gathered from the cluster
//   3  r_i = Z[rows_i] - f_i for its sampled coefficients, S = scatter(r)
//   4  T = C^T S_all for its image rows, S_all gathered    (column transform back)
//   5  G = T C for its rows                                (row transform back)
// C lives in shared memory once per block with rows padded to n + 4 floats, so
// that a warp reading a column of C four entries at a time (phase 1) and a
// warp reading a row (phases 2-5) both hit distinct banks.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace tvcs {

namespace {

constexpr int DCT_THREADS = 256;

template <int NN, int CL>
struct DctShape {
    static constexpr int R = NN / CL;
    static constexpr int LD = NN + 4;              // padded row stride of C
    static constexpr size_t O_C = 0;               // NN x LD
    static constexpr size_t O_ALL = O_C + (size_t)NN * LD * 4;    // NN x NN gathered rows
    static constexpr size_t O_U = O_ALL + (size_t)NN * NN * 4;    // R x NN each below
    static constexpr size_t O_Y = O_U + (size_t)R * NN * 4;       // cluster-visible
    static constexpr size_t O_S = O_Y + (size_t)R * NN * 4;       // cluster-visible
    static constexpr size_t O_T = O_S + (size_t)R * NN * 4;
    static constexpr size_t O_RED = O_T + (size_t)R * NN * 4;     // doubles
    static constexpr size_t SMEM = O_RED + (32 + 2 * 16) * 8;
    static_assert(NN % CL == 0 && NN % 4 == 0, "whole rows per block, float4 rows");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// out[i][c] = sum_j left(i, j) right[j][c], i < R, c < NN; right rows at stride NN
// (float4), left(i, j) a warp-uniform scalar per (i, j).  Each thread: one row i,
// four columns.
template <int NN, int R, typename Left>
__device__ __forceinline__ void left_times_right(Left left, const float* right, float* out, int tid,
                                                 int nthr)
{
    constexpr int C4 = NN / 4;
    for (int o = tid; o < R * C4; o += nthr) {
        const int i = o / C4, c4 = o - i * C4;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4* rb = reinterpret_cast<const float4*>(right) + c4;
#pragma unroll 4
        for (int j = 0; j < NN; ++j) {
            const float a = left(i, j);
            const float4 b = rb[(size_t)j * C4];
            acc.x = fmaf(a, b.x, acc.x);
            acc.y = fmaf(a, b.y, acc.y);
            acc.z = fmaf(a, b.z, acc.z);
            acc.w = fmaf(a, b.w, acc.w);
        }
        reinterpret_cast<float4*>(out)[o] = acc;
    }
}

}  // namespace

template <int NN, int CL>
__global__ void __launch_bounds__(DCT_THREADS, 1)
k_dct_products(const float* __restrict__ Cg, const float* __restrict__ x,
               const float* __restrict__ y, const int* __restrict__ sidx,
               const int* __restrict__ sperm, const int* __restrict__ rowptr,
               float* __restrict__ r, float* __restrict__ g, Ctrl* __restrict__ ctrl, int mode,
               cudaGraphConditionalHandle cond, int set_cond)
{
    using S = DctShape<NN, CL>;
    constexpr int R = S::R, LD = S::LD;
    extern __shared__ __align__(16) unsigned char smem[];
    float* sC = reinterpret_cast<float*>(smem + S::O_C);
    float* sAll = reinterpret_cast<float*>(smem + S::O_ALL);
    float* sU = reinterpret_cast<float*>(smem + S::O_U);
    float* sY = reinterpret_cast<float*>(smem + S::O_Y);
    float* sS = reinterpret_cast<float*>(smem + S::O_S);
    float* sT = reinterpret_cast<float*>(smem + S::O_T);
    double* red = reinterpret_cast<double*>(smem + S::O_RED);   // [32]
    double* cred = red + 32;                                    // [CL] cluster partials

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int r0 = rank * R;

    pdl_wait();
    if (mode == MODE_ITER) {
        const int skip = ctrl->skip;
        // the next u-solve writes skip before its own wait: release it only now
        pdl_release();
        if (rank == 0 && tid == 0) {
            if (!skip && ctrl->algo == 0) ctrl->pending = 1;
            if (set_cond) {
                const int lc = ++ctrl->loops;
                const int cont =
                    (!ctrl->done && ctrl->error == ERR_NONE && lc < ctrl->loops_max) ? 1 : 0;
                cudaGraphSetConditional(cond, (unsigned)cont);
            }
        }
        if (skip) return;   // uniform across the cluster
    } else {
        pdl_release();
    }

    // C (padded rows) and this block's rows of u
    constexpr int CPR = NN / 4;
    for (int i = tid; i < NN * CPR; i += nthr) {
        const int k = i / CPR, c4 = i - k * CPR;
        cp_async16(sC + k * LD + 4 * c4, Cg + (size_t)k * NN + 4 * c4);
    }
    for (int i = tid; i < R * CPR; i += nthr) cp_async16(sU + 4 * i, x + (size_t)r0 * NN + 4 * i);
    cp_async_wait_all();
    __syncthreads();

    // 1: Y[i][k] = sum_c U[i][c] C[k][c]; each thread one k, several rows, C read
    //    down a column four entries at a time
    for (int o = tid; o < R * NN; o += nthr) {
        const int i = o / NN, k = o - i * NN;
        const float4* cr = reinterpret_cast<const float4*>(sC + k * LD);
        const float4* ur = reinterpret_cast<const float4*>(sU + i * NN);
        float acc = 0.f;
#pragma unroll 4
        for (int c4 = 0; c4 < CPR; ++c4) {
            const float4 a = ur[c4], b = cr[c4];
            acc = fmaf(a.x, b.x, acc);
            acc = fmaf(a.y, b.y, acc);
            acc = fmaf(a.z, b.z, acc);
            acc = fmaf(a.w, b.w, acc);
        }
        sY[o] = acc;
    }
    cluster.sync();   // every block's rows of Y are complete

    // 2: Z = C Y_all for coefficient rows r0 .. r0+R-1
    for (int i = tid; i < NN * CPR; i += nthr) {
        const int row = i / CPR, c4 = i - row * CPR;
        const float4* src = reinterpret_cast<const float4*>(cluster.map_shared_rank(sY, row / R));
        reinterpret_cast<float4*>(sAll)[i] = src[(row % R) * CPR + c4];
    }
    __syncthreads();
    left_times_right<NN, R>([&](int i, int j) { return sC[(r0 + i) * LD + j]; }, sAll, sT, tid,
                            nthr);   // sT holds Z for now
    __syncthreads();

    // 3: residuals of this block's sampled coefficients, S = scatter(r)
    for (int i = tid; i < R * NN; i += nthr) sS[i] = 0.f;
    __syncthreads();
    double r2 = 0.0;
    const int e0 = rowptr[r0], e1 = rowptr[r0 + R];
    for (int e = e0 + tid; e < e1; e += nthr) {
        const int idx = sidx[e] - r0 * NN;   // local position in the block's rows
        const int q = sperm[e];              // caller's order of the measurement
        const float rv = y ? sT[idx] - y[q] : sT[idx];
        r[q] = rv;
        sS[idx] = rv;
        r2 += (double)rv * (double)rv;
    }
    const double br2 = block_sum(r2, red);
    if (tid == 0) {
        double* dst = cluster.map_shared_rank(cred, 0);
        dst[rank] = br2;
    }
    cluster.sync();   // every block's rows of S (and its ||r||^2 partial) are complete

    // 4: T = C^T S_all for image rows r0 .. r0+R-1
    for (int i = tid; i < NN * CPR; i += nthr) {
        const int row = i / CPR, c4 = i - row * CPR;
        const float4* src = reinterpret_cast<const float4*>(cluster.map_shared_rank(sS, row / R));
        reinterpret_cast<float4*>(sAll)[i] = src[(row % R) * CPR + c4];
    }
    __syncthreads();
    left_times_right<NN, R>([&](int i, int j) { return sC[j * LD + r0 + i]; }, sAll, sT, tid, nthr);
    __syncthreads();

    // 5: G = T C for image rows r0 .. r0+R-1 (C's rows read at the padded stride)
    {
        constexpr int C4 = NN / 4;
        for (int o = tid; o < R * C4; o += nthr) {
            const int i = o / C4, c4 = o - i * C4;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int j = 0; j < NN; ++j) {
                const float a = sT[i * NN + j];
                const float4 b = reinterpret_cast<const float4*>(sC + j * LD)[c4];
                acc.x = fmaf(a, b.x, acc.x);
                acc.y = fmaf(a, b.y, acc.y);
                acc.z = fmaf(a, b.z, acc.z);
                acc.w = fmaf(a, b.w, acc.w);
            }
            reinterpret_cast<float4*>(g + (size_t)r0 * NN)[o] = acc;
        }
    }
    if (rank == 0 && tid == 0) {
        double t = 0.0;
        for (int k = 0; k < CL; ++k) t += cred[k];
        ctrl->r2 = t;
    }
    cluster.sync();   // the peers' gathers from this block's shared memory are done
}

// ---------------------------------------------------------------------------
// Host side.  Cluster of 16 blocks (8 for n = 16).
// ---------------------------------------------------------------------------
#define TVCS_DCT_TABLE(X) X(16, 8) X(32, 16) X(48, 16) X(64, 16) X(96, 16) X(128, 16)

template <int NN, int CL>
static bool dct_configure_t()
{
    using S = DctShape<NN, CL>;
    if (cudaFuncSetAttribute(k_dct_products<NN, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::SMEM) != cudaSuccess ||
        (CL > 8 && cudaFuncSetAttribute(k_dct_products<NN, CL>,
                                        cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    return true;
}

bool dct_supported(int n)
{
#define X(NN, CL) \
    if (n == NN) return true;
    TVCS_DCT_TABLE(X)
#undef X
    return false;
}

bool dct_configure(int n)
{
#define X(NN, CL) \
    if (n == NN) return dct_configure_t<NN, CL>();
    TVCS_DCT_TABLE(X)
#undef X
    return false;
}

template <int NN, int CL>
static void launch_dct_t(const DctArgs& a, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(DCT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = DctShape<NN, CL>::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_dct_products<NN, CL>, a.C, a.x, a.y, a.sidx, a.sperm, a.rowptr, a.r,
                       a.g, a.ctrl, a.mode, (cudaGraphConditionalHandle)a.cond, a.set_cond);
}

void launch_dct_products(int n, const DctArgs& a, cudaStream_t s)
{
#define X(NN, CL)                     \
    if (n == NN) {                    \
        launch_dct_t<NN, CL>(a, s);   \
        return;                       \
    }
    TVCS_DCT_TABLE(X)
#undef X
}

}  // namespace tvcs
