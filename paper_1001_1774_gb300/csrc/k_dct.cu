// Products with the partial-DCT encoder (Sec. 3.2; reading C18): A is a set of
// m rows of the orthonormal 2D DCT-II, A u = (C U C^T)[rows], C[k][j] =
// a_k cos(pi (2j+1) k / (2n)).  Then
//   r = A u - f,  g = A^T r = C^T S C,  S zero except S[rows_i] = r_i,
// with no matrix of size m x n^2 anywhere: four dense n x n transforms of the
// image (the two matrix-vector products of eq. (line) for this encoder).
//
// One thread-block cluster of CL blocks; block q owns image rows (and
// coefficient rows) [q R, (q+1) R), R = n / CL (a multiple of 4).  Per block:
//   1  Y = U C^T for its rows of u                       (row transform)
//   2  Z = C Y_all for its coefficient rows, Y_all gathered from the cluster
//   3  r_i = Z[rows_i] - f_i for its sampled coefficients, S = scatter(r)
//   4  T = C^T S_all for its image rows, S_all gathered    (column transform back)
//   5  G = T C for its rows                                (row transform back)
// Every transform has the form out[i][c] = sum_j A[j][i] B[j][c] over the
// block's R rows i: A is C, C^T or a transposed band (u, T) and B is C, C^T or
// a gathered n x n matrix, all in shared memory.  A thread accumulates a 4 x 4
// tile over one of KS slices of j (one float4 of A, broadcast across the warp,
// and one of B per 16 FMAs); the KS partial tiles are summed afterwards.  C and
// C^T are constants and are copied in before waiting on the preceding kernel.
// The bands of Y and S are exchanged through global scratch (L2): each block
// stores its band, and after a cluster barrier copies the whole matrix in,
// which moves data faster than loads from the peers' shared memory.
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
    static constexpr int RG = R / 4, CG = NN / 4, TILES = RG * CG;
    static constexpr int KS0 = DCT_THREADS / TILES;
    static constexpr int KS = KS0 < CG ? KS0 : CG;    // slices of the summation index
    static constexpr int JL = (NN + KS - 1) / KS;     // slice length
    static constexpr size_t NSQ = (size_t)NN * NN * 4;
    static constexpr size_t BAND = (size_t)R * NN * 4;
    static constexpr size_t O_C = 0;                  // C, n x n
    static constexpr size_t O_CT = O_C + NSQ;         // C^T, n x n
    static constexpr size_t O_ALL = O_CT + NSQ;       // gathered n x n (Y_all, then S_all)
    static constexpr size_t O_UT = O_ALL + NSQ;       // u band transposed (n x R), later T^T
    static constexpr size_t O_S = O_UT + BAND;        // S band
    static constexpr size_t O_P = O_S + BAND;         // KS partial bands
    static constexpr size_t O_RED = O_P + (size_t)KS * BAND;   // float2
    static constexpr size_t SMEM = O_RED + (32 + 16) * 8;
    static_assert(NN % CL == 0 && R % 4 == 0 && CL <= 16, "whole 4-row groups per block");
    static_assert(KS >= 1 && TILES * KS <= DCT_THREADS, "one tile slice per thread at most");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// P[ks][i][c] = sum over j in slice ks of A[j * lda + i] B[j * NN + c], i < R,
// c < NN; one 4 x 4 tile per thread.
template <int NN, int CL>
__device__ __forceinline__ void tile_partials(const float* A, int lda, const float* B, float* P,
                                              int tid)
{
    using S = DctShape<NN, CL>;
    constexpr int CG = S::CG, RG = S::RG, R = S::R;
    if (tid >= S::TILES * S::KS) return;
    const int cg = tid % CG, rest = tid / CG, rg = rest % RG, ks = rest / RG;
    const int j0 = ks * S::JL, j1 = min(NN, j0 + S::JL);
    const float* ap = A + 4 * rg;
    const float* bp = B + 4 * cg;
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[t][v] = 0.f;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const float4 a = *reinterpret_cast<const float4*>(ap + (size_t)j * lda);
        const float4 b = *reinterpret_cast<const float4*>(bp + (size_t)j * NN);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            acc[t][0] = fmaf(av[t], b.x, acc[t][0]);
            acc[t][1] = fmaf(av[t], b.y, acc[t][1]);
            acc[t][2] = fmaf(av[t], b.z, acc[t][2]);
            acc[t][3] = fmaf(av[t], b.w, acc[t][3]);
        }
    }
    float* pp = P + ((size_t)ks * R + 4 * rg) * NN + 4 * cg;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        *reinterpret_cast<float4*>(pp + (size_t)t * NN) =
            make_float4(acc[t][0], acc[t][1], acc[t][2], acc[t][3]);
}

// Sum of the KS partial bands at float4 position o (row o / (NN/4)).
template <int NN, int CL>
__device__ __forceinline__ float4 partial_sum4(const float* P, int o)
{
    using S = DctShape<NN, CL>;
    float4 t = reinterpret_cast<const float4*>(P)[o];
#pragma unroll
    for (int ks = 1; ks < S::KS; ++ks) {
        const float4 v = reinterpret_cast<const float4*>(P + (size_t)ks * S::R * NN)[o];
        t.x += v.x;
        t.y += v.y;
        t.z += v.z;
        t.w += v.w;
    }
    return t;
}

// dst (n x n, shared memory) = src (n x n, global), asynchronous 16-byte copies
// that bypass L1 (the bands were written by other blocks in this launch).
template <int NN>
__device__ __forceinline__ void copy_matrix_async(const float* src, float* dst, int tid)
{
    for (int i = tid; i < NN * NN / 4; i += DCT_THREADS) cp_async16(dst + 4 * i, src + 4 * i);
}

// dst[c * R + 4 rg + t] = sum over slices of P[ks][4 rg + t][c]: the summed
// band stored transposed (n x R), one column and four rows per thread.
template <int NN, int CL>
__device__ __forceinline__ void partial_sum_transposed(const float* P, float* dst, int tid)
{
    using S = DctShape<NN, CL>;
    constexpr int R = S::R;
    for (int o = tid; o < NN * S::RG; o += DCT_THREADS) {
        const int c = o % NN, rg = o / NN;
        float t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v = P[(size_t)(4 * rg + k) * NN + c];
#pragma unroll
            for (int ks = 1; ks < S::KS; ++ks) v += P[((size_t)ks * R + 4 * rg + k) * NN + c];
            t[k] = v;
        }
        *reinterpret_cast<float4*>(dst + (size_t)c * R + 4 * rg) = make_float4(t[0], t[1], t[2], t[3]);
    }
}

}  // namespace

template <int NN, int CL>
__global__ void __launch_bounds__(DCT_THREADS, 1)
k_dct_products(const float* __restrict__ Cg, const float* __restrict__ x,
               const float* __restrict__ y, const int* __restrict__ sidx,
               const int* __restrict__ sperm, const int* __restrict__ rowptr,
               float* __restrict__ r, float* __restrict__ g, float* __restrict__ scratch,
               Ctrl* __restrict__ ctrl, int mode, cudaGraphConditionalHandle cond, int set_cond)
{
    using S = DctShape<NN, CL>;
    constexpr int R = S::R, C4 = NN / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    float* sC = reinterpret_cast<float*>(smem + S::O_C);
    float* sCt = reinterpret_cast<float*>(smem + S::O_CT);
    float* sAll = reinterpret_cast<float*>(smem + S::O_ALL);
    float* sUt = reinterpret_cast<float*>(smem + S::O_UT);
    float* sS = reinterpret_cast<float*>(smem + S::O_S);
    float* sP = reinterpret_cast<float*>(smem + S::O_P);
    float2* red = reinterpret_cast<float2*>(smem + S::O_RED);   // [32]
    float2* cred = red + 32;                                    // [CL] cluster partials

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    float* Yg = scratch;                    // n x n, bands of Y
    float* Sg = scratch + (size_t)NN * NN;  // n x n, bands of S
    const int tid = threadIdx.x;
    const int r0 = rank * R;

    // C and C^T (2 n^2 floats), the sampled positions of this block's rows and
    // their measurements: constants during a solve, fetched while the preceding
    // kernel finishes
    for (int i = tid; i < 2 * NN * C4; i += DCT_THREADS) cp_async16(sC + 4 * i, Cg + 4 * i);
    constexpr int EMAX = (R * NN + DCT_THREADS - 1) / DCT_THREADS;
    const int e0 = rowptr[r0], e1 = rowptr[r0 + R];
    int eidx[EMAX], eq[EMAX];
    float ey[EMAX];
#pragma unroll
    for (int k = 0; k < EMAX; ++k) {
        const int e = e0 + tid + k * DCT_THREADS;
        eidx[k] = -1;
        if (e < e1) {
            eidx[k] = sidx[e] - r0 * NN;   // local position in the block's rows
            eq[k] = sperm[e];              // caller's order of the measurement
            ey[k] = y ? y[eq[k]] : 0.f;
        }
    }

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
        if (skip) {   // uniform across the cluster; leave no copy in flight
            cp_async_wait_all();
            return;
        }
    } else {
        pdl_release();
    }

    // this block's rows of u, transposed: sUt[c][i] = u[r0 + i][c]
    for (int o = tid; o < NN * S::RG; o += DCT_THREADS) {
        const int c = o % NN, rg = o / NN;
        const float* xr = x + (size_t)(r0 + 4 * rg) * NN + c;
        *reinterpret_cast<float4*>(sUt + (size_t)c * R + 4 * rg) =
            make_float4(xr[0], xr[NN], xr[2 * NN], xr[3 * NN]);
    }
    cp_async_wait_all();
    __syncthreads();

    // 1: Y[i][k] = sum_c U[i][c] C[k][c] = sum_c Ut[c][i] Ct[c][k]
    tile_partials<NN, CL>(sUt, R, sCt, sP, tid);
    __syncthreads();
    for (int o = tid; o < R * C4; o += DCT_THREADS)
        reinterpret_cast<float4*>(Yg + (size_t)r0 * NN)[o] = partial_sum4<NN, CL>(sP, o);
    cluster_arrive();
    for (int i = tid; i < R * NN; i += DCT_THREADS) sS[i] = 0.f;
    cluster_wait();   // every block's rows of Y are in Yg

    // 2: Z[i][c] = sum_k C[r0+i][k] Y[k][c] = sum_k Ct[k][r0+i] Y_all[k][c], left as partials
    copy_matrix_async<NN>(Yg, sAll, tid);
    cp_async_wait_all();
    __syncthreads();
    tile_partials<NN, CL>(sCt + r0, NN, sAll, sP, tid);
    __syncthreads();

    // 3: residuals of this block's sampled coefficients, S = scatter(r)
    float2 r2 = make_float2(0.f, 0.f);   // double-single ||r||^2
#pragma unroll
    for (int k = 0; k < EMAX; ++k) {
        const int idx = eidx[k];
        if (idx >= 0) {
            float z = sP[idx];
#pragma unroll
            for (int ks = 1; ks < S::KS; ++ks) z += sP[(size_t)ks * R * NN + idx];
            const float rv = z - ey[k];
            r[eq[k]] = rv;
            sS[idx] = rv;
            r2 = ds_add(r2, ds_sq(rv));
        }
    }
    __syncthreads();
    for (int o = tid; o < R * C4; o += DCT_THREADS)
        reinterpret_cast<float4*>(Sg + (size_t)r0 * NN)[o] = reinterpret_cast<const float4*>(sS)[o];
    cluster_arrive();
    cluster_wait();   // every block's rows of S are in Sg

    // 4: T[i][c] = sum_k C[k][r0+i] S_all[k][c]; stored transposed into sUt.  The
    // ||r||^2 partial goes to block 0 while the copy of S is in flight.
    copy_matrix_async<NN>(Sg, sAll, tid);
    const float2 br2 = block_sum_ds(r2, red);
    if (tid == 0) {   // read by block 0 after the last barrier
        float2* dst = cluster.map_shared_rank(cred, 0);
        dst[rank] = br2;
    }
    cluster_arrive();   // the partial is written; the matching wait is the last step
    cp_async_wait_all();
    __syncthreads();
    tile_partials<NN, CL>(sC + r0, NN, sAll, sP, tid);
    __syncthreads();
    partial_sum_transposed<NN, CL>(sP, sUt, tid);
    __syncthreads();

    // 5: G[i][c] = sum_j T[i][j] C[j][c] = sum_j Tt[j][i] C[j][c]
    tile_partials<NN, CL>(sUt, R, sC, sP, tid);
    __syncthreads();
    for (int o = tid; o < R * C4; o += DCT_THREADS)
        reinterpret_cast<float4*>(g + (size_t)r0 * NN)[o] = partial_sum4<NN, CL>(sP, o);
    cluster_wait();   // every block's ||r||^2 partial is in block 0
    if (rank == 0 && tid == 0) {
        float2 t = cred[0];
        for (int k = 1; k < CL; ++k) t = ds_add(t, cred[k]);
        ctrl->r2 = ds_value(t);
    }
}

// ---------------------------------------------------------------------------
// Host side.  Clusters of up to 16 blocks with 4 or 8 rows each.
// ---------------------------------------------------------------------------
#define TVCS_DCT_TABLE(X) X(16, 4) X(32, 8) X(48, 12) X(64, 16) X(96, 12) X(128, 16)

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
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(DCT_THREADS, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_dct_products<NN, CL>, &cfg) != cudaSuccess ||
        clusters < 1) {
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
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k_dct_products<NN, CL>, a.C, a.x, a.y, a.sidx, a.sperm, a.rowptr, a.r,
                       a.g, a.scratch, a.ctrl, a.mode, (cudaGraphConditionalHandle)a.cond, a.set_cond);
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
