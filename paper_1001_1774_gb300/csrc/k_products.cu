// Rows a6-a7: r = A x - y and g = A^T r in ONE pass over A (Xiao & Yang,
// eq. (line): g_k = A^T (A u^k - f); two products per iteration, Sec. 3.1).
//
// Each block owns a contiguous range of rows of A (row-major binary32).  Thread
// 0 streams the rows into a 3-stage shared-memory ring with bulk asynchronous
// copies (TMA, non-tensor form, one mbarrier per stage; A is read once per
// call, with an L2 evict-first hint), the first stages before the dependency
// wait on the preceding kernel, together with an L2 prefetch of the next 1 MB
// of the block's rows.  All 512 threads own fixed columns: for each
// row they form the dot product with x (warp shuffles + one named barrier),
// compute r_i = dot - y_i, and fold r_i * A_i into per-thread accumulators of
// A^T r.  Row i's data is used twice from shared memory and read from HBM once,
// so the algorithmic traffic is one pass over A.  Each block writes its partial
// A^T r (N floats); with g_out set, a grid barrier (cooperative launch) follows
// and every block sums its slice of the P partials in a fixed order
// (deterministic), otherwise a later kernel does.
//
// Shapes: 512 threads in RL row lanes of TPR = 512/RL threads; a thread holds V
// float4 columns of x and of the accumulator (N = 4*TPR*V).  RS rows per stage,
// 3 stages: one block per SM, and the grid leaves 16 SMs free for the u-solve.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace tvcs {

constexpr int PROD_CONS = 512;           // 16 warps; thread 0 also issues the TMA copies
constexpr int PROD_THREADS = PROD_CONS;
constexpr int PROD_NST = 3;
// Rows of A prefetched into L2 per block before the dependency wait, beyond the
// ring: 1 MB (16 rows at n = 128; 136 blocks then hold about L2's capacity).
constexpr size_t PROD_PF_BYTES = 1024 * 1024;
// Bulk copies per stage of the ring.
constexpr int PROD_TMA_PIECES = 1;
// Stages ahead of each refill that are also prefetched into L2 while streaming
// (0: only the pre-wait prefetch).
constexpr int PROD_PF_STREAM = 0;

template <int V, int RL, int RS>
struct ProdShape {
    static constexpr int TPR = PROD_CONS / RL;
    static constexpr int WPR = TPR / 32;
    static constexpr int N = 4 * TPR * V;
    static constexpr size_t STAGE_FLOATS = (size_t)RS * N;
    static constexpr int YMAX = 1024;   // rows of y prefetched into shared memory
    static constexpr size_t SMEM = PROD_NST * STAGE_FLOATS * 4 + 2 * PROD_NST * 8 +
                                   2 * RL * WPR * 4 + 32 * 8 + 16 + YMAX * 4;
    static_assert(RS % RL == 0, "rows per stage must be a multiple of the row lanes");
    static_assert(TPR % 32 == 0, "row lanes must be whole warps");
};

// One block of 16 warps per SM (a three-stage ring of rows fills shared memory);
// the grid leaves 16 SMs to the u-solve cluster of the same iteration, which
// runs there while this kernel streams A.
template <int V, int RL, int RS>
__global__ void __maxnreg__(128)
    k_products(const float* __restrict__ A, int m, const float* __restrict__ x,
               const float* __restrict__ y, float* __restrict__ r, float* __restrict__ gpart,
               float* __restrict__ g_out, float2* __restrict__ r2part, Ctrl* __restrict__ ctrl,
               int mode, cudaGraphConditionalHandle cond, int set_cond, long long budget, int pf,
               int bar_extra)
{
    using S = ProdShape<V, RL, RS>;
    constexpr int N = S::N;
    constexpr int TPR = S::TPR;
    constexpr int WPR = S::WPR;
    extern __shared__ __align__(128) unsigned char smem[];
    float* stage = reinterpret_cast<float*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + PROD_NST * S::STAGE_FLOATS * 4);
    uint64_t* empty = full + PROD_NST;
    float* red = reinterpret_cast<float*>(empty + PROD_NST);        // [2][RL][WPR]
    float2* dred = reinterpret_cast<float2*>(red + 2 * RL * WPR);   // [32]
    int* sflag = reinterpret_cast<int*>(dred + 32);                 // [4]
    float* sy = reinterpret_cast<float*>(sflag + 4);                // [YMAX]

    const int tid = threadIdx.x;
    const int G = gridDim.x;
    const int i0 = (int)(((long long)m * blockIdx.x) / G);
    const int i1 = (int)(((long long)m * (blockIdx.x + 1)) / G);
    const int nrows = i1 - i0;
    const int nst = (nrows + RS - 1) / RS;

    if (tid == 0) {
        for (int s = 0; s < PROD_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], PROD_CONS / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // The TMA copies are issued by thread 0.  A does not depend on the preceding
    // kernel: the first PROD_NST stages go out before the dependency wait, so
    // that under a programmatic dependent launch they stream in while the
    // u-solve still runs.
    const uint64_t pol = l2_policy_evict_first();
    auto issue = [&](int s) {
        const int slot = s % PROD_NST;
        const int rows = min(RS, nrows - s * RS);
        const uint32_t bytes = (uint32_t)rows * N * 4u;
        mbar_arrive_expect_tx(&full[slot], bytes);
        tma_load_1d_split(stage + slot * S::STAGE_FLOATS, A + (size_t)(i0 + s * RS) * N, bytes,
                          &full[slot], pol, PROD_TMA_PIECES);
    };
    // The pf stages after the ring are prefetched into L2 before the wait as
    // well (nothing waits for them): while the u-solve still runs, HBM streams
    // more of A than the ring holds, and the ring's later copies find those
    // rows in L2.  (Prefetching further ahead during the stream measured slower.)
    auto prefetch = [&](int s) {
        const int rows = min(RS, nrows - s * RS);
        prefetch_l2_bulk(A + (size_t)(i0 + s * RS) * N, (uint32_t)rows * N * 4u);
    };
    const int pre = min(PROD_NST, nst);
    int issued = 0;   // stages issued (thread 0)
    if (tid == 0) {
        for (; issued < pre; ++issued) issue(issued);
        for (int s = pre; s < min(pre + pf, nst); ++s) prefetch(s);
    }
    pdl_wait();   // x and the control block come from the preceding u-solve
    if (mode == MODE_ITER) {
        const int skip = ctrl->skip;
        // The next u-solve writes skip before its own wait: release it only now.
        pdl_release();
        if (blockIdx.x == 0 && tid == 0) {
            if (!skip && ctrl->algo == 0) ctrl->pending = 1;
            if (set_cond) {
                // The loop ends when the run is done; `loops` bounds it independently.
                const int lc = ++ctrl->loops;
                const int cont =
                    (!ctrl->done && ctrl->error == ERR_NONE && lc < ctrl->loops_max) ? 1 : 0;
                cudaGraphSetConditional(cond, (unsigned)cont);
            }
        }
        if (skip) {   // leave no copy in flight
            if (tid == 0)
                for (int s = 0; s < pre; ++s) mbar_wait(&full[s], 0u, drain_budget(budget));
            return;
        }
    } else {
        pdl_release();
    }

    // ---------------- consumers ----------------
    // y of this block's rows, prefetched so that r_i = dot - y_i waits on no global load.
    const bool y_in_smem = (y != nullptr) && nrows <= S::YMAX;
    if (y_in_smem)
        for (int i = tid; i < nrows; i += PROD_CONS) sy[i] = y[i0 + i];
    const int lane_row = tid / TPR;
    const int ltid = tid - lane_row * TPR;
    const int warp_in_row = ltid >> 5;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float4 xu[V], acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        xu[v] = x4[ltid + v * TPR];
        acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float2 r2 = make_float2(0.f, 0.f);   // double-single ||r||^2 of this thread's rows
    bool ok = true;
    int step = 0;
    for (int s = 0; s < nst; ++s) {
        const int slot = s % PROD_NST;
        if (ok && !mbar_wait(&full[slot], (s / PROD_NST) & 1, budget)) {
            set_error(ctrl, ERR_TIMEOUT);
            ok = false;
        }
        const float* sb = stage + slot * S::STAGE_FLOATS;
        const int rows = min(RS, nrows - s * RS);
#pragma unroll 1
        for (int st = 0; st < RS / RL; ++st, ++step) {
            const int rl = st * RL + lane_row;
            const bool valid = ok && rl < rows;
            const float4* a4 = reinterpret_cast<const float4*>(sb + (size_t)rl * N);
            const int li = s * RS + rl;   // row index within the block
            float yi = 0.f;
            if (valid && y != nullptr && !y_in_smem) yi = y[i0 + li];
            float d = 0.f;
            if (valid) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float4 a = a4[ltid + v * TPR];
                    d = fmaf(a.x, xu[v].x, d);
                    d = fmaf(a.y, xu[v].y, d);
                    d = fmaf(a.z, xu[v].z, d);
                    d = fmaf(a.w, xu[v].w, d);
                }
            }
            d = warp_sum(d);
            float* rb = red + (step & 1) * RL * WPR;
            if ((tid & 31) == 0) rb[lane_row * WPR + warp_in_row] = d;
            named_barrier(1, PROD_CONS);
            if (valid) {
                float dot = 0.f;
#pragma unroll
                for (int w = 0; w < WPR; ++w) dot += rb[lane_row * WPR + w];
                const int gi = i0 + li;
                if (y_in_smem) yi = sy[li];
                const float ri = dot - yi;
                if (ltid == 0) {
                    r[gi] = ri;
                    r2 = ds_add(r2, ds_sq(ri));
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float4 a = a4[ltid + v * TPR];
                    acc[v].x = fmaf(ri, a.x, acc[v].x);
                    acc[v].y = fmaf(ri, a.y, acc[v].y);
                    acc[v].z = fmaf(ri, a.z, acc[v].z);
                    acc[v].w = fmaf(ri, a.w, acc[v].w);
                }
            }
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[slot]);
        // refill this slot with stage s + PROD_NST once every warp is done with it
        if (tid == 0 && s + PROD_NST < nst) {
            if (ok && !mbar_wait(&empty[slot], (s / PROD_NST) & 1, budget)) {
                set_error(ctrl, ERR_TIMEOUT);
                ok = false;
            }
            if (ok) {
                issue(s + PROD_NST);
                ++issued;
                // while streaming, prefetch into L2 the stage PROD_PF_STREAM stages past
                // the one just issued
                if (PROD_PF_STREAM > 0 && s + PROD_NST + PROD_PF_STREAM < nst)
                    prefetch(s + PROD_NST + PROD_PF_STREAM);
            }
        }
    }
    if (tid == 0 && !ok)   // a wait gave up: let the copies still in flight land (bounded)
        for (int s = max(0, issued - PROD_NST); s < issued; ++s)
            mbar_wait(&full[s % PROD_NST], (s / PROD_NST) & 1, drain_budget(budget));

    // ---------------- epilogue: partial A^T r and ||r||^2 ----------------
    named_barrier(1, PROD_CONS);   // every consumer is done with the stage ring
    float4* out4 = reinterpret_cast<float4*>(gpart + (size_t)blockIdx.x * N);
    if constexpr (RL == 1) {
#pragma unroll
        for (int v = 0; v < V; ++v) out4[ltid + v * TPR] = acc[v];
    } else {
        float4* scr = reinterpret_cast<float4*>(stage);   // (RL-1) x N/4 float4
        if (lane_row > 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) scr[(lane_row - 1) * (N / 4) + ltid + v * TPR] = acc[v];
        }
        named_barrier(1, PROD_CONS);
        if (lane_row == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float4 t = acc[v];
                for (int l = 1; l < RL; ++l) {
                    const float4 o = scr[(l - 1) * (N / 4) + ltid + v * TPR];
                    t.x += o.x; t.y += o.y; t.z += o.z; t.w += o.w;
                }
                out4[ltid + v * TPR] = t;
            }
        }
    }
    // ||r||^2: one double-single value per row lane (held by ltid == 0)
    if (ltid == 0) dred[lane_row] = r2;
    named_barrier(1, PROD_CONS);
    if (tid == 0) {
        float2 s = dred[0];
        for (int l = 1; l < RL; ++l) s = ds_add(s, dred[l]);
        r2part[blockIdx.x] = s;
        // without the grid barrier below, the last block to arrive sums the partials
        sflag[0] = (g_out == nullptr && last_block_arrive(&ctrl->ticket_prod)) ? 1 : 0;
    }
    named_barrier(1, PROD_CONS);
    // ||r||^2 = sum of the G partials with all consumer warps (G <= 512), fixed order
    auto sum_r2 = [&]() {
        float2 v = tid < G ? __ldcg(r2part + tid) : make_float2(0.f, 0.f);
        v = warp_sum_ds(v);
        if ((tid & 31) == 0) dred[tid >> 5] = v;
        named_barrier(1, PROD_CONS);
        if (tid == 0) {
            float2 t = dred[0];
            for (int w = 1; w < PROD_CONS / 32; ++w) t = ds_add(t, dred[w]);
            ctrl->r2 = ds_value(t);
        }
    };
    if (sflag[0]) sum_r2();
    if (g_out == nullptr) return;

    // ---------------- grid barrier, then g = sum of the G partials ----------------
    // All G blocks are co-resident (cooperative launch, one block per SM), so
    // a bounded spin on a monotone arrival counter is a grid barrier.
    named_barrier(1, PROD_CONS);
    if (tid == 0) {
        __threadfence();
        const unsigned long long t = atomicAdd(&ctrl->gbar, 1ull);
        // bar_extra (0 outside the timeout test) raises the target beyond what the
        // grid's arrivals reach, so that only this bounded spin runs out
        const unsigned long long target =
            (t / (unsigned long long)G + 1ull) * (unsigned long long)G + (unsigned)bar_extra;
        const long long t0 = clock64();
        while (ld_acquire_u64(&ctrl->gbar) < target) {
            if (clock64() - t0 > budget) {
                set_error(ctrl, ERR_TIMEOUT);
                break;
            }
        }
        __threadfence();
    }
    named_barrier(1, PROD_CONS);
    if (blockIdx.x == 0) sum_r2();   // every block's partial is visible after the barrier
    // This block's slice of float4 columns; warp w sums partials w, w+16, ... and
    // warp 0 adds the 16 warp sums in order (deterministic).
    const int N4 = N / 4;
    const int c0 = (int)(((long long)N4 * blockIdx.x) / G);
    const int c1 = (int)(((long long)N4 * (blockIdx.x + 1)) / G);
    const float4* gp4 = reinterpret_cast<const float4*>(gpart);
    float4* sred = reinterpret_cast<float4*>(stage);   // [16][32], the stage ring is free
    float4* g4 = reinterpret_cast<float4*>(g_out);
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NWC = PROD_CONS / 32;   // consumer warps
    constexpr int BATCH = 10;             // partials in flight per thread (G <= 160: one round)
    for (int base = c0; base < c1; base += 32) {
        const int c = base + lane;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < c1) {
            for (int p0 = warp; p0 < G; p0 += NWC * BATCH) {
                float4 v[BATCH];
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {   // all loads issued before the first add
                    const int p = p0 + k * NWC;
                    v[k] = p < G ? __ldcg(gp4 + (size_t)p * N4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < BATCH; ++k) {   // partials in increasing order, as before
                    s.x += v[k].x; s.y += v[k].y; s.z += v[k].z; s.w += v[k].w;
                }
            }
        }
        sred[warp * 32 + lane] = s;
        named_barrier(1, PROD_CONS);
        if (warp == 0 && c < c1) {
            float4 t = sred[lane];
#pragma unroll
            for (int w = 1; w < PROD_CONS / 32; ++w) {
                const float4 v = sred[w * 32 + lane];
                t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
            }
            g4[c] = t;
        }
        named_barrier(1, PROD_CONS);
    }
}

// ---------------------------------------------------------------------------
// Shape table: n -> (V, RL, RS).  N = n^2 = 4 * (512/RL) * V.
// ---------------------------------------------------------------------------
template <int V, int RL, int RS>
static cudaError_t launch_prod_t(int grid, const ProdArgs& a, cudaStream_t s)
{
    using S = ProdShape<V, RL, RS>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(PROD_THREADS, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (a.g_out) {   // the grid barrier needs co-resident blocks
        attr[na].id = cudaLaunchAttributeCooperative;
        attr[na].val.cooperative = 1;
        ++na;
    }
    if (a.pdl) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    const int pf = (int)(PROD_PF_BYTES / (S::STAGE_FLOATS * 4));
    return cudaLaunchKernelEx(&cfg, k_products<V, RL, RS>, a.A, a.m, a.x, a.y, a.r, a.gpart,
                              a.g_out, a.r2part, a.ctrl, a.mode,
                              (cudaGraphConditionalHandle)a.cond, a.set_cond, a.budget, pf,
                              a.bar_extra);
}

template <int V, int RL, int RS>
static cudaError_t configure_t()
{
    using S = ProdShape<V, RL, RS>;
    return cudaFuncSetAttribute(k_products<V, RL, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)S::SMEM);
}

#define TVCS_PROD_TABLE(X)   \
    X(16, 1, 8, 64)          \
    X(32, 2, 4, 16)          \
    X(48, 9, 8, 8)           \
    X(64, 4, 2, 4)           \
    X(96, 9, 2, 2)           \
    X(128, 8, 1, 1)

bool prod_supported(int n)
{
    switch (n) {
#define X(NN, V, RL, RS) case NN: return true;
        TVCS_PROD_TABLE(X)
#undef X
        default: return false;
    }
}

static int prod_rl(int n)
{
    switch (n) {
#define X(NN, V, RL, RS) case NN: return RL;
        TVCS_PROD_TABLE(X)
#undef X
        default: return 1;
    }
}

int prod_grid(int n, int m, int num_sms)
{
    const int rl = prod_rl(n);
    int g = (m + rl - 1) / rl;
    const int cap = num_sms > 32 ? num_sms - 16 : num_sms;   // 16 SMs stay free for the u-solve cluster
    return g < cap ? g : cap;
}

cudaError_t prod_configure(int n)
{
    switch (n) {
#define X(NN, V, RL, RS) case NN: return configure_t<V, RL, RS>();
        TVCS_PROD_TABLE(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_products(int n, int grid, const ProdArgs& a, cudaStream_t s)
{
    switch (n) {
#define X(NN, V, RL, RS) case NN: return launch_prod_t<V, RL, RS>(grid, a, s);
        TVCS_PROD_TABLE(X)
#undef X
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Gather of the partials, normalisation, fill.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gather(const float* __restrict__ gpart, int P, int N,
                                                float scale, float* __restrict__ out,
                                                double* __restrict__ part, Ctrl* __restrict__ ctrl)
{
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (i < N) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int p = 0;
        for (; p + 4 <= P; p += 4) {
            s0 += gpart[(size_t)p * N + i];
            s1 += gpart[(size_t)(p + 1) * N + i];
            s2 += gpart[(size_t)(p + 2) * N + i];
            s3 += gpart[(size_t)(p + 3) * N + i];
        }
        for (; p < P; ++p) s0 += gpart[(size_t)p * N + i];
        const float v = scale * ((s0 + s1) + (s2 + s3));
        out[i] = v;
        sq = (double)v * (double)v;
    }
    const double s = block_sum(sq, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    __shared__ int is_last;
    if (!last_block_all(&ctrl->ticket_gather, &is_last)) return;
    const double t = block_sum_array(part, gridDim.x, 1, red);
    if (threadIdx.x == 0) ctrl->vec2 = t;
}

// g = sum over the P per-block partials, in a fixed order.  A block covers 32
// float4 columns with 8 partial slices (one warp each); slice k sums partials
// k, k+8, ..., then slice 0 adds the 8 slice sums in order.
__global__ void __launch_bounds__(256) k_greduce(const float4* __restrict__ gpart, int P, int N4,
                                                 float4* __restrict__ g,
                                                 const Ctrl* __restrict__ ctrl, int mode)
{
    __shared__ float4 acc[8][32];
    if (mode == MODE_ITER && ctrl->skip) return;
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < N4) {
        for (int p = slice; p < P; p += 8) {
            const float4 v = gpart[(size_t)p * N4 + c];
            s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
        }
    }
    acc[slice][lane] = s;
    __syncthreads();
    if (slice == 0 && c < N4) {
        float4 t = acc[0][lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) {
            const float4 v = acc[k][lane];
            t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
        }
        g[c] = t;
    }
}

cudaError_t launch_greduce(const float* gpart, int P, int N, float* g, const Ctrl* ctrl, int mode,
                           cudaStream_t s)
{
    const int N4 = N / 4;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((N4 + 31) / 32, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    return cudaLaunchKernelEx(&cfg, k_greduce, reinterpret_cast<const float4*>(gpart), P, N4,
                              reinterpret_cast<float4*>(g), ctrl, mode);
}

__global__ void k_normalize(const float* __restrict__ z, float* __restrict__ v, int N,
                            const Ctrl* __restrict__ ctrl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double nrm = sqrt(ctrl->vec2);
    if (i < N) v[i] = (float)((double)z[i] / nrm);
}

__global__ void k_fill(float* __restrict__ v, int N, float value)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) v[i] = value;
}

// Start of a run: the loop bookkeeping of the control block, set on the device
// (no host round trip before the loop); the other fields keep their values.
__global__ void k_run_begin(Ctrl* __restrict__ c, int max_iter, int loops_max, double tol, int algo)
{
    c->it = 0;
    c->max_iter = max_iter;
    c->done = 0;
    c->skip = 0;
    c->stop_by_tol = 0;
    c->loops = 0;
    c->loops_max = loops_max;
    c->tol = tol;
    c->error = 0;
    c->algo = algo;
    c->ticket_fft = c->ticket_prod = c->ticket_fin = c->ticket_w = c->ticket_gather = 0u;
}

void launch_run_begin(Ctrl* c, int max_iter, int loops_max, double tol, int algo, cudaStream_t s)
{
    k_run_begin<<<1, 1, 0, s>>>(c, max_iter, loops_max, tol, algo);
}

void launch_gather(const float* gpart, int P, int N, float scale, float* out, double* part,
                   Ctrl* ctrl, cudaStream_t s)
{
    k_gather<<<(N + 255) / 256, 256, 0, s>>>(gpart, P, N, scale, out, part, ctrl);
}

void launch_normalize(const float* z, float* v, int N, const Ctrl* ctrl, cudaStream_t s)
{
    k_normalize<<<(N + 255) / 256, 256, 0, s>>>(z, v, N, ctrl);
}

void launch_fill(float* v, int N, float value, cudaStream_t s)
{
    k_fill<<<(N + 255) / 256, 256, 0, s>>>(v, N, value);
}

}  // namespace tvcs
