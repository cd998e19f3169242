// Products with the encoding matrix regenerated inside the kernel (row a9):
//   r = A x - y,  g = A^T r,
// A_ij = binary32(z(i N + j) * binary32(1/sqrt(m))), z the counter-based
// Gaussian stream of gen.cuh -- the values the input generator writes, so the
// products read no byte of A from memory (the two matrix-vector products of
// eq. (line), Sec. 2.1, with A given by its seed).
//
// A cluster of CS blocks splits each row's N columns into CS slices of
// W = N / CS; block `rank` reads x's slice through the read-only cache and
// accumulates its slice of A^T r in shared memory.  A tile is up to 16 consecutive rows.  Per tile:
//   gen     each thread generates four-element groups (one Philox block each)
//           of one row, stores them in the tile buffer and accumulates the
//           row's dot product with x;
//   exch    every block reads the per-row partial dots of all blocks of its
//           cluster (distributed shared memory) and adds them in rank order,
//           so all blocks hold the same r_i;
//   update  g_slice += A_tile^T r_tile from the tile buffer.
// With two tile buffers, split cluster barriers (arrive after the partial
// dots of tile t, wait before reading them) let the generation of tile t+1
// run while the exchange of tile t completes; with one, the shared memory
// halves and the other blocks resident on the SM cover the wait.  Each
// element of A is generated once per launch.
//
// Many problems (own m, N, seed, x, y) share one launch.  Problem p's rows are
// cut into `chunks` chunks; the chunks of the active problems are numbered in
// problem order (T in all) and cluster q takes chunks [q T / Q, (q+1) T / Q).
// A run of consecutive chunks of one problem inside a cluster's range sums
// into one slice, stored at the end of the run in the slot of the run's first
// chunk.  k_regen_reduce finds the same run heads from (T, Q) and adds the
// slots in chunk order: the result does not depend on timing.
#include <cooperative_groups.h>

#include "common.cuh"
#include "gen.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace tvcs {

namespace {

constexpr int RG_THREADS = 256;
constexpr int RG_RTMAX = 16;                 // rows per tile at most
constexpr int RG_NWMAX = RG_THREADS / 32;    // warps sharing one row at most
constexpr int RG_QMAX = 1024;                // clusters per launch at most

__host__ __device__ __forceinline__ int range_start(int q, int T, int Q)
{
    return (int)(((long long)q * T) / Q);
}

__host__ __device__ __forceinline__ int tile_rows_for(int W, int tile_cap)
{
    int rt = RG_RTMAX;
    while (rt > 1 && rt * W > tile_cap) rt >>= 1;
    return rt;
}

// pre[p] = number of active chunks before problem p, pre[P] = T (all threads).
__device__ int active_prefix(const RegenProb* __restrict__ probs, int P, int mode, int* pre,
                             int* scan)
{
    const int tid = threadIdx.x;
    int cnt[4];
    int local = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = tid * 4 + k;
        int c = 0;
        if (p < P) {
            c = probs[p].chunks;
            if (mode == MODE_ITER && probs[p].ctrl && probs[p].ctrl->skip) c = 0;
        }
        cnt[k] = c;
        local += c;
    }
    scan[tid] = local;
    __syncthreads();
    for (int off = 1; off < RG_THREADS; off <<= 1) {
        const int v = tid >= off ? scan[tid - off] : 0;
        __syncthreads();
        scan[tid] += v;
        __syncthreads();
    }
    int run = scan[tid] - local;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = tid * 4 + k;
        if (p < P) pre[p] = run;
        run += cnt[k];
    }
    if (tid == RG_THREADS - 1) pre[P] = scan[tid];
    __syncthreads();
    return pre[P];
}

struct TileMeta {
    int p, i0, nr, rt, W, head, last;   // last: the run of the slice ends with this tile
};

__device__ __forceinline__ void fma4(float4& acc, const float4& a, float s)
{
    acc.x = fmaf(a.x, s, acc.x);
    acc.y = fmaf(a.y, s, acc.y);
    acc.z = fmaf(a.z, s, acc.z);
    acc.w = fmaf(a.w, s, acc.w);
}

}  // namespace

// MINB: blocks per SM the registers are budgeted for (2: up to 128 registers
// a thread, 3: up to 80, 4: up to 64).  NBUF: tile buffers; with 2 the generation of tile
// t+1 overlaps the exchange of tile t inside a block, with 1 the shared memory
// halves and other resident blocks fill the wait.  The tuner picks the variant.
template <int MINB, int NBUF>
__global__ void __launch_bounds__(RG_THREADS, MINB)
k_regen_products(const RegenProb* __restrict__ probs, int P, int mode, int wmax, int tile_cap,
                 int pcap, int* __restrict__ pre_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int* pre = reinterpret_cast<int*>(smem);                    // pcap + 4 (pcap >= P, multiple of 4)
    int* scan = pre + pcap + 4;                                 // RG_THREADS
    float* gs = reinterpret_cast<float*>(scan + RG_THREADS);    // A^T r slice, wmax
    float* tile = gs + wmax;                                    // NBUF x tile_cap
    float* wpart = tile + NBUF * tile_cap;                      // 2 x RTMAX x NWMAX
    float* slotv = wpart + 2 * RG_RTMAX * RG_NWMAX;             // 2 x RTMAX, read by the peers
    float* rvec = slotv + 2 * RG_RTMAX;                         // 2 x RTMAX

    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int Q = gridDim.x / CS;
    const int cq = blockIdx.x / CS;
    const int tid = threadIdx.x;

    const int T = active_prefix(probs, P, mode, pre, scan);
    if (blockIdx.x == 0)
        for (int p = tid; p <= P; p += RG_THREADS) pre_out[p] = pre[p];
    int j = range_start(cq, T, Q);
    const int j1 = range_start(cq + 1, T, Q);
    if (j >= j1) return;   // the whole cluster has no chunk

    for (int i = tid; i < wmax; i += RG_THREADS) gs[i] = 0.f;

    // cursor: chunk j = chunk c of problem p, next row `row` of rows [.., cend)
    int p = 0;
    while (pre[p + 1] <= j) ++p;
    const RegenProb* pr = probs + p;
    int c = j - pre[p];
    int N = pr->N, m = pr->m, RC = pr->rows_per_chunk;
    int W = N / CS;
    int rt = tile_rows_for(W, tile_cap);
    int row = c * RC;
    int cend = min(m, row + RC);
    int head = c;

    float2 r2acc = make_float2(0.f, 0.f);   // double-single ||r||^2 of the problem
    // exch + update of tile tm: partial dots from slot buffer sb, entries from tile buffer tb
    auto finish = [&](const TileMeta& tm, int sb, int tb) {
        cluster_wait();   // every block's partial dots of tile tm are visible
        const RegenProb* pp = probs + tm.p;
        if (tid < tm.nr) {
            float s = 0.f;
            for (int k = 0; k < CS; ++k) s += cluster.map_shared_rank(slotv, k)[sb * RG_RTMAX + tid];
            const int i = tm.i0 + tid;
            const float rv = pp->y ? s - pp->y[i] : s;
            rvec[sb * RG_RTMAX + tid] = rv;
            if (rank == 0) {
                pp->r[i] = rv;
                r2acc = ds_add(r2acc, ds_sq(rv));
            }
        }
        __syncthreads();
        const float4* tbuf = reinterpret_cast<const float4*>(tile + tb * tile_cap);
        float4* g4 = reinterpret_cast<float4*>(gs);
        const int G = tm.W / 4;
        for (int q4 = tid; q4 < G; q4 += RG_THREADS) {
            float4 acc = g4[q4];
            for (int rr = 0; rr < tm.nr; ++rr) fma4(acc, tbuf[rr * G + q4], rvec[sb * RG_RTMAX + rr]);
            g4[q4] = acc;
        }
        if (tm.last) {   // each thread stores and clears the groups it accumulated
            float4* dst = reinterpret_cast<float4*>(pp->gslot + (size_t)tm.head * pp->N +
                                                    (size_t)rank * tm.W);
            for (int q4 = tid; q4 < G; q4 += RG_THREADS) {
                dst[q4] = g4[q4];
                g4[q4] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (rank == 0 && tid < 32) {   // r2acc lives in threads < 16 of block 0
                const float2 v = warp_sum_ds(r2acc);
                if (tid == 0) pp->r2slot[tm.head] = v;
            }
            r2acc = make_float2(0.f, 0.f);
        }
    };

    TileMeta prev{};
    bool have_prev = false;
    for (int t = 0;; ++t) {
        const bool have_cur = j < j1;
        const int sb = t & 1;                  // partial-dot and r buffers
        const int tb = NBUF == 2 ? sb : 0;     // tile buffer
        TileMeta cur{};
        if (have_cur) {
            cur.p = p;
            cur.i0 = row;
            cur.nr = min(rt, cend - row);
            cur.rt = rt;
            cur.W = W;
            cur.head = head;
            // gen: rows of the tile, tpr threads per row
            {
                const int tpr = RG_THREADS / rt;
                const int rr = tid / tpr, lane = tid - rr * tpr;
                const int G = W / 4;
                float dot = 0.f;
                if (rr < cur.nr) {
                    const unsigned long long i = (unsigned long long)(cur.i0 + rr);
                    const unsigned long long b0 =
                        (i * (unsigned long long)N + (unsigned long long)rank * W) >> 2;
                    float4* trow = reinterpret_cast<float4*>(tile + tb * tile_cap) + rr * G;
                    // x slice through the read-only path: L1 keeps it across the tile's rows
                    const float4* x4 = reinterpret_cast<const float4*>(pr->x + (size_t)rank * W);
                    const float scale = pr->scale;
                    const unsigned long long seed = pr->seed;
                    auto emit = [&](int q, const float4& z) {
                        float4 a;
                        a.x = __fmul_rn(z.x, scale);
                        a.y = __fmul_rn(z.y, scale);
                        a.z = __fmul_rn(z.z, scale);
                        a.w = __fmul_rn(z.w, scale);
                        trow[q] = a;
                        const float4 xv = __ldg(x4 + q);
                        dot = fmaf(a.x, xv.x, dot);
                        dot = fmaf(a.y, xv.y, dot);
                        dot = fmaf(a.z, xv.z, dot);
                        dot = fmaf(a.w, xv.w, dot);
                    };
                    // two independent Philox blocks in flight per thread (latency hiding)
                    int q4 = lane;
                    for (; q4 + tpr < G; q4 += 2 * tpr) {
                        const float4 z0 = gen_normals4(seed, 0u, b0 + q4);
                        const float4 z1 = gen_normals4(seed, 0u, b0 + q4 + tpr);
                        emit(q4, z0);
                        emit(q4 + tpr, z1);
                    }
                    if (q4 < G) emit(q4, gen_normals4(seed, 0u, b0 + q4));
                }
                const int wl = tpr < 32 ? tpr : 32;
                for (int off = wl >> 1; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                if (rr < cur.nr && (lane & (wl - 1)) == 0)
                    wpart[(sb * RG_RTMAX + rr) * RG_NWMAX + (lane >> 5)] = dot;
            }
            // advance the cursor
            row += cur.nr;
            if (row >= cend) {
                ++j;
                if (j < j1) {
                    ++c;
                    if (j >= pre[p + 1]) {   // first chunk of the next active problem
                        do ++p;
                        while (pre[p + 1] <= j);
                        c = j - pre[p];
                        pr = probs + p;
                        N = pr->N;
                        m = pr->m;
                        RC = pr->rows_per_chunk;
                        W = N / CS;
                        rt = tile_rows_for(W, tile_cap);
                        head = c;
                    }
                    row = c * RC;
                    cend = min(m, row + RC);
                }
            }
            cur.last = (j >= j1 || p != cur.p) ? 1 : 0;
        }
        if (NBUF == 2 && have_prev) finish(prev, sb ^ 1, tb ^ 1);
        if (!have_cur) break;
        __syncthreads();   // partial dots of this tile complete; the other tile buffer is free
        if (tid < cur.nr) {
            const int nw = (RG_THREADS / cur.rt) / 32;
            float s = 0.f;
            for (int w = 0; w < (nw > 0 ? nw : 1); ++w) s += wpart[(sb * RG_RTMAX + tid) * RG_NWMAX + w];
            slotv[sb * RG_RTMAX + tid] = s;
        }
        cluster_arrive();
        if (NBUF == 1) {
            finish(cur, sb, 0);
            __syncthreads();   // the tile buffer is free for the next tile
        } else {
            prev = cur;
            have_prev = true;
        }
    }
    // the peers may still read this block's slots: leave together
    cluster_arrive();
    cluster_wait();
}

// g = sum of the run slots (chunk order), ctrl->r2 = sum of the run r2 slots.
// Grid (ceil(maxN / 1024), P), 256 threads, one float4 per thread.
__global__ void __launch_bounds__(256)
k_regen_reduce(const RegenProb* __restrict__ probs, int P, int Q, const int* __restrict__ pre,
               cudaGraphConditionalHandle cond, int set_cond)
{
    __shared__ int heads[RG_QMAX + 1];
    __shared__ int nh;
    const int p = blockIdx.y;
    const int tid = threadIdx.x;
    const RegenProb& pr = probs[p];
    if (set_cond && p == 0 && blockIdx.x == 0 && tid == 0) {
        Ctrl* c = pr.ctrl;
        const int lc = ++c->loops;
        const int cont = (!c->done && c->error == ERR_NONE && lc < c->loops_max) ? 1 : 0;
        cudaGraphSetConditional(cond, (unsigned)cont);
    }
    const int s = pre[p], K = pre[p + 1] - s;
    if (K == 0) return;   // inactive in this launch
    const int T = pre[P];
    if (tid == 0) {
        int n = 0;
        heads[n++] = 0;
        for (int q = 1; q < Q; ++q) {
            const int st = range_start(q, T, Q);
            if (st > s && st < s + K && st - s != heads[n - 1]) heads[n++] = st - s;
        }
        nh = n;
    }
    __syncthreads();
    const int n4 = pr.N / 4;
    const int q4 = blockIdx.x * blockDim.x + tid;
    if (q4 < n4) {
        const float4* slot = reinterpret_cast<const float4*>(pr.gslot);
        float4 acc = slot[(size_t)heads[0] * n4 + q4];
        for (int h = 1; h < nh; ++h) {
            const float4 v = slot[(size_t)heads[h] * n4 + q4];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        reinterpret_cast<float4*>(pr.g)[q4] = acc;
    }
    if (blockIdx.x == 0 && tid == 0 && pr.ctrl) {
        float2 v = pr.r2slot[heads[0]];
        for (int h = 1; h < nh; ++h) v = ds_add(v, pr.r2slot[heads[h]]);
        pr.ctrl->r2 = ds_value(v);
    }
}

static size_t regen_smem(int wmax, int tile_cap, int nbuf, int pcap)
{
    return sizeof(int) * ((size_t)pcap + 4 + RG_THREADS) +
           sizeof(float) * ((size_t)wmax + (size_t)nbuf * tile_cap + 2 * RG_RTMAX * RG_NWMAX +
                            4 * RG_RTMAX);
}

int regen_tile_rows(const RegenPlan& plan, int N)
{
    return tile_rows_for(N / plan.cs, plan.tile_cap);
}

template <int MINB, int NBUF>
static bool configure_t(RegenPlan* plan, int optin)
{
    if (cudaFuncSetAttribute(k_regen_products<MINB, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin) != cudaSuccess ||
        cudaFuncSetAttribute(k_regen_products<MINB, NBUF>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                             1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan->cs, 1, 1);
    cfg.blockDim = dim3(RG_THREADS, 1, 1);
    cfg.dynamicSmemBytes = plan->smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan->cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_regen_products<MINB, NBUF>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (n > RG_QMAX) n = RG_QMAX;
    plan->clusters = n;
    return n >= 1;
}

bool regen_configure(RegenPlan* plan)
{
    plan->clusters = 0;
    if (plan->cs < 1 || plan->cs > 16 || plan->wmax <= 0 || plan->wmax % 4 != 0 ||
        plan->tile_cap < plan->wmax || plan->tile_cap % 4 != 0 ||
        plan->minb < 2 || plan->minb > 4 || (plan->nbuf != 1 && plan->nbuf != 2) ||
        plan->pcap < 1 || plan->pcap > REGEN_PMAX)
        return false;
    plan->pcap = (plan->pcap + 3) / 4 * 4;
    plan->smem = regen_smem(plan->wmax, plan->tile_cap, plan->nbuf, plan->pcap);
    // The attributes are per kernel, not per plan: allow the largest opt-in
    // size once, so that plans of different sizes can alternate.
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (plan->smem > (size_t)optin) return false;
    if (plan->minb == 2)
        return plan->nbuf == 2 ? configure_t<2, 2>(plan, optin) : configure_t<2, 1>(plan, optin);
    if (plan->minb == 3)
        return plan->nbuf == 2 ? configure_t<3, 2>(plan, optin) : configure_t<3, 1>(plan, optin);
    return plan->nbuf == 2 ? configure_t<4, 2>(plan, optin) : configure_t<4, 1>(plan, optin);
}

void launch_regen(const RegenProb* probs, int P, int mode, const RegenPlan& plan, int* pre_out,
                  cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.clusters * plan.cs, 1, 1);
    cfg.blockDim = dim3(RG_THREADS, 1, 1);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto k = plan.minb == 4   ? (plan.nbuf == 2 ? k_regen_products<4, 2> : k_regen_products<4, 1>)
             : plan.minb == 3 ? (plan.nbuf == 2 ? k_regen_products<3, 2> : k_regen_products<3, 1>)
                              : (plan.nbuf == 2 ? k_regen_products<2, 2> : k_regen_products<2, 1>);
    cudaLaunchKernelEx(&cfg, k, probs, P, mode, plan.wmax, plan.tile_cap, plan.pcap, pre_out);
}

void launch_regen_reduce(const RegenProb* probs, int P, int maxN, int mode, const RegenPlan& plan,
                         const int* pre, unsigned long long cond, int set_cond, cudaStream_t s)
{
    (void)mode;
    const dim3 grid((maxN / 4 + 255) / 256, P);
    k_regen_reduce<<<grid, 256, 0, s>>>(probs, P, plan.clusters, pre,
                                        (cudaGraphConditionalHandle)cond, set_cond);
}

}  // namespace tvcs
