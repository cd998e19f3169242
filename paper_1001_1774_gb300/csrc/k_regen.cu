// Products with the encoding matrix regenerated inside the kernel (row a9):
//   r = A x - y,  g = A^T r,
// A_ij = binary32(z(i N + j) * binary32(1/sqrt(m))), z the counter-based
// Gaussian stream of gen.cuh -- the values the input generator writes, so the
// products read no byte of A from memory (the two matrix-vector products of
// eq. (line), Sec. 2.1, with A given by its seed).
//
// A cluster of CS blocks (4, 8 or 16) splits each row's N columns into CS slices
// of W = N / CS; block `rank` reads x's slice through the read-only cache and
// accumulates its slice of A^T r in shared memory.  A tile is up to 16
// consecutive rows.  Per tile:
//   gen     the warps take (row, segment) items: a segment is one sixteenth of
//           a row (N / 16 columns, so a block owns 16 / CS of them); lane L
//           generates the four-element groups L, L+32, L+64, ... of the segment
//           (one Philox block each, two in flight), stores them in the tile
//           buffer and adds them into its dot product with x in that order; a
//           fixed shuffle tree adds the 32 lanes;
//   exch    every block reads the 16 segment dots of each row from the blocks of
//           its cluster (distributed shared memory) and adds them in segment
//           order, so all blocks hold the same r_i;
//   update  g_slice += A_tile^T r_tile from the tile buffer, row after row.
// With two tile buffers, split cluster barriers (arrive after the partial
// dots of tile t, wait before reading them) let the generation of tile t+1
// run while the exchange of tile t completes; with one, the shared memory
// halves and the other blocks resident on the SM cover the wait.  Each
// element of A is generated once per launch.
//
// Many problems (own m, N, seed, x, y) share one launch.  Problem p's rows are
// cut into chunks of a fixed number of rows (about 2^21 entries, and at least
// 16 chunks when the problem has the rows: fixed by the problem, not by the
// launch shape); the chunks of the active problems are numbered in problem
// order, and cluster q of Q takes the chunks that start in the q-th of Q equal
// shares of the active problems' entries.
// Every chunk stores its slice of A^T r and its ||r||^2 (added row after row)
// in a slot of its own; k_regen_reduce adds a problem's slots in chunk order.
// So every sum has an order fixed by the problem alone: the results do not
// depend on the cluster size, tile height, kernel variant or number of clusters
// the tuner picks, nor on which other problems share the launch.
#include <cooperative_groups.h>

#include "common.cuh"
#include "gen.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace tvcs {

namespace {

constexpr int RG_THREADS = 256;
constexpr int RG_RTMAX = 16;                 // rows per tile at most
constexpr int RG_NWARP = RG_THREADS / 32;
constexpr int RG_NSEG = 16;                  // segments of a row (fixed summation order)
constexpr int RG_SEGMAX = 4;                 // segments of a row per block (cluster size >= 4)
constexpr int RG_QMAX = 1024;                // clusters per launch at most

__host__ __device__ __forceinline__ int tile_rows_for(int W, int tile_cap)
{
    int rt = RG_RTMAX;
    while (rt > 1 && rt * W > tile_cap) rt >>= 1;
    return rt;
}

// pre[p] = number of active chunks before problem p, pre[P] = T; prew[p] = entries
// of A of the active problems before p, prew[P] = E (all threads).
__device__ int active_prefix(const RegenProb* __restrict__ probs, int P, int mode, int* pre,
                             int* scan, long long* prew, long long* wscan)
{
    const int tid = threadIdx.x;
    int cnt[4];
    long long wk[4];
    int local = 0;
    long long wlocal = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = tid * 4 + k;
        int c = 0;
        long long w = 0;
        if (p < P) {
            c = probs[p].chunks;
            if (mode == MODE_ITER && probs[p].ctrl && probs[p].ctrl->skip) c = 0;
            if (c > 0) w = (long long)probs[p].m * probs[p].N;
        }
        cnt[k] = c;
        wk[k] = w;
        local += c;
        wlocal += w;
    }
    scan[tid] = local;
    wscan[tid] = wlocal;
    __syncthreads();
    for (int off = 1; off < RG_THREADS; off <<= 1) {
        const int v = tid >= off ? scan[tid - off] : 0;
        const long long wv = tid >= off ? wscan[tid - off] : 0;
        __syncthreads();
        scan[tid] += v;
        wscan[tid] += wv;
        __syncthreads();
    }
    int run = scan[tid] - local;
    long long wrun = wscan[tid] - wlocal;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = tid * 4 + k;
        if (p < P) {
            pre[p] = run;
            prew[p] = wrun;
        }
        run += cnt[k];
        wrun += wk[k];
    }
    if (tid == RG_THREADS - 1) {
        pre[P] = scan[tid];
        prew[P] = wscan[tid];
    }
    __syncthreads();
    return pre[P];
}

// The first active chunk whose first entry lies at or after work offset t (T when
// t is at or past the end).  Cluster q takes the chunks starting in
// [q E / Q, (q+1) E / Q): ranges of equal work, whatever the chunk sizes.
__device__ int chunk_at_work(const RegenProb* __restrict__ probs, int P, const int* pre,
                             const long long* prew, long long t)
{
    if (t >= prew[P]) return pre[P];
    int lo = 0, hi = P - 1;   // the problem p with prew[p] <= t < prew[p+1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prew[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int p = lo;
    const long long cw = (long long)probs[p].rows_per_chunk * probs[p].N;
    const long long k = (t - prew[p] + cw - 1) / cw;
    return pre[p] + (int)k;
}

struct TileMeta {
    int p, i0, nr, rt, W, chunk, last;   // last: the tile ends its chunk
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
    long long* prew = reinterpret_cast<long long*>(scan + RG_THREADS);   // pcap + 4
    long long* wscan = prew + pcap + 4;                         // RG_THREADS
    float* gs = reinterpret_cast<float*>(wscan + RG_THREADS);   // A^T r slice, wmax
    float* tile = gs + wmax;                                    // NBUF x tile_cap
    float* wpart = tile + NBUF * tile_cap;                      // 2 x RTMAX x SEGMAX, this block's
    float* slotv = wpart + 2 * RG_RTMAX * RG_SEGMAX;            // the same, read by the peers
    float* rvec = slotv + 2 * RG_RTMAX * RG_SEGMAX;             // 2 x RTMAX

    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int Q = gridDim.x / CS;
    const int cq = blockIdx.x / CS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int segs = RG_NSEG / CS;   // segments of a row this block owns

    active_prefix(probs, P, mode, pre, scan, prew, wscan);
    if (blockIdx.x == 0)
        for (int p = tid; p <= P; p += RG_THREADS) pre_out[p] = pre[p];
    const long long E = prew[P];
    int j = chunk_at_work(probs, P, pre, prew, (long long)cq * E / Q);
    const int j1 = chunk_at_work(probs, P, pre, prew, (long long)(cq + 1) * E / Q);
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

    float2 r2acc = make_float2(0.f, 0.f);   // double-single ||r||^2 of the chunk (block 0, thread 0)
    // exch + update of tile tm: partial dots from slot buffer sb, entries from tile buffer tb
    auto finish = [&](const TileMeta& tm, int sb, int tb) {
        cluster_wait();   // every block's segment dots of tile tm are visible
        const RegenProb* pp = probs + tm.p;
        if (tid < tm.nr) {
            float s = 0.f;   // segments 0 .. 15 in order: block k holds k segs .. (k+1) segs - 1
            for (int k = 0; k < CS; ++k) {
                const float* pv = cluster.map_shared_rank(slotv, k) + (sb * RG_RTMAX + tid) * RG_SEGMAX;
                for (int q = 0; q < segs; ++q) s += pv[q];
            }
            const int i = tm.i0 + tid;
            const float rv = pp->y ? s - pp->y[i] : s;
            rvec[sb * RG_RTMAX + tid] = rv;
            if (rank == 0) pp->r[i] = rv;
        }
        __syncthreads();
        if (rank == 0 && tid == 0)   // ||r||^2 of the chunk, row after row
            for (int rr = 0; rr < tm.nr; ++rr) r2acc = ds_add(r2acc, ds_sq(rvec[sb * RG_RTMAX + rr]));
        const float4* tbuf = reinterpret_cast<const float4*>(tile + tb * tile_cap);
        float4* g4 = reinterpret_cast<float4*>(gs);
        const int G = tm.W / 4;
        for (int q4 = tid; q4 < G; q4 += RG_THREADS) {
            float4 acc = g4[q4];
            for (int rr = 0; rr < tm.nr; ++rr) fma4(acc, tbuf[rr * G + q4], rvec[sb * RG_RTMAX + rr]);
            g4[q4] = acc;
        }
        if (tm.last) {   // the chunk ends: each thread stores and clears the groups it accumulated
            float4* dst = reinterpret_cast<float4*>(pp->gslot + (size_t)tm.chunk * pp->N +
                                                    (size_t)rank * tm.W);
            for (int q4 = tid; q4 < G; q4 += RG_THREADS) {
                dst[q4] = g4[q4];
                g4[q4] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (rank == 0 && tid == 0) {
                pp->r2slot[tm.chunk] = r2acc;
                r2acc = make_float2(0.f, 0.f);
            }
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
            cur.chunk = c;
            // gen: (row, segment) items over the warps
            {
                const int Gs = N / (4 * RG_NSEG);   // groups of a segment
                const int G = W / 4;                // groups of the block's slice of a row
                float4* tbase = reinterpret_cast<float4*>(tile + tb * tile_cap);
                const float4* xbase = reinterpret_cast<const float4*>(pr->x + (size_t)rank * W);
                const float scale = pr->scale;
                const unsigned long long seed = pr->seed;
                for (int it = warp; it < cur.nr * segs; it += RG_NWARP) {
                    const int rr = it / segs, sl = it - rr * segs;
                    const unsigned long long i = (unsigned long long)(cur.i0 + rr);
                    const int g0 = sl * Gs;
                    const unsigned long long b0 =
                        ((i * (unsigned long long)N + (unsigned long long)rank * W) >> 2) + g0;
                    float4* trow = tbase + rr * G + g0;
                    // x slice through the read-only path: L1 keeps it across the tile's rows
                    const float4* x4 = xbase + g0;
                    float dot = 0.f;
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
                    // groups lane, lane+32, lane+64, ... in this order, two Philox blocks in
                    // flight (four measured slower: 21.0 against 20.3 ms over the 64 problems)
                    int q = lane;
                    for (; q + 32 < Gs; q += 64) {
                        const float4 z0 = gen_normals4(seed, 0u, b0 + q);
                        const float4 z1 = gen_normals4(seed, 0u, b0 + q + 32);
                        emit(q, z0);
                        emit(q + 32, z1);
                    }
                    if (q < Gs) emit(q, gen_normals4(seed, 0u, b0 + q));
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                    if (lane == 0) wpart[(sb * RG_RTMAX + rr) * RG_SEGMAX + sl] = dot;
                }
            }
            // advance the cursor
            row += cur.nr;
            cur.last = row >= cend ? 1 : 0;
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
                    }
                    row = c * RC;
                    cend = min(m, row + RC);
                }
            }
        }
        if (NBUF == 2 && have_prev) finish(prev, sb ^ 1, tb ^ 1);
        if (!have_cur) break;
        __syncthreads();   // segment dots of this tile complete; the other tile buffer is free
        // Published only now: the peers read slotv[sb] of tile t-2 until they arrive
        // for tile t-1, which finish(prev) above has waited for.
        if (tid < cur.nr * segs) {
            const int rr = tid / segs, sl = tid - rr * segs;
            slotv[(sb * RG_RTMAX + rr) * RG_SEGMAX + sl] = wpart[(sb * RG_RTMAX + rr) * RG_SEGMAX + sl];
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

// g = sum of the chunk slots in chunk order, ctrl->r2 = sum of the chunk r2 slots.
// Grid (ceil(maxN / 1024), P), 256 threads, one float4 per thread.
__global__ void __launch_bounds__(256)
k_regen_reduce(const RegenProb* __restrict__ probs, int P, const int* __restrict__ pre,
               cudaGraphConditionalHandle cond, int set_cond)
{
    const int p = blockIdx.y;
    const int tid = threadIdx.x;
    const RegenProb& pr = probs[p];
    if (set_cond && p == 0 && blockIdx.x == 0 && tid == 0) {
        Ctrl* c = pr.ctrl;
        const int lc = ++c->loops;
        const int cont = (!c->done && c->error == ERR_NONE && lc < c->loops_max) ? 1 : 0;
        cudaGraphSetConditional(cond, (unsigned)cont);
    }
    const int K = pre[p + 1] - pre[p];
    if (K == 0) return;   // inactive in this launch
    const int n4 = pr.N / 4;
    const int q4 = blockIdx.x * blockDim.x + tid;
    if (q4 < n4) {
        const float4* slot = reinterpret_cast<const float4*>(pr.gslot);
        float4 acc = slot[q4];
        for (int h = 1; h < K; ++h) {
            const float4 v = slot[(size_t)h * n4 + q4];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        reinterpret_cast<float4*>(pr.g)[q4] = acc;
    }
    if (blockIdx.x == 0 && tid == 0 && pr.ctrl) {
        float2 v = pr.r2slot[0];
        for (int h = 1; h < K; ++h) v = ds_add(v, pr.r2slot[h]);
        pr.ctrl->r2 = ds_value(v);
    }
}

static size_t regen_smem(int wmax, int tile_cap, int nbuf, int pcap)
{
    return sizeof(int) * ((size_t)pcap + 4 + RG_THREADS) +
           sizeof(long long) * ((size_t)pcap + 4 + RG_THREADS) +
           sizeof(float) * ((size_t)wmax + (size_t)nbuf * tile_cap + 4 * RG_RTMAX * RG_SEGMAX +
                            2 * RG_RTMAX);
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
    if ((plan->cs != 4 && plan->cs != 8 && plan->cs != 16) || plan->wmax <= 0 ||
        plan->wmax % 4 != 0 || tile_rows_for(plan->wmax, plan->tile_cap) < plan->cs / 2 ||
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
    (void)plan;
    const dim3 grid((maxN / 4 + 255) / 256, P);
    k_regen_reduce<<<grid, 256, 0, s>>>(probs, P, pre, (cudaGraphConditionalHandle)cond, set_cond);
}

}  // namespace tvcs
