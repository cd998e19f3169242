// Rows a6-a7 with A in reduced or split precision, and for images whose rows
// are too long for one block: r = A x - y, partials of g = A^T r, one pass
// over A (Xiao & Yang, eq. (line): g_k = A^T (A u^k - f)).
//
// Storage of A (m x N, row-major planes):
//   FP32      one binary32 plane;
//   BF16X2    A = hi + lo, hi = bf16(A), lo = bf16(A - hi) (both round to
//             nearest even); hi + lo is exact in binary32 and within 2^-16 |A|;
//   FP8_BF16  A = s_i q + c, s_i = max_j |A_ij| / 448 per row, q = e4m3(A / s_i)
//             (round to nearest even, saturating), c = bf16(A - s_i q).
// Products accumulate in binary32; ||r||^2 as binary32 double-single pairs.
//
// A cluster of CS blocks shares each row: block k of the cluster owns columns
// [k N/CS, (k+1) N/CS).  Each streams its column slice of the rows through a
// shared-memory ring filled by bulk asynchronous copies (TMA, one mbarrier per
// stage), forms its part of every row's dot product, and sends it to every
// block of the cluster: an asynchronous store into the peer's shared memory
// whose 4 bytes complete on the peer's mbarrier (st.async; a remote arrival with
// a cluster-scope release per part stalled the block's own bulk copies of A and
// held the binary32 storage at 87 % of the copy peak).  Each block waits, with a
// bounded spin, for the CS parts of a row, adds them in rank order (every block
// gets the same r_i), and folds r_i times its slice of the row (decoded again
// from shared memory) into per-thread accumulators.  The exchange is software-
// pipelined: the part of row s+1 is sent before the parts of row s are awaited.
// Cluster c writes its partial of A^T r to gpart[c]; the partials are summed
// afterwards in a fixed order.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"

namespace tvcs {

constexpr int QPROD_YMAX = 1024;
// Bulk copies per storage plane and stage (the binary32 plane, twice the bytes, takes twice as many).
constexpr int QPROD_TMA_PIECES = 1;

template <int PREC>
struct QPrec;

template <>
struct QPrec<0> {   // binary32
    static constexpr int PLANE_BYTES_NUM = 4;   // bytes per element in the stage
};
template <>
struct QPrec<1> {   // bf16 hi + lo
    static constexpr int PLANE_BYTES_NUM = 4;
};
template <>
struct QPrec<2> {   // fp8 e4m3 + bf16 correction
    static constexpr int PLANE_BYTES_NUM = 3;
};

template <int PREC, int V, int CS, int CONS, int NST>
struct QShape {
    static constexpr int NS = 4 * CONS * V;        // columns per block (the slice)
    static constexpr int N = NS * CS;
    static constexpr int THREADS = CONS + 64;   // consumers, the producer warp, the exchange warp
    static constexpr size_t STAGE_BYTES = (size_t)NS * QPrec<PREC>::PLANE_BYTES_NUM;
    static constexpr size_t O_BAR = NST * STAGE_BYTES;   // full[NST], empty[NST], xbar[4], partbar[2]
    static constexpr size_t O_RED = O_BAR + (2 * NST + 6) * 8;       // [2][CONS/32] floats
    static constexpr size_t O_XRED = O_RED + 2 * (CONS / 32) * 4;    // [4][CS] floats
    static constexpr size_t O_DRED = ((O_XRED + 4 * CS * 4 + 15) / 16) * 16;   // [32] float2
    static constexpr size_t O_Y = O_DRED + 32 * 8;                   // y of the rows
    static constexpr size_t O_S = O_Y + QPROD_YMAX * 4;              // row scales (FP8)
    static constexpr size_t SMEM = O_S + QPROD_YMAX * 4 + 16;
    static_assert(STAGE_BYTES % 16 == 0, "TMA sizes are multiples of 16 bytes");
    static_assert(CONS % 32 == 0 && CONS <= 512, "consumer warps");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t map_remote(uint32_t local_smem, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_smem), "r"(rank));
    return r;
}

// Store v at shared::cluster address `addr` (any block of the cluster) and count
// its 4 bytes on the barrier at `bar` in that block (complete_tx): the value is
// visible to the threads that observe the barrier's phase, with no release fence
// (a cluster-scope release per row stalled this block's bulk copies of A).
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr),
                 "f"(v), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

__device__ __forceinline__ float bf16_lo_f(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

template <int PREC, int V, int CS, int CONS, int NST>
__global__ void __launch_bounds__(CONS + 64, 1)
    k_products_q(const unsigned char* __restrict__ P0, const unsigned char* __restrict__ P1,
                 const float* __restrict__ rscale, int m, const float* __restrict__ x,
                 const float* __restrict__ y, float* __restrict__ r, float* __restrict__ gpart,
                 float2* __restrict__ r2part, Ctrl* __restrict__ ctrl, int mode,
                 cudaGraphConditionalHandle cond, int set_cond, long long budget)
{
    using S = QShape<PREC, V, CS, CONS, NST>;
    constexpr int NS = S::NS, N = S::N, WARPS = CONS / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::O_BAR);
    uint64_t* empty = full + NST;
    uint64_t* xbar = empty + NST;                                   // [4]
    uint64_t* partbar = xbar + 4;                                   // [2]
    float* red = reinterpret_cast<float*>(smem + S::O_RED);         // [2][WARPS]
    float* xred = reinterpret_cast<float*>(smem + S::O_XRED);       // [4][CS]
    float2* dred = reinterpret_cast<float2*>(smem + S::O_DRED);
    float* sy = reinterpret_cast<float*>(smem + S::O_Y);
    float* ss = reinterpret_cast<float*>(smem + S::O_S);
    int* sflag = reinterpret_cast<int*>(smem + S::O_S + QPROD_YMAX * 4);

    const int tid = threadIdx.x;
    const uint32_t rank = CS > 1 ? cluster_rank() : 0u;
    const int cidx = blockIdx.x / CS;          // cluster index = partial index
    const int G = gridDim.x / CS;              // number of clusters
    if (mode == MODE_ITER) {
        const int skip = ctrl->skip;
        if (blockIdx.x == 0 && tid == 0) {
            if (!skip && ctrl->algo == 0) ctrl->pending = 1;
            if (set_cond) {
                const int lc = ++ctrl->loops;
                const int cont =
                    (!ctrl->done && ctrl->error == ERR_NONE && lc < ctrl->loops_max) ? 1 : 0;
                cudaGraphSetConditional(cond, (unsigned)cont);
            }
        }
        if (skip) return;   // uniform over the grid
    }
    const int i0 = (int)(((long long)m * cidx) / G);
    const int i1 = (int)(((long long)m * (cidx + 1)) / G);
    const int nrows = i1 - i0;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], WARPS);
        }
        for (int b = 0; b < 4; ++b) mbar_init(&xbar[b], 1);   // the exchange warp's arrival (+ CS parts' bytes)
        for (int b = 0; b < 2; ++b) mbar_init(&partbar[b], WARPS);
        fence_mbar_init();
    }
    __syncthreads();
    if constexpr (CS > 1) cluster_sync_all();   // peers' barriers exist before any remote store

    if (tid >= CONS + 32) {
        // ---------------- exchange warp: the block's part of every row to the cluster ----
        // The warps' parts of row s (red[s & 1], complete when partbar[s & 1] completes)
        // are read by lanes 0 .. WARPS-1 and added by a fixed shuffle tree; lane 0 arms
        // this block's slot s mod 4 for the CS parts (one arrival, CS x 4 bytes) and lane
        // k < CS stores the sum into block k's slot with an asynchronous store that
        // counts its bytes on block k's barrier.  Slot s mod 4 is armed for row s only
        // once this block's warps have passed row s-2, hence row s-4: its previous phase
        // is complete (a peer's bytes may land before the arming, which the barrier's
        // transaction count allows).  All reads of red[] for row s precede every send of
        // row s, so the consumers, which reuse red[s & 1] for row s+2 only after this
        // block's own part of row s reached them, never overwrite a part that is still
        // to be read.
        const int lane = tid & 31;
        const uint32_t xr = CS > 1 ? map_remote(smem_u32(xred), (uint32_t)(lane % CS)) : 0u;
        const uint32_t xb = CS > 1 ? map_remote(smem_u32(xbar), (uint32_t)(lane % CS)) : 0u;
        bool eok = true;
        for (int s = 0; s < nrows; ++s) {
            if (eok && !mbar_wait(&partbar[s & 1], (uint32_t)((s >> 1) & 1), budget)) {
                set_error(ctrl, ERR_TIMEOUT);
                eok = false;
            }
            float part = lane < WARPS ? red[(s & 1) * WARPS + lane] : 0.f;
            part = warp_sum(part);
            const int b = s & 3;
            if constexpr (CS > 1) {
                if (lane == 0) mbar_arrive_expect_tx(&xbar[b], (uint32_t)CS * 4u);
                if (lane < CS) st_async_f32(xr + (uint32_t)((b * CS + rank) * 4), part, xb + (uint32_t)(b * 8));
            } else if (lane == 0) {
                xred[b] = part;
                mbar_arrive(&xbar[b]);
            }
            __syncwarp();
        }
        if constexpr (CS > 1) cluster_sync_all();
        return;
    }
    if (tid >= CONS) {
        // ---------------- producer warp: row slices into the ring ----------------
        if (tid == CONS) {
            const uint64_t pol = l2_policy_evict_first();
            const size_t col0 = (size_t)rank * NS;
            int issued = 0;
            for (int s = 0; s < nrows; ++s) {
                const int slot = s % NST;
                if (s >= NST && !mbar_wait(&empty[slot], ((s / NST) - 1) & 1, budget)) {
                    set_error(ctrl, ERR_TIMEOUT);
                    break;
                }
                const size_t row = (size_t)(i0 + s);
                unsigned char* dst = smem + (size_t)slot * S::STAGE_BYTES;
                if constexpr (PREC == 0) {
                    mbar_arrive_expect_tx(&full[slot], NS * 4u);
                    tma_load_1d_split(dst, P0 + (row * N + col0) * 4, NS * 4u, &full[slot], pol,
                                      QPROD_TMA_PIECES * 2);
                } else if constexpr (PREC == 1) {
                    mbar_arrive_expect_tx(&full[slot], NS * 4u);
                    tma_load_1d_split(dst, P0 + (row * N + col0) * 2, NS * 2u, &full[slot], pol,
                                      QPROD_TMA_PIECES);
                    tma_load_1d_split(dst + (size_t)NS * 2, P1 + (row * N + col0) * 2, NS * 2u,
                                      &full[slot], pol, QPROD_TMA_PIECES);
                } else {
                    mbar_arrive_expect_tx(&full[slot], NS * 3u);
                    tma_load_1d_split(dst, P0 + (row * N + col0), NS * 1u, &full[slot], pol,
                                      QPROD_TMA_PIECES);
                    tma_load_1d_split(dst + (size_t)NS, P1 + (row * N + col0) * 2, NS * 2u,
                                      &full[slot], pol, QPROD_TMA_PIECES);
                }
                ++issued;
            }
            // the last copy of every slot has landed before the block may leave (bounded),
            // also when a wait gave up
            for (int s = max(0, issued - NST); s < issued; ++s)
                mbar_wait(&full[s % NST], (s / NST) & 1, drain_budget(budget));
        }
        __syncwarp();
        // stay for the final cluster barrier: no block leaves while peers may still write to it
        if constexpr (CS > 1) cluster_sync_all();
        return;
    }

    // ---------------- consumers ----------------
    const int lane = tid & 31, warp = tid >> 5;
    const bool y_in_smem = (y != nullptr) && nrows <= QPROD_YMAX;
    const bool s_in_smem = (PREC == 2) && nrows <= QPROD_YMAX;
    if (y_in_smem)
        for (int i = tid; i < nrows; i += CONS) sy[i] = y[i0 + i];
    if (s_in_smem)
        for (int i = tid; i < nrows; i += CONS) ss[i] = rscale[i0 + i];
    const float4* x4 = reinterpret_cast<const float4*>(x + (size_t)rank * NS);
    float4 xu[V], acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        xu[v] = x4[tid + v * CONS];
        acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    named_barrier(1, CONS);
    float2 r2 = make_float2(0.f, 0.f);   // double-single ||r||^2 (block 0, thread 0)
    bool ok = true;
    int s_nowait = -1;   // first row whose parts this thread did not wait for (a wait gave up)
    auto row_scale = [&](int s) -> float {
        if constexpr (PREC == 2) return s_in_smem ? ss[s] : rscale[i0 + s];
        return 1.0f;
    };
    // Row s, first use: this warp's part of the block's dot product over its column
    // slice; lane 0 stores it in red[s & 1] and arrives on partbar[s & 1].  No
    // block-wide barrier: only the exchange warp waits for all warps (the consumer
    // warps otherwise run apart by up to the exchange's bound).
    auto warp_part = [&](int s) {
        const int slot = s % NST;
        if (ok && !mbar_wait(&full[slot], (s / NST) & 1, budget)) {
            set_error(ctrl, ERR_TIMEOUT);
            ok = false;
            s_nowait = s > 0 ? s - 1 : 0;   // the exchange of row s-1 is not awaited either
        }
        const unsigned char* sb = smem + (size_t)slot * S::STAGE_BYTES;
        float d0 = 0.f, d1 = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int ch = tid + v * CONS;
            if constexpr (PREC == 0) {
                const float4 a = reinterpret_cast<const float4*>(sb)[ch];
                d0 = fmaf(a.x, xu[v].x, d0);
                d1 = fmaf(a.y, xu[v].y, d1);
                d0 = fmaf(a.z, xu[v].z, d0);
                d1 = fmaf(a.w, xu[v].w, d1);
            } else if constexpr (PREC == 1) {   // hi + lo, each product exact-free of a join
                const uint2 h = reinterpret_cast<const uint2*>(sb)[ch];
                const uint2 l = reinterpret_cast<const uint2*>(sb + (size_t)NS * 2)[ch];
                d0 = fmaf(bf16_lo_f(h.x), xu[v].x, d0);
                d1 = fmaf(bf16_lo_f(l.x), xu[v].x, d1);
                d0 = fmaf(bf16_hi_f(h.x), xu[v].y, d0);
                d1 = fmaf(bf16_hi_f(l.x), xu[v].y, d1);
                d0 = fmaf(bf16_lo_f(h.y), xu[v].z, d0);
                d1 = fmaf(bf16_lo_f(l.y), xu[v].z, d1);
                d0 = fmaf(bf16_hi_f(h.y), xu[v].w, d0);
                d1 = fmaf(bf16_hi_f(l.y), xu[v].w, d1);
            } else {   // s q + c: the e4m3 part (d0, scaled once per row) and the correction (d1)
                const uint32_t q = reinterpret_cast<const uint32_t*>(sb)[ch];
                const uint2 c = reinterpret_cast<const uint2*>(sb + (size_t)NS)[ch];
                const float2 a01 = __half22float2(__half2(
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q & 0xffffu), __NV_E4M3)));
                const float2 a23 = __half22float2(__half2(
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q >> 16), __NV_E4M3)));
                d0 = fmaf(a01.x, xu[v].x, d0);
                d1 = fmaf(bf16_lo_f(c.x), xu[v].x, d1);
                d0 = fmaf(a01.y, xu[v].y, d0);
                d1 = fmaf(bf16_hi_f(c.x), xu[v].y, d1);
                d0 = fmaf(a23.x, xu[v].z, d0);
                d1 = fmaf(bf16_lo_f(c.y), xu[v].z, d1);
                d0 = fmaf(a23.y, xu[v].w, d0);
                d1 = fmaf(bf16_hi_f(c.y), xu[v].w, d1);
            }
        }
        float d;
        if constexpr (PREC == 2)
            d = fmaf(row_scale(s), d0, d1);
        else
            d = d0 + d1;
        d = warp_sum(d);
        if (lane == 0) {
            red[(s & 1) * WARPS + warp] = d;
            mbar_arrive(&partbar[s & 1]);
        }
    };
    // Software pipeline: the part of row s+1 is computed (and sent by the exchange
    // warp) before the cluster's parts of row s are awaited, hiding the exchange
    // latency.  Slot reuse: a peer writes slot s mod 4 for row s+4 only after it
    // has received this block's part of row s+2, which is sent only once all of
    // this block's warps have passed row s; the red[] and partbar[] pairs are
    // reused two rows later under the same argument.
    if (nrows > 0) warp_part(0);
    for (int s = 0; s < nrows; ++s) {
        if (s + 1 < nrows) warp_part(s + 1);
        const int b = s & 3;
        const uint32_t phase = (uint32_t)((s >> 2) & 1);
        if (ok) {
            bool got;
            if constexpr (CS > 1) got = mbar_try_wait_cluster(&xbar[b], phase);
            else got = mbar_try_wait(&xbar[b], phase);
            if (!got) {
                const long long t0 = clock64();
                for (;;) {
                    if constexpr (CS > 1) got = mbar_try_wait_cluster(&xbar[b], phase);
                    else got = mbar_try_wait(&xbar[b], phase);
                    if (got) break;
                    if (clock64() - t0 > budget) {
                        set_error(ctrl, ERR_TIMEOUT);
                        ok = false;
                        s_nowait = s;
                        break;
                    }
                }
            }
        }
        float dot = 0.f;
#pragma unroll
        for (int k = 0; k < CS; ++k) dot += xred[b * CS + k];
        float yi = 0.f;
        if (y != nullptr) yi = y_in_smem ? sy[s] : y[i0 + s];
        const float ri = dot - yi;
        if (rank == 0 && tid == 0) {
            r[i0 + s] = ri;
            r2 = ds_add(r2, ds_sq(ri));
        }
        const int slot = s % NST;
        const unsigned char* sb = smem + (size_t)slot * S::STAGE_BYTES;
        // Second use of row s: acc += r_i A_i over this block's columns.
        float rs = ri;
        if constexpr (PREC == 2) rs = ri * row_scale(s);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int ch = tid + v * CONS;
            if constexpr (PREC == 0) {
                const float4 a = reinterpret_cast<const float4*>(sb)[ch];
                acc[v].x = fmaf(ri, a.x, acc[v].x);
                acc[v].y = fmaf(ri, a.y, acc[v].y);
                acc[v].z = fmaf(ri, a.z, acc[v].z);
                acc[v].w = fmaf(ri, a.w, acc[v].w);
            } else if constexpr (PREC == 1) {
                const uint2 h = reinterpret_cast<const uint2*>(sb)[ch];
                const uint2 l = reinterpret_cast<const uint2*>(sb + (size_t)NS * 2)[ch];
                acc[v].x = fmaf(ri, bf16_lo_f(h.x) + bf16_lo_f(l.x), acc[v].x);
                acc[v].y = fmaf(ri, bf16_hi_f(h.x) + bf16_hi_f(l.x), acc[v].y);
                acc[v].z = fmaf(ri, bf16_lo_f(h.y) + bf16_lo_f(l.y), acc[v].z);
                acc[v].w = fmaf(ri, bf16_hi_f(h.y) + bf16_hi_f(l.y), acc[v].w);
            } else {   // (r_i s_i) q + r_i c
                const uint32_t q = reinterpret_cast<const uint32_t*>(sb)[ch];
                const uint2 c = reinterpret_cast<const uint2*>(sb + (size_t)NS)[ch];
                const float2 a01 = __half22float2(__half2(
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q & 0xffffu), __NV_E4M3)));
                const float2 a23 = __half22float2(__half2(
                    __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q >> 16), __NV_E4M3)));
                acc[v].x = fmaf(ri, bf16_lo_f(c.x), fmaf(rs, a01.x, acc[v].x));
                acc[v].y = fmaf(ri, bf16_hi_f(c.x), fmaf(rs, a01.y, acc[v].y));
                acc[v].z = fmaf(ri, bf16_lo_f(c.y), fmaf(rs, a23.x, acc[v].z));
                acc[v].w = fmaf(ri, bf16_hi_f(c.y), fmaf(rs, a23.y, acc[v].w));
            }
        }
        // this warp is done with row s: release its slot to the producer
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
    }

    // ---------------- epilogue ----------------
    float4* out4 = reinterpret_cast<float4*>(gpart + (size_t)cidx * N + (size_t)rank * NS);
#pragma unroll
    for (int v = 0; v < V; ++v) out4[tid + v * CONS] = acc[v];
    if (tid == 0) {
        sflag[0] = 0;
        if (rank == 0) {   // one arrival per cluster: the last of the G clusters sums ||r||^2
            r2part[cidx] = r2;
            __threadfence();
            const unsigned t = atomicAdd(&ctrl->ticket_prod, 1u);
            if (t == (unsigned)G - 1u) {
                __threadfence();
                ctrl->ticket_prod = 0u;
                sflag[0] = 1;
            }
        }
    }
    named_barrier(1, CONS);
    if (sflag[0]) {
        float2 v = make_float2(0.f, 0.f);
        for (int b = tid; b < G; b += CONS) v = ds_add(v, __ldcg(r2part + b));
        v = warp_sum_ds(v);
        if ((tid & 31) == 0) dred[tid >> 5] = v;
        named_barrier(1, CONS);
        if (tid == 0) {
            float2 t = dred[0];
            for (int w = 1; w < WARPS; ++w) t = ds_add(t, dred[w]);
            ctrl->r2 = ds_value(t);
        }
    }
    __syncwarp();
    if constexpr (CS > 1) {
        cluster_sync_all();
        // After a wait gave up, parts of the rows no longer awaited may still be on their
        // way into this block's shared memory (stores that complete on its barriers).
        // Every block has issued all of its parts by the cluster barrier above, so thread
        // 0 waits for them (bounded) before the block retires.
        if (tid == 0 && s_nowait >= 0)
            for (int s = s_nowait; s < nrows; ++s)
                mbar_wait(&xbar[s & 3], (uint32_t)((s >> 2) & 1), drain_budget(budget));
    }
}

// ---------------------------------------------------------------------------
// Quantisation of a binary32 A into the split / reduced storages.
// ---------------------------------------------------------------------------
__global__ void k_split_bf16x2(const float4* __restrict__ A, uint2* __restrict__ hi,
                               uint2* __restrict__ lo, long long total4)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 a = A[i];
        const float av[4] = {a.x, a.y, a.z, a.w};
        unsigned short h[4], l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat16 hb = __float2bfloat16_rn(av[k]);
            const float rem = av[k] - __bfloat162float(hb);    // exact
            const __nv_bfloat16 lb = __float2bfloat16_rn(rem);
            h[k] = __bfloat16_as_ushort(hb);
            l[k] = __bfloat16_as_ushort(lb);
        }
        hi[i] = make_uint2((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16));
        lo[i] = make_uint2((uint32_t)l[0] | ((uint32_t)l[1] << 16), (uint32_t)l[2] | ((uint32_t)l[3] << 16));
    }
}

// One block per row: s = max|A_i.| / 448, q = e4m3(A / s), c = bf16(A - s q).
__global__ void __launch_bounds__(256) k_quant_fp8(const float* __restrict__ A, int N,
                                                   unsigned char* __restrict__ q,
                                                   unsigned short* __restrict__ c,
                                                   float* __restrict__ scale)
{
    __shared__ float wmax[8];
    const float* a = A + (size_t)blockIdx.x * N;
    float mx = 0.f;
    for (int j = threadIdx.x; j < N; j += blockDim.x) mx = fmaxf(mx, fabsf(a[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t = fmaxf(t, wmax[w]);
        wmax[0] = t;
    }
    __syncthreads();
    const float s = wmax[0] > 0.f ? wmax[0] / 448.0f : 1.0f;
    if (threadIdx.x == 0) scale[blockIdx.x] = s;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float v = a[j];
        const __nv_fp8_storage_t qq = __nv_cvt_float_to_fp8(v / s, __NV_SATFINITE, __NV_E4M3);
        const float qf = __half2float(__half(__nv_cvt_fp8_to_halfraw(qq, __NV_E4M3)));
        const float rem = __fmaf_rn(-s, qf, v);   // one rounding of v - s q
        q[(size_t)blockIdx.x * N + j] = (unsigned char)qq;
        c[(size_t)blockIdx.x * N + j] = __bfloat16_as_ushort(__float2bfloat16_rn(rem));
    }
}

void launch_split_bf16x2(const float* A, void* hi, void* lo, long long count, cudaStream_t s)
{
    const long long total4 = count / 4;
    int grid = (int)((total4 + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    k_split_bf16x2<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(A),
                                        reinterpret_cast<uint2*>(hi), reinterpret_cast<uint2*>(lo),
                                        total4);
}

void launch_quant_fp8(const float* A, int m, int N, void* q, void* c, float* scale, cudaStream_t s)
{
    k_quant_fp8<<<m, 256, 0, s>>>(A, N, reinterpret_cast<unsigned char*>(q),
                                  reinterpret_cast<unsigned short*>(c), scale);
}

// ---------------------------------------------------------------------------
// Shape table: (precision, n) -> (V, CS, CONS, NST).  N = n^2 = 4 CONS V CS.
// ---------------------------------------------------------------------------
#define TVCS_QPROD_TABLE(X)                                                              \
    X(0, 192, 9, 2, 512, 3) X(0, 256, 8, 4, 512, 3)                                      \
    X(1, 32, 1, 1, 256, 3) X(1, 64, 2, 1, 512, 3) X(1, 128, 8, 1, 512, 3)                \
    X(1, 192, 9, 2, 512, 3) X(1, 256, 8, 4, 512, 3)                                      \
    X(2, 32, 1, 1, 256, 4) X(2, 64, 2, 1, 512, 4) X(2, 128, 8, 1, 512, 4)                \
    X(2, 192, 9, 2, 512, 4) X(2, 256, 8, 4, 512, 4)

template <int PREC, int V, int CS, int CONS, int NST>
static cudaError_t qconfigure_t()
{
    using S = QShape<PREC, V, CS, CONS, NST>;
    return cudaFuncSetAttribute(k_products_q<PREC, V, CS, CONS, NST>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
}

template <int PREC, int V, int CS, int CONS, int NST>
static int qmax_clusters_t()
{
    using S = QShape<PREC, V, CS, CONS, NST>;
    if (qconfigure_t<PREC, V, CS, CONS, NST>() != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (CS == 1) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return sms;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS, 1, 1);
    cfg.blockDim = dim3(S::THREADS, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_products_q<PREC, V, CS, CONS, NST>, &cfg) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int PREC, int V, int CS, int CONS, int NST>
static void qlaunch_t(int clusters, const QProdArgs& a, cudaStream_t s)
{
    using S = QShape<PREC, V, CS, CONS, NST>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * CS, 1, 1);
    cfg.blockDim = dim3(S::THREADS, 1, 1);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = CS > 1 ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_products_q<PREC, V, CS, CONS, NST>, a.P0, a.P1, a.rscale, a.m, a.x,
                       a.y, a.r, a.gpart, a.r2part, a.ctrl, a.mode,
                       (cudaGraphConditionalHandle)a.cond, a.set_cond, a.budget);
}

bool qprod_supported(int prec, int n)
{
#define X(PR, NN, V, CS, CONS, NST) \
    if (prec == PR && n == NN) return true;
    TVCS_QPROD_TABLE(X)
#undef X
    return false;
}

int qprod_cluster_size(int prec, int n)
{
#define X(PR, NN, V, CS, CONS, NST) \
    if (prec == PR && n == NN) return CS;
    TVCS_QPROD_TABLE(X)
#undef X
    return 0;
}

// Number of clusters (= partials) to launch: every row group on the GPU at once.
int qprod_grid_clusters(int prec, int n, int m)
{
#define X(PR, NN, V, CS, CONS, NST)                                   \
    if (prec == PR && n == NN) {                                      \
        int c = qmax_clusters_t<PR, V, CS, CONS, NST>();              \
        if (c <= 0) return 0;                                         \
        return c < m ? c : m;                                         \
    }
    TVCS_QPROD_TABLE(X)
#undef X
    return 0;
}

void launch_qproducts(int prec, int n, int clusters, const QProdArgs& a, cudaStream_t s)
{
#define X(PR, NN, V, CS, CONS, NST)                          \
    if (prec == PR && n == NN) {                             \
        qlaunch_t<PR, V, CS, CONS, NST>(clusters, a, s);     \
        return;                                              \
    }
    TVCS_QPROD_TABLE(X)
#undef X
}

}  // namespace tvcs
