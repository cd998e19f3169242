// Shared device definitions of the TV/L2 solver library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tvcs {

// Device-side control block of one handle.  Written by single threads at
// kernel boundaries (never concurrently within one kernel), read by all.
struct Ctrl {
    int it;            // iterations completed in the current run
    int max_iter;      // cap of the current run
    int done;          // 1: the run has ended; later iterations are skipped
    int skip;          // 1: the current iteration is skipped (copied from done by the w-step)
    int pending;       // 1: the multiplier update of eq. (udlamb) for the last u is pending
    int stop_by_tol;   // 1: eq. (stop) ended the run
    int loops;         // executions of the graph loop body (hard bound on the loop)
    int loops_max;
    unsigned ticket_fft;   // last-block tickets of the reducing kernels
    unsigned ticket_prod;
    unsigned ticket_fin;
    unsigned ticket_w;
    unsigned ticket_gather;
    int wpar;          // which copy of the double-buffered w/lambda is current
    int error;         // ERR_* below, first error wins
    int algo;          // 0 IADM, 1 FTVCS
    double tol;
    double du2;        // ||u^{k+1} - u^k||^2 of the last iteration
    double u2;         // ||u^k||^2 of the last iteration
    double r2;         // ||A u - f||^2 at the current u
    double tv;         // sum_i ||D_i u||
    double kkt_p2;     // ||w - D u||^2
    double kkt_d2;     // ||D^T lambda + mu g||^2
    double lam_max;    // max_i ||lambda_i||
    double vec2;       // ||g||^2 of the last gathered vector (power iteration)
    unsigned long long gbar;  // monotone arrival counter of the product kernel's grid barrier
    int nact;          // batch control block: images still iterating (the GEMMs' active columns)
};

// sqrt(du2 / u2), the relative change of eq. (stop) (host side).
inline double ctrl_relchg(const Ctrl& c)
{
    return c.u2 > 0.0 ? sqrt(c.du2 / c.u2) : (c.du2 > 0.0 ? INFINITY : 0.0);
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

enum { ERR_NONE = 0, ERR_TIMEOUT = 1, ERR_NONFINITE = 2 };

// Iteration-kernel modes.
enum { MODE_PLAIN = 0, MODE_ITER = 1 };

__device__ __forceinline__ void set_error(Ctrl* c, int code)
{
    atomicCAS(&c->error, ERR_NONE, code);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier (PTX ISA, "Parallel Synchronization and Communication") ----
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t tx)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(tx)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of an mbarrier: false when `budget` SM cycles pass.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// Bound of the waits that let a block's own asynchronous copies (or MMAs) land
// after another wait gave up: never below 2^31 SM cycles (about a second), so
// that a short timeout_cycles cannot make a block retire while its copies are
// still writing to its shared memory.
constexpr long long DRAIN_FLOOR_CYCLES = 1LL << 31;
__device__ __forceinline__ long long drain_budget(long long budget)
{
    return budget > DRAIN_FLOOR_CYCLES ? budget : DRAIN_FLOOR_CYCLES;
}

// ---- bulk asynchronous copy global -> shared (TMA, non-tensor form) ----
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                            uint64_t* bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// The same copy issued as `pieces` bulk copies of nearly equal size (each a
// multiple of 16 bytes; bytes must be one), completing on the same barrier.
__device__ __forceinline__ void tma_load_1d_split(void* dst_smem, const void* src_gmem,
                                                  uint32_t bytes, uint64_t* bar, uint64_t policy,
                                                  int pieces)
{
    const uint32_t piece = ((bytes / (uint32_t)pieces) + 15u) & ~15u;
    for (uint32_t off = 0; off < bytes; off += piece) {
        const uint32_t len = bytes - off < piece ? bytes - off : piece;
        tma_load_1d(static_cast<unsigned char*>(dst_smem) + off,
                    static_cast<const unsigned char*>(src_gmem) + off, len, bar, policy);
    }
}

// ---- bulk prefetch global -> L2 (no completion to wait for) ----
// src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void* src_gmem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src_gmem), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Programmatic dependent launch.  pdl_wait: until the preceding grid in the
// stream has completed and its memory is visible (a no-op when the launch had
// no programmatic dependency).  pdl_release: the next grid may be launched
// from now on (it still waits for this grid's completion before it reads
// what this grid writes).
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The two halves of a cluster barrier, executed by every thread of the cluster:
// writes before arrive (shared, distributed shared, global) are visible after wait.
__device__ __forceinline__ void cluster_arrive()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void pdl_release()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_wait_then_release()
{
    pdl_wait();
    pdl_release();
}

// Named barrier over `count` threads (a multiple of 32).
__device__ __forceinline__ void named_barrier(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of squares in binary32 double-single arithmetic: a value is the
// unevaluated pair hi + lo.  ds_sq gives x^2 exactly (the FMA residual of the
// rounded product), ds_add is Knuth's TwoSum followed by a fast
// renormalisation, so a sum of non-negative terms keeps about 44 significant
// bits.  Binary64 arithmetic runs at a small fraction of the binary32 rate on
// this part, so reductions stay in binary32 and only ds_value converts.  The
// _rn intrinsics keep the compiler from contracting the error terms into FMAs.
__device__ __forceinline__ float2 ds_sq(float x)
{
    const float p = __fmul_rn(x, x);
    return make_float2(p, __fmaf_rn(x, x, -p));
}

__device__ __forceinline__ float2 ds_add(float2 a, float2 b)
{
    const float s = __fadd_rn(a.x, b.x);
    const float v = __fsub_rn(s, a.x);
    const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v));
    const float t = __fadd_rn(__fadd_rn(a.y, b.y), e);
    const float h = __fadd_rn(s, t);
    return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}

__device__ __forceinline__ double ds_value(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 warp_sum_ds(float2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.x, o),
                                     __shfl_xor_sync(0xffffffffu, v.y, o));
        v = ds_add(v, w);
    }
    return v;
}

// Block-wide double-single sums of two values per thread (one pair of
// barriers); results valid in thread 0.  `scratch` holds >= 64 float2.
__device__ __forceinline__ void block_sum_ds2(float2& a, float2& b, float2* scratch)
{
    a = warp_sum_ds(a);
    b = warp_sum_ds(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        scratch[wid] = a;
        scratch[32 + wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 1; i < nw; ++i) {
            a = ds_add(a, scratch[i]);
            b = ds_add(b, scratch[32 + i]);
        }
    }
}

__device__ __forceinline__ float2 block_sum_ds(float2 a, float2* scratch)
{
    a = warp_sum_ds(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 1; i < nw; ++i) a = ds_add(a, scratch[i]);
    }
    return a;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
// `scratch` holds >= 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* scratch)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += scratch[i];
    }
    return s;
}

__device__ __forceinline__ double block_max(double v, double* scratch)
{
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s = fmax(s, scratch[i]);
    }
    return s;
}

// Block-wide sum over an array of per-block binary64 partials (fixed order
// per thread, fixed tree across threads: deterministic).  All threads call;
// result valid in thread 0.
__device__ __forceinline__ double block_sum_array(const double* __restrict__ a, int count,
                                                  int stride, double* scratch)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += a[(size_t)i * stride];
    return block_sum(s, scratch);
}

__device__ __forceinline__ double block_max_array(const double* __restrict__ a, int count,
                                                  int stride, double* scratch)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s = fmax(s, a[(size_t)i * stride]);
    return block_max(s, scratch);
}

// Last-block detection over the gridDim.x blocks that share `ticket` (one row
// of the grid; batched kernels give every image, grid row y, its own ticket):
// returns true in exactly one block (the last to arrive), after the prior
// global writes of every block are visible to it.  The ticket is reset by that
// block.  Call from thread 0 only.
__device__ __forceinline__ bool last_block_arrive(unsigned* ticket)
{
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    const bool last = (t == gridDim.x - 1);
    if (last) {
        __threadfence();
        *ticket = 0u;
    }
    return last;
}

// Whole-block version: every thread calls it after the block's partials are
// written; returns true in every thread of the last block.
__device__ __forceinline__ bool last_block_all(unsigned* ticket, int* sflag)
{
    __syncthreads();
    if (threadIdx.x == 0) *sflag = last_block_arrive(ticket) ? 1 : 0;
    __syncthreads();
    return *sflag != 0;
}

}  // namespace tvcs
