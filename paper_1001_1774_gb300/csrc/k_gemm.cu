// Row a8: the two products of many images that share one encoding matrix, as
// tensor-core GEMMs (Xiao & Yang, eq. (line) for every image at once):
//     R = A U - F        (m x B,  K = n^2)
//     G = A^T R          (n^2 x B, K = m)
// with U = [u_1 ... u_B], F = [f_1 ... f_B].  Both run as K-major ("TN") GEMMs
// D = X Y^T with the operand X = A (m x n^2) or A^T (n^2 x m) held in
// tile-contiguous planes (k_tile_planes): each 128 x 64 tile of X is one
// contiguous 16 KB block, so that a TMA load reads whole DRAM pages instead of
// 128 pieces of 128 bytes a row pitch apart.
//
// Precision: every operand is split into bfloat16 hi + lo planes (hi =
// bf16(v), lo = bf16(v - hi), round to nearest even) and
//     D = X_hi Y_hi + X_hi Y_lo + X_lo Y_hi
// accumulates in binary32 in tensor memory (the dropped X_lo Y_lo term is
// below 2^-16 of |X||Y|).
//
// Kernel: one 128 x BN output tile per MMA (tcgen05.mma, cta_group::1,
// kind::f16, BF16 inputs, FP32 accumulator in TMEM), K in blocks of 64.  Warp 0
// streams the four operand tiles of a K block into a 2-stage shared-memory ring
// with tiled TMA loads (128-byte swizzle, the canonical K-major layout of the
// MMA's shared-memory descriptors); one thread of warp 1 issues the 12 MMAs of
// a K block and commits them to the stage's "empty" barrier; warps 2-5 drain a
// finished accumulator (tcgen05.ld) into a workspace.  Work is split by
// "stream-K": the tiles x K-blocks iterations are divided evenly over the
// blocks, so a block may own the tail of one tile and the head of the next
// (two accumulators in TMEM let the MMAs of the second start while the first
// drains).  Each (block, segment) writes a partial tile; a fix-up kernel adds
// the partials of every tile in K order (deterministic) and applies the
// epilogue.  Every wait is bounded; on a timeout the kernel records the error,
// lets its copies land and frees its tensor memory.  k_gemm_bf16x3_pair runs the
// same GEMM on clusters of two blocks (tcgen05 cta_group::2, 256-row tiles).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace tvcs {

constexpr int GM_BM = 128;
constexpr int GM_BK = 64;
constexpr int GM_BN = 256;
constexpr int GM_NST = 2;
constexpr uint32_t GM_A_BYTES = GM_BM * GM_BK * 2;            // 16 KB
constexpr uint32_t GM_B_BYTES = GM_BN * GM_BK * 2;            // 32 KB
constexpr uint32_t GM_YBOX_BYTES = GEMM_Y_BOX * GM_BK * 2;    // one 32-row box of a Y tile (4 KB)
constexpr uint32_t GM_STAGE = 2 * GM_A_BYTES + 2 * GM_B_BYTES; // 96 KB
constexpr uint32_t GM_TMEM_COLS = 2 * GM_BN;                  // two accumulators
constexpr size_t GM_SMEM = 1024 + GM_NST * GM_STAGE + 256;

// ---- tcgen05 / TMA wrappers (PTX ISA: tcgen05 family, cp.async.bulk.tensor) ----
// Tiled 2D TMA load with an L2 cache policy (createpolicy): the operand A streams
// through once per GEMM (evict first), the small image operand is re-read by every
// block (evict last), so that A does not push it, or the partial tiles, out of L2.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile with 128-byte swizzle,
// 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = nb
// (a multiple of 16, at most BN).
__host__ __device__ constexpr uint32_t gemm_idesc(int nb)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nb >> 3) << 17) |
           ((uint32_t)(GM_BM >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// The GEMM.  tiles_m output tiles of 128 rows, kblocks K blocks of 64; block c
// owns iterations [c W / G, (c+1) W / G) of W = tiles_m * kblocks.  Partial
// tile (c, j) goes to ws + (c * smax + j) * BN * 128 as [column][row].  Only
// the first nb = roundup(min(ncols, *nact), 32) columns take part: the Y tile
// is loaded as ceil(nb / 64) boxes of 64 rows, the MMAs run with N = nb and the
// partial tiles get nb columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(192, 1)
    k_gemm_bf16x3(const __grid_constant__ CUtensorMap tXh, const __grid_constant__ CUtensorMap tXl,
                  const __grid_constant__ CUtensorMap tYh, const __grid_constant__ CUtensorMap tYl,
                  int tiles_m, int kblocks, float* __restrict__ ws, int smax,
                  Ctrl* __restrict__ ctrl, int check_skip, long long budget,
                  int ncols, const int* __restrict__ nact)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + GM_NST * GM_STAGE);
    uint64_t* empty = full + GM_NST;
    uint64_t* tfull = empty + GM_NST;    // [2] accumulator ready
    uint64_t* tempty = tfull + 2;        // [2] accumulator drained
    uint64_t* mdrain = tempty + 2;       // the issuer's MMAs have finished (after a timeout)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mdrain + 1);

    if (check_skip && ctrl->skip) return;
    int nb = min(ncols, GM_BN);   // columns of the MMAs and of the partial tiles
    if (nact) nb = min(nb, *nact);
    nb = min(GM_BN, max(32, (nb + 31) & ~31));
    const int ybox = (nb + GEMM_Y_BOX - 1) / GEMM_Y_BOX;
    const uint32_t stage_bytes = 2 * GM_A_BYTES + 2 * (uint32_t)ybox * GM_YBOX_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long W = (long long)tiles_m * kblocks;
    const int G = gridDim.x;
    const long long w0 = W * blockIdx.x / G, w1 = W * (blockIdx.x + 1) / G;

    if (tid == 0) {
        for (int s = 0; s < GM_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);
        }
        mbar_init(mdrain, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(GM_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            bool ok = true;
            const uint64_t pol_x = l2_policy_evict_first(), pol_y = l2_policy_evict_last();
            auto load_x = [&](long long it_, long long w) {   // X: tile-contiguous A or A^T
                const int s = (int)(it_ % GM_NST);
                const int t = (int)(w / kblocks), kb = (int)(w % kblocks);
                unsigned char* st = smem + (size_t)s * GM_STAGE;
                mbar_arrive_expect_tx(&full[s], stage_bytes);
                const int xrow = (t * kblocks + kb) * GM_BM;
                tma_load_2d(st, &tXh, 0, xrow, &full[s], pol_x);
                tma_load_2d(st + GM_A_BYTES, &tXl, 0, xrow, &full[s], pol_x);
            };
            auto load_y = [&](long long it_, long long w) {   // Y: the images' planes
                const int s = (int)(it_ % GM_NST);
                const int kb = (int)(w % kblocks);
                unsigned char* st = smem + (size_t)s * GM_STAGE;
                for (int j = 0; j < ybox; ++j) {   // 32-row boxes, 1024-byte aligned
                    tma_load_2d(st + 2 * GM_A_BYTES + j * GM_YBOX_BYTES, &tYh, kb * GM_BK,
                                j * GEMM_Y_BOX, &full[s], pol_y);
                    tma_load_2d(st + 2 * GM_A_BYTES + GM_B_BYTES + j * GM_YBOX_BYTES, &tYl,
                                kb * GM_BK, j * GEMM_Y_BOX, &full[s], pol_y);
                }
            };
            // The first stages' X halves do not depend on the preceding kernel: under a
            // programmatic dependent launch they stream in before its end; Y (the
            // images' planes it writes) only after the wait.
            const long long npre = min((long long)GM_NST, w1 - w0);
            for (long long j = 0; j < npre; ++j) load_x(j, w0 + j);
            pdl_wait();
            for (long long j = 0; j < npre; ++j) load_y(j, w0 + j);
            long long it = npre;
            for (long long w = w0 + npre; w < w1; ++w, ++it) {
                const int s = (int)(it % GM_NST);
                if (!mbar_wait(&empty[s], (uint32_t)((it / GM_NST) - 1) & 1u, budget)) {
                    set_error(ctrl, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                load_x(it, w);
                load_y(it, w);
            }
            // leave no copy in flight
            const long long n_issued = it;
            for (long long j = (n_issued > GM_NST ? n_issued - GM_NST : 0); j < n_issued; ++j)
                mbar_wait(&full[j % GM_NST], (uint32_t)(j / GM_NST) & 1u, drain_budget(budget));
            (void)ok;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = gemm_idesc(nb);
            bool ok = true;
            long long it = 0;
            int seg = 0;
            long long w = w0;
            while (w < w1 && ok) {
                const int t = (int)(w / kblocks);
                const long long wend = min(w1, (long long)(t + 1) * kblocks);
                const int acc = seg & 1;
                if (seg >= 2 && !mbar_wait(&tempty[acc], (uint32_t)((seg >> 1) - 1) & 1u, budget)) {
                    set_error(ctrl, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * GM_BN);
                bool first = true;
                for (; w < wend; ++w, ++it) {
                    const int s = (int)(it % GM_NST);
                    if (!mbar_wait(&full[s], (uint32_t)(it / GM_NST) & 1u, budget)) {
                        set_error(ctrl, ERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + (size_t)s * GM_STAGE);
                    const uint32_t xh = base, xl = base + GM_A_BYTES;
                    const uint32_t yh = base + 2 * GM_A_BYTES, yl = yh + GM_B_BYTES;
#pragma unroll
                    for (int k = 0; k < GM_BK / 16; ++k) {
                        const uint32_t off = k * 32;   // 16 bf16 along K
                        tc_mma(dt, sw128_desc(xh + off), sw128_desc(yh + off), idesc, first ? 0u : 1u);
                        first = false;
                        tc_mma(dt, sw128_desc(xh + off), sw128_desc(yl + off), idesc, 1u);
                        tc_mma(dt, sw128_desc(xl + off), sw128_desc(yh + off), idesc, 1u);
                    }
                    tc_commit(&empty[s]);   // frees the stage when these MMAs finish
                }
                if (!ok) break;
                tc_commit(&tfull[acc]);     // accumulator ready when all MMAs finish
                ++seg;
            }
            if (!ok) {   // a wait gave up: the MMAs already issued finish before TMEM is freed
                tc_commit(mdrain);
                mbar_wait(mdrain, 0u, drain_budget(budget));
            }
        }
    } else {
        // ---------------- epilogue warps 2..5: TMEM -> workspace ----------------
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        int seg = 0;
        long long w = w0;
        bool ok = true;
        while (w < w1 && ok) {
            const int t = (int)(w / kblocks);
            const long long wend = min(w1, (long long)(t + 1) * kblocks);
            const int acc = seg & 1;
            if (!mbar_wait(&tfull[acc], (uint32_t)(seg >> 1) & 1u, budget)) {
                set_error(ctrl, ERR_TIMEOUT);
                ok = false;
                break;
            }
            tc_fence_after();
            float* dst = ws + ((size_t)blockIdx.x * smax + seg) * (size_t)GM_BN * GM_BM;
            for (int c0 = 0; c0 < nb; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * GM_BN + c0), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[(size_t)(c0 + j) * GM_BM + q * 32 + lane] = v[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            w = wend;
            ++seg;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(GM_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// The same GEMM on CTA pairs (cta_group::2): a cluster of two blocks computes a
// 256 x BN tile with M = 256 MMAs issued by the even block.  Each block holds
// its 128 rows of the X tile and half of the Y tile (rows [rank nb/2, (rank+1)
// nb/2) of the nb running columns); the MMA reads the X half of each block and
// both Y halves, and writes each block's 128 rows of the accumulator into that
// block's tensor memory.  Per block and K block the ring then holds 64 KB (three
// stages) and the MMAs read 96 KB of shared memory instead of 144 KB, the Y
// operand is fetched once per pair, and the two blocks' epilogues drain their
// own halves.
//   Barriers: both blocks' producers fill their own stages with tensor copies
// that complete on the even block's "full" barrier (cta_group::2 copies may
// signal a barrier in either block of the pair), which the even block's
// producer arms with both blocks' bytes, so the even block's MMAs start when
// both halves are in and no thread hands a stage from one block to the other.
// The MMA commits arrive on the "empty" and "accumulator ready" barriers of
// both blocks (multicast); the odd block's epilogue warps arrive on the even
// block's "accumulator drained" barrier.  Stream-K over pairs: pair p owns
// iterations [p W / P, (p+1) W / P) of W = tiles x kblocks (256-row tiles);
// block c of the grid writes its partial tiles to ws + (c smax + j) BN 128, the
// 128-row half tile 2 t + rank of the pair's tile t.
// ---------------------------------------------------------------------------
// NT: N tiles of 256 columns (images) per X tile, 1 or 2.  With two, TMEM holds
// one accumulator per N tile (512 columns) and A is streamed once for up to 512
// images.  A stage holds the X tile and this block's half of each N tile's
// running columns in 32-row boxes, so its size follows the running images (64 KB
// for 256, 72 KB for 300, 96 KB for 512), and the ring takes as many stages of
// that size as 225 KB hold (at most six).
constexpr uint32_t GP_RING_BYTES = 225 * 1024;
constexpr int GP_NST_MAX = 6;
constexpr size_t GP_SMEM = 1024 + GP_RING_BYTES + 256;
template <int NT>
struct PairCfg {
    static constexpr int NSETS = 2 / NT;                              // accumulator sets in TMEM
};

__device__ __forceinline__ void tc_mma_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the barrier at the same shared-memory offset in every block of the
// cluster named in cta_mask once the MMAs issued so far have finished.
__device__ __forceinline__ void tc_commit_pair(uint64_t* bar, uint16_t cta_mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(smem_u32(bar)),
        "h"(cta_mask)
        : "memory");
}

__device__ __forceinline__ uint32_t gemm_cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t gemm_map_peer(const void* local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}

// Tensor copy into this block's shared memory that completes on the barrier at
// shared::cluster address `bar` in either block of the CTA pair (cta_group::2):
// both blocks' copies of a stage complete on the even block's barrier.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void gemm_arrive_remote(uint32_t addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr)
                 : "memory");
}

// Bounded wait with cluster-scope acquire: the phase may have been completed by
// the other block of the pair (its arrival or an MMA commit it issued).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, long long budget)
{
    auto try_once = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (try_once()) return true;
    const long long t0 = clock64();
    while (!try_once()) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

__device__ __forceinline__ void gemm_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// Instruction descriptor of the pair's MMA: M = 256 (128 rows in each block).
__host__ __device__ constexpr uint32_t gemm_idesc_pair(int nb)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nb >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

template <int NT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(192, 1)
    k_gemm_bf16x3_pair(const __grid_constant__ CUtensorMap tXh, const __grid_constant__ CUtensorMap tXl,
                       const __grid_constant__ CUtensorMap tYh, const __grid_constant__ CUtensorMap tYl,
                       int tiles, int kblocks, float* __restrict__ ws, int smax,
                       Ctrl* __restrict__ ctrl, int check_skip, long long budget, int ncols,
                       const int* __restrict__ nact)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int NSETS = PairCfg<NT>::NSETS;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + GP_RING_BYTES);
    uint64_t* empty = full + GP_NST_MAX;
    uint64_t* tfull = empty + GP_NST_MAX;   // [NSETS] accumulator set ready
    uint64_t* tempty = tfull + 2;        // [NSETS] accumulator set drained (both blocks; used on the even one)
    uint64_t* mdrain = tempty + 2;       // the issuer's MMAs have finished (after a timeout)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mdrain + 1);

    if (check_skip && ctrl->skip) return;   // the same for every block of the grid
    int ntot = min(ncols, NT * GM_BN);      // running columns
    if (nact) ntot = min(ntot, *nact);
    // per N tile: MMA columns, Y rows per block, 32-row boxes, offset in a stage
    int nbj[NT], nbh[NT], ybox[NT];
    uint32_t yoff[NT];
    uint32_t stage_bytes = 2 * GM_A_BYTES;   // a multiple of 4 KB: stages stay 1024-byte aligned
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int rem = ntot - j * GM_BN;
        nbj[j] = j == 0 ? min(GM_BN, max(32, (rem + 31) & ~31))
                        : (rem > 0 ? min(GM_BN, (rem + 31) & ~31) : 0);
        nbh[j] = nbj[j] / 2;
        ybox[j] = (nbh[j] + GEMM_Y_BOX - 1) / GEMM_Y_BOX;
        yoff[j] = stage_bytes;   // hi plane, then lo plane
        stage_bytes += 2 * (uint32_t)ybox[j] * GM_YBOX_BYTES;
    }
    const int GP_NST = min(GP_NST_MAX, (int)(GP_RING_BYTES / stage_bytes));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = gemm_cluster_rank();
    const bool lead = rank == 0;
    const long long W = (long long)tiles * kblocks;
    const int P = gridDim.x >> 1, pair = blockIdx.x >> 1;
    const long long w0 = W * pair / P, w1 = W * (pair + 1) / P;

    if (tid == 0) {
        for (int s = 0; s < GP_NST_MAX; ++s) {
            mbar_init(&full[s], 1);   // even block: its producer's arrival, both blocks' bytes
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NSETS; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 8);
        }
        mbar_init(mdrain, 1);
        fence_mbar_init();
    }
    if (warp == 1) {   // one warp of each block of the pair, together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(GM_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    gemm_cluster_sync();   // both blocks' barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both blocks) ----------------
            bool ok = true;
            const uint64_t pol_x = l2_policy_evict_first(), pol_y = l2_policy_evict_last();
            // every copy of a stage, in either block, completes on the even block's
            // full barrier, which its producer arms with both blocks' bytes
            const uint32_t full_lead = gemm_map_peer(full, 0);
            auto load_x = [&](long long it_, long long w) {
                const int s = (int)(it_ % GP_NST);
                const int t = (int)(w / kblocks), kb = (int)(w % kblocks);
                unsigned char* st = smem + (size_t)s * stage_bytes;
                if (lead) mbar_arrive_expect_tx(&full[s], 2 * stage_bytes);
                // 128-row tile 2 t + rank of the tile-contiguous X (past the last one: zeros)
                const int xrow = ((2 * t + (int)rank) * kblocks + kb) * GM_BM;
                const uint32_t fb = full_lead + (uint32_t)(s * 8);
                tma_load_2d_pair(st, &tXh, 0, xrow, fb, pol_x);
                tma_load_2d_pair(st + GM_A_BYTES, &tXl, 0, xrow, fb, pol_x);
            };
            auto load_y = [&](long long it_, long long w) {
                const int s = (int)(it_ % GP_NST);
                const int kb = (int)(w % kblocks);
                unsigned char* st = smem + (size_t)s * stage_bytes;
                const uint32_t fb = full_lead + (uint32_t)(s * 8);
#pragma unroll
                for (int n = 0; n < NT; ++n) {       // this block's half of each N tile
                    unsigned char* yst = st + yoff[n];
                    for (int j = 0; j < ybox[n]; ++j) {   // 32-row boxes, 1024-byte aligned
                        const int yrow = n * GM_BN + (int)rank * nbh[n] + j * GEMM_Y_BOX;
                        tma_load_2d_pair(yst + j * GM_YBOX_BYTES, &tYh, kb * GM_BK, yrow, fb, pol_y);
                        tma_load_2d_pair(yst + (ybox[n] + j) * GM_YBOX_BYTES, &tYl, kb * GM_BK, yrow, fb,
                                         pol_y);
                    }
                }
            };
            // the first stages' X halves before the wait on the preceding kernel, Y after it
            const long long npre = min((long long)GP_NST, w1 - w0);
            for (long long j = 0; j < npre; ++j) load_x(j, w0 + j);
            pdl_wait();
            for (long long j = 0; j < npre; ++j) load_y(j, w0 + j);
            long long it = npre;
            for (long long w = w0 + npre; w < w1; ++w, ++it) {
                const int s = (int)(it % GP_NST);
                if (!mbar_wait_cluster(&empty[s], (uint32_t)((it / GP_NST) - 1) & 1u, budget)) {
                    set_error(ctrl, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                load_x(it, w);
                load_y(it, w);
            }
            // leave no copy in flight: the even block's full barriers count both
            // blocks' bytes; the odd block's copies of a stage have landed once the
            // even block has consumed it (its commit arrives on this block's empty)
            const long long n_issued = it;
            const long long j0 = n_issued > GP_NST ? n_issued - GP_NST : 0;
            if (lead)
                for (long long j = j0; j < n_issued; ++j)
                    mbar_wait_cluster(&full[j % GP_NST], (uint32_t)(j / GP_NST) & 1u, drain_budget(budget));
            // and no MMA-commit arrival still on its way to this block's barriers
            if (ok || !lead)
                for (long long j = j0; j < n_issued; ++j)
                    mbar_wait_cluster(&empty[j % GP_NST], (uint32_t)(j / GP_NST) & 1u,
                                      drain_budget(budget));
        }
    } else if (warp == 1) {
        if (lane == 0 && lead) {
            // ---------------- MMA issuer (even block) ----------------
            uint32_t idesc[NT];
#pragma unroll
            for (int n = 0; n < NT; ++n) idesc[n] = gemm_idesc_pair(nbj[n] > 0 ? nbj[n] : 32);
            bool ok = true;
            long long it = 0;
            int seg = 0;
            long long w = w0;
            while (w < w1 && ok) {
                const int t = (int)(w / kblocks);
                const long long wend = min(w1, (long long)(t + 1) * kblocks);
                const int acc = seg % NSETS;
                if (seg >= NSETS &&
                    !mbar_wait_cluster(&tempty[acc], (uint32_t)((seg / NSETS) - 1) & 1u, budget)) {
                    set_error(ctrl, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * NT * GM_BN);   // N tile n at + n BN
                bool first = true;
                for (; w < wend; ++w, ++it) {
                    const int s = (int)(it % GP_NST);
                    if (!mbar_wait_cluster(&full[s], (uint32_t)(it / GP_NST) & 1u, budget)) {
                        set_error(ctrl, ERR_TIMEOUT);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + (size_t)s * stage_bytes);
                    const uint32_t xh = base, xl = base + GM_A_BYTES;
#pragma unroll
                    for (int k = 0; k < GM_BK / 16; ++k) {
                        const uint32_t off = k * 32;   // 16 bf16 along K
#pragma unroll
                        for (int n = 0; n < NT; ++n) {
                            if (nbj[n] == 0) continue;
                            const uint32_t yh = base + yoff[n], yl = yh + (uint32_t)ybox[n] * GM_YBOX_BYTES;
                            const uint32_t d = dt + (uint32_t)(n * GM_BN);
                            tc_mma_pair(d, sw128_desc(xh + off), sw128_desc(yh + off), idesc[n], first ? 0u : 1u);
                            tc_mma_pair(d, sw128_desc(xh + off), sw128_desc(yl + off), idesc[n], 1u);
                            tc_mma_pair(d, sw128_desc(xl + off), sw128_desc(yh + off), idesc[n], 1u);
                        }
                        first = false;
                    }
                    tc_commit_pair(&empty[s], 3);   // frees the stage in both blocks
                }
                if (!ok) break;
                tc_commit_pair(&tfull[acc], 3);     // both halves of the accumulator ready
                ++seg;
            }
            if (!ok) {   // a wait gave up: the MMAs already issued finish before TMEM is freed
                tc_commit_pair(mdrain, 1);
                mbar_wait(mdrain, 0u, drain_budget(budget));
            }
        }
    } else {
        // ---------------- epilogue warps 2..5 (both blocks): TMEM -> workspace ----------------
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const uint32_t lead_tempty = gemm_map_peer(tempty, 0);
        int seg = 0;
        long long w = w0;
        while (w < w1) {
            const int t = (int)(w / kblocks);
            const long long wend = min(w1, (long long)(t + 1) * kblocks);
            const int acc = seg % NSETS;
            if (!mbar_wait_cluster(&tfull[acc], (uint32_t)(seg / NSETS) & 1u, budget)) {
                set_error(ctrl, ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            float* dst = ws + ((size_t)blockIdx.x * smax + seg) * (size_t)(NT * GM_BN) * GM_BM;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                for (int c0 = 0; c0 < nbj[n]; c0 += 32) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((acc * NT + n) * GM_BN + c0), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        dst[(size_t)(n * GM_BN + c0 + j) * GM_BM + q * 32 + lane] = v[j];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (lead)
                    mbar_arrive(&tempty[acc]);
                else
                    gemm_arrive_remote(lead_tempty + (uint32_t)(acc * 8));
            }
            w = wend;
            ++seg;
        }
    }
    tc_fence_before();
    __syncthreads();
    gemm_cluster_sync();   // neither block leaves while the pair's MMAs or arrivals may touch it
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(GM_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Fix-up: D = sum of a tile's partials (in K order), then the epilogue.
// Block (t, j): rows [128 t, 128 t + 128) of the columns 8 j .. 8 j + 7; column c
// belongs to image slot_img[c] (c itself when slot_img is null), and with nact
// set only columns below *nact take part.
// mode 1: R = D - F, R planes (column order), ||r_b||^2 partial;  mode 2: G = D.
// ---------------------------------------------------------------------------
constexpr int FX_B = 4;     // images per fix-up block
constexpr int FX_SEG = GEMM_FX_SEG;   // segments a tile usually has at most (more are added in a second pass)

__global__ void __launch_bounds__(128) k_gemm_fixup(
    const float* __restrict__ ws, const int* __restrict__ tile_seg_begin,
    const int* __restrict__ seg_slot, int M, int ws_cols, int count, const float* __restrict__ F, int ldf,
    float* __restrict__ out, int ldo, __nv_bfloat16* __restrict__ out_hi,
    __nv_bfloat16* __restrict__ out_lo, int ldh, float2* __restrict__ r2part, int tiles_m,
    const Ctrl* __restrict__ ctrl, int check_skip, const int* __restrict__ slot_img,
    const int* __restrict__ nact)
{
    __shared__ float2 red[4][FX_B];
    pdl_release();   // the next GEMM may start its independent prologue (it waits before reading R)
    if (check_skip && ctrl->skip) return;
    const int t = blockIdx.x, b0 = blockIdx.y * FX_B;
    if (nact) count = min(count, *nact);
    if (b0 >= count) return;   // uniform across the block
    const int row = t * GM_BM + threadIdx.x;
    const int s0 = tile_seg_begin[t], s1 = tile_seg_begin[t + 1];
    const int ns = s1 - s0;
    // every image's first FX_SEG partials are loaded before any is added
    int slot[FX_SEG];
#pragma unroll
    for (int q = 0; q < FX_SEG; ++q) slot[q] = q < ns ? seg_slot[s0 + q] : 0;
    float v[FX_B][FX_SEG];
#pragma unroll
    for (int k = 0; k < FX_B; ++k)
#pragma unroll
        for (int q = 0; q < FX_SEG; ++q)
            v[k][q] = (q < ns && b0 + k < count)
                          ? ws[((size_t)slot[q] * ws_cols + b0 + k) * GM_BM + threadIdx.x]
                          : 0.f;
    // the columns' images and their F entries, loaded with the partials
    int img[FX_B];
    float fv[FX_B];
#pragma unroll
    for (int k = 0; k < FX_B; ++k) {
        const int c = b0 + k;
        img[k] = c < count ? (slot_img ? __ldg(slot_img + c) : c) : 0;
        fv[k] = (F && c < count && row < M) ? __ldg(F + (size_t)img[k] * ldf + row) : 0.f;
    }
    float2 sq[FX_B];   // double-single squares
#pragma unroll
    for (int k = 0; k < FX_B; ++k) {
        const int c = b0 + k;   // column
        sq[k] = make_float2(0.f, 0.f);
        if (c >= count) continue;
        const int b = img[k];
        float d = 0.f;   // the tile's segments in K order
#pragma unroll
        for (int q = 0; q < FX_SEG; ++q) d += v[k][q];
        for (int s = s0 + FX_SEG; s < s1; ++s)
            d += ws[((size_t)seg_slot[s] * ws_cols + c) * GM_BM + threadIdx.x];
        if (row < M) {
            d -= fv[k];
            out[(size_t)b * ldo + row] = d;
            if (out_hi) {
                const __nv_bfloat16 h = __float2bfloat16_rn(d);
                out_hi[(size_t)c * ldh + row] = h;
                out_lo[(size_t)c * ldh + row] = __float2bfloat16_rn(d - __bfloat162float(h));
            }
            sq[k] = ds_sq(d);
        }
    }
    if (r2part) {   // per image: the sum over the tile's rows (fixed order)
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < FX_B; ++k) {
            const float2 v = warp_sum_ds(sq[k]);
            if (lane == 0) red[w][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < FX_B && b0 + (int)threadIdx.x < count) {
            const int k = threadIdx.x;
            const int b = slot_img ? slot_img[b0 + k] : b0 + k;
            r2part[(size_t)b * tiles_m + t] =
                ds_add(ds_add(ds_add(red[0][k], red[1][k]), red[2][k]), red[3][k]);
        }
    }
}

// v (count x len binary32, row pitch ld) -> bf16 hi/lo planes (row pitch ldh).
__global__ void k_split_rows(const float* __restrict__ v, int len, int ld,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldh)
{
    const int b = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        const float x = v[(size_t)b * ld + i];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[(size_t)b * ldh + i] = h;
        lo[(size_t)b * ldh + i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// Tile-contiguous bf16 planes of the operand X of a batched GEMM: X = A
// (trans = 0, m x N) or X = A^T (trans = 1, N x m), both from A's hi and lo
// planes (m x N, row-major).  Tile (t, kb) of X -- rows [128 t, 128 t + 128),
// columns [64 kb, 64 kb + 64) -- is stored as 128 rows of 64 values (16 KB, one
// TMA box read from contiguous memory) at tile index t * kblocks + kb; entries
// past X's edge are zero.  One block per tile.
__global__ void __launch_bounds__(256) k_tile_planes(const unsigned short* __restrict__ Ph,
                                                     const unsigned short* __restrict__ Pl, int m,
                                                     int N, int trans, unsigned short* __restrict__ Th,
                                                     unsigned short* __restrict__ Tl, int kblocks)
{
    __shared__ unsigned short sh[2][GM_BK][GM_BM + 2];   // [plane][column of X][row of X]
    const int tile = blockIdx.x;
    const int t = tile / kblocks, kb = tile - t * kblocks;
    const size_t out = (size_t)tile * GM_BM * GM_BK;
    if (!trans) {   // X row 128 t + r is A row 128 t + r: 128-byte pieces, copied as they are
        for (int i = threadIdx.x; i < GM_BM * GM_BK; i += blockDim.x) {
            const int r = i / GM_BK, c = i - r * GM_BK;
            const int R = t * GM_BM + r, C = kb * GM_BK + c;
            const bool in = R < m && C < N;
            const size_t src = (size_t)R * N + C;
            Th[out + i] = in ? Ph[src] : (unsigned short)0;
            Tl[out + i] = in ? Pl[src] : (unsigned short)0;
        }
    } else {        // X[128 t + r][64 kb + c] = A[64 kb + c][128 t + r]: through shared memory
        for (int i = threadIdx.x; i < GM_BK * GM_BM; i += blockDim.x) {
            const int c = i / GM_BM, r = i - c * GM_BM;
            const int R = kb * GM_BK + c, C = t * GM_BM + r;   // A's row and column
            const bool in = R < m && C < N;
            const size_t src = (size_t)R * N + C;
            sh[0][c][r] = in ? Ph[src] : (unsigned short)0;
            sh[1][c][r] = in ? Pl[src] : (unsigned short)0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < GM_BM * GM_BK; i += blockDim.x) {
            const int r = i / GM_BK, c = i - r * GM_BK;
            Th[out + i] = sh[0][c][r];
            Tl[out + i] = sh[1][c][r];
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2D bf16 tensor [rows][inner] (row pitch ld elements), box [box_rows][64], 128B swizzle.
bool make_bf16_map(CUtensorMap* map, const void* base, int inner, int rows, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)GM_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

void gemm_plan(int M, int K, int grid, GemmPlan* p, bool pair, int nt)
{
    p->pair = pair ? 1 : 0;
    p->nt = pair && nt == 2 ? 2 : 1;
    p->tiles_m = (M + GM_BM - 1) / GM_BM;
    p->tiles = pair ? (M + 2 * GM_BM - 1) / (2 * GM_BM) : p->tiles_m;
    p->kblocks = (K + GM_BK - 1) / GM_BK;
    const long long W = (long long)p->tiles * p->kblocks;
    long long units = pair ? grid / 2 : grid;   // blocks, or pairs of blocks
    if (units > W) units = W;
    if (units < 1) units = 1;
    p->grid = (int)(pair ? 2 * units : units);
    // segments of each unit and, per 128-row tile, its (block, segment) slots in K order
    std::vector<std::vector<long long>> per_tile(p->tiles_m);
    int smax = 1;
    for (long long c = 0; c < units; ++c) {
        const long long w0 = W * c / units, w1 = W * (c + 1) / units;
        int j = 0;
        long long w = w0;
        while (w < w1) {
            const int t = (int)(w / p->kblocks);
            if (pair) {   // the even block holds rows [0, 128) of the pair's tile, the odd one the rest
                per_tile[2 * t].push_back((2 * c) * 1000000 + j);
                if (2 * t + 1 < p->tiles_m) per_tile[2 * t + 1].push_back((2 * c + 1) * 1000000 + j);
            } else {
                per_tile[t].push_back(c * 1000000 + j);
            }
            w = std::min(w1, (long long)(t + 1) * p->kblocks);
            ++j;
        }
        smax = std::max(smax, j);
    }
    p->smax = smax;
    p->tile_seg_begin.assign(p->tiles_m + 1, 0);
    p->seg_slot.clear();
    for (int t = 0; t < p->tiles_m; ++t) {
        p->tile_seg_begin[t] = (int)p->seg_slot.size();
        for (long long code : per_tile[t])
            p->seg_slot.push_back((int)((code / 1000000) * smax + code % 1000000));
    }
    p->tile_seg_begin[p->tiles_m] = (int)p->seg_slot.size();
    p->ws_floats = (size_t)p->grid * smax * (p->nt * GM_BN) * GM_BM;
}

cudaError_t gemm_configure()
{
    cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GM_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_gemm_bf16x3_pair<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GP_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gemm_bf16x3_pair<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)GP_SMEM);
}

int gemm_pair_max_clusters(int num_sms)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(num_sms & ~1), 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = GP_SMEM;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)k_gemm_bf16x3_pair<1>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

void launch_gemm(const CUtensorMap* xh, const CUtensorMap* xl, const CUtensorMap* yh,
                 const CUtensorMap* yl, const GemmPlan& p, float* ws, Ctrl* ctrl, int check_skip,
                 long long budget, cudaStream_t s, int ncols, const int* nact, int pdl)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.grid, 1, 1);
    cfg.blockDim = dim3(192, 1, 1);
    cfg.dynamicSmemBytes = p.pair ? GP_SMEM : GM_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (p.pair && p.nt == 2)
        cudaLaunchKernelEx(&cfg, k_gemm_bf16x3_pair<2>, *xh, *xl, *yh, *yl, p.tiles, p.kblocks, ws,
                           p.smax, ctrl, check_skip, budget, ncols, nact);
    else if (p.pair)
        cudaLaunchKernelEx(&cfg, k_gemm_bf16x3_pair<1>, *xh, *xl, *yh, *yl, p.tiles, p.kblocks, ws,
                           p.smax, ctrl, check_skip, budget, ncols, nact);
    else
        cudaLaunchKernelEx(&cfg, k_gemm_bf16x3, *xh, *xl, *yh, *yl, p.tiles, p.kblocks, ws, p.smax,
                           ctrl, check_skip, budget, ncols, nact);
}

void launch_gemm_fixup(const float* ws, const int* tile_seg_begin, const int* seg_slot, int M,
                       int tiles_m, int ws_cols, int count, const float* F, int ldf, float* out,
                       int ldo, void* out_hi, void* out_lo, int ldh, float2* r2part, const Ctrl* ctrl,
                       int check_skip, cudaStream_t s, const int* slot_img, const int* nact)
{
    dim3 grid(tiles_m, (count + FX_B - 1) / FX_B);
    k_gemm_fixup<<<grid, 128, 0, s>>>(ws, tile_seg_begin, seg_slot, M, ws_cols, count, F, ldf, out, ldo,
                                      reinterpret_cast<__nv_bfloat16*>(out_hi),
                                      reinterpret_cast<__nv_bfloat16*>(out_lo), ldh, r2part,
                                      tiles_m, ctrl, check_skip, slot_img, nact);
}

void launch_split_rows(const float* v, int count, int len, int ld, void* hi, void* lo, int ldh,
                       cudaStream_t s)
{
    dim3 grid((len + 255) / 256 < 64 ? (len + 255) / 256 : 64, count);
    k_split_rows<<<grid, 256, 0, s>>>(v, len, ld, reinterpret_cast<__nv_bfloat16*>(hi),
                                      reinterpret_cast<__nv_bfloat16*>(lo), ldh);
}

void launch_tile_planes(const void* Ph, const void* Pl, int m, int N, int trans, void* Th,
                        void* Tl, int tiles_m, int kblocks, cudaStream_t s)
{
    k_tile_planes<<<tiles_m * kblocks, 256, 0, s>>>(
        static_cast<const unsigned short*>(Ph), static_cast<const unsigned short*>(Pl), m, N, trans,
        static_cast<unsigned short*>(Th), static_cast<unsigned short*>(Tl), kblocks);
}

}  // namespace tvcs
