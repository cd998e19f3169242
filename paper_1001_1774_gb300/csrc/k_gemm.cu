// Row a8: the two products of many images that share one encoding matrix, as
// tensor-core GEMMs (Xiao & Yang, eq. (line) for every image at once):
//     R = A U - F        (m x B,  K = n^2)
//     G = A^T R          (n^2 x B, K = m)
// with U = [u_1 ... u_B], F = [f_1 ... f_B].  Both run as K-major ("TN") GEMMs
// D = X Y^T because A is stored twice, as A (m x n^2) and as A^T (n^2 x m).
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
// lets its copies land and frees its tensor memory.
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
constexpr uint32_t GM_YBOX_BYTES = GEMM_Y_BOX * GM_BK * 2;    // one 64-row box of a Y tile
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
            long long it = 0;
            const uint64_t pol_x = l2_policy_evict_first(), pol_y = l2_policy_evict_last();
            for (long long w = w0; w < w1; ++w, ++it) {
                const int s = (int)(it % GM_NST);
                if (it >= GM_NST && !mbar_wait(&empty[s], (uint32_t)((it / GM_NST) - 1) & 1u, budget)) {
                    set_error(ctrl, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                const int t = (int)(w / kblocks), kb = (int)(w % kblocks);
                unsigned char* st = smem + (size_t)s * GM_STAGE;
                mbar_arrive_expect_tx(&full[s], stage_bytes);
                tma_load_2d(st, &tXh, kb * GM_BK, t * GM_BM, &full[s], pol_x);
                tma_load_2d(st + GM_A_BYTES, &tXl, kb * GM_BK, t * GM_BM, &full[s], pol_x);
                for (int j = 0; j < ybox; ++j) {   // 64-row boxes, 1024-byte aligned
                    tma_load_2d(st + 2 * GM_A_BYTES + j * GM_YBOX_BYTES, &tYh, kb * GM_BK,
                                j * GEMM_Y_BOX, &full[s], pol_y);
                    tma_load_2d(st + 2 * GM_A_BYTES + GM_B_BYTES + j * GM_YBOX_BYTES, &tYl,
                                kb * GM_BK, j * GEMM_Y_BOX, &full[s], pol_y);
                }
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
// Fix-up: D = sum of a tile's partials (in K order), then the epilogue.
// Block (t, j): rows [128 t, 128 t + 128) of the columns 8 j .. 8 j + 7; column c
// belongs to image slot_img[c] (c itself when slot_img is null), and with nact
// set only columns below *nact take part.
// mode 1: R = D - F, R planes (column order), ||r_b||^2 partial;  mode 2: G = D.
// ---------------------------------------------------------------------------
constexpr int FX_B = 4;     // images per fix-up block
constexpr int FX_SEG = 6;   // segments a tile usually has at most (more are added in a second pass)

__global__ void __launch_bounds__(128) k_gemm_fixup(
    const float* __restrict__ ws, const int* __restrict__ tile_seg_begin,
    const int* __restrict__ seg_slot, int M, int count, const float* __restrict__ F, int ldf,
    float* __restrict__ out, int ldo, __nv_bfloat16* __restrict__ out_hi,
    __nv_bfloat16* __restrict__ out_lo, int ldh, float2* __restrict__ r2part, int tiles_m,
    const Ctrl* __restrict__ ctrl, int check_skip, const int* __restrict__ slot_img,
    const int* __restrict__ nact)
{
    __shared__ float2 red[4][FX_B];
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
                          ? ws[((size_t)slot[q] * GM_BN + b0 + k) * GM_BM + threadIdx.x]
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
            d += ws[((size_t)seg_slot[s] * GM_BN + c) * GM_BM + threadIdx.x];
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

// A (m x N binary32) -> A^T hi/lo planes (N x ldt bf16), 32 x 32 tiles.
__global__ void k_transpose_split(const float* __restrict__ A, int m, int N,
                                  __nv_bfloat16* __restrict__ th, __nv_bfloat16* __restrict__ tl,
                                  int ldt)
{
    __shared__ float tile[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k, j = j0 + threadIdx.x;
        tile[k][threadIdx.x] = (i < m && j < N) ? A[(size_t)i * N + j] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int j = j0 + k, i = i0 + threadIdx.x;
        if (j < N && i < ldt) {
            const float x = i < m ? tile[threadIdx.x][k] : 0.f;
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            th[(size_t)j * ldt + i] = h;
            tl[(size_t)j * ldt + i] = __float2bfloat16_rn(x - __bfloat162float(h));
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

void gemm_plan(int M, int K, int num_sms, GemmPlan* p)
{
    p->tiles_m = (M + GM_BM - 1) / GM_BM;
    p->kblocks = (K + GM_BK - 1) / GM_BK;
    const long long W = (long long)p->tiles_m * p->kblocks;
    p->grid = (int)(W < num_sms ? W : num_sms);
    // segments of each block and, per tile, its (block, segment) slots in K order
    std::vector<std::vector<int>> per_tile(p->tiles_m);
    int smax = 1;
    for (int c = 0; c < p->grid; ++c) {
        const long long w0 = W * c / p->grid, w1 = W * (c + 1) / p->grid;
        int j = 0;
        long long w = w0;
        while (w < w1) {
            const int t = (int)(w / p->kblocks);
            per_tile[t].push_back(c * 1000000 + j);   // decoded below once smax is known
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
        for (int code : per_tile[t]) p->seg_slot.push_back((code / 1000000) * smax + code % 1000000);
    }
    p->tile_seg_begin[p->tiles_m] = (int)p->seg_slot.size();
    p->ws_floats = (size_t)p->grid * smax * GM_BN * GM_BM;
}

cudaError_t gemm_configure()
{
    return cudaFuncSetAttribute(k_gemm_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)GM_SMEM);
}

void launch_gemm(const CUtensorMap* xh, const CUtensorMap* xl, const CUtensorMap* yh,
                 const CUtensorMap* yl, const GemmPlan& p, float* ws, Ctrl* ctrl, int check_skip,
                 long long budget, cudaStream_t s, int ncols, const int* nact)
{
    k_gemm_bf16x3<<<p.grid, 192, GM_SMEM, s>>>(*xh, *xl, *yh, *yl, p.tiles_m, p.kblocks, ws,
                                               p.smax, ctrl, check_skip, budget, ncols, nact);
}

void launch_gemm_fixup(const float* ws, const int* tile_seg_begin, const int* seg_slot, int M,
                       int tiles_m, int count, const float* F, int ldf, float* out, int ldo,
                       void* out_hi, void* out_lo, int ldh, float2* r2part, const Ctrl* ctrl,
                       int check_skip, cudaStream_t s, const int* slot_img, const int* nact)
{
    dim3 grid(tiles_m, (count + FX_B - 1) / FX_B);
    k_gemm_fixup<<<grid, 128, 0, s>>>(ws, tile_seg_begin, seg_slot, M, count, F, ldf, out, ldo,
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

void launch_transpose_split(const float* A, int m, int N, void* th, void* tl, int ldt,
                            cudaStream_t s)
{
    dim3 grid((N + 31) / 32, (ldt + 31) / 32);
    k_transpose_split<<<grid, dim3(32, 8), 0, s>>>(A, m, N, reinterpret_cast<__nv_bfloat16*>(th),
                                                   reinterpret_cast<__nv_bfloat16*>(tl), ldt);
}

}  // namespace tvcs
