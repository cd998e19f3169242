// Many images sharing one encoding matrix (row a8): IADM for every image at
// once, with the two products of all images as tcgen05 BF16x3 GEMMs (k_gemm.cu)
// and the u-steps as one batched thread-block-cluster launch (k_usolve.cu).
//
// Loop body (a CUDA graph with a WHILE node): batched u-solve (rows a1-a5 per
// image, with per-image mu, stop test and control block) -> GEMM R = A U - F ->
// fix-up (R, its bf16 planes, ||r_b||^2) -> GEMM G = A^T R -> fix-up (G) ->
// loop condition (any image still running).  Images that met eq. (stop) skip
// their u-steps; the GEMMs keep all columns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "kernels.h"

namespace tvcs {

// Continue while any image runs and the loop bound holds.  With slot tables
// (count <= blockDim.x = BATCH_MAX): the running images, in image order, take slots
// 0 .. nact-1 for the next iteration (a block-wide exclusive prefix sum of the
// running flags); an image that stopped gets slot -1.  img_slot_prev (nullable)
// keeps each image's slot of the iteration that just ended (its column in that
// iteration's GEMMs).
__global__ void k_batch_cond(const Ctrl* __restrict__ ctrls, int count, Ctrl* __restrict__ bctrl,
                             cudaGraphConditionalHandle cond, int set_cond,
                             int* __restrict__ slot_img, int* __restrict__ img_slot,
                             int* __restrict__ img_slot_prev)
{
    __shared__ int any;
    __shared__ int wtot[BATCH_MAX / 32];
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < count; b += blockDim.x)
        if (!ctrls[b].done && ctrls[b].error == ERR_NONE) atomicOr(&any, 1);
    if (slot_img) {
        const int b = threadIdx.x, lane = b & 31, w = b >> 5;
        const bool run = b < count && !ctrls[b].done && ctrls[b].error == ERR_NONE;
        const unsigned m = __ballot_sync(0xffffffffu, run);
        if (lane == 0) wtot[w] = __popc(m);
        __syncthreads();
        int base = 0, total = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            if (k < w) base += wtot[k];
            total += wtot[k];
        }
        const int slot = base + __popc(m & ((1u << lane) - 1u));
        if (b < count) {
            if (img_slot_prev) img_slot_prev[b] = img_slot[b];   // read and rewritten by thread b only
            img_slot[b] = run ? slot : -1;
            if (run) slot_img[slot] = b;
        }
        if (b == 0) bctrl->nact = total;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int lc = ++bctrl->loops;
        const int cont = (any && lc < bctrl->loops_max) ? 1 : 0;
        bctrl->done = !cont;
        bctrl->skip = !cont;   // the GEMMs and fix-ups of later iterations in the body
        if (set_cond) cudaGraphSetConditional(cond, (unsigned)cont);
    }
}

void launch_batch_cond(const Ctrl* ctrls, int count, Ctrl* bctrl, unsigned long long cond,
                       int set_cond, cudaStream_t s, int* slot_img, int* img_slot,
                       int* img_slot_prev)
{
    k_batch_cond<<<1, BATCH_MAX, 0, s>>>(ctrls, count, bctrl, (cudaGraphConditionalHandle)cond,
                                         set_cond, slot_img, img_slot, img_slot_prev);
}

// End-of-run residual of every image, r_b = A_eff u_b - f_b with A_eff = hi + lo
// (the stored matrix, exact in binary32), on the CUDA cores in binary32 with a
// three-level sum: 32 products from zero, 16 such chunks, then the running total
// (the tensor-core products keep 16 bits of u and add in one long binary32 chain,
// which is accurate for the iteration but not for ||r||^2 of a converged image).
// Block: 64 rows x 64 images, 256 threads of 4 x 4 outputs; K in chunks of 32.
constexpr int RS_BM = 64, RS_BB = 64, RS_BK = 32;

__global__ void __launch_bounds__(256)
    k_batch_resid(const unsigned short* __restrict__ hi, const unsigned short* __restrict__ lo,
                  int m, int N, const float* __restrict__ U, const float* __restrict__ F,
                  int count, float* __restrict__ R)
{
    __shared__ float As[RS_BK][RS_BM + 4];
    __shared__ float Us[RS_BK][RS_BB + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;              // images tx*4.., rows ty*4..
    const int i0 = blockIdx.x * RS_BM, b0 = blockIdx.y * RS_BB;
    float c[4][4], l1[4][4], l2[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) l1[a][b] = l2[a][b] = 0.f;
    const int lr = tid >> 2, lg = (tid & 3) * 8;         // loader: row / image lr, columns lg..lg+7
    int chunk = 0;
    for (int k0 = 0; k0 < N; k0 += RS_BK, ++chunk) {
        {   // A_eff tile (transposed) and U tile (transposed)
            const int i = i0 + lr;
            float av[8];
            if (i < m) {
                const uint4 h = *reinterpret_cast<const uint4*>(hi + (size_t)i * N + k0 + lg);
                const uint4 l = *reinterpret_cast<const uint4*>(lo + (size_t)i * N + k0 + lg);
                const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    av[2 * q] = __uint_as_float(hw[q] << 16) + __uint_as_float(lw[q] << 16);
                    av[2 * q + 1] = __uint_as_float(hw[q] & 0xffff0000u) +
                                    __uint_as_float(lw[q] & 0xffff0000u);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) av[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) As[lg + q][lr] = av[q];
            const int b = b0 + lr;
            float uv[8];
            if (b < count) {
                const float4 u0 = *reinterpret_cast<const float4*>(U + (size_t)b * N + k0 + lg);
                const float4 u1 = *reinterpret_cast<const float4*>(U + (size_t)b * N + k0 + lg + 4);
                uv[0] = u0.x; uv[1] = u0.y; uv[2] = u0.z; uv[3] = u0.w;
                uv[4] = u1.x; uv[5] = u1.y; uv[6] = u1.z; uv[7] = u1.w;
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) uv[q] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) Us[lg + q][lr] = uv[q];
        }
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) c[a][b] = 0.f;
#pragma unroll 8
        for (int k = 0; k < RS_BK; ++k) {
            const float4 a4 = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
            const float4 u4 = *reinterpret_cast<const float4*>(&Us[k][tx * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, uv[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) c[a][b] = fmaf(av[a], uv[b], c[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) l1[a][b] += c[a][b];
        if ((chunk & 15) == 15) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    l2[a][b] += l1[a][b];
                    l1[a][b] = 0.f;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = i0 + ty * 4 + a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int img = b0 + tx * 4 + b;
            if (img < count) R[(size_t)img * m + i] = (l2[a][b] + l1[a][b]) - F[(size_t)img * m + i];
        }
    }
}

// ctrls[b].r2 = ||R_b||^2 (double-single, fixed order), one block per image.
__global__ void k_batch_resid_r2(const float* __restrict__ R, int m, Ctrl* __restrict__ ctrls)
{
    __shared__ float2 red[32];
    float2 s = make_float2(0.f, 0.f);
    const float* r = R + (size_t)blockIdx.x * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s = ds_add(s, ds_sq(r[i]));
    s = block_sum_ds(s, red);
    if (threadIdx.x == 0) ctrls[blockIdx.x].r2 = ds_value(s);
}

namespace {

#define BCK(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_last_error(e_ == cudaErrorMemoryAllocation ? TVCS_ERR_OOM : TVCS_ERR_CUDA, \
                                  "%s failed: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

#define BCKS(expr)                                  \
    do {                                            \
        tvcs_status s_ = (expr);                    \
        if (s_ != TVCS_OK) return s_;               \
    } while (0)

tvcs_status balloc(void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_last_error(TVCS_ERR_OOM, "cudaMalloc of %zu bytes failed", bytes);
    }
    return TVCS_OK;
}

void free_buffers(tvcs_batch* b)
{
    void* bufs[] = {b->U, b->W, b->L, b->G, b->R, b->F, b->mu, b->Uh, b->Ul, b->Rh, b->Rl,
                    b->ctrls, b->bctrl, b->r2part, b->part, b->ws, b->tsb1, b->ss1, b->tsb2, b->ss2,
                    b->slot_img, b->img_slot, b->img_slot_prev};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (b->hctrls) cudaFreeHost(b->hctrls);
    if (b->hbctrl) cudaFreeHost(b->hbctrl);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->U = b->W = b->L = b->G = b->R = b->F = b->mu = nullptr;
    b->Uh = b->Ul = b->Rh = b->Rl = nullptr;
    b->ctrls = b->bctrl = b->hctrls = b->hbctrl = nullptr;
    b->r2part = nullptr;
    b->part = nullptr;
    b->slot_img = b->img_slot = b->img_slot_prev = nullptr;
    b->ws = nullptr;
    b->tsb1 = b->ss1 = b->tsb2 = b->ss2 = nullptr;
    b->exec = nullptr;
    b->graph = nullptr;
    b->cap = 0;
}

// True when p[i] = p[0] + i * len for every i and the whole range lies in one
// allocation (pageable host memory, or one device / pinned allocation), so that
// one copy can move all images.
template <typename T>
bool contiguous(T* const* p, int count, size_t len)
{
    for (int i = 1; i < count; ++i)
        if (p[i] != p[0] + (size_t)i * len) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p[0]) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeUnregistered) return true;
    // the driver's address-range query, looked up at run time (the library links no
    // driver symbol, so that it loads where no driver is installed)
    typedef CUresult (*RangeFn)(CUdeviceptr*, size_t*, CUdeviceptr);
    static RangeFn range_fn = nullptr;
    if (!range_fn) {
        void* fp = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fp, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fp) {
            cudaGetLastError();
            return false;
        }
        range_fn = reinterpret_cast<RangeFn>(fp);
    }
    CUdeviceptr base = 0;
    size_t size = 0;
    const CUdeviceptr a = (CUdeviceptr)(uintptr_t)p[0];
    if (range_fn(&base, &size, a) != CUDA_SUCCESS) return false;
    return a + (CUdeviceptr)(sizeof(T) * len * (size_t)count) <= base + size;
}

tvcs_status sync_check(tvcs_ctx* h, const char* what)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(TVCS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return TVCS_OK;
}

tvcs_status upload_plan(const GemmPlan& p, int** tsb, int** ss, cudaStream_t s)
{
    BCKS(balloc((void**)tsb, sizeof(int) * p.tile_seg_begin.size()));
    BCKS(balloc((void**)ss, sizeof(int) * (p.seg_slot.size() ? p.seg_slot.size() : 1)));
    BCK(cudaMemcpyAsync(*tsb, p.tile_seg_begin.data(), sizeof(int) * p.tile_seg_begin.size(),
                        cudaMemcpyHostToDevice, s));
    if (!p.seg_slot.empty())
        BCK(cudaMemcpyAsync(*ss, p.seg_slot.data(), sizeof(int) * p.seg_slot.size(),
                            cudaMemcpyHostToDevice, s));
    return TVCS_OK;
}

tvcs_status make_maps(tvcs_ctx* h, int count)
{
    tvcs_batch* b = h->batch;
    // the X operands in their tile-contiguous planes: rows of 64 values, boxes of 128 rows
    const int rows1 = b->tiles1 * b->kb1 * 128, rows2 = b->tiles2 * b->kb2 * 128;
    bool ok = make_bf16_map(&b->mAh, b->Tah, 64, rows1, 64, 128) &&
              make_bf16_map(&b->mAl, b->Tal, 64, rows1, 64, 128) &&
              make_bf16_map(&b->mAth, b->Tth, 64, rows2, 64, 128) &&
              make_bf16_map(&b->mAtl, b->Ttl, 64, rows2, 64, 128) &&
              make_bf16_map(&b->mUh, b->Uh, h->N, count, h->N, GEMM_Y_BOX) &&
              make_bf16_map(&b->mUl, b->Ul, h->N, count, h->N, GEMM_Y_BOX) &&
              make_bf16_map(&b->mRh, b->Rh, h->m, count, b->mpad, GEMM_Y_BOX) &&
              make_bf16_map(&b->mRl, b->Rl, h->m, count, b->mpad, GEMM_Y_BOX);
    if (!ok) return set_last_error(TVCS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return TVCS_OK;
}

// N tiles of 256 images per X tile of the GEMMs: two above 256 images.
int gemm_nt(int count) { return count > 256 ? 2 : 1; }

// Launch shapes the GEMM tuner tries: one block per SM and 7/8, 3/4, 1/2 of
// that, on single blocks and (where the device holds clusters of two of them)
// on CTA pairs.
struct GemmShape {
    int grid = 0, pair = 0;
};

std::vector<GemmShape> gemm_shape_candidates(int num_sms, int pair_clusters, int nt)
{
    std::vector<GemmShape> v;
    if (nt == 1)   // the single-block kernel takes at most 256 images
        for (int g : {num_sms, num_sms * 7 / 8, num_sms * 3 / 4, num_sms / 2}) v.push_back({g, 0});
    const int pc = std::min(pair_clusters, num_sms / 2);
    if (pc > 0)
        for (int c : {pc, pc * 7 / 8, pc * 3 / 4, pc / 2})
            if (c > 0) v.push_back({2 * c, 1});
    return v;
}

std::mutex g_gemm_tune_mutex;
std::map<std::tuple<int, int, int, int>, std::pair<GemmShape, GemmShape>> g_gemm_shapes;   // (device, m, N, nt)

// Picks the launch shape of each GEMM (persistent blocks or pairs, and with it
// the stream-K split of its tiles x K-blocks) by timing every candidate, GEMM
// and fix-up together, over five launches each (median), on the handle's own
// operands; cached per device and (m, n).  opt.autotune = 0 keeps one block
// per SM; a shape set through tvcs_test_gemm_shape takes precedence.  A
// different split regroups the K sums of a tile, so results agree to binary32
// rounding with the default shape, not bitwise.
tvcs_status tune_gemms(tvcs_ctx* h, int count)
{
    tvcs_batch* b = h->batch;
    cudaStream_t s = h->stream;
    const int nt = gemm_nt(count);
    const GemmShape dflt = nt == 1 ? GemmShape{h->num_sms, 0}
                                   : GemmShape{2 * std::min(b->pair_clusters, h->num_sms / 2), 1};
    GemmShape g1 = dflt, g2 = dflt;
    if (h->gemm_force[0] > 0) {
        g1 = {h->gemm_force[0], h->gemm_force[1]};
        g2 = {h->gemm_force[2], h->gemm_force[3]};
        if (nt == 2 && (!g1.pair || !g2.pair))
            return set_last_error(TVCS_ERR_INVALID_ARG,
                                  "more than 256 images need the GEMMs on CTA pairs (tvcs_test_gemm_shape)");
    } else if (h->opt.autotune) {
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_gemm_tune_mutex);
            auto it = g_gemm_shapes.find({h->dev, h->m, h->N, nt});
            if (it != g_gemm_shapes.end()) {
                g1 = it->second.first;
                g2 = it->second.second;
                cached = true;
            }
        }
        if (!cached) {
            const long long budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : (1LL << 31);
            for (int which = 0; which < 2; ++which) {
                const int M = which == 0 ? h->m : h->N, K = which == 0 ? h->N : h->m;
                float best = -1.f;
                for (GemmShape g : gemm_shape_candidates(h->num_sms, b->pair_clusters, nt)) {
                    GemmPlan p;
                    gemm_plan(M, K, g.grid, &p, g.pair != 0, nt);
                    int *tsb = nullptr, *ss = nullptr;
                    BCKS(upload_plan(p, &tsb, &ss, s));
                    float t[5];
                    for (int rep = -1; rep < 5; ++rep) {
                        if (rep >= 0) BCK(cudaEventRecord(h->ev0, s));
                        if (which == 0) {
                            launch_gemm(&b->mAh, &b->mAl, &b->mUh, &b->mUl, p, b->ws, b->bctrl, 0,
                                        budget, s, count);
                            launch_gemm_fixup(b->ws, tsb, ss, h->m, p.tiles_m, p.nt * 256, count, b->F, h->m,
                                              b->R, h->m, b->Rh, b->Rl, b->mpad, b->r2part, b->bctrl,
                                              0, s);
                        } else {
                            launch_gemm(&b->mAth, &b->mAtl, &b->mRh, &b->mRl, p, b->ws, b->bctrl, 0,
                                        budget, s, count);
                            launch_gemm_fixup(b->ws, tsb, ss, h->N, p.tiles_m, p.nt * 256, count, nullptr, 0,
                                              b->G, h->N, nullptr, nullptr, 0, nullptr, b->bctrl, 0,
                                              s);
                        }
                        if (rep >= 0) {
                            BCK(cudaEventRecord(h->ev1, s));
                            BCK(cudaEventSynchronize(h->ev1));
                            BCK(cudaEventElapsedTime(&t[rep], h->ev0, h->ev1));
                        }
                    }
                    BCKS(sync_check(h, "tuning the batched GEMMs"));
                    cudaFree(tsb);
                    cudaFree(ss);
                    std::sort(t, t + 5);
                    if (best < 0.f || t[2] < best) {
                        best = t[2];
                        (which == 0 ? g1 : g2) = g;
                    }
                }
            }
            std::lock_guard<std::mutex> lk(g_gemm_tune_mutex);
            g_gemm_shapes[{h->dev, h->m, h->N, nt}] = {g1, g2};
        }
    }
    GemmPlan q1, q2;
    gemm_plan(h->m, h->N, g1.grid, &q1, g1.pair != 0, nt);
    gemm_plan(h->N, h->m, g2.grid, &q2, g2.pair != 0, nt);
    if (q1.grid != b->p1.grid || q1.pair != b->p1.pair || q1.nt != b->p1.nt ||
        q2.grid != b->p2.grid || q2.pair != b->p2.pair || q2.nt != b->p2.nt) {
        cudaFree(b->tsb1);
        cudaFree(b->ss1);
        cudaFree(b->tsb2);
        cudaFree(b->ss2);
        b->tsb1 = b->ss1 = b->tsb2 = b->ss2 = nullptr;
        b->p1 = q1;
        b->p2 = q2;
        BCKS(upload_plan(b->p1, &b->tsb1, &b->ss1, s));
        BCKS(upload_plan(b->p2, &b->tsb2, &b->ss2, s));
        BCKS(sync_check(h, "uploading the tuned GEMM plans"));
    }
    return TVCS_OK;
}

// Buffers for `count` images (reallocated when count grows), A^T planes, plans.
tvcs_status ensure_batch(tvcs_ctx* h, int count)
{
    if (h->opt.precision != TVCS_PREC_BF16X2)
        return set_last_error(TVCS_ERR_UNSUPPORTED,
                              "the shared-A batched path needs A stored as bf16 hi+lo "
                              "(precision TVCS_PREC_BF16X2)");
    if (count > batch_max(h))
        return set_last_error(TVCS_ERR_INVALID_ARG, "at most %d images per batch", batch_max(h));
    if (h->N % 128 != 0)
        return set_last_error(TVCS_ERR_UNSUPPORTED, "batched path needs n*n a multiple of 128");
    if (!h->batch) {
        h->batch = new (std::nothrow) tvcs_batch();
        if (!h->batch) return set_last_error(TVCS_ERR_OOM, "host allocation failed");
    }
    tvcs_batch* b = h->batch;
    cudaStream_t s = h->stream;
    const size_t N = h->N, m = h->m;
    if (b->ucluster == 0) {
        // Many images in flight: one block per image where n allows it, else
        // 8-block clusters (they pack the SMs more densely than 16).
        b->uimg = usolve_img_configure(h->n);
        b->ureg = h->n == 128 && usolve_reg_configure();
        b->gfused = b->ureg;   // 128 x 128 images: GEMM tile t of G = A^T R is image row t
        b->ucluster = usolve_cluster_fits(h->n, 8) ? 8 : h->ucluster;
        usolve_cluster_fits(h->n, b->ucluster);   // kernel attributes of the chosen size
    }
    if (!b->Tah) {
        // A and A^T as tile-contiguous hi/lo planes (each GEMM tile of the X operand is
        // one contiguous 16 KB block in HBM)
        b->mpad = (int)((m + 7) / 8 * 8);
        BCK(gemm_configure());
        b->pair_clusters = std::min(batch_pair_clusters(h), h->num_sms / 2);
        b->tiles1 = (int)((m + 127) / 128);
        b->kb1 = (int)((N + 63) / 64);
        b->tiles2 = (int)((N + 127) / 128);
        b->kb2 = (int)((m + 63) / 64);
        const size_t e1 = (size_t)b->tiles1 * b->kb1 * 128 * 64, e2 = (size_t)b->tiles2 * b->kb2 * 128 * 64;
        BCKS(balloc((void**)&b->Tah, sizeof(unsigned short) * e1));
        BCKS(balloc((void**)&b->Tal, sizeof(unsigned short) * e1));
        BCKS(balloc((void**)&b->Tth, sizeof(unsigned short) * e2));
        BCKS(balloc((void**)&b->Ttl, sizeof(unsigned short) * e2));
        launch_tile_planes(h->P0, h->P1, h->m, h->N, 0, b->Tah, b->Tal, b->tiles1, b->kb1, s);
        launch_tile_planes(h->P0, h->P1, h->m, h->N, 1, b->Tth, b->Ttl, b->tiles2, b->kb2, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess)
            return set_last_error(TVCS_ERR_CUDA, "building the tiled planes of A and A^T: %s",
                                  cudaGetErrorString(e));
    }
    if (b->cap < count) {
        // keep the tiled planes of A and A^T, replace the per-image buffers
        free_buffers(b);
        const size_t B = (size_t)count;
        gemm_plan(h->m, h->N, h->num_sms, &b->p1);
        gemm_plan(h->N, h->m, h->num_sms, &b->p2);
        BCKS(upload_plan(b->p1, &b->tsb1, &b->ss1, s));
        BCKS(upload_plan(b->p2, &b->tsb2, &b->ss2, s));
        // the workspace holds the partial tiles of every candidate shape the tuner may pick
        size_t wsf = 0;
        for (int nt = 1; nt <= gemm_nt(count); ++nt) {
            std::vector<GemmShape> shapes = gemm_shape_candidates(h->num_sms, b->pair_clusters, nt);
            if (h->gemm_force[0] > 0) {
                shapes.push_back({h->gemm_force[0], h->gemm_force[1]});
                shapes.push_back({h->gemm_force[2], h->gemm_force[3]});
            }
            for (GemmShape g : shapes) {
                GemmPlan q1, q2;
                gemm_plan(h->m, h->N, g.grid, &q1, g.pair != 0, nt);
                gemm_plan(h->N, h->m, g.grid, &q2, g.pair != 0, nt);
                wsf = std::max(wsf, std::max(q1.ws_floats, q2.ws_floats));
            }
        }
        BCKS(balloc((void**)&b->ws, sizeof(float) * wsf));
        BCKS(balloc((void**)&b->U, sizeof(float) * B * N));
        BCKS(balloc((void**)&b->G, sizeof(float) * B * N));
        BCKS(balloc((void**)&b->W, sizeof(float) * B * 4 * N));
        BCKS(balloc((void**)&b->L, sizeof(float) * B * 4 * N));
        BCKS(balloc((void**)&b->R, sizeof(float) * B * m));
        BCKS(balloc((void**)&b->F, sizeof(float) * B * m));
        BCKS(balloc((void**)&b->mu, sizeof(float) * B));
        BCKS(balloc((void**)&b->Uh, sizeof(unsigned short) * B * N));
        BCKS(balloc((void**)&b->Ul, sizeof(unsigned short) * B * N));
        BCKS(balloc((void**)&b->Rh, sizeof(unsigned short) * B * b->mpad));
        BCKS(balloc((void**)&b->Rl, sizeof(unsigned short) * B * b->mpad));
        BCKS(balloc((void**)&b->ctrls, sizeof(Ctrl) * B));
        BCKS(balloc((void**)&b->bctrl, sizeof(Ctrl)));
        BCKS(balloc((void**)&b->r2part, sizeof(float2) * B * b->p1.tiles_m));
        BCKS(balloc((void**)&b->part, sizeof(double) * B * 2 * ((N + 255) / 256)));
        BCKS(balloc((void**)&b->slot_img, sizeof(int) * B));
        BCKS(balloc((void**)&b->img_slot, sizeof(int) * B));
        BCKS(balloc((void**)&b->img_slot_prev, sizeof(int) * B));
        BCK(cudaMallocHost((void**)&b->hctrls, sizeof(Ctrl) * B));
        BCK(cudaMallocHost((void**)&b->hbctrl, sizeof(Ctrl)));
        BCK(cudaMemsetAsync(b->Rh, 0, sizeof(unsigned short) * B * b->mpad, s));
        BCK(cudaMemsetAsync(b->Rl, 0, sizeof(unsigned short) * B * b->mpad, s));
        BCK(cudaMemsetAsync(b->Uh, 0, sizeof(unsigned short) * B * N, s));
        BCK(cudaMemsetAsync(b->Ul, 0, sizeof(unsigned short) * B * N, s));
        BCK(cudaMemsetAsync(b->F, 0, sizeof(float) * B * m, s));
        b->cap = count;
        b->tuned = false;
    }
    if (b->exec && b->graph_count != count) {   // the loop graph's launch shapes depend on count
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    b->last_count = count;
    BCKS(make_maps(h, count));
    if (b->p1.nt != gemm_nt(count)) b->tuned = false;   // 256 or 512 columns per X tile
    if (!b->tuned) {
        BCKS(tune_gemms(h, count));
        b->tuned = true;
    }
    return TVCS_OK;
}

// R = A U - F (R planes, ||r||^2 partials), then G = A^T R, for `count` images.
// compact: the GEMMs take the first bctrl->nact columns, column j being image
// slot_img[j] (the U and R planes are stored in that column order).  in_loop:
// the kernels return at once when bctrl->skip is set (every image has stopped).
void batch_products(tvcs_ctx* h, int count, bool subtract_f, cudaStream_t s, bool compact = false,
                    bool in_loop = false, bool g_partials = false)
{
    tvcs_batch* b = h->batch;
    const long long budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : (1LL << 31);
    const int* nact = compact ? &b->bctrl->nact : nullptr;
    const int* slot = compact ? b->slot_img : nullptr;
    const int chk = in_loop ? 1 : 0;
    // in the loop both GEMMs overlap the tail of the preceding kernel (the u-solve, R's
    // fix-up) with their first copies of A
    const int pdl = in_loop && h->pdl ? 1 : 0;
    launch_gemm(&b->mAh, &b->mAl, &b->mUh, &b->mUl, b->p1, b->ws, b->bctrl, chk, budget, s, count,
                nact, pdl);
    launch_gemm_fixup(b->ws, b->tsb1, b->ss1, h->m, b->p1.tiles_m, b->p1.nt * 256, count,
                      subtract_f ? b->F : nullptr, h->m, b->R, h->m, b->Rh, b->Rl, b->mpad,
                      b->r2part, b->bctrl, chk, s, slot, nact);
    launch_gemm(&b->mAth, &b->mAtl, &b->mRh, &b->mRl, b->p2, b->ws, b->bctrl, chk, budget, s, count,
                nact, pdl);
    if (g_partials) return;   // the next u-solve adds G's partial tiles itself
    launch_gemm_fixup(b->ws, b->tsb2, b->ss2, h->N, b->p2.tiles_m, b->p2.nt * 256, count, nullptr, 0, b->G, h->N,
                      nullptr, nullptr, 0, nullptr, b->bctrl, chk, s, slot, nact);
}

TvArgs batch_tv_args(tvcs_ctx* h, int count, int mode, bool compact = false)
{
    tvcs_batch* b = h->batch;
    TvArgs a{};
    a.u = b->U;
    a.w = b->W;
    a.lam = b->L;
    a.g = b->G;
    a.rhs_out = nullptr;
    a.tw = h->tw;
    a.s2 = h->s2;
    a.part = b->part;
    a.beta = (float)h->beta;
    a.mu_over_tau = (float)(h->mu / h->tau);
    a.mu = (float)h->mu;
    a.ctrl = b->ctrls;
    a.mode = mode;
    a.nimg = count;
    a.mu_img = b->mu;
    a.tau = (float)h->tau;
    a.u_hi = b->Uh;
    a.u_lo = b->Ul;
    a.img_slot = compact ? b->img_slot : nullptr;
    if (b->gfused) {   // g from the partial tiles of G = A^T R (k_usolve_reg128)
        a.gws = b->ws;
        a.gtsb = b->tsb2;
        a.gss = b->ss2;
        a.gws_cols = b->p2.nt * 256;
        a.img_slot_prev = compact ? b->img_slot_prev : nullptr;
    }
    return a;
}

void batch_usolve(tvcs_ctx* h, const TvArgs& a, cudaStream_t s)
{
    if (h->batch->ureg)
        launch_usolve_reg128(a, s);
    else if (h->batch->uimg)
        launch_usolve_img(h->n, a, s);
    else
        launch_usolve(h->n, h->batch->ucluster, a, s);
}

constexpr int BATCH_ITERS_PER_BODY = 4;

tvcs_status build_batch_graph(tvcs_ctx* h, int count)
{
    tvcs_batch* b = h->batch;
    if (b->exec) return TVCS_OK;
    BCK(cudaGraphCreate(&b->graph, 0));
    cudaGraphConditionalHandle ch;
    BCK(cudaGraphConditionalHandleCreate(&ch, b->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    BCK(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cs = h->cap_stream;
    BCK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
    // BATCH_ITERS_PER_BODY iterations per body (each pass through the WHILE node
    // costs several microseconds); once every image has stopped, the rest of the
    // body is skipped (the u-solves per image, the GEMMs and fix-ups on bctrl->skip)
    const bool compact = h->opt.batch_compact != 0;
    TvArgs a = batch_tv_args(h, count, MODE_ITER, compact);
    for (int k = 0; k < BATCH_ITERS_PER_BODY; ++k) {
        batch_usolve(h, a, cs);
        batch_products(h, count, true, cs, compact, true, b->gfused);
        launch_batch_cond(b->ctrls, count, b->bctrl, (unsigned long long)ch,
                          k + 1 == BATCH_ITERS_PER_BODY ? 1 : 0, cs,
                          compact ? b->slot_img : nullptr, compact ? b->img_slot : nullptr,
                          compact && b->gfused ? b->img_slot_prev : nullptr);
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    if (e != cudaSuccess)
        return set_last_error(TVCS_ERR_CUDA, "capture of the batched loop: %s", cudaGetErrorString(e));
    BCK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->graph_count = count;
    return TVCS_OK;
}

}  // namespace

int batch_pair_clusters(tvcs_ctx* h)
{
    if (h->pair_clusters < 0)
        h->pair_clusters = gemm_configure() == cudaSuccess ? gemm_pair_max_clusters(h->num_sms) : 0;
    return h->pair_clusters;
}

int batch_max(tvcs_ctx* h) { return batch_pair_clusters(h) > 0 ? BATCH_MAX : 256; }

void free_batch(tvcs_ctx* h)
{
    if (!h || !h->batch) return;
    tvcs_batch* b = h->batch;
    free_buffers(b);
    for (void* p : {(void*)b->Tah, (void*)b->Tal, (void*)b->Tth, (void*)b->Ttl})
        if (p) cudaFree(p);
    delete b;
    h->batch = nullptr;
}

// Back-to-back launches of one part of a batched iteration on the current batch
// state, between two events: 3 the two GEMM kernels, 4 their two fix-ups, 5 the
// batched u-solve.
tvcs_status time_batch_stage(tvcs_ctx* h, int stage, int reps, double* ms)
{
    tvcs_batch* b = h->batch;
    if (!b || b->cap == 0 || b->last_count <= 0)
        return set_last_error(TVCS_ERR_INVALID_ARG, "no batched state: call tvcs_solve_batched first");
    const int count = b->last_count;
    cudaStream_t s = h->stream;
    const long long budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : (1LL << 31);
    TvArgs a = batch_tv_args(h, count, MODE_PLAIN);
    BCK(cudaEventRecord(h->ev0, s));
    for (int i = 0; i < reps; ++i) {
        if (stage == 3) {
            launch_gemm(&b->mAh, &b->mAl, &b->mUh, &b->mUl, b->p1, b->ws, b->bctrl, 0, budget, s, count);
            launch_gemm(&b->mAth, &b->mAtl, &b->mRh, &b->mRl, b->p2, b->ws, b->bctrl, 0, budget, s, count);
        } else if (stage == 4) {
            launch_gemm_fixup(b->ws, b->tsb1, b->ss1, h->m, b->p1.tiles_m, b->p1.nt * 256, count, b->F, h->m, b->R,
                              h->m, b->Rh, b->Rl, b->mpad, b->r2part, b->bctrl, 0, s);
            if (!b->gfused)   // else the u-solve adds G's partials: no second fix-up in the loop
                launch_gemm_fixup(b->ws, b->tsb2, b->ss2, h->N, b->p2.tiles_m, b->p2.nt * 256, count, nullptr,
                                  0, b->G, h->N, nullptr, nullptr, 0, nullptr, b->bctrl, 0, s);
        } else {
            batch_usolve(h, a, s);
        }
    }
    BCK(cudaEventRecord(h->ev1, s));
    BCKS(sync_check(h, "timing a batched stage"));
    float t = 0.f;
    BCK(cudaEventElapsedTime(&t, h->ev0, h->ev1));
    *ms = t;
    return TVCS_OK;
}

tvcs_status apply_batch(tvcs_ctx* h, int count, const float* X, const float* Y, float* R, float* G)
{
    BCKS(ensure_batch(h, count));
    tvcs_batch* b = h->batch;
    cudaStream_t s = h->stream;
    const size_t N = h->N, m = h->m;
    BCK(cudaMemcpyAsync(b->U, X, sizeof(float) * count * N, cudaMemcpyDefault, s));
    if (Y) BCK(cudaMemcpyAsync(b->F, Y, sizeof(float) * count * m, cudaMemcpyDefault, s));
    BCK(cudaMemsetAsync(&b->bctrl->error, 0, sizeof(int), s));   // bounded waits report here
    launch_split_rows(b->U, count, h->N, h->N, b->Uh, b->Ul, h->N, s);
    batch_products(h, count, Y != nullptr, s);
    BCK(cudaMemcpyAsync(R, b->R, sizeof(float) * count * m, cudaMemcpyDefault, s));
    BCK(cudaMemcpyAsync(G, b->G, sizeof(float) * count * N, cudaMemcpyDefault, s));
    BCK(cudaMemcpyAsync(b->hbctrl, b->bctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    BCKS(sync_check(h, "batched products"));
    if (b->hbctrl->error == ERR_TIMEOUT)
        return set_last_error(TVCS_ERR_TIMEOUT, "a bounded device wait gave up");
    return TVCS_OK;
}

tvcs_status solve_batch(tvcs_ctx* h, int count, const float* const* f, float* const* u,
                        const double* mu, tvcs_result* res)
{
    BCKS(ensure_batch(h, count));
    tvcs_batch* b = h->batch;
    cudaStream_t s = h->stream;
    const size_t N = h->N, m = h->m;
    if (contiguous(f, count, m)) {   // one copy when the caller's arrays are back to back
        BCK(cudaMemcpyAsync(b->F, f[0], sizeof(float) * m * count, cudaMemcpyDefault, s));
    } else {
        for (int i = 0; i < count; ++i)
            BCK(cudaMemcpyAsync(b->F + i * m, f[i], sizeof(float) * m, cudaMemcpyDefault, s));
    }
    std::vector<float> mus(count);
    for (int i = 0; i < count; ++i) mus[i] = (float)(mu ? mu[i] : h->mu);
    BCK(cudaMemcpyAsync(b->mu, mus.data(), sizeof(float) * count, cudaMemcpyHostToDevice, s));
    BCK(cudaMemsetAsync(b->W, 0, sizeof(float) * count * 4 * N, s));
    BCK(cudaMemsetAsync(b->L, 0, sizeof(float) * count * 4 * N, s));
    memset(b->hctrls, 0, sizeof(Ctrl) * count);
    for (int i = 0; i < count; ++i) {
        b->hctrls[i].max_iter = h->opt.max_iter;
        b->hctrls[i].tol = h->tol;
        b->hctrls[i].algo = h->opt.algo;
    }
    BCK(cudaMemcpyAsync(b->ctrls, b->hctrls, sizeof(Ctrl) * count, cudaMemcpyHostToDevice, s));
    memset(b->hbctrl, 0, sizeof(Ctrl));
    b->hbctrl->loops_max = h->opt.max_iter + 2;
    b->hbctrl->nact = count;   // every image starts in its own column (identity slots)
    {
        std::vector<int> ident(count);
        for (int i = 0; i < count; ++i) ident[i] = i;
        BCK(cudaMemcpyAsync(b->slot_img, ident.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(b->img_slot, ident.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(b->img_slot_prev, ident.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
        BCK(cudaStreamSynchronize(s));   // the host vector goes out of scope
    }
    BCK(cudaMemcpyAsync(b->bctrl, b->hbctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    // u^0 = A^T f (reading C3) or 0: G = A^T F through the second GEMM.
    if (h->opt.init == TVCS_INIT_ZERO) {
        BCK(cudaMemsetAsync(b->U, 0, sizeof(float) * count * N, s));
    } else {
        launch_split_rows(b->F, count, h->m, h->m, b->Rh, b->Rl, b->mpad, s);
        const long long budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : (1LL << 31);
        launch_gemm(&b->mAth, &b->mAtl, &b->mRh, &b->mRl, b->p2, b->ws, b->bctrl, 0, budget, s, count);
        launch_gemm_fixup(b->ws, b->tsb2, b->ss2, h->N, b->p2.tiles_m, b->p2.nt * 256, count, nullptr, 0, b->U,
                          h->N, nullptr, nullptr, 0, nullptr, b->bctrl, 0, s);
    }
    launch_split_rows(b->U, count, h->N, h->N, b->Uh, b->Ul, h->N, s);
    batch_products(h, count, true, s, false, false, b->gfused);
    BCKS(build_batch_graph(h, count));
    BCK(cudaEventRecord(h->ev0, s));
    if (h->opt.max_iter > 0) BCK(cudaGraphLaunch(b->exec, s));
    BCK(cudaEventRecord(h->ev1, s));
    if (b->gfused) {
        // G = A^T R of every image at its final iterate (the loop left G in partial
        // tiles, in the columns of each iteration): R's planes in image order, the
        // second GEMM and its fix-up, the same values the loop's fix-ups wrote before
        const long long budget = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : (1LL << 31);
        launch_split_rows(b->R, count, h->m, h->m, b->Rh, b->Rl, b->mpad, s);
        launch_gemm(&b->mAth, &b->mAtl, &b->mRh, &b->mRl, b->p2, b->ws, b->bctrl, 0, budget, s, count);
        launch_gemm_fixup(b->ws, b->tsb2, b->ss2, h->N, b->p2.tiles_m, b->p2.nt * 256, count, nullptr, 0, b->G,
                          h->N, nullptr, nullptr, 0, nullptr, b->bctrl, 0, s);
    }
    // end of run, per image: ||r||^2 of the image's own residual recomputed on the CUDA
    // cores, final multiplier update, objective, residuals
    k_batch_resid<<<dim3((h->m + RS_BM - 1) / RS_BM, (count + RS_BB - 1) / RS_BB), 256, 0, s>>>(
        reinterpret_cast<const unsigned short*>(h->P0), reinterpret_cast<const unsigned short*>(h->P1),
        h->m, h->N, b->U, b->F, count, b->R);
    k_batch_resid_r2<<<count, 256, 0, s>>>(b->R, h->m, b->ctrls);
    TvArgs a = batch_tv_args(h, count, MODE_PLAIN);
    launch_tv(h->n, a, 4, s);
    launch_tv(h->n, a, 5, s);
    if (contiguous(u, count, N)) {
        BCK(cudaMemcpyAsync(u[0], b->U, sizeof(float) * N * count, cudaMemcpyDefault, s));
    } else {
        for (int i = 0; i < count; ++i)
            BCK(cudaMemcpyAsync(u[i], b->U + i * N, sizeof(float) * N, cudaMemcpyDefault, s));
    }
    BCK(cudaMemcpyAsync(b->hctrls, b->ctrls, sizeof(Ctrl) * count, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(b->hbctrl, b->bctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    BCKS(sync_check(h, "batched solve"));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    tvcs_status worst = TVCS_OK, err = TVCS_OK;
    for (int i = 0; i < count; ++i) {
        const Ctrl& c = b->hctrls[i];
        tvcs_status st = TVCS_OK;
        if (c.error == ERR_TIMEOUT)
            st = TVCS_ERR_TIMEOUT;
        else if (c.error == ERR_NONFINITE || !isfinite(c.tv) || !isfinite(c.r2))
            st = TVCS_ERR_DIVERGED;
        else if (h->tol > 0.0 && !c.stop_by_tol)
            st = TVCS_NOT_CONVERGED;
        if (st < 0)
            err = st;
        else if (st > worst)
            worst = st;
        if (res) {
            tvcs_result& r = res[i];
            r.iters = c.it;
            r.status = st;
            r.stopped_by_tol = c.stop_by_tol;
            r.rel_change = ctrl_relchg(c);
            r.tv = c.tv;
            r.resid2 = c.r2;
            r.objective = c.tv + 0.5 * mus[i] * c.r2;
            r.kkt_primal = sqrt(c.kkt_p2);
            r.kkt_dual = sqrt(c.kkt_d2);
            r.lambda_max_norm = c.lam_max;
            r.ms = ms;
        }
    }
    if (err < 0) return set_last_error(err, "an image of the batch failed (see its result)");
    return worst;
}

}  // namespace tvcs
