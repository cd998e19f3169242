// The solver handle (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "tvcs.h"

#include <vector>

// Device state of the batched path (many images sharing the handle's A).
struct tvcs_batch {
    int cap = 0;                   // images the buffers hold
    int mpad = 0;                  // m rounded up to a multiple of 8 (bf16 row pitch)
    // the GEMMs' X operands, A (m x N) and A^T (N x m), as tile-contiguous bf16 hi/lo
    // planes: tiles x kb tiles of 128 x 64 values, 16 KB each (launch_tile_planes)
    unsigned short *Tah = nullptr, *Tal = nullptr, *Tth = nullptr, *Ttl = nullptr;
    int tiles1 = 0, kb1 = 0, tiles2 = 0, kb2 = 0;
    float *U = nullptr, *W = nullptr, *L = nullptr, *G = nullptr, *R = nullptr, *F = nullptr;
    float* mu = nullptr;           // per-image mu
    unsigned short *Uh = nullptr, *Ul = nullptr, *Rh = nullptr, *Rl = nullptr;
    tvcs::Ctrl* ctrls = nullptr;         // per image
    tvcs::Ctrl* hctrls = nullptr;        // pinned host mirror
    tvcs::Ctrl* bctrl = nullptr;         // loop control of the batch
    tvcs::Ctrl* hbctrl = nullptr;
    float2* r2part = nullptr;   // double-single ||r||^2 partials
    double* part = nullptr;
    float* ws = nullptr;           // stream-K partial tiles
    tvcs::GemmPlan p1, p2;               // R = A U - F (M = m, K = N) and G = A^T R (M = N, K = m)
    int *tsb1 = nullptr, *ss1 = nullptr, *tsb2 = nullptr, *ss2 = nullptr;
    int *slot_img = nullptr, *img_slot = nullptr;   // compaction: column -> image, image -> column
    int* img_slot_prev = nullptr;  // image -> column in the GEMMs of the iteration that just ended
    CUtensorMap mAh, mAl, mAth, mAtl, mUh, mUl, mRh, mRl;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_count = 0;           // images the loop graph was built for
    int last_count = 0;            // images of the last batched call
    int ucluster = 0;              // cluster size of the batched u-solve
    bool uimg = false;             // the u-solve runs one block per image (k_usolve_img)
    bool ureg = false;             // n = 128: one block per image, transforms in registers (k_usolve_reg.cu)
    bool gfused = false;           // the u-solve adds the partial tiles of G = A^T R (no second fix-up in the loop)
    bool tuned = false;            // the GEMM launch shapes have been picked for these buffers
    int pair_clusters = 0;         // clusters of two GEMM blocks resident at once (0: no pair kernel)
};

// Products with A regenerated in the kernel (handles created with
// TVCS_A_REGENERATE): a small device table of (x, y, r, g) pointer sets, one
// per call pattern of the handle, and the partial-slot buffers.
struct tvcs_regen {
    tvcs::RegenPlan plan;
    tvcs::RegenProb* dtab = nullptr;       // device entries
    std::vector<tvcs::RegenProb> htab;     // host copies, same order
    float* gslot = nullptr;
    float2* r2slot = nullptr;    // double-single ||r||^2 partials
    int* pre = nullptr;
};
struct tvcs_uneven;   // state of the uneven batch (regen.cu)

struct tvcs_ctx {
    int dev = 0, num_sms = 0, ucluster = 0;
    int pdl = 1;                   // the loop's product launch overlaps the u-solve's tail
    int m = 0, n = 0, N = 0, P = 0;
    double mu = 0, beta = 0, tol = 0, tau = 0;
    tvcs_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    // device buffers
    float* A = nullptr;            // binary32 A for the single-block-row product kernel (n <= 128)
    bool use_q = false;            // products by clusters / reduced precision (k_products_q)
    unsigned char *P0 = nullptr, *P1 = nullptr;   // storage planes of A on that path
    float* rscale = nullptr;       // per-row scales of the fp8 storage
    float *f = nullptr, *u = nullptr, *w = nullptr, *lam = nullptr, *g = nullptr, *r = nullptr,
          *rhs = nullptr, *zeroN = nullptr;
    float *tx = nullptr, *ty = nullptr, *tr = nullptr, *tg = nullptr;
    float2* spec = nullptr;
    float2* tw = nullptr;
    float* s2 = nullptr;
    float *gpart = nullptr, *gpart2 = nullptr;
    float2* r2part = nullptr;   // double-single ||r||^2 partials
    double* part = nullptr;
    tvcs::Ctrl* ctrl = nullptr;
    tvcs::Ctrl* hctrl = nullptr;  // pinned host mirror
    // loop graph (a WHILE node over bodies of 16 iterations) and the graphs of
    // 1..15 iterations that end a run whose length is not a multiple of 16
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t tail[16] = {};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool state_ready = false;
    tvcs_batch* batch = nullptr;
    uint64_t seed = 0;
    tvcs_regen* regen = nullptr;   // set for TVCS_A_REGENERATE
    bool dct = false;              // partial-DCT encoder (tvcs_create_partial_dct)
    float* dctC = nullptr;         // n x n DCT matrix, its transpose, 2 n x n scratch
    int *dsidx = nullptr, *dsperm = nullptr, *drowptr = nullptr;
    tvcs_uneven* uneven = nullptr; // uneven batch whose first handle is this one
    int bar_extra = 0;             // timeout test hook (tvcs_test_hold_grid_barrier), else 0
    int gemm_force[4] = {0, 0, 0, 0};   // tvcs_test_gemm_shape: grid, pair of each batched GEMM (0: tuner)
    int pair_clusters = -1;        // clusters of two GEMM blocks that fit (-1: not asked yet)
};

namespace tvcs {
// Images one shared-A batch holds (one thread per image in the batch condition
// kernel's slot tables); larger calls run in groups.  Above 256 images the GEMMs
// need the CTA-pair kernel (two N tiles per X tile), so a device on which that
// kernel cannot run holds 256 (batch_max).
constexpr int BATCH_MAX = 512;
int batch_max(tvcs_ctx* h);
// Clusters of two GEMM blocks that fit on the handle's device (0: none).
int batch_pair_clusters(tvcs_ctx* h);
tvcs_status set_last_error(tvcs_status s, const char* fmt, ...);
void free_batch(tvcs_ctx* h);
// Many images with the handle's A (all handles of a tvcs_solve_batched call equal).
tvcs_status solve_batch(tvcs_ctx* h, int count, const float* const* f, float* const* u,
                        const double* mu, tvcs_result* res);
tvcs_status apply_batch(tvcs_ctx* h, int count, const float* X, const float* Y, float* R,
                        float* G);
tvcs_status time_batch_stage(tvcs_ctx* h, int stage, int reps, double* ms);
// Regenerated-A products of one handle (regen.cu).
tvcs_status regen_init(tvcs_ctx* h);
void regen_products(tvcs_ctx* h, const float* x, const float* y, float* r, float* g, int mode,
                    unsigned long long cond, int set_cond, cudaStream_t s);
void free_regen(tvcs_ctx* h);
// Many problems of different sizes, all with regenerated A, in one loop graph.
bool uneven_eligible(const tvcs_handle* hs, int count);
tvcs_status solve_uneven(const tvcs_handle* hs, int count, const float* const* f, float* const* u,
                         const double* mu, tvcs_result* res);
tvcs_status time_uneven_stage(tvcs_ctx* h, int stage, int reps, double* ms);
}  // namespace tvcs
