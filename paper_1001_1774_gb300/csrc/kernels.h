// Host-side launchers of the solver kernels (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace tvcs {

struct Ctrl;

// Arguments of the TV / FFT kernels (rows a1-a5) and the end-of-run kernels.
struct TvArgs {
    float* u;
    float* w;           // 2 copies x 2 planes x N
    float* lam;         // 2 copies x 2 planes x N
    const float* g;     // g = A^T (A u - f), N values
    float* rhs_out;     // nullable
    float2* spec;       // n x (n/2+1)
    const float2* tw;   // n twiddles (cos, sin)(2 pi t / n)
    const float* s2;    // n values 4 sin^2(pi k / n)
    double* part;       // per-block binary64 partials (>= 2 * max blocks)
    float beta, mu_over_tau, mu;
    Ctrl* ctrl;                 // per image when nimg > 1 (ctrl + b)
    int mode;
    // batches of images (the u-solve and the end-of-run kernels)
    int nimg;                   // images (grid y); 0 or 1 for one image
    const float* mu_img;        // nullable: per-image mu
    const float* tau_img;       // nullable: per-image tau (used with mu_img)
    float tau;
    unsigned short* u_hi;       // nullable: bf16 hi/lo planes of the new u
    unsigned short* u_lo;
    const int* img_slot;        // nullable: row of image b's planes (compacted batch), else b
    int pdl;                    // launch with a programmatic dependency on the preceding grid
    // k_usolve_reg128 only: g read as the sum of the stream-K partial tiles of the
    // G = A^T R GEMM (tile t = image row t), in the order the fix-up adds them, when
    // gws is set; the image's column in that GEMM is img_slot_prev[b] (else b)
    const float* gws;
    const int* gtsb;            // per tile: first segment (the GEMM plan's tile_seg_begin)
    const int* gss;             // workspace slot of each segment (seg_slot)
    int gws_cols;               // columns of a partial tile
    const int* img_slot_prev;
};

bool tv_supported(int n);
// which: 4 final1 (pending multiplier update, TV, ||w - D u||), 5 final2 (dual residual)
void launch_tv(int n, const TvArgs& a, int which, cudaStream_t s);

// Rows a1-a5 (multiplier update, shrink, right-hand side, FFT u-solve, stop
// norms) as one thread-block-cluster launch.  usolve_choose_cluster returns the
// cluster size used for n on the current device (16 or 8), 0 if none fits;
// it also sets the kernel attributes and must run before launch_usolve.
int usolve_choose_cluster(int n);
bool usolve_cluster_fits(int n, int c);   // also sets the kernel attributes
void launch_usolve(int n, int cluster, const TvArgs& a, cudaStream_t s);
// The same rows for batches, one block per image (k_usolve_img.cu, n <= 128):
// usolve_img_configure sets the kernel attributes, false if n has no variant.
bool usolve_img_configure(int n);
void launch_usolve_img(int n, const TvArgs& a, cudaStream_t s);
// The same rows for batches of 128 x 128 images with the 128-point transforms in
// the registers of one warp (k_usolve_reg.cu): no block barrier inside a phase.
bool usolve_reg_configure();
void launch_usolve_reg128(const TvArgs& a, cudaStream_t s);

// Fused single-pass products r = A x - y, gpart = per-block partials of A^T r.
struct ProdArgs {
    const float* A;
    int m;
    const float* x;
    const float* y;     // nullable
    float* r;
    float* gpart;       // grid x N
    float* g_out;       // nullable: when set, the blocks meet at a grid barrier (cooperative
                        // launch) and reduce the partials into g_out = A^T r themselves
    float2* r2part;     // grid, double-single ||r||^2 partials
    Ctrl* ctrl;
    int mode;           // MODE_PLAIN or MODE_ITER
    unsigned long long cond;  // cudaGraphConditionalHandle (MODE_ITER inside the loop graph)
    int set_cond;
    long long budget;   // spin-wait bound, SM cycles
    int pdl;            // launch with a programmatic dependency on the preceding grid
    int bar_extra;      // 0; > 0 only in the timeout test: the grid barrier's target is
                        // raised by this many arrivals, which never come
};

bool prod_supported(int n);
int prod_grid(int n, int m, int num_sms);   // number of blocks = number of partials P
cudaError_t prod_configure(int n);          // opt-in shared memory size (call once per device)
// Both return the launch's own status.
cudaError_t launch_products(int n, int grid, const ProdArgs& a, cudaStream_t s);
// g = sum_p gpart[p] (fixed order), wide grid; skipped when mode == MODE_ITER and ctrl->skip.
cudaError_t launch_greduce(const float* gpart, int P, int N, float* g, const Ctrl* ctrl, int mode,
                           cudaStream_t s);

// Products with A in binary32 (n = 192, 256), bf16 hi+lo, or fp8 e4m3 + bf16
// correction: clusters of CS blocks split each row's columns.
struct QProdArgs {
    const unsigned char* P0;  // binary32 plane | bf16 hi plane | e4m3 plane
    const unsigned char* P1;  // unused | bf16 lo plane | bf16 correction plane
    const float* rscale;      // per-row scale (fp8 storage), else unused
    int m;
    const float* x;
    const float* y;           // nullable
    float* r;
    float* gpart;             // clusters x N
    float2* r2part;           // clusters, double-single ||r||^2 partials
    Ctrl* ctrl;
    int mode;
    unsigned long long cond;
    int set_cond;
    long long budget;
};
bool qprod_supported(int prec, int n);
int qprod_cluster_size(int prec, int n);
int qprod_grid_clusters(int prec, int n, int m);   // sets kernel attributes; 0 if none fits
void launch_qproducts(int prec, int n, int clusters, const QProdArgs& a, cudaStream_t s);
void launch_split_bf16x2(const float* A, void* hi, void* lo, long long count, cudaStream_t s);
void launch_quant_fp8(const float* A, int m, int N, void* q, void* c, float* scale, cudaStream_t s);

// Batched products as tcgen05 BF16x3 GEMMs with stream-K scheduling (k_gemm.cu).
struct GemmPlan {
    int tiles_m = 0, kblocks = 0, grid = 0, smax = 1;   // tiles_m: 128-row tiles of the fix-up
    int pair = 0;    // 1: CTA pairs (k_gemm_bf16x3_pair) on 256-row tiles
    int nt = 1;      // N tiles of 256 columns per X tile (2: up to 512 images, pairs only)
    int tiles = 0;   // the kernel's tiles (128 or 256 rows)
    std::vector<int> tile_seg_begin;   // tiles_m + 1 offsets into seg_slot
    std::vector<int> seg_slot;         // workspace slot of each segment, per tile in K order
    size_t ws_floats = 0;
};
// grid: blocks of the launch (pair: rounded down to whole pairs); every plan
// covers W = tiles x kblocks with at most W units (blocks or pairs).
void gemm_plan(int M, int K, int grid, GemmPlan* p, bool pair = false, int nt = 1);
cudaError_t gemm_configure();
// Clusters of two GEMM blocks that fit on the device at once (0: the pair
// kernel cannot run).
int gemm_pair_max_clusters(int num_sms);
bool make_bf16_map(CUtensorMap* map, const void* base, int inner, int rows, int ld, int box_rows);
// The Y operand's tensor maps use boxes of GEMM_Y_BOX rows.  ncols: columns
// (images) of Y; nact (nullable): the number of leading columns that take part,
// read on the device.  The MMAs run with N = min(ncols, nact) rounded up to 32.
constexpr int GEMM_Y_BOX = 32;
// The fix-up adds a tile's first GEMM_FX_SEG partials (zeros past the last
// segment) and then the rest, each from 0 in K order; readers of the partials
// that stand in for the fix-up add them the same way.
constexpr int GEMM_FX_SEG = 6;
void launch_gemm(const CUtensorMap* xh, const CUtensorMap* xl, const CUtensorMap* yh,
                 const CUtensorMap* yl, const GemmPlan& p, float* ws, Ctrl* ctrl, int check_skip,
                 long long budget, cudaStream_t s, int ncols, const int* nact = nullptr,
                 int pdl = 0);
// Column j of the GEMM is image slot_img[j] (identity when slot_img is null) for
// F, out and r2part; the bf16 planes out_hi/out_lo stay in column order.  With
// nact set, only the first *nact columns are processed.
// pdl: launch with a programmatic dependency on the preceding kernel (the GEMM issues
// its first stages' copies of A before it waits for that kernel's output).
// ws_cols: columns of a partial tile in the workspace (256 x the plan's nt).
void launch_gemm_fixup(const float* ws, const int* tile_seg_begin, const int* seg_slot, int M,
                       int tiles_m, int ws_cols, int count, const float* F, int ldf, float* out, int ldo,
                       void* out_hi, void* out_lo, int ldh, float2* r2part, const Ctrl* ctrl,
                       int check_skip, cudaStream_t s, const int* slot_img = nullptr,
                       const int* nact = nullptr);
void launch_split_rows(const float* v, int count, int len, int ld, void* hi, void* lo, int ldh,
                       cudaStream_t s);
// Tile-contiguous hi/lo planes of X = A (trans 0) or A^T (trans 1) for the
// batched GEMMs, from A's planes Ph/Pl (m x N): tiles_m x kblocks tiles of
// 128 x 64, tile (t, kb) at index t * kblocks + kb (k_gemm.cu).
void launch_tile_planes(const void* Ph, const void* Pl, int m, int N, int trans, void* Th,
                        void* Tl, int tiles_m, int kblocks, cudaStream_t s);

// Products with A regenerated inside the kernel (k_regen.cu): r = A x - y and
// g = A^T r for many problems of different sizes in one persistent launch.
// Problem p's rows are cut into `chunks` chunks of rows_per_chunk rows; the
// clusters take contiguous ranges of the active chunks.  A cluster keeps one
// partial A^T r per run of consecutive chunks of one problem, written to the
// slot of the run's first chunk; k_regen_reduce adds the slots in chunk order.
struct RegenProb {
    unsigned long long seed;
    const float* x;      // N
    const float* y;      // m, nullable (y = 0)
    float* r;            // m
    float* g;            // N, written by the reduction
    float* gslot;        // chunks x N partial slots
    float2* r2slot;      // chunks, double-single ||r||^2 partials
    Ctrl* ctrl;          // receives r2; with MODE_ITER, ctrl->skip marks a problem as inactive
    int m, N;
    int rows_per_chunk, chunks;
    float scale;         // binary32(1/sqrt(m))
    int pad;
};
struct RegenPlan {
    int cs = 8;          // cluster size (blocks splitting each row's columns)
    int tile_cap = 0;    // floats of one tile buffer (rows per tile = tile_cap / (N / cs), power of 2)
    int wmax = 0;        // max over problems of N / cs
    int minb = 2;        // kernel variant: registers budgeted for 2, 3 or 4 blocks per SM
    int nbuf = 2;        // kernel variant: tile buffers (2: generation overlaps the exchange)
    int pcap = 1;        // problems a launch may carry (<= REGEN_PMAX; sizes a shared-memory table)
    int clusters = 0;    // persistent grid, in clusters
    size_t smem = 0;
};
constexpr int REGEN_PMAX = 1024;   // problems per launch
// Fills plan->clusters and plan->smem for (cs, tile_cap, wmax); false if no cluster fits.
bool regen_configure(RegenPlan* plan);
// Rows per tile for a problem of N columns under `plan` (a power of 2 <= 16).
int regen_tile_rows(const RegenPlan& plan, int N);
void launch_regen(const RegenProb* probs, int P, int mode, const RegenPlan& plan, int* pre_out,
                  cudaStream_t s);
// g of every active problem from its slots, ctrl->r2 from its r2 slots; with
// set_cond, probs[0].ctrl drives the loop condition (single-problem loops).
void launch_regen_reduce(const RegenProb* probs, int P, int maxN, int mode, const RegenPlan& plan,
                         const int* pre, unsigned long long cond, int set_cond, cudaStream_t s);

// Products with the partial-DCT encoder (k_dct.cu): r = (C U C^T)[rows] - y and
// g = C^T S C, one thread-block cluster.  The sampled coefficients are given in
// increasing index order (sidx) with their positions in the caller's order
// (sperm); rowptr[k] = first sorted entry with index >= k n (n + 1 values).
struct DctArgs {
    const float* C;      // n x n orthonormal DCT-II matrix, then its transpose, binary32
    const float* x;      // n*n
    const float* y;      // m, nullable
    const int* sidx;
    const int* sperm;
    const int* rowptr;
    float* r;            // m (caller's order)
    float* g;            // n*n
    float* scratch;      // 2 n*n, exchange of the bands between the cluster's blocks
    Ctrl* ctrl;          // receives r2; MODE_ITER bookkeeping as the other product kernels
    int mode;
    unsigned long long cond;
    int set_cond;
    int pdl;             // launched as a programmatic dependent of the preceding kernel
};
bool dct_supported(int n);
bool dct_configure(int n);   // kernel attributes (call once per device)
void launch_dct_products(int n, const DctArgs& a, cudaStream_t s);

// Loop condition of a batch: continue while any of ctrls[0..count) runs and
// bctrl->loops stays below bctrl->loops_max (batch.cu).
// With slot_img / img_slot set (count <= 512), also packs the running images
// into the leading slots in image order: slot_img[0 .. nact), img_slot[b] (-1 for
// an image that stopped), bctrl->nact; img_slot_prev (nullable) receives the
// slots of the iteration that just ended.
void launch_batch_cond(const Ctrl* ctrls, int count, Ctrl* bctrl, unsigned long long cond,
                       int set_cond, cudaStream_t s, int* slot_img = nullptr,
                       int* img_slot = nullptr, int* img_slot_prev = nullptr);

// gather: out = scale * sum_p gpart[p], ctrl->vec2 = ||out||^2 (binary64)
void launch_gather(const float* gpart, int P, int N, float scale, float* out, double* part,
                   Ctrl* ctrl, cudaStream_t s);
// v = z / sqrt(ctrl->vec2)
void launch_normalize(const float* z, float* v, int N, const Ctrl* ctrl, cudaStream_t s);
void launch_fill(float* v, int N, float value, cudaStream_t s);
// it, max_iter, done, skip, stop_by_tol, loops, loops_max, tol, error, algo and the
// tickets of a control block for a new run
void launch_run_begin(Ctrl* c, int max_iter, int loops_max, double tol, int algo, cudaStream_t s);

// Gaussian encoding matrix rows from the counter-based generator.
void launch_gen_gauss(float* A, int m, int64_t N, uint64_t seed, float scale, cudaStream_t s);

}  // namespace tvcs
