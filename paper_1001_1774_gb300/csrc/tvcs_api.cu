// C ABI of the solver (declared in include/tvcs.h): handle lifetime, the
// iteration loop as a CUDA graph with a device-driven WHILE node, state access
// and the products entry point.  All arithmetic happens in the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "kernels.h"
#include "tvcs.h"

using namespace tvcs;

namespace {

thread_local std::string g_last_error;

tvcs_status fail(tvcs_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? TVCS_ERR_OOM : TVCS_ERR_CUDA,       \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                      \
        }                                                                                     \
    } while (0)

#define CKS(expr)                                  \
    do {                                           \
        tvcs_status s_ = (expr);                   \
        if (s_ != TVCS_OK) return s_;              \
    } while (0)

std::mutex g_cfg_mutex;
std::set<std::pair<int, int>> g_configured;  // (device, n) with the product kernel configured

}  // namespace

namespace {

long long budget_of(const tvcs_ctx* h)
{
    return h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : (1LL << 31);
}

TvArgs tv_args(tvcs_ctx* h, int mode, bool stage_outputs)
{
    TvArgs a{};
    a.u = h->u;
    a.w = h->w;
    a.lam = h->lam;
    a.g = h->g;
    a.rhs_out = stage_outputs ? h->rhs : nullptr;
    a.spec = h->spec;
    a.tw = h->tw;
    a.s2 = h->s2;
    a.part = h->part;
    a.beta = (float)h->beta;
    a.mu_over_tau = (float)(h->mu / h->tau);
    a.mu = (float)h->mu;
    a.ctrl = h->ctrl;
    a.mode = mode;
    return a;
}

// r = A x - y and the partials of A^T r into gpart; then g = their sum when g != NULL.
void products(tvcs_ctx* h, const float* x, const float* y, float* r, float* gpart, float* g,
              int mode, unsigned long long cond, int set_cond, cudaStream_t s, int pdl = 0)
{
    if (h->regen) {   // A regenerated in the kernel; A^T r whole in g, else in gpart (P = 1)
        regen_products(h, x, y, r, g ? g : gpart, mode, cond, set_cond, s);
        return;
    }
    if (h->dct) {     // partial-DCT encoder; A^T r whole in g, else in gpart (P = 1)
        DctArgs d{};
        d.C = h->dctC;
        d.scratch = h->dctC + 2 * (size_t)h->n * h->n;
        d.x = x;
        d.y = y;
        d.sidx = h->dsidx;
        d.sperm = h->dsperm;
        d.rowptr = h->drowptr;
        d.r = r;
        d.g = g ? g : gpart;
        d.ctrl = h->ctrl;
        d.mode = mode;
        d.cond = cond;
        d.set_cond = set_cond;
        d.pdl = pdl;
        launch_dct_products(h->n, d, s);
        return;
    }
    if (h->use_q) {
        QProdArgs q{};
        q.P0 = h->P0;
        q.P1 = h->P1;
        q.rscale = h->rscale;
        q.m = h->m;
        q.x = x;
        q.y = y;
        q.r = r;
        q.gpart = gpart;
        q.r2part = h->r2part;
        q.ctrl = h->ctrl;
        q.mode = mode;
        q.cond = cond;
        q.set_cond = set_cond;
        q.budget = budget_of(h);
        launch_qproducts(h->opt.precision, h->n, h->P, q, s);
        if (g) launch_greduce(gpart, h->P, h->N, g, h->ctrl, mode, s);
        return;
    }
    ProdArgs a{};
    a.A = h->A;
    a.m = h->m;
    a.x = x;
    a.y = y;
    a.r = r;
    a.gpart = gpart;
    a.r2part = h->r2part;
    a.ctrl = h->ctrl;
    a.mode = mode;
    a.cond = cond;
    a.set_cond = set_cond;
    a.g_out = g;
    a.budget = budget_of(h);
    a.pdl = pdl;
    a.bar_extra = h->bar_extra;
    launch_products(h->n, h->P, a, s);
}

// One iteration (rows a1-a7), MODE_ITER: the cluster u-solve, then the products
// with the reduction of their partials into g.  With pdl_first the
// u-solve is launched with a programmatic dependency on the preceding product
// kernel (inside a graph body; not across the WHILE node's iterations).
void launch_iteration(tvcs_ctx* h, unsigned long long cond, int set_cond, cudaStream_t s,
                      bool pdl_first)
{
    TvArgs a = tv_args(h, MODE_ITER, false);
    a.pdl = (pdl_first && h->pdl) ? 1 : 0;
    launch_usolve(h->n, h->ucluster, a, s);
    products(h, h->u, h->f, h->r, h->gpart, h->g, MODE_ITER, cond, set_cond, s, h->pdl);
}

tvcs_status sync_and_check(tvcs_ctx* h, const char* what)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(TVCS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TVCS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return TVCS_OK;
}

tvcs_status read_ctrl(tvcs_ctx* h)
{
    CK(cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    return sync_and_check(h, "reading the control block");
}

// Writes selected control fields from the host (the rest are preserved).
tvcs_status write_ctrl(tvcs_ctx* h)
{
    CK(cudaMemcpyAsync(h->ctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
    return TVCS_OK;
}

// The loop graphs capture launch arguments (beta, mu, test hooks): destroyed
// whenever one of them changes, rebuilt on the next run.
void drop_loop_graphs(tvcs_ctx* h)
{
    if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    for (cudaGraphExec_t& t : h->tail)
        if (t) { cudaGraphExecDestroy(t); t = nullptr; }
}

void free_ctx(tvcs_ctx* h)
{
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_batch(h);
    free_regen(h);
    drop_loop_graphs(h);
    void* bufs[] = {h->A, h->f, h->u, h->w, h->lam, h->g, h->r, h->rhs, h->zeroN, h->tx, h->ty,
                    h->tr, h->tg, h->spec, h->tw, h->s2, h->gpart, h->gpart2, h->r2part, h->part,
                    h->ctrl, h->P0, h->P1, h->rscale, h->dctC, h->dsidx, h->dsperm, h->drowptr};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (h->hctrl) cudaFreeHost(h->hctrl);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

tvcs_status alloc(void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(TVCS_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    return TVCS_OK;
}

// Runs the iteration body in a loop graph: K1 -> column pass -> inverse rows ->
// products; the products kernel sets the WHILE condition from ctrl->done.
constexpr int ITERS_PER_BODY = 16;

tvcs_status build_tail(tvcs_ctx* h, int iters);

// The WHILE graph and the graphs of 1 .. 15 iterations that end runs whose
// length is not a multiple of the body, all built (and uploaded to the device)
// at once, so that no later call pays for a capture or a first-launch upload.
tvcs_status build_graph(tvcs_ctx* h)
{
    if (h->exec) return TVCS_OK;
    CK(cudaGraphCreate(&h->graph, 0));
    cudaGraphConditionalHandle ch;
    CK(cudaGraphConditionalHandleCreate(&ch, h->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, h->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    // ITERS_PER_BODY iterations per body, so that all kernel boundaries but the
    // one across the WHILE node are programmatic; the rest of a body is skipped
    // once an iteration ends the run
    for (int k = 0; k < ITERS_PER_BODY; ++k)
        launch_iteration(h, (unsigned long long)ch, k + 1 == ITERS_PER_BODY ? 1 : 0,
                         h->cap_stream, k > 0);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &captured);
    if (e != cudaSuccess) return fail(TVCS_ERR_CUDA, "capture of the loop body: %s", cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&h->exec, h->graph, 0));
    CK(cudaGraphUpload(h->exec, h->stream));
    for (int r = 1; r < ITERS_PER_BODY; ++r) CKS(build_tail(h, r));
    return TVCS_OK;
}

// A plain graph of `iters` (1..15) iterations: the end of a run whose length is
// not a multiple of the loop body, so that a run launches exactly its iterations.
tvcs_status build_tail(tvcs_ctx* h, int iters)
{
    if (h->tail[iters]) return TVCS_OK;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < iters; ++k) launch_iteration(h, 0ull, 0, h->cap_stream, k > 0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) return fail(TVCS_ERR_CUDA, "capture of the run's last iterations: %s",
                                      cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->tail[iters], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->tail[iters] = nullptr;
        return fail(TVCS_ERR_CUDA, "instantiating the run's last iterations: %s",
                    cudaGetErrorString(e));
    }
    CK(cudaGraphUpload(h->tail[iters], h->stream));
    return TVCS_OK;
}

// (Re)computes r = A u - f and the partials of g = A^T r for the current u.
void refresh_products(tvcs_ctx* h)
{
    products(h, h->u, h->f, h->r, h->gpart, h->g, MODE_PLAIN, 0ull, 0, h->stream);
}

tvcs_status init_state(tvcs_ctx* h, int init)
{
    const size_t N = (size_t)h->N;
    if (init == TVCS_INIT_GIVEN) {
        // Warm start: keep the caller's u and lambda (tvcs_set_state), w^0 = 0.
        if (!h->state_ready) return fail(TVCS_ERR_INVALID_ARG, "INIT_GIVEN needs tvcs_set_state(U) first");
        refresh_products(h);
        CKS(read_ctrl(h));   // after the kernels: the host copy is current
        const int par = h->hctrl->wpar;
        CK(cudaMemsetAsync(h->w + (size_t)par * 2 * N, 0, sizeof(float) * 2 * N, h->stream));
        h->hctrl->pending = 0;
        h->hctrl->error = 0;
        return write_ctrl(h);
    }
    CK(cudaMemsetAsync(h->w, 0, sizeof(float) * 4 * N, h->stream));
    CK(cudaMemsetAsync(h->lam, 0, sizeof(float) * 4 * N, h->stream));
    if (init == TVCS_INIT_ATF) {
        // u^0 = A^T f (reading C3): the products at x = 0 give A^T (0 - f).
        products(h, h->zeroN, h->f, h->r, h->gpart, nullptr, MODE_PLAIN, 0ull, 0, h->stream);
        launch_gather(h->gpart, h->P, h->N, -1.0f, h->u, h->part, h->ctrl, h->stream);
    } else if (init == TVCS_INIT_ZERO) {
        CK(cudaMemsetAsync(h->u, 0, sizeof(float) * N, h->stream));
    }
    refresh_products(h);
    CKS(read_ctrl(h));
    h->hctrl->pending = 0;
    h->hctrl->wpar = 0;
    h->hctrl->error = 0;
    CKS(write_ctrl(h));
    h->state_ready = true;
    return TVCS_OK;
}

// Runs up to `iters` iterations from the current state; tol > 0 enables eq. (stop).
tvcs_status run_loop(tvcs_ctx* h, int iters, double tol, tvcs_result* res)
{
    // whole loop bodies in the WHILE graph, the remainder in a graph of its own
    const int nbody = iters / ITERS_PER_BODY, rest = iters % ITERS_PER_BODY;
    if (!h->opt.host_loop) CKS(build_graph(h));
    Ctrl& c = *h->hctrl;
    // loops_max: bodies of the WHILE graph (each ends by checking this bound)
    launch_run_begin(h->ctrl, iters, nbody, tol, h->opt.algo, h->stream);
    CK(cudaEventRecord(h->ev0, h->stream));
    if (iters > 0) {
        if (h->opt.host_loop) {
            // Same kernels launched from the host, one iteration at a time (for
            // profilers that cannot look inside graphs with conditional nodes).
            for (int k = 0; k < iters; ++k) launch_iteration(h, 0ull, 0, h->stream, false);
        } else {
            if (nbody > 0) CK(cudaGraphLaunch(h->exec, h->stream));
            if (rest > 0) CK(cudaGraphLaunch(h->tail[rest], h->stream));
        }
    }
    CK(cudaEventRecord(h->ev1, h->stream));
    // End of run: final multiplier update, objective and optimality residuals.
    TvArgs a = tv_args(h, MODE_PLAIN, false);
    launch_tv(h->n, a, 4, h->stream);
    launch_tv(h->n, a, 5, h->stream);
    CKS(read_ctrl(h));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    tvcs_status st = TVCS_OK;
    if (c.error == ERR_TIMEOUT)
        st = fail(TVCS_ERR_TIMEOUT, "a bounded device wait gave up");
    else if (c.error == ERR_NONFINITE || !isfinite(c.tv) || !isfinite(c.r2))
        st = fail(TVCS_ERR_DIVERGED, "non-finite iterate");
    else if (tol > 0.0 && !c.stop_by_tol)
        st = TVCS_NOT_CONVERGED;
    if (res) {
        res->iters = c.it;
        res->status = st;
        res->stopped_by_tol = c.stop_by_tol;
        res->rel_change = ctrl_relchg(c);
        res->tv = c.tv;
        res->resid2 = c.r2;
        res->objective = c.tv + 0.5 * h->mu * c.r2;
        res->kkt_primal = sqrt(c.kkt_p2);
        res->kkt_dual = sqrt(c.kkt_d2);
        res->lambda_max_norm = c.lam_max;
        res->ms = ms;
    }
    return st;
}

tvcs_status power_tau(tvcs_ctx* h, int iters, double* tau_out)
{
    const int N = h->N;
    launch_fill(h->tx, N, (float)(1.0 / sqrt((double)N)), h->stream);
    for (int it = 0; it < iters; ++it) {
        products(h, h->tx, nullptr, h->tr, h->gpart2, nullptr, MODE_PLAIN, 0ull, 0, h->stream);
        launch_gather(h->gpart2, h->P, N, 1.0f, h->tg, h->part, h->ctrl, h->stream);
        launch_normalize(h->tg, h->tx, N, h->ctrl, h->stream);
    }
    products(h, h->tx, nullptr, h->tr, h->gpart2, nullptr, MODE_PLAIN, 0ull, 0, h->stream);
    CKS(read_ctrl(h));
    const double lmax = h->hctrl->r2;
    if (!(lmax > 0.0) || !isfinite(lmax))
        return fail(TVCS_ERR_DIVERGED, "power iteration gave lambda_max = %g", lmax);
    *tau_out = 1.0 / (1.01 * lmax);
    return TVCS_OK;
}

tvcs_status check_handle(tvcs_handle h)
{
    if (!h) return fail(TVCS_ERR_INVALID_ARG, "null handle");
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return fail(TVCS_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return TVCS_OK;
}

// The partial-DCT encoder's tables: C[k][j] = a_k cos(pi (2j+1) k / (2n)) (binary64 at
// the exactly reduced angle, then rounded), the sampled indices in increasing order
// with their caller positions, and the first entry of each coefficient row.
tvcs_status dct_init(tvcs_ctx* h, const int32_t* rows)
{
    const int n = h->n, m = h->m;
    if (!dct_configure(n)) return fail(TVCS_ERR_UNSUPPORTED, "no partial-DCT kernel fits for n = %d", n);
    std::vector<float> C(2 * (size_t)n * n);   // C, then C^T
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < n; ++k) {
        const double a = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
        for (int j = 0; j < n; ++j) {
            const long t = ((long)(2 * j + 1) * k) % (4L * n);
            const float c = (float)(a * cos(2.0 * pi * (double)t / (4.0 * n)));
            C[(size_t)k * n + j] = c;
            C[(size_t)n * n + (size_t)j * n + k] = c;
        }
    }
    std::vector<std::pair<int, int>> e(m);
    for (int i = 0; i < m; ++i) e[i] = {rows[i], i};
    std::sort(e.begin(), e.end());
    std::vector<int> sidx(m), sperm(m), rowptr(n + 1);
    for (int i = 0; i < m; ++i) {
        sidx[i] = e[i].first;
        sperm[i] = e[i].second;
    }
    for (int k = 0, i = 0; k <= n; ++k) {
        while (i < m && sidx[i] < k * n) ++i;
        rowptr[k] = i;
    }
    CKS(alloc((void**)&h->dctC, 4 * sizeof(float) * (size_t)n * n));   // C, C^T, 2 n^2 scratch
    CKS(alloc((void**)&h->dsidx, sizeof(int) * (size_t)m));
    CKS(alloc((void**)&h->dsperm, sizeof(int) * (size_t)m));
    CKS(alloc((void**)&h->drowptr, sizeof(int) * (size_t)(n + 1)));
    CK(cudaMemcpy(h->dctC, C.data(), 2 * sizeof(float) * (size_t)n * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->dsidx, sidx.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->dsperm, sperm.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->drowptr, rowptr.data(), sizeof(int) * (size_t)(n + 1), cudaMemcpyHostToDevice));
    return TVCS_OK;
}

tvcs_status create_impl(tvcs_ctx* h, const float* A, uint64_t seed, const int32_t* dct_rows = nullptr)
{
    CK(cudaGetDevice(&h->dev));
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev));
    {
        std::lock_guard<std::mutex> lk(g_cfg_mutex);
        if (prod_supported(h->n) && !g_configured.count({h->dev, h->n})) {
            CK(prod_configure(h->n));
            g_configured.insert({h->dev, h->n});
        }
    }
    if (h->opt.stream) {
        h->stream = (cudaStream_t)h->opt.stream;
    } else {
        CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&h->ev0));
    CK(cudaEventCreate(&h->ev1));
    const size_t m = (size_t)h->m, N = (size_t)h->N;
    const int prec = h->opt.precision;
    const bool regen = h->opt.a_mode == TVCS_A_REGENERATE;
    h->dct = dct_rows != nullptr;
    const bool noA = regen || h->dct;   // no stored matrix
    h->use_q = !noA && !(prec == TVCS_PREC_FP32 && prod_supported(h->n));
    if (noA) {
        h->P = 1;   // these products leave A^T r whole
    } else if (h->use_q) {
        h->P = qprod_grid_clusters(prec, h->n, h->m);
        if (h->P == 0)
            return fail(TVCS_ERR_UNSUPPORTED, "no cluster of the product kernel fits (n = %d)", h->n);
    } else {
        h->P = prod_grid(h->n, h->m, h->num_sms);
    }
    h->ucluster = usolve_choose_cluster(h->n);
    if (h->ucluster == 0)
        return fail(TVCS_ERR_UNSUPPORTED, "no thread-block cluster of 8 or 16 fits for n = %d", h->n);
    const size_t nparts = 2 * (size_t)((N + 255) / 256 + 1024);
    // A: binary32 for the classic path and as the source of the split storages.
    if (!noA) CKS(alloc((void**)&h->A, sizeof(float) * m * N));
    CKS(alloc((void**)&h->f, sizeof(float) * m));
    CKS(alloc((void**)&h->r, sizeof(float) * m));
    CKS(alloc((void**)&h->ty, sizeof(float) * m));
    CKS(alloc((void**)&h->tr, sizeof(float) * m));
    CKS(alloc((void**)&h->u, sizeof(float) * N));
    CKS(alloc((void**)&h->g, sizeof(float) * N));
    CKS(alloc((void**)&h->rhs, sizeof(float) * N));
    CKS(alloc((void**)&h->zeroN, sizeof(float) * N));
    CKS(alloc((void**)&h->tx, sizeof(float) * N));
    CKS(alloc((void**)&h->tg, sizeof(float) * N));
    CKS(alloc((void**)&h->w, sizeof(float) * 4 * N));
    CKS(alloc((void**)&h->lam, sizeof(float) * 4 * N));
    CKS(alloc((void**)&h->spec, sizeof(float2) * (size_t)h->n * (h->n / 2 + 1)));
    CKS(alloc((void**)&h->tw, sizeof(float2) * (size_t)h->n));
    CKS(alloc((void**)&h->s2, sizeof(float) * (size_t)h->n));
    CKS(alloc((void**)&h->gpart, sizeof(float) * N * (size_t)h->P));
    CKS(alloc((void**)&h->gpart2, sizeof(float) * N * (size_t)h->P));
    CKS(alloc((void**)&h->r2part, sizeof(float2) * (size_t)h->P));
    CKS(alloc((void**)&h->part, sizeof(double) * nparts));
    CKS(alloc((void**)&h->ctrl, sizeof(Ctrl)));
    CK(cudaMallocHost((void**)&h->hctrl, sizeof(Ctrl)));
    memset(h->hctrl, 0, sizeof(Ctrl));
    h->hctrl->algo = h->opt.algo;
    CK(cudaMemcpyAsync(h->ctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->zeroN, 0, sizeof(float) * N, h->stream));
    CK(cudaMemsetAsync(h->u, 0, sizeof(float) * N, h->stream));
    CK(cudaMemsetAsync(h->f, 0, sizeof(float) * m, h->stream));

    // Twiddles (cos, sin)(2 pi t/n) and 4 sin^2(pi k/n) (eigenvalues of the 1D
    // periodic difference operator, Sec. 2.1), in binary64 then rounded.
    std::vector<float2> tw(h->n);
    std::vector<float> s2(h->n);
    const double pi = 3.14159265358979323846;
    for (int t = 0; t < h->n; ++t) {
        tw[t] = make_float2((float)cos(2.0 * pi * t / h->n), (float)sin(2.0 * pi * t / h->n));
        const double sv = sin(pi * t / h->n);
        s2[t] = (float)(4.0 * sv * sv);
    }
    CK(cudaMemcpyAsync(h->tw, tw.data(), sizeof(float2) * h->n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->s2, s2.data(), sizeof(float) * h->n, cudaMemcpyHostToDevice, h->stream));

    if (h->dct) {
        CKS(dct_init(h, dct_rows));
    } else if (regen) {
        CKS(sync_and_check(h, "tvcs_create"));
        CKS(regen_init(h));
    } else if (A) {
        CK(cudaMemcpyAsync(h->A, A, sizeof(float) * m * N, cudaMemcpyDefault, h->stream));
    } else {
        const float scale = (float)(1.0 / sqrt((double)h->m));
        launch_gen_gauss(h->A, h->m, (int64_t)N, seed, scale, h->stream);
    }
    CKS(sync_and_check(h, "uploading A"));
    if (h->use_q && !noA) {
        if (prec == TVCS_PREC_FP32) {
            h->P0 = reinterpret_cast<unsigned char*>(h->A);   // the plane is A itself
            h->A = nullptr;
        } else if (prec == TVCS_PREC_BF16X2) {
            CKS(alloc((void**)&h->P0, sizeof(uint16_t) * m * N));
            CKS(alloc((void**)&h->P1, sizeof(uint16_t) * m * N));
            launch_split_bf16x2(h->A, h->P0, h->P1, (long long)(m * N), h->stream);
        } else {
            CKS(alloc((void**)&h->P0, m * N));
            CKS(alloc((void**)&h->P1, sizeof(uint16_t) * m * N));
            CKS(alloc((void**)&h->rscale, sizeof(float) * m));
            launch_quant_fp8(h->A, h->m, h->N, h->P0, h->P1, h->rscale, h->stream);
        }
        CKS(sync_and_check(h, "storing A"));
        if (h->A) {   // the binary32 copy is no longer needed
            cudaFree(h->A);
            h->A = nullptr;
        }
    }
    if (h->opt.tau > 0.0) {
        h->tau = h->opt.tau;
    } else {
        CKS(power_tau(h, h->opt.power_iters > 0 ? h->opt.power_iters : 100, &h->tau));
    }
    return sync_and_check(h, "tvcs_create");
}

tvcs_status copy_in(tvcs_ctx* h, float* dst, const float* src, size_t count)
{
    CK(cudaMemcpyAsync(dst, src, sizeof(float) * count, cudaMemcpyDefault, h->stream));
    return TVCS_OK;
}

tvcs_status copy_out(tvcs_ctx* h, float* dst, const float* src, size_t count)
{
    CK(cudaMemcpyAsync(dst, src, sizeof(float) * count, cudaMemcpyDefault, h->stream));
    return TVCS_OK;
}

bool valid_n(int n, int prec)
{
    if (!tv_supported(n)) return false;
    if (prec == TVCS_PREC_FP32) return prod_supported(n) || qprod_supported(prec, n);
    return qprod_supported(prec, n);
}

}  // namespace

namespace tvcs {
// Sets the calling thread's tvcs_last_error() message (used by other translation units).
tvcs_status set_last_error(tvcs_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}
}  // namespace tvcs

extern "C" {

void tvcs_default_options(tvcs_options* opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->algo = TVCS_ALGO_IADM;
    opt->tau = 0.0;
    opt->max_iter = 500;
    opt->precision = TVCS_PREC_FP32;
    opt->init = TVCS_INIT_ATF;
    opt->stream = nullptr;
    opt->power_iters = 100;
    opt->timeout_cycles = 0;
    opt->host_loop = 0;
    opt->a_mode = TVCS_A_STORED;
    opt->batch_compact = 1;
    opt->autotune = 1;
}

const char* tvcs_last_error(void)
{
    return g_last_error.c_str();
}

tvcs_status tvcs_create(tvcs_handle* out, const float* A, uint64_t seed, int m, int n, double mu,
                        double beta, double tol, const tvcs_options* opt)
{
    if (!out) return fail(TVCS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (m < 1 || m > (1 << 24)) return fail(TVCS_ERR_INVALID_ARG, "m = %d outside [1, 2^24]", m);
    if (!(mu > 0.0) || !isfinite(mu)) return fail(TVCS_ERR_INVALID_ARG, "mu must be > 0");
    if (!(beta > 0.0) || !isfinite(beta)) return fail(TVCS_ERR_INVALID_ARG, "beta must be > 0");
    if (!(tol >= 0.0) || !isfinite(tol)) return fail(TVCS_ERR_INVALID_ARG, "tol must be >= 0");
    tvcs_options o;
    tvcs_default_options(&o);
    if (opt) o = *opt;
    if (o.algo != TVCS_ALGO_IADM && o.algo != TVCS_ALGO_FTVCS)
        return fail(TVCS_ERR_INVALID_ARG, "unknown algo %d", o.algo);
    if (o.init < TVCS_INIT_ATF || o.init > TVCS_INIT_GIVEN)
        return fail(TVCS_ERR_INVALID_ARG, "unknown init %d", o.init);
    if (o.precision < TVCS_PREC_FP32 || o.precision > TVCS_PREC_FP8_BF16)
        return fail(TVCS_ERR_INVALID_ARG, "unknown precision %d", o.precision);
    if (o.a_mode != TVCS_A_STORED && o.a_mode != TVCS_A_REGENERATE)
        return fail(TVCS_ERR_INVALID_ARG, "unknown a_mode %d", o.a_mode);
    if (o.a_mode == TVCS_A_REGENERATE && (A || o.precision != TVCS_PREC_FP32))
        return fail(TVCS_ERR_INVALID_ARG,
                    "TVCS_A_REGENERATE needs A = NULL (A comes from the seed) and precision "
                    "TVCS_PREC_FP32");
    if (o.a_mode == TVCS_A_REGENERATE ? !tv_supported(n) : !valid_n(n, o.precision))
        return fail(TVCS_ERR_INVALID_ARG,
                    "n = %d not supported with precision %d (binary32: 16, 32, 48, 64, 96, 128, 192, "
                    "256; bf16x2 / fp8: 32, 64, 128, 192, 256)",
                    n, o.precision);
    if (!isfinite(o.tau)) return fail(TVCS_ERR_INVALID_ARG, "tau must be finite");
    if (o.max_iter <= 0) o.max_iter = 500;
    tvcs_ctx* h = new (std::nothrow) tvcs_ctx();
    if (!h) return fail(TVCS_ERR_OOM, "host allocation failed");
    h->m = m;
    h->n = n;
    h->N = n * n;
    h->mu = mu;
    h->beta = beta;
    h->tol = tol;
    h->opt = o;
    h->seed = seed;
    tvcs_status st = create_impl(h, A, seed);
    if (st != TVCS_OK) {
        std::string msg = g_last_error;
        free_ctx(h);
        g_last_error = msg;
        return st;
    }
    *out = h;
    return TVCS_OK;
}

tvcs_status tvcs_create_partial_dct(tvcs_handle* out, const int32_t* rows, int m, int n, double mu,
                                    double beta, double tol, const tvcs_options* opt)
{
    if (!out) return fail(TVCS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!rows) return fail(TVCS_ERR_INVALID_ARG, "rows is NULL");
    if (!dct_supported(n) || !tv_supported(n))
        return fail(TVCS_ERR_INVALID_ARG, "n = %d not supported by the partial-DCT encoder "
                                          "(16, 32, 48, 64, 96, 128)", n);
    const long long N = (long long)n * n;
    if (m < 1 || m > N) return fail(TVCS_ERR_INVALID_ARG, "m = %d outside [1, n*n]", m);
    if (!(mu > 0.0) || !isfinite(mu)) return fail(TVCS_ERR_INVALID_ARG, "mu must be > 0");
    if (!(beta > 0.0) || !isfinite(beta)) return fail(TVCS_ERR_INVALID_ARG, "beta must be > 0");
    if (!(tol >= 0.0) || !isfinite(tol)) return fail(TVCS_ERR_INVALID_ARG, "tol must be >= 0");
    {
        std::vector<int32_t> sorted(rows, rows + m);
        std::sort(sorted.begin(), sorted.end());
        if (sorted[0] < 0 || sorted[m - 1] >= N)
            return fail(TVCS_ERR_INVALID_ARG, "a coefficient index lies outside [0, n*n)");
        for (int i = 1; i < m; ++i)
            if (sorted[i] == sorted[i - 1])
                return fail(TVCS_ERR_INVALID_ARG, "coefficient index %d appears twice", sorted[i]);
    }
    tvcs_options o;
    tvcs_default_options(&o);
    if (opt) o = *opt;
    if (o.algo != TVCS_ALGO_IADM && o.algo != TVCS_ALGO_FTVCS)
        return fail(TVCS_ERR_INVALID_ARG, "unknown algo %d", o.algo);
    if (o.init < TVCS_INIT_ATF || o.init > TVCS_INIT_GIVEN)
        return fail(TVCS_ERR_INVALID_ARG, "unknown init %d", o.init);
    if (o.precision != TVCS_PREC_FP32 || o.a_mode != TVCS_A_STORED)
        return fail(TVCS_ERR_INVALID_ARG, "the partial-DCT encoder computes in binary32 and stores "
                                          "no matrix (precision FP32, a_mode STORED)");
    if (!isfinite(o.tau)) return fail(TVCS_ERR_INVALID_ARG, "tau must be finite");
    if (o.max_iter <= 0) o.max_iter = 500;
    tvcs_ctx* h = new (std::nothrow) tvcs_ctx();
    if (!h) return fail(TVCS_ERR_OOM, "host allocation failed");
    h->m = m;
    h->n = n;
    h->N = n * n;
    h->mu = mu;
    h->beta = beta;
    h->tol = tol;
    h->opt = o;
    tvcs_status st = create_impl(h, nullptr, 0, rows);
    if (st != TVCS_OK) {
        std::string msg = g_last_error;
        free_ctx(h);
        g_last_error = msg;
        return st;
    }
    *out = h;
    return TVCS_OK;
}

tvcs_status tvcs_destroy(tvcs_handle h)
{
    if (!h) return TVCS_OK;
    free_ctx(h);
    return TVCS_OK;
}

tvcs_status tvcs_get_tau(tvcs_handle h, double* tau)
{
    CKS(check_handle(h));
    if (!tau) return fail(TVCS_ERR_INVALID_ARG, "tau is NULL");
    *tau = h->tau;
    return TVCS_OK;
}

tvcs_status tvcs_solve(tvcs_handle h, const float* f, float* u, tvcs_result* res)
{
    CKS(check_handle(h));
    if (!f || !u) return fail(TVCS_ERR_INVALID_ARG, "f and u must be non-NULL");
    CKS(copy_in(h, h->f, f, (size_t)h->m));
    CKS(init_state(h, h->opt.init));
    tvcs_status st = run_loop(h, h->opt.max_iter, h->tol, res);
    if (st < 0) return st;
    CKS(copy_out(h, u, h->u, (size_t)h->N));
    CKS(sync_and_check(h, "tvcs_solve"));
    return st;
}

tvcs_status tvcs_solve_continuation(tvcs_handle h, const float* f, float* u, const double* betas,
                                    int nbeta, tvcs_result* res)
{
    CKS(check_handle(h));
    if (!f || !u || !betas || nbeta < 1)
        return fail(TVCS_ERR_INVALID_ARG, "f, u and betas must be non-NULL and nbeta >= 1");
    for (int k = 0; k < nbeta; ++k)
        if (!(betas[k] > 0.0) || !isfinite(betas[k]))
            return fail(TVCS_ERR_INVALID_ARG, "betas[%d] must be > 0", k);
    const double beta0 = h->beta;
    auto drop_graph = [&]() { drop_loop_graphs(h); };   // beta is captured in the loop graphs
    CKS(copy_in(h, h->f, f, (size_t)h->m));
    tvcs_status worst = TVCS_OK;
    for (int k = 0; k < nbeta; ++k) {
        if (betas[k] != h->beta) {
            h->beta = betas[k];
            drop_graph();
        }
        // stage 0 from the handle's initial point; later stages warm-started from the
        // previous stage's u (and lambda), with w restarted at 0
        tvcs_status st = init_state(h, k == 0 ? h->opt.init : TVCS_INIT_GIVEN);
        if (st == TVCS_OK) st = run_loop(h, h->opt.max_iter, h->tol, res ? &res[k] : nullptr);
        if (st < 0) {
            h->beta = beta0;
            drop_graph();
            return st;
        }
        if (st > worst) worst = st;
    }
    if (h->beta != beta0) {
        h->beta = beta0;
        drop_graph();
    }
    CKS(copy_out(h, u, h->u, (size_t)h->N));
    CKS(sync_and_check(h, "tvcs_solve_continuation"));
    return worst;
}

tvcs_status tvcs_solve_batched(const tvcs_handle* hs, int count, const float* const* f,
                               float* const* u, const double* mu, tvcs_result* res)
{
    if (count < 0) return fail(TVCS_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return TVCS_OK;
    if (!hs || !f || !u) return fail(TVCS_ERR_INVALID_ARG, "hs, f and u must be non-NULL");
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || !f[i] || !u[i]) return fail(TVCS_ERR_INVALID_ARG, "entry %d is NULL", i);
        if (mu && (!(mu[i] > 0.0) || !isfinite(mu[i])))
            return fail(TVCS_ERR_INVALID_ARG, "mu[%d] must be finite and > 0", i);
    }
    bool shared = hs[0]->opt.precision == TVCS_PREC_BF16X2 && hs[0]->N % 128 == 0;
    for (int i = 1; i < count && shared; ++i) shared = hs[i] == hs[0];
    if (shared) {
        CKS(check_handle(hs[0]));
        if (count <= tvcs::batch_max(hs[0])) return solve_batch(hs[0], count, f, u, mu, res);
        // More images than one batch holds: groups of nearly equal size (the larger
        // ones first, so that the loop graph is rebuilt at most once), each through
        // the same tensor-core path.  A group whose images report a per-image
        // failure does not stop the later groups.
        const int gmax = tvcs::batch_max(hs[0]);
        const int groups = (count + gmax - 1) / gmax;
        const int base = count / groups, extra = count % groups;
        tvcs_status worst = TVCS_OK, err = TVCS_OK;
        for (int gi = 0, off = 0; gi < groups; ++gi) {
            const int c = base + (gi < extra ? 1 : 0);
            tvcs_status st = solve_batch(hs[0], c, f + off, u + off, mu ? mu + off : nullptr,
                                         res ? res + off : nullptr);
            if (st == TVCS_ERR_DIVERGED || st == TVCS_ERR_TIMEOUT) {
                if (err == TVCS_OK) err = st;
            } else if (st < 0) {
                return st;
            } else if (st > worst) {
                worst = st;
            }
            off += c;
        }
        if (err < 0) return fail(err, "an image of the batch failed (see its result)");
        return worst;
    }
    if (uneven_eligible(hs, count)) {
        CKS(check_handle(hs[0]));
        return solve_uneven(hs, count, f, u, mu, res);
    }
    tvcs_status worst = TVCS_OK;
    for (int i = 0; i < count; ++i) {
        tvcs_ctx* h = hs[i];
        const double mu0 = h->mu;
        if (mu && mu[i] != h->mu) {
            // mu is baked into the loop graph: rebuild it for this problem.
            h->mu = mu[i];
            drop_loop_graphs(h);
        }
        tvcs_status st = tvcs_solve(h, f[i], u[i], res ? &res[i] : nullptr);
        if (h->mu != mu0) {
            h->mu = mu0;
            drop_loop_graphs(h);
        }
        if (st < 0) return st;
        if (st > worst) worst = st;
    }
    return worst;
}

tvcs_status tvcs_get_state(tvcs_handle h, int which, float* dst)
{
    CKS(check_handle(h));
    if (!dst) return fail(TVCS_ERR_INVALID_ARG, "dst is NULL");
    CKS(read_ctrl(h));
    const size_t N = (size_t)h->N;
    const int par = h->hctrl->wpar;
    switch (which) {
        case TVCS_STATE_U: CKS(copy_out(h, dst, h->u, N)); break;
        case TVCS_STATE_W: CKS(copy_out(h, dst, h->w + (size_t)par * 2 * N, 2 * N)); break;
        case TVCS_STATE_LAMBDA: CKS(copy_out(h, dst, h->lam + (size_t)par * 2 * N, 2 * N)); break;
        case TVCS_STATE_G: CKS(copy_out(h, dst, h->g, N)); break;
        case TVCS_STATE_R: CKS(copy_out(h, dst, h->r, (size_t)h->m)); break;
        case TVCS_STATE_RHS: CKS(copy_out(h, dst, h->rhs, N)); break;
        case TVCS_STATE_F: CKS(copy_out(h, dst, h->f, (size_t)h->m)); break;
        default: return fail(TVCS_ERR_INVALID_ARG, "unknown state %d", which);
    }
    return sync_and_check(h, "tvcs_get_state");
}

tvcs_status tvcs_set_state(tvcs_handle h, int which, const float* src)
{
    CKS(check_handle(h));
    if (!src) return fail(TVCS_ERR_INVALID_ARG, "src is NULL");
    const size_t N = (size_t)h->N;
    if (which == TVCS_STATE_U || which == TVCS_STATE_F) {
        if (!h->state_ready) {
            CK(cudaMemsetAsync(h->w, 0, sizeof(float) * 4 * N, h->stream));
            CK(cudaMemsetAsync(h->lam, 0, sizeof(float) * 4 * N, h->stream));
            h->state_ready = true;
        }
        CKS(copy_in(h, which == TVCS_STATE_U ? h->u : h->f, src, which == TVCS_STATE_U ? N : (size_t)h->m));
        refresh_products(h);
        return sync_and_check(h, "tvcs_set_state");
    }
    if (which == TVCS_STATE_LAMBDA) {
        CKS(read_ctrl(h));
        CKS(copy_in(h, h->lam + (size_t)h->hctrl->wpar * 2 * N, src, 2 * N));
        h->hctrl->pending = 0;
        CKS(write_ctrl(h));
        return sync_and_check(h, "tvcs_set_state");
    }
    return fail(TVCS_ERR_INVALID_ARG, "state %d cannot be set", which);
}

tvcs_status tvcs_iterate(tvcs_handle h, int iters, tvcs_result* res)
{
    CKS(check_handle(h));
    if (iters < 0) return fail(TVCS_ERR_INVALID_ARG, "iters < 0");
    if (!h->state_ready) return fail(TVCS_ERR_INVALID_ARG, "no state: call tvcs_set_state or tvcs_solve first");
    tvcs_status st = run_loop(h, iters, 0.0, res);
    if (st < 0) return st;
    return sync_and_check(h, "tvcs_iterate");
}

tvcs_status tvcs_run_stage(tvcs_handle h, int stage)
{
    CKS(check_handle(h));
    if (!h->state_ready) return fail(TVCS_ERR_INVALID_ARG, "no state: call tvcs_set_state or tvcs_solve first");
    if (stage == 1) {
        TvArgs a = tv_args(h, MODE_PLAIN, true);
        launch_usolve(h->n, h->ucluster, a, h->stream);
    } else if (stage == 2) {
        refresh_products(h);
        if (h->opt.algo == TVCS_ALGO_IADM) {
            CKS(read_ctrl(h));
            h->hctrl->pending = 1;
            CKS(write_ctrl(h));
        }
    } else {
        return fail(TVCS_ERR_INVALID_ARG, "unknown stage %d", stage);
    }
    return sync_and_check(h, "tvcs_run_stage");
}

tvcs_status tvcs_time_stage(tvcs_handle h, int stage, int reps, double* ms)
{
    CKS(check_handle(h));
    if (!ms || reps < 1) return fail(TVCS_ERR_INVALID_ARG, "ms must be non-NULL and reps >= 1");
    if (stage >= 3 && stage <= 5) return time_batch_stage(h, stage, reps, ms);
    if (stage == 6 || stage == 7) return time_uneven_stage(h, stage, reps, ms);
    if (stage < 1 || stage > 2) return fail(TVCS_ERR_INVALID_ARG, "unknown stage %d", stage);
    if (!h->state_ready) return fail(TVCS_ERR_INVALID_ARG, "no state: call tvcs_set_state or tvcs_solve first");
    TvArgs a = tv_args(h, MODE_PLAIN, false);
    CK(cudaEventRecord(h->ev0, h->stream));
    for (int i = 0; i < reps; ++i) {
        if (stage == 1)
            launch_usolve(h->n, h->ucluster, a, h->stream);
        else
            refresh_products(h);
    }
    CK(cudaEventRecord(h->ev1, h->stream));
    CKS(sync_and_check(h, "tvcs_time_stage"));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->ev0, h->ev1));
    *ms = t;
    return TVCS_OK;
}

tvcs_status tvcs_apply_batched(tvcs_handle h, int count, const float* X, const float* Y,
                               float* R, float* G)
{
    CKS(check_handle(h));
    if (count < 1) return fail(TVCS_ERR_INVALID_ARG, "count must be >= 1");
    if (!X || !R || !G) return fail(TVCS_ERR_INVALID_ARG, "X, R and G must be non-NULL");
    // groups of at most batch_max images (nearly equal sizes, the larger first)
    const int gmax = tvcs::batch_max(h);
    const int groups = (count + gmax - 1) / gmax;
    const int base = count / groups, extra = count % groups;
    const size_t N = (size_t)h->N, m = (size_t)h->m;
    for (int gi = 0, off = 0; gi < groups; ++gi) {
        const int c = base + (gi < extra ? 1 : 0);
        CKS(apply_batch(h, c, X + off * N, Y ? Y + off * m : nullptr, R + off * m, G + off * N));
        off += c;
    }
    return TVCS_OK;
}

tvcs_status tvcs_test_hold_grid_barrier(tvcs_handle h, int extra)
{
    CKS(check_handle(h));
    if (extra < 0) return fail(TVCS_ERR_INVALID_ARG, "extra must be >= 0");
    if (h->use_q || h->regen || h->dct)
        return fail(TVCS_ERR_UNSUPPORTED, "the hook acts on the binary32 product kernel (n <= 128)");
    if (h->bar_extra != extra) {
        h->bar_extra = extra;
        drop_loop_graphs(h);   // the loop graphs captured the old value
    }
    return TVCS_OK;
}

tvcs_status tvcs_test_gemm_shape(tvcs_handle h, int grid1, int pair1, int grid2, int pair2)
{
    CKS(check_handle(h));
    if (grid1 < 0 || grid2 < 0 || (grid1 == 0) != (grid2 == 0))
        return fail(TVCS_ERR_INVALID_ARG, "grids must both be > 0, or both 0 (the tuner decides)");
    if (grid1 > 0) {
        const int pc = std::min(tvcs::batch_pair_clusters(h), h->num_sms / 2);
        const int grid[2] = {grid1, grid2}, pair[2] = {pair1, pair2};
        for (int i = 0; i < 2; ++i) {
            if (pair[i] != 0 && pair[i] != 1) return fail(TVCS_ERR_INVALID_ARG, "pair must be 0 or 1");
            if (pair[i] && grid[i] % 2 != 0)
                return fail(TVCS_ERR_INVALID_ARG, "a grid of pairs is an even number of blocks");
            if (pair[i] && grid[i] / 2 > pc)
                return fail(TVCS_ERR_UNSUPPORTED, "%d pairs requested, %d fit on the device", grid[i] / 2,
                            pc);
            if (!pair[i] && grid[i] > h->num_sms)
                return fail(TVCS_ERR_INVALID_ARG, "at most %d persistent blocks", h->num_sms);
        }
    }
    h->gemm_force[0] = grid1;
    h->gemm_force[1] = grid1 > 0 ? pair1 : 0;
    h->gemm_force[2] = grid2;
    h->gemm_force[3] = grid2 > 0 ? pair2 : 0;
    if (h->batch) {   // the next batched call re-plans and resizes the workspace
        h->batch->tuned = false;
        h->batch->cap = 0;
    }
    return TVCS_OK;
}

tvcs_status tvcs_apply(tvcs_handle h, const float* x, const float* y, float* r, float* g)
{
    CKS(check_handle(h));
    if (!x || !r || !g) return fail(TVCS_ERR_INVALID_ARG, "x, r and g must be non-NULL");
    CKS(copy_in(h, h->tx, x, (size_t)h->N));
    if (y) CKS(copy_in(h, h->ty, y, (size_t)h->m));
    // the kernels record a bounded wait that gave up in the control block's error word
    CK(cudaMemsetAsync(&h->ctrl->error, 0, sizeof(int), h->stream));
    products(h, h->tx, y ? h->ty : nullptr, h->tr, h->gpart2, h->tg, MODE_PLAIN, 0ull, 0,
             h->stream);
    CKS(copy_out(h, r, h->tr, (size_t)h->m));
    CKS(copy_out(h, g, h->tg, (size_t)h->N));
    CKS(read_ctrl(h));
    if (h->hctrl->error == ERR_TIMEOUT)
        return fail(TVCS_ERR_TIMEOUT, "a bounded device wait gave up");
    return TVCS_OK;
}

}  // extern "C"
