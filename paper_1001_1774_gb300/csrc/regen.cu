// Host side of the products with regenerated A (row a9).
//
// One handle (tvcs_create with TVCS_A_REGENERATE): A is never stored; every
// product of the handle (iteration, start point, power iteration, tvcs_apply)
// is one k_regen_products launch over a single problem plus its reduction.
// The launch arguments live in a small device table, one entry per pointer
// pattern the handle uses, written before any graph capture.
//
// Uneven batch (tvcs_solve_batched over regenerating handles): problems of
// different n, m, seed, mu and tau iterate together.  Images are grouped by
// n; the loop graph's body is one batched u-solve launch per n (rows a1-a5,
// per-image mu, tau, control block and stop test), then ONE persistent
// product launch over all problems (rows a6-a7 with in-kernel A), its
// reduction, and the loop condition (a WHILE node, as in the other paths).
// Problems that met eq. (stop) drop out of the product launch's work list.
//
// Tiles are chosen by measurement: every candidate of cluster size (4, 8, 16),
// tile height (1, 2, 4, 8 rows of the largest problem, at least half the
// cluster size) and kernel variant (registers for 2, 3 or 4 blocks per SM; one
// or two tile buffers) is timed on the actual problem set and the fastest is
// kept.  Every candidate adds in the same order (fixed row segments and
// chunks), so the choice changes the time, not the results.
#include <algorithm>
#include <utility>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "kernels.h"

namespace {

struct UClass {            // the images of one side length n
    int n = 0, N = 0, cnt = 0, off = 0, ucl = 0;
    float *U = nullptr, *W = nullptr, *L = nullptr, *G = nullptr, *mu = nullptr, *tau = nullptr;
    double* part = nullptr;
    float2* tw = nullptr;
    float* s2 = nullptr;
};

struct ProbSig {           // what the batch state was built for
    unsigned long long seed;
    int m, n, max_iter, algo;
    double mu, tau, tol;
    bool operator==(const ProbSig& o) const
    {
        return seed == o.seed && m == o.m && n == o.n && max_iter == o.max_iter && algo == o.algo &&
               mu == o.mu && tau == o.tau && tol == o.tol;
    }
};

}  // namespace

struct tvcs_uneven {
    std::vector<ProbSig> sig;      // per caller index
    std::vector<int> order;        // class order -> caller index
    std::vector<long long> moff;   // per class-order problem: offset in R and F
    std::vector<UClass> cls;
    int P = 0, maxN = 0, init = 0;
    double beta = 0;
    float *R = nullptr, *F = nullptr, *zero = nullptr, *gslot = nullptr;
    float2* r2slot = nullptr;
    int* pre = nullptr;
    tvcs::RegenProb *dtab = nullptr, *dtab0 = nullptr;
    tvcs::RegenPlan plan;
    long long elems = 0;           // sum over problems of m N (entries of A per product)
    tvcs::Ctrl *ctrls = nullptr, *hctrls = nullptr, *bctrl = nullptr, *hbctrl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace tvcs {

namespace {

#define RCK(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_last_error(e_ == cudaErrorMemoryAllocation ? TVCS_ERR_OOM : TVCS_ERR_CUDA, \
                                  "%s failed: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

#define RCKS(expr)                                  \
    do {                                            \
        tvcs_status s_ = (expr);                    \
        if (s_ != TVCS_OK) return s_;               \
    } while (0)

__global__ void k_negate(const float* __restrict__ in, float* __restrict__ out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = -in[i];
}

tvcs_status ralloc(void** p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_last_error(TVCS_ERR_OOM, "cudaMalloc of %zu bytes failed", bytes);
    }
    return TVCS_OK;
}

// Rows per chunk: about 2^21 entries of A, and at most m/16 rows so that a small
// problem still spreads over 16 clusters; fixed by the problem alone, so that
// the chunk slots (and with them the order of every sum of A^T r and ||r||^2)
// do not depend on the launch shape.  The kernel balances the clusters by
// entries, so chunks of different problems may differ in size.
constexpr long long kChunkEntries = 1LL << 21;

void chunking(int m, int N, int* rpc, int* chunks)
{
    long long rows = (kChunkEntries + N - 1) / N;
    const long long cap = (m + 15) / 16;
    if (rows > cap) rows = cap;
    if (rows < 1) rows = 1;
    *rpc = (int)rows;
    *chunks = (int)((m + rows - 1) / rows);
}

std::vector<RegenPlan> candidates(int maxN, int P)
{
    std::vector<RegenPlan> out;
    const int variants[6][2] = {{2, 2}, {2, 1}, {3, 2}, {3, 1}, {4, 2}, {4, 1}};   // (blocks/SM, tile buffers)
    for (const auto& v : variants)
        for (int cs : {4, 8, 16})
            for (int rt : {1, 2, 4, 8}) {
                RegenPlan p;
                p.cs = cs;
                p.minb = v[0];
                p.nbuf = v[1];
                p.pcap = P;
                p.wmax = maxN / cs;
                p.tile_cap = rt * p.wmax;
                if (maxN % (4 * cs) != 0) continue;
                if (regen_configure(&p)) out.push_back(p);
            }
    return out;
}

// Chunk layout of a problem set under a plan: rows per chunk, chunks, slot offsets.
struct Layout {
    std::vector<int> rpc, chunks;
    std::vector<size_t> gofs, rofs;
    size_t gfloats = 0, rslots = 0;
};

Layout layout_for(const std::vector<RegenProb>& probs)
{
    Layout L;
    for (const RegenProb& p : probs) {
        int rpc = 0, ch = 0;
        chunking(p.m, p.N, &rpc, &ch);
        L.rpc.push_back(rpc);
        L.chunks.push_back(ch);
        L.gofs.push_back(L.gfloats);
        L.rofs.push_back(L.rslots);
        L.gfloats += (size_t)ch * p.N;
        L.rslots += (size_t)ch;
    }
    return L;
}

void apply_layout(const Layout& L, float* gslot, float2* r2slot, std::vector<RegenProb>* probs)
{
    for (size_t i = 0; i < probs->size(); ++i) {
        RegenProb& p = (*probs)[i];
        p.rows_per_chunk = L.rpc[i];
        p.chunks = L.chunks[i];
        p.gslot = gslot + L.gofs[i];
        p.r2slot = r2slot + L.rofs[i];
    }
}

// Times each candidate plan on the problem set (one warm-up launch, one timed)
// and returns the fastest.  The chunk layout is the same for every plan (and so
// are the results); gslot / r2slot hold it.
tvcs_status autotune(std::vector<RegenProb> probs, int maxN, RegenProb* dtab, float* gslot,
                     float2* r2slot, int* pre, cudaStream_t s, RegenPlan* best, bool timed = true)
{
    std::vector<RegenPlan> cands = candidates(maxN, (int)probs.size());
    if (cands.empty()) return set_last_error(TVCS_ERR_UNSUPPORTED, "no cluster of the regenerating product kernel fits");
    if (!timed) {   // the first candidate, untimed
        *best = cands[0];
        regen_configure(best);
        return TVCS_OK;
    }
    cudaEvent_t e0, e1;
    RCK(cudaEventCreate(&e0));
    RCK(cudaEventCreate(&e1));
    const int P = (int)probs.size();
    // one timed launch (after one untimed) per candidate; the reps-launch minimum
    apply_layout(layout_for(probs), gslot, r2slot, &probs);
    RCK(cudaMemcpyAsync(dtab, probs.data(), sizeof(RegenProb) * P, cudaMemcpyHostToDevice, s));
    auto time_plan = [&](const RegenPlan& c, int reps, float* out) -> tvcs_status {
        launch_regen(dtab, P, MODE_PLAIN, c, pre, s);
        launch_regen_reduce(dtab, P, maxN, MODE_PLAIN, c, pre, 0ull, 0, s);
        float best = -1.f;
        for (int k = 0; k < reps; ++k) {
            cudaEventRecord(e0, s);
            launch_regen(dtab, P, MODE_PLAIN, c, pre, s);
            launch_regen_reduce(dtab, P, maxN, MODE_PLAIN, c, pre, 0ull, 0, s);
            cudaEventRecord(e1, s);
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess)
                return set_last_error(TVCS_ERR_CUDA, "tuning the regenerating products: %s",
                                      cudaGetErrorString(e));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0.f || ms < best) best = ms;
        }
        *out = best;
        return TVCS_OK;
    };
    // a pass over every candidate, then the three fastest again with three launches
    // each, so that one noisy launch does not decide
    std::vector<std::pair<float, int>> first;
    for (int i = 0; i < (int)cands.size(); ++i) {
        float ms = 0.f;
        const tvcs_status st = time_plan(cands[i], 1, &ms);
        if (st != TVCS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        first.push_back({ms, i});
    }
    std::sort(first.begin(), first.end());
    float best_ms = -1.f;
    for (int k = 0; k < (int)first.size() && k < 3; ++k) {
        float ms = 0.f;
        const tvcs_status st = time_plan(cands[first[k].second], 3, &ms);
        if (st != TVCS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return st;
        }
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            *best = cands[first[k].second];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms < 0.f) return set_last_error(TVCS_ERR_CUDA, "tuning the regenerating products failed");
    regen_configure(best);   // kernel attributes of the chosen plan
    return TVCS_OK;
}

std::mutex g_plan_mutex;
std::map<std::tuple<int, int, int>, RegenPlan> g_plans;   // (device, N, m) -> tuned plan

constexpr int kTab = 8;   // call patterns per handle

int find_entry(tvcs_regen* g, const float* x, const float* y, float* r, float* gout)
{
    for (size_t i = 0; i < g->htab.size(); ++i) {
        const RegenProb& p = g->htab[i];
        if (p.x == x && p.y == y && p.r == r && p.g == gout) return (int)i;
    }
    return -1;
}

tvcs_status add_entry(tvcs_ctx* h, const float* x, const float* y, float* r, float* gout)
{
    tvcs_regen* g = h->regen;
    if (find_entry(g, x, y, r, gout) >= 0) return TVCS_OK;
    if ((int)g->htab.size() >= kTab) return set_last_error(TVCS_ERR_INVALID_ARG, "too many product patterns");
    RegenProb p = g->htab.empty() ? RegenProb{} : g->htab[0];
    p.x = x;
    p.y = y;
    p.r = r;
    p.g = gout;
    g->htab.push_back(p);
    RCK(cudaMemcpy(g->dtab + (g->htab.size() - 1), &p, sizeof(RegenProb), cudaMemcpyHostToDevice));
    return TVCS_OK;
}

}  // namespace

tvcs_status regen_init(tvcs_ctx* h)
{
    tvcs_regen* g = new (std::nothrow) tvcs_regen();
    if (!g) return set_last_error(TVCS_ERR_OOM, "host allocation failed");
    h->regen = g;
    h->P = 1;   // products leave A^T r whole in gpart
    RegenProb base{};
    base.seed = h->seed;
    base.m = h->m;
    base.N = h->N;
    base.scale = (float)(1.0 / sqrt((double)h->m));
    base.ctrl = h->ctrl;
    base.x = h->tx;
    base.y = nullptr;
    base.r = h->tr;
    base.g = h->tg;
    std::vector<RegenProb> one(1, base);
    const Layout L0 = layout_for(one);
    if (candidates(h->N, 1).empty())
        return set_last_error(TVCS_ERR_UNSUPPORTED, "no cluster of the regenerating product kernel fits");
    RCKS(ralloc((void**)&g->gslot, sizeof(float) * L0.gfloats));
    RCKS(ralloc((void**)&g->r2slot, sizeof(float2) * L0.rslots));
    RCKS(ralloc((void**)&g->pre, sizeof(int) * 4));
    RCKS(ralloc((void**)&g->dtab, sizeof(RegenProb) * kTab));
    RegenPlan plan;
    bool cached = false;
    if (h->opt.autotune) {
        std::lock_guard<std::mutex> lk(g_plan_mutex);
        auto it = g_plans.find({h->dev, h->N, h->m});
        if (it != g_plans.end()) {
            plan = it->second;
            cached = true;
        }
    }
    if (cached) {
        regen_configure(&plan);
    } else {
        launch_fill(h->tx, h->N, (float)(1.0 / sqrt((double)h->N)), h->stream);
        RCKS(autotune(one, h->N, g->dtab, g->gslot, g->r2slot, g->pre, h->stream, &plan,
                      h->opt.autotune != 0));
        if (h->opt.autotune) {
            std::lock_guard<std::mutex> lk(g_plan_mutex);
            g_plans[{h->dev, h->N, h->m}] = plan;
        }
    }
    g->plan = plan;
    apply_layout(L0, g->gslot, g->r2slot, &one);
    g->htab.clear();
    g->htab.push_back(one[0]);
    RCK(cudaMemcpy(g->dtab, &one[0], sizeof(RegenProb), cudaMemcpyHostToDevice));
    // every pointer pattern the handle uses, before any capture
    RCKS(add_entry(h, h->u, h->f, h->r, h->g));           // iteration, refresh
    RCKS(add_entry(h, h->zeroN, h->f, h->r, h->gpart));   // u^0 = A^T f
    RCKS(add_entry(h, h->tx, nullptr, h->tr, h->gpart2)); // power iteration
    RCKS(add_entry(h, h->tx, h->ty, h->tr, h->tg));       // tvcs_apply with y
    return TVCS_OK;
}

void regen_products(tvcs_ctx* h, const float* x, const float* y, float* r, float* g, int mode,
                    unsigned long long cond, int set_cond, cudaStream_t s)
{
    tvcs_regen* rg = h->regen;
    int i = find_entry(rg, x, y, r, g);
    if (i < 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (cs != cudaStreamCaptureStatusNone || add_entry(h, x, y, r, g) != TVCS_OK) {
            set_last_error(TVCS_ERR_INVALID_ARG, "unregistered product pattern");
            return;
        }
        i = find_entry(rg, x, y, r, g);
    }
    launch_regen(rg->dtab + i, 1, mode, rg->plan, rg->pre, s);
    launch_regen_reduce(rg->dtab + i, 1, h->N, mode, rg->plan, rg->pre, cond, set_cond, s);
}

namespace {

void free_uneven_state(tvcs_uneven* u)
{
    if (!u) return;
    if (u->exec) cudaGraphExecDestroy(u->exec);
    if (u->graph) cudaGraphDestroy(u->graph);
    for (UClass& c : u->cls) {
        void* b[] = {c.U, c.W, c.L, c.G, c.mu, c.tau, c.part, c.tw, c.s2};
        for (void* p : b)
            if (p) cudaFree(p);
    }
    void* b[] = {u->R, u->F, u->zero, u->gslot, u->r2slot, u->pre, u->dtab, u->dtab0, u->ctrls,
                 u->bctrl};
    for (void* p : b)
        if (p) cudaFree(p);
    if (u->hctrls) cudaFreeHost(u->hctrls);
    if (u->hbctrl) cudaFreeHost(u->hbctrl);
    delete u;
}

}  // namespace

void free_regen(tvcs_ctx* h)
{
    if (h->uneven) {
        free_uneven_state(h->uneven);
        h->uneven = nullptr;
    }
    if (!h->regen) return;
    tvcs_regen* g = h->regen;
    void* b[] = {g->gslot, g->r2slot, g->pre, g->dtab};
    for (void* p : b)
        if (p) cudaFree(p);
    delete g;
    h->regen = nullptr;
}

bool uneven_eligible(const tvcs_handle* hs, int count)
{
    if (count < 1 || count > REGEN_PMAX) return false;
    const tvcs_ctx* h0 = hs[0];
    if (!h0->regen) return false;
    for (int i = 0; i < count; ++i) {
        const tvcs_ctx* h = hs[i];
        if (!h->regen || h->dev != h0->dev || h->opt.algo != h0->opt.algo || h->beta != h0->beta ||
            h->opt.init != h0->opt.init || h->opt.init == TVCS_INIT_GIVEN)
            return false;
    }
    return true;
}

namespace {

TvArgs class_args(const tvcs_uneven* u, const UClass& c, int mode)
{
    TvArgs a{};
    a.u = c.U;
    a.w = c.W;
    a.lam = c.L;
    a.g = c.G;
    a.tw = c.tw;
    a.s2 = c.s2;
    a.part = c.part;
    a.beta = (float)u->beta;
    a.mu_over_tau = 1.0f;   // per image from mu_img / tau_img
    a.mu = 1.0f;
    a.ctrl = u->ctrls + c.off;
    a.mode = mode;
    a.nimg = c.cnt;
    a.mu_img = c.mu;
    a.tau_img = c.tau;
    a.tau = 1.0f;
    return a;
}

// Builds the state for the problem set: classes, buffers, tuned plan, tables.
tvcs_status build_uneven(const tvcs_handle* hs, int count, const double* mu, tvcs_uneven* u)
{
    tvcs_ctx* h0 = hs[0];
    cudaStream_t s = h0->stream;
    u->P = count;
    u->beta = h0->beta;
    u->init = h0->opt.init;
    for (int i = 0; i < count; ++i) {
        const tvcs_ctx* h = hs[i];
        u->sig.push_back({h->seed, h->m, h->n, h->opt.max_iter, h->opt.algo, mu ? mu[i] : h->mu,
                          h->tau, h->tol});
    }
    // classes by n (ascending), problems in caller order inside a class
    std::map<int, std::vector<int>> by_n;
    for (int i = 0; i < count; ++i) by_n[hs[i]->n].push_back(i);
    long long mtot = 0;
    for (auto& kv : by_n) {
        UClass c;
        c.n = kv.first;
        c.N = c.n * c.n;
        c.cnt = (int)kv.second.size();
        c.off = (int)u->order.size();
        c.ucl = hs[kv.second[0]]->ucluster;
        if (c.N > u->maxN) u->maxN = c.N;
        for (int i : kv.second) {
            u->order.push_back(i);
            u->moff.push_back(mtot);
            mtot += hs[i]->m;
        }
        u->cls.push_back(c);
    }
    for (UClass& c : u->cls) {
        const size_t B = (size_t)c.cnt, N = (size_t)c.N;
        RCKS(ralloc((void**)&c.U, sizeof(float) * B * N));
        RCKS(ralloc((void**)&c.G, sizeof(float) * B * N));
        RCKS(ralloc((void**)&c.W, sizeof(float) * B * 4 * N));
        RCKS(ralloc((void**)&c.L, sizeof(float) * B * 4 * N));
        RCKS(ralloc((void**)&c.mu, sizeof(float) * B));
        RCKS(ralloc((void**)&c.tau, sizeof(float) * B));
        RCKS(ralloc((void**)&c.part, sizeof(double) * B * 2 * ((N + 255) / 256)));
        RCKS(ralloc((void**)&c.tw, sizeof(float2) * c.n));
        RCKS(ralloc((void**)&c.s2, sizeof(float) * c.n));
        const tvcs_ctx* hc = hs[u->order[c.off]];
        RCK(cudaMemcpyAsync(c.tw, hc->tw, sizeof(float2) * c.n, cudaMemcpyDeviceToDevice, s));
        RCK(cudaMemcpyAsync(c.s2, hc->s2, sizeof(float) * c.n, cudaMemcpyDeviceToDevice, s));
        std::vector<float> mus(c.cnt), taus(c.cnt);
        for (int b = 0; b < c.cnt; ++b) {
            const int i = u->order[c.off + b];
            mus[b] = (float)u->sig[i].mu;
            taus[b] = (float)u->sig[i].tau;
        }
        RCK(cudaMemcpy(c.mu, mus.data(), sizeof(float) * c.cnt, cudaMemcpyHostToDevice));
        RCK(cudaMemcpy(c.tau, taus.data(), sizeof(float) * c.cnt, cudaMemcpyHostToDevice));
        RCK(cudaMemsetAsync(c.U, 0, sizeof(float) * B * N, s));
    }
    RCKS(ralloc((void**)&u->R, sizeof(float) * mtot));
    RCKS(ralloc((void**)&u->F, sizeof(float) * mtot));
    RCKS(ralloc((void**)&u->zero, sizeof(float) * u->maxN));
    RCK(cudaMemsetAsync(u->zero, 0, sizeof(float) * u->maxN, s));
    RCK(cudaMemsetAsync(u->F, 0, sizeof(float) * mtot, s));
    RCKS(ralloc((void**)&u->ctrls, sizeof(Ctrl) * count));
    RCK(cudaMallocHost((void**)&u->hctrls, sizeof(Ctrl) * count));
    RCKS(ralloc((void**)&u->bctrl, sizeof(Ctrl)));
    RCK(cudaMallocHost((void**)&u->hbctrl, sizeof(Ctrl)));
    memset(u->hctrls, 0, sizeof(Ctrl) * count);
    RCK(cudaMemcpyAsync(u->ctrls, u->hctrls, sizeof(Ctrl) * count, cudaMemcpyHostToDevice, s));
    RCKS(ralloc((void**)&u->pre, sizeof(int) * (count + 4)));
    RCKS(ralloc((void**)&u->dtab, sizeof(RegenProb) * count));
    RCKS(ralloc((void**)&u->dtab0, sizeof(RegenProb) * count));
    // problem table in class order: iteration pattern (x = U, y = F)
    std::vector<RegenProb> probs(count);
    for (const UClass& c : u->cls)
        for (int b = 0; b < c.cnt; ++b) {
            const int k = c.off + b;
            const tvcs_ctx* h = hs[u->order[k]];
            RegenProb& p = probs[k];
            p = RegenProb{};
            p.seed = h->seed;
            p.m = h->m;
            p.N = c.N;
            p.scale = (float)(1.0 / sqrt((double)h->m));
            p.x = c.U + (size_t)b * c.N;
            p.y = u->F + u->moff[k];
            p.r = u->R + u->moff[k];
            p.g = c.G + (size_t)b * c.N;
            p.ctrl = u->ctrls + k;
            u->elems += (long long)h->m * c.N;
        }
    const Layout L = layout_for(probs);
    RCKS(ralloc((void**)&u->gslot, sizeof(float) * L.gfloats));
    RCKS(ralloc((void**)&u->r2slot, sizeof(float2) * L.rslots));
    RCKS(autotune(probs, u->maxN, u->dtab, u->gslot, u->r2slot, u->pre, s, &u->plan,
                  h0->opt.autotune != 0));
    apply_layout(L, u->gslot, u->r2slot, &probs);
    RCK(cudaMemcpy(u->dtab, probs.data(), sizeof(RegenProb) * count, cudaMemcpyHostToDevice));
    for (RegenProb& p : probs) p.x = u->zero;   // start point: A^T (0 - f)
    RCK(cudaMemcpy(u->dtab0, probs.data(), sizeof(RegenProb) * count, cudaMemcpyHostToDevice));
    return TVCS_OK;
}

tvcs_status build_uneven_graph(tvcs_ctx* h0, tvcs_uneven* u)
{
    if (u->exec) return TVCS_OK;
    RCK(cudaGraphCreate(&u->graph, 0));
    cudaGraphConditionalHandle ch;
    RCK(cudaGraphConditionalHandleCreate(&ch, u->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    RCK(cudaGraphAddNode(&node, u->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    cudaStream_t cs = h0->cap_stream;
    RCK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    for (const UClass& c : u->cls) launch_usolve(c.n, c.ucl, class_args(u, c, MODE_ITER), cs);
    launch_regen(u->dtab, u->P, MODE_ITER, u->plan, u->pre, cs);
    launch_regen_reduce(u->dtab, u->P, u->maxN, MODE_ITER, u->plan, u->pre, 0ull, 0, cs);
    launch_batch_cond(u->ctrls, u->P, u->bctrl, (unsigned long long)ch, 1, cs);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    if (e != cudaSuccess)
        return set_last_error(TVCS_ERR_CUDA, "capture of the uneven loop: %s", cudaGetErrorString(e));
    RCK(cudaGraphInstantiate(&u->exec, u->graph, 0));
    return TVCS_OK;
}

}  // namespace

tvcs_status solve_uneven(const tvcs_handle* hs, int count, const float* const* f, float* const* u_out,
                         const double* mu, tvcs_result* res)
{
    tvcs_ctx* h0 = hs[0];
    RCK(cudaSetDevice(h0->dev));
    cudaStream_t s = h0->stream;
    // reuse the state when the problem set is the same
    bool same = h0->uneven && h0->uneven->P == count;
    for (int i = 0; i < count && same; ++i) {
        const tvcs_ctx* h = hs[i];
        const ProbSig sg{h->seed, h->m, h->n, h->opt.max_iter, h->opt.algo, mu ? mu[i] : h->mu,
                         h->tau, h->tol};
        same = h0->uneven->sig[i] == sg && h0->uneven->beta == h->beta && h0->uneven->init == h->opt.init;
    }
    if (!same) {
        cudaStreamSynchronize(s);
        free_uneven_state(h0->uneven);
        h0->uneven = new (std::nothrow) tvcs_uneven();
        if (!h0->uneven) return set_last_error(TVCS_ERR_OOM, "host allocation failed");
        tvcs_status st = build_uneven(hs, count, mu, h0->uneven);
        if (st != TVCS_OK) {
            cudaStreamSynchronize(s);
            free_uneven_state(h0->uneven);
            h0->uneven = nullptr;
            return st;
        }
    }
    tvcs_uneven* u = h0->uneven;
    const int P = u->P;
    for (int k = 0; k < P; ++k) {
        const int i = u->order[k];
        RCK(cudaMemcpyAsync(u->F + u->moff[k], f[i], sizeof(float) * hs[i]->m, cudaMemcpyDefault, s));
    }
    int maxit = 0;
    memset(u->hctrls, 0, sizeof(Ctrl) * P);
    for (int k = 0; k < P; ++k) {
        const ProbSig& sg = u->sig[u->order[k]];
        u->hctrls[k].max_iter = sg.max_iter;
        u->hctrls[k].tol = sg.tol;
        u->hctrls[k].algo = sg.algo;
        if (sg.max_iter > maxit) maxit = sg.max_iter;
    }
    RCK(cudaMemcpyAsync(u->ctrls, u->hctrls, sizeof(Ctrl) * P, cudaMemcpyHostToDevice, s));
    memset(u->hbctrl, 0, sizeof(Ctrl));
    u->hbctrl->loops_max = maxit + 2;
    RCK(cudaMemcpyAsync(u->bctrl, u->hbctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    for (const UClass& c : u->cls) {
        RCK(cudaMemsetAsync(c.W, 0, sizeof(float) * 4 * (size_t)c.cnt * c.N, s));
        RCK(cudaMemsetAsync(c.L, 0, sizeof(float) * 4 * (size_t)c.cnt * c.N, s));
    }
    // u^0: A^T f (reading C3) from the products at x = 0, or zero
    if (u->init == TVCS_INIT_ATF) {
        launch_regen(u->dtab0, P, MODE_PLAIN, u->plan, u->pre, s);
        launch_regen_reduce(u->dtab0, P, u->maxN, MODE_PLAIN, u->plan, u->pre, 0ull, 0, s);
        for (const UClass& c : u->cls)
            k_negate<<<152 * 4, 256, 0, s>>>(c.G, c.U, (long long)c.cnt * c.N);
    } else {
        for (const UClass& c : u->cls)
            RCK(cudaMemsetAsync(c.U, 0, sizeof(float) * (size_t)c.cnt * c.N, s));
    }
    launch_regen(u->dtab, P, MODE_PLAIN, u->plan, u->pre, s);
    launch_regen_reduce(u->dtab, P, u->maxN, MODE_PLAIN, u->plan, u->pre, 0ull, 0, s);
    RCKS(build_uneven_graph(h0, u));
    RCK(cudaEventRecord(h0->ev0, s));
    if (maxit > 0) RCK(cudaGraphLaunch(u->exec, s));
    RCK(cudaEventRecord(h0->ev1, s));
    for (const UClass& c : u->cls) {
        TvArgs a = class_args(u, c, MODE_PLAIN);
        launch_tv(c.n, a, 4, s);
        launch_tv(c.n, a, 5, s);
    }
    for (const UClass& c : u->cls)
        for (int b = 0; b < c.cnt; ++b) {
            const int i = u->order[c.off + b];
            RCK(cudaMemcpyAsync(u_out[i], c.U + (size_t)b * c.N, sizeof(float) * c.N,
                                cudaMemcpyDefault, s));
        }
    RCK(cudaMemcpyAsync(u->hctrls, u->ctrls, sizeof(Ctrl) * P, cudaMemcpyDeviceToHost, s));
    RCK(cudaStreamSynchronize(s));
    RCK(cudaGetLastError());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h0->ev0, h0->ev1);
    tvcs_status worst = TVCS_OK, err = TVCS_OK;
    for (int k = 0; k < P; ++k) {
        const int i = u->order[k];
        const Ctrl& c = u->hctrls[k];
        const ProbSig& sg = u->sig[i];
        tvcs_status st = TVCS_OK;
        if (c.error == ERR_TIMEOUT)
            st = TVCS_ERR_TIMEOUT;
        else if (c.error == ERR_NONFINITE || !isfinite(c.tv) || !isfinite(c.r2))
            st = TVCS_ERR_DIVERGED;
        else if (sg.tol > 0.0 && !c.stop_by_tol)
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
            r.objective = c.tv + 0.5 * sg.mu * c.r2;
            r.kkt_primal = sqrt(c.kkt_p2);
            r.kkt_dual = sqrt(c.kkt_d2);
            r.lambda_max_norm = c.lam_max;
            r.ms = ms;
        }
    }
    if (err < 0) return set_last_error(err, "a problem of the batch failed (see its result)");
    return worst;
}

// 6: the regenerating products over every problem of the last uneven batch;
// 7: the u-solve launches of all its image sizes.
tvcs_status time_uneven_stage(tvcs_ctx* h, int stage, int reps, double* ms)
{
    tvcs_uneven* u = h->uneven;
    if (!u) return set_last_error(TVCS_ERR_INVALID_ARG, "no uneven batch: call tvcs_solve_batched first");
    cudaStream_t s = h->stream;
    RCK(cudaEventRecord(h->ev0, s));
    for (int k = 0; k < reps; ++k) {
        if (stage == 6) {
            launch_regen(u->dtab, u->P, MODE_PLAIN, u->plan, u->pre, s);
            launch_regen_reduce(u->dtab, u->P, u->maxN, MODE_PLAIN, u->plan, u->pre, 0ull, 0, s);
        } else {
            for (const UClass& c : u->cls) launch_usolve(c.n, c.ucl, class_args(u, c, MODE_PLAIN), s);
        }
    }
    RCK(cudaEventRecord(h->ev1, s));
    RCK(cudaStreamSynchronize(s));
    RCK(cudaGetLastError());
    float t = 0.f;
    RCK(cudaEventElapsedTime(&t, h->ev0, h->ev1));
    *ms = t;
    return TVCS_OK;
}

}  // namespace tvcs
