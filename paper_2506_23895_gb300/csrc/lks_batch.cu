// Batches of contexts (lks_batch_*): many D2Q9 FP32 problems advanced in lock step.
#include "lks_engine.h"

using namespace lks;
using namespace lks::eng;

// ================================================================ batches of contexts
// Many D2Q9 FP32 contexts (designs, finite-difference perturbations, grids of different sizes)
// advanced in lock step: one checkpoint schedule, every phase of a step one persistent launch
// over all instances, runs of steps captured into CUDA graphs on the batch's own stream, tile
// shapes of the fused kernels picked by timing every candidate on the batch itself.

struct lks_batch {
    std::vector<lks_ctx*> cs;
    cudaStream_t user_st = nullptr;   // the contexts' stream
    cudaStream_t st = nullptr;        // own stream: graphs need a capturable stream
    cudaEvent_t ev = nullptr;
    char* dmem = nullptr;
    Inst* dinst = nullptr;
    int* dpre = nullptr;
    int* nbase = nullptr;
    Plan plan;
    bool have_plan = false;
    std::vector<int> gens;
    GraphCache graphs;
    bool use_graphs = true;
    int tile_req[2] = {-1, -1};       // requested tile shapes, -1 = autotune
    int tile[2] = {-1, -1};           // in use
    float tune_ms[2][kTileCfgs];
    long long launches = 0;
    std::string err;
};

namespace {

lks_status bfail(lks_batch* b, lks_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->err = buf;
    return s;
}

#define BCU(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail(b, LKS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

// Copy the first failing context's message into the batch.
lks_status bcollect(lks_batch* b, lks_status s) {
    if (s == LKS_OK) return s;
    for (size_t i = 0; i < b->cs.size(); ++i)
        if (!b->cs[i]->err.empty()) {
            b->err = "instance " + std::to_string(i) + ": " + b->cs[i]->err;
            return s;
        }
    b->err = "batch run failed";
    return s;
}

lks_status batch_prepare(lks_batch* b, int n_steps) {
    for (size_t i = 0; i < b->cs.size(); ++i) {
        lks_ctx* c = b->cs[i];
        c->err.clear();
        if (!c->have_design || !c->have_motion)
            return bfail(b, LKS_ERR_ORDER, "instance %zu: set_design and set_motion must precede forward", i);
        if (n_steps < 1 || n_steps > c->cfg.max_steps)
            return bfail(b, LKS_ERR_ARG, "n_steps must be in [1, max_steps]");
    }
    bool stale = !b->have_plan;
    for (size_t i = 0; i < b->cs.size(); ++i) stale = stale || b->gens[i] != b->cs[i]->geo_gen;
    if (stale) {
        b->graphs.clear();
        BCU(build_plan(b->cs, b->dinst, b->dpre, b->nbase, b->st, b->plan));
        for (size_t i = 0; i < b->cs.size(); ++i) b->gens[i] = b->cs[i]->geo_gen;
        b->have_plan = true;
        b->tile[0] = b->tile[1] = -1;
    }
    // autotune: time every tile shape of the fused step and adjoint kernels on this batch
    if (b->tile[0] < 0 || b->tile[1] < 0) {
        for (int w = 0; w < 2; ++w) {
            if (b->tile_req[w] >= 0) {
                b->tile[w] = b->tile_req[w];
                continue;
            }
            BCU(launch_set_int(b->nbase, 0, b->st));
            BCU(launch_t_design_pos(b->plan, 1, b->st));
            BCU(launch_t_transfer2d(b->plan, 1, -1, false, b->st));
            for (lks_ctx* c : b->cs) {
                BCU(cudaMemsetAsync(c->lam[0], 0, c->snap_bytes, b->st));
                BCU(cudaMemsetAsync(c->lam[1], 0, c->snap_bytes, b->st));
            }
            cudaEvent_t e0, e1;
            BCU(cudaEventCreate(&e0));
            BCU(cudaEventCreate(&e1));
            int best = 0;
            const int ncfg = w == 0 ? kTileCfgs : kAdjCfgs;
            for (int k = 0; k < kTileCfgs; ++k) b->tune_ms[w][k] = -1.f;
            for (int k = 0; k < ncfg; ++k) {
                auto run = [&]() -> cudaError_t {
                    return w == 0 ? launch_t_step2d(b->plan, k, BUF_INIT, BUF_S1, -1, b->st)
                                  : launch_t_adj2d(b->plan, k, 1, BUF_LAM0, BUF_LAM1, BUF_INIT,
                                                   BUF_INIT, -1, b->st);
                };
                cudaError_t e = cudaSuccess;
                for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run();
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->st);
                for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = run();
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return bfail(b, LKS_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
                }
                b->tune_ms[w][k] = ms / 5.f;
                if (b->tune_ms[w][k] < b->tune_ms[w][best]) best = k;
                b->launches += 7;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            b->tile[w] = best;
            b->launches += 3;
        }
        b->graphs.clear();
    }
    return LKS_OK;
}

Group batch_group(lks_batch* b) {
    Group G;
    G.cs = b->cs.data();
    G.count = (int)b->cs.size();
    G.table = true;
    G.plan = &b->plan;
    G.nbase = b->nbase;
    G.tile_fwd = b->tile[0];
    G.tile_adj = b->tile[1];
    G.graphs = b->use_graphs ? &b->graphs : nullptr;
    G.st = b->st;
    return G;
}

}  // namespace

extern "C" {

lks_status lks_batch_create(lks_ctx* const* ctxs, int n, lks_batch** out) {
    if (!out) return LKS_ERR_ARG;
    *out = nullptr;
    if (!ctxs || n < 1) return LKS_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        lks_ctx* c = ctxs[i];
        if (!c) return LKS_ERR_ARG;
        if (!c->fused2d) {
            fprintf(stderr, "lks_batch_create: instance %d is not a D2Q9 FP32 context on the "
                            "fused kernels\n", i);
            return LKS_ERR_ARG;
        }
        if (c->cfg.max_steps != ctxs[0]->cfg.max_steps || c->pool_slots != ctxs[0]->pool_slots ||
            c->st != ctxs[0]->st) {
            fprintf(stderr, "lks_batch_create: instances need equal max_steps, snapshot slots "
                            "and stream (instance %d differs)\n", i);
            return LKS_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) {
                fprintf(stderr, "lks_batch_create: instance %d repeats instance %d\n", i, j);
                return LKS_ERR_ARG;
            }
    }
    lks_batch* b = new lks_batch();
    b->cs.assign(ctxs, ctxs + n);
    b->gens.assign(n, -1);
    b->user_st = ctxs[0]->st;
    const size_t inst_bytes = align256(sizeof(Inst) * n);
    const size_t pre_bytes = align256(sizeof(int) * U_COUNT * (n + 1));
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        dev_alloc((void**)&b->dmem, inst_bytes + pre_bytes + 256) != cudaSuccess) {
        cudaGetLastError();
        lks_batch_destroy(b);
        return LKS_ERR_NOMEM;
    }
    b->dinst = (Inst*)b->dmem;
    b->dpre = (int*)(b->dmem + inst_bytes);
    b->nbase = (int*)(b->dmem + inst_bytes + pre_bytes);
    *out = b;
    return LKS_OK;
}

lks_status lks_batch_set_options(lks_batch* b, int use_graphs, int tile_fwd, int tile_adj) {
    if (!b) return LKS_ERR_ARG;
    if (tile_fwd < -1 || tile_fwd >= kTileCfgs || tile_adj < -1 || tile_adj >= kAdjCfgs)
        return bfail(b, LKS_ERR_ARG, "tile shape index out of range");
    b->use_graphs = use_graphs != 0;
    b->tile_req[0] = tile_fwd;
    b->tile_req[1] = tile_adj;
    b->tile[0] = b->tile[1] = -1;
    b->graphs.clear();
    return LKS_OK;
}

lks_status lks_batch_forward(lks_batch* b, int n_steps, double* J_out) {
    if (!b) return LKS_ERR_ARG;
    b->err.clear();
    BCU(cudaEventRecord(b->ev, b->user_st));
    BCU(cudaStreamWaitEvent(b->st, b->ev, 0));
    b->launches = 0;
    lks_status s = batch_prepare(b, n_steps);
    if (s == LKS_OK) {
        Group G = batch_group(b);
        s = bcollect(b, do_forward<float>(G, n_steps));
        b->launches += G.launches;
        for (lks_ctx* c : b->cs) b->launches += c->stats[4];
    }
    BCU(cudaEventRecord(b->ev, b->st));
    BCU(cudaStreamWaitEvent(b->user_st, b->ev, 0));
    if (s != LKS_OK) return s;
    if (J_out)
        for (size_t i = 0; i < b->cs.size(); ++i) J_out[i] = b->cs[i]->J;
    return LKS_OK;
}

lks_status lks_batch_adjoint(lks_batch* b, double* const* dJdgamma, int on_device) {
    if (!b) return LKS_ERR_ARG;
    b->err.clear();
    for (size_t i = 0; i < b->cs.size(); ++i)
        if (!b->cs[i]->fwd_valid)
            return bfail(b, LKS_ERR_ORDER, "instance %zu: adjoint needs a preceding forward run", i);
    BCU(cudaEventRecord(b->ev, b->user_st));
    BCU(cudaStreamWaitEvent(b->st, b->ev, 0));
    Group G = batch_group(b);
    long long before = 0;
    for (lks_ctx* c : b->cs) before += c->stats[4];
    lks_status s = bcollect(b, do_adjoint<float>(G));
    b->launches += G.launches;
    for (lks_ctx* c : b->cs) b->launches += c->stats[4];
    b->launches -= before;
    if (s == LKS_OK && dJdgamma) {
        for (size_t i = 0; i < b->cs.size(); ++i) {
            lks_ctx* c = b->cs[i];
            if (c->d.nd == 0 || !dJdgamma[i]) continue;
            BCU(cudaMemcpyAsync(dJdgamma[i], design_gradient(c, b->st), (size_t)c->d.nd * 8,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                b->st));
        }
        BCU(cudaStreamSynchronize(b->st));
    }
    BCU(cudaEventRecord(b->ev, b->st));
    BCU(cudaStreamWaitEvent(b->user_st, b->ev, 0));
    return s;
}

int lks_batch_tile_shapes(int* txty, int cap) {
    if (cap < 0 || (!txty && cap > 0)) return -1;
    for (int k = 0; k < kTileCfgs && k < cap; ++k) {
        txty[2 * k] = tile_tx(k);
        txty[2 * k + 1] = tile_ty(k);
    }
    return kTileCfgs;
}

lks_status lks_batch_tuning(const lks_batch* b, int* chosen2, float* ms) {
    if (!b || !chosen2) return LKS_ERR_ARG;
    chosen2[0] = b->tile[0];
    chosen2[1] = b->tile[1];
    if (ms)
        for (int w = 0; w < 2; ++w)
            for (int k = 0; k < kTileCfgs; ++k)
                ms[w * kTileCfgs + k] =
                    (b->tile_req[w] < 0 && b->tile[w] >= 0) ? b->tune_ms[w][k] : -1.f;
    return LKS_OK;
}

lks_status lks_batch_stats(const lks_batch* b, long long* stats3) {
    if (!b || !stats3) return LKS_ERR_ARG;
    stats3[0] = b->launches;
    stats3[1] = (long long)b->graphs.execs.size();
    long long nodes = 0;
    for (const auto& kv : b->graphs.nodes) nodes += kv.second;
    stats3[2] = nodes;
    return LKS_OK;
}

const char* lks_batch_last_error(const lks_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lks_batch_destroy(lks_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    b->graphs.clear();
    if (b->dmem) cudaFree(b->dmem);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

}  // extern "C"

