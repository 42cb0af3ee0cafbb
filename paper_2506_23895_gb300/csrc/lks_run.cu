// Run machinery of the host engine: the rigid motion of each step, transfers (with the 3D
// side-stream prefetch), the forward and adjoint steps on the per-context and instance-table
// kernels, runs of steps over a group of contexts (captured into CUDA graphs on the table path),
// and the forward and reverse execution of the binomial checkpoint schedule (Algorithm 1 with
// the objective of Sec. 2.5; the exact discrete adjoint in the structure of Algorithm 2).
#include "lks_engine.h"

namespace lks {
namespace eng {

bool timing_begin(lks_ctx* c, int n, int which) {
    if (c->timing_stride <= 0 || (n % c->timing_stride) != 0) return false;
    std::vector<cudaEvent_t>& v = c->tev[which];
    if (c->tused[which] + 2 > v.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return false;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return false;
        }
        v.push_back(a);
        v.push_back(b);
    }
    cudaEventRecord(v[c->tused[which]], c->st);
    return true;
}

void timing_end(lks_ctx* c, int which) {
    cudaEventRecord(c->tev[which][c->tused[which] + 1], c->st);
    c->tused[which] += 2;
}

Motion motion_row(const lks_ctx* c, int n) {
    const double* r = c->motion.data() + 8 * (size_t)n;
    Motion m;
    m.c = std::cos(r[0]);
    m.s = std::sin(r[0]);
    m.om = r[1];
    for (int a = 0; a < 3; ++a) {
        m.xG[a] = r[2 + a];
        m.uG[a] = r[5 + a];
        m.ugf[a] = (float)m.uG[a];
    }
    m.ch = (float)m.c;
    m.cl = (float)(m.c - (double)m.ch);
    m.sh = (float)m.s;
    m.sl = (float)(m.s - (double)m.sh);
    for (int a = 0; a < 2; ++a) {
        const double fl = std::floor(m.xG[a]);
        m.xgi[a] = (int)fl;
        m.xgh[a] = (float)(m.xG[a] - fl);
        m.xgl[a] = (float)((m.xG[a] - fl) - (double)m.xgh[a]);
        m.xgf[a] = (float)m.xG[a];
    }
    m.cf = (float)m.c;
    m.sf = (float)m.s;
    m.omf = (float)m.om;
    // R(theta) about the unit axis a by Rodrigues' formula (the z axis gives the plane rotation)
    const double* a = c->axis;
    const double cc = m.c, ss = m.s, oc = 1.0 - cc;
    if (!c->gaxis) {
        const double Rz[9] = {cc, -ss, 0.0, ss, cc, 0.0, 0.0, 0.0, 1.0};
        for (int k = 0; k < 9; ++k) m.R[k] = Rz[k];
        m.ax[0] = 0.0;
        m.ax[1] = 0.0;
        m.ax[2] = 1.0;
    } else {
        m.R[0] = cc + oc * a[0] * a[0];
        m.R[1] = oc * a[0] * a[1] - ss * a[2];
        m.R[2] = oc * a[0] * a[2] + ss * a[1];
        m.R[3] = oc * a[1] * a[0] + ss * a[2];
        m.R[4] = cc + oc * a[1] * a[1];
        m.R[5] = oc * a[1] * a[2] - ss * a[0];
        m.R[6] = oc * a[2] * a[0] - ss * a[1];
        m.R[7] = oc * a[2] * a[1] + ss * a[0];
        m.R[8] = cc + oc * a[2] * a[2];
        for (int k = 0; k < 3; ++k) m.ax[k] = a[k];
    }
    return m;
}

// ---------------------------------------------------------------- single-context steps

// The transfer of step n into buffer set x on stream st (3D and plain 2D paths).
template <class T>
lks_status transfer_into(lks_ctx* c, int n, const lks_ctx::XSlot& x, cudaStream_t st) {
    const Motion m = motion_row(c, n);
    if (c->gaxis) {
        launch_transfer_axis<T>(c->d, c->g, m, x.as, (const T*)c->kref, st4<T>(x.kus), st);
        LAUNCHED();
        c->stats[4] += 2;
        return LKS_OK;
    }
    launch_design_pos<T>(c->d, c->g, m, x.ts, st);
    LAUNCHED();
    launch_transfer<T>(c->d, c->g, m, x.ts, (const T*)c->kref_t, (T*)x.k2, st4<T>(x.kus), st);
    LAUNCHED();
    return LKS_OK;
}

void use_set(lks_ctx* c, int i) {
    c->xcur = i;
    c->kus = c->xs[i].kus;
    c->k2 = c->xs[i].k2;
    c->ts = c->xs[i].ts;
    c->as = c->xs[i].as;
}

// The streams and events of a 3D context's overlapped work, created once: the run stream at
// the highest priority, the side stream at the lowest.
lks_status ensure_streams(lks_ctx* c) {
    if (c->run_st) return LKS_OK;
    int least = 0, greatest = 0;
    CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CU(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, least));
    for (cudaEvent_t* e : {&c->ev_main, &c->ev_pf, &c->ev_join, &c->ev_adj, &c->ev_sens[0],
                           &c->ev_sens[1], &c->ev_fork, &c->ev_back})
        CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    CU(cudaStreamCreateWithPriority(&c->run_st, cudaStreamNonBlocking, greatest));
    return LKS_OK;
}

// Fork a 3D context's run onto its high-priority stream (after the work on the caller's
// stream) and join it back afterwards.
lks_status run_fork(lks_ctx* c) {
    c->user_st = c->st;
    if (!c->pf_on) return LKS_OK;
    lks_status s = ensure_streams(c);
    if (s != LKS_OK) return s;
    CU(cudaEventRecord(c->ev_fork, c->user_st));
    CU(cudaStreamWaitEvent(c->run_st, c->ev_fork, 0));
    c->st = c->run_st;
    return LKS_OK;
}

lks_status run_join(lks_ctx* c, lks_status s) {
    if (c->pf_on && c->st == c->run_st && c->run_st) {
        cudaError_t e1 = cudaEventRecord(c->ev_back, c->run_st);
        cudaError_t e2 = cudaStreamWaitEvent(c->user_st, c->ev_back, 0);
        c->st = c->user_st;
        if (s == LKS_OK && (e1 != cudaSuccess || e2 != cudaSuccess))
            return fail(c, LKS_ERR_CUDA, "join of the run's stream failed");
    }
    c->st = c->user_st;
    return s;
}

// The context's stream waits for all side-stream work (prefetches, sensitivity gathers); a
// prefetch in flight is dropped, the current set keeps its step.
lks_status transfer_settle(lks_ctx* c) {
    if (c->side) {
        CU(cudaEventRecord(c->ev_join, c->side));
        CU(cudaStreamWaitEvent(c->st, c->ev_join, 0));
    }
    c->pf_step = -1;
    return LKS_OK;
}

// Settle and forget the current set too: no side work outlives a run, and the next run
// (after a possible change of design or motion) starts from fresh transfers.
lks_status transfer_join(lks_ctx* c) {
    lks_status s = transfer_settle(c);
    c->cur_step = -1;
    c->pf_last = -1;
    c->pf_dir = 0;
    return s;
}

// kappa and u_S of step n in the current buffer set.  3D: the transfer depends on the motion
// and the design only, so while the step n kernels run, the transfer of the step the run is
// heading to (n + 1 going forward, n - 1 going backward) is computed into the other set on a
// side stream, ordered by events; a later request for that step swaps the sets.  A request for
// the step the current set already holds (the adjoint's first step after a tape segment)
// launches nothing.
template <class T>
lks_status transfer_at(lks_ctx* c, int n) {
    if (c->d.nd == 0 || c->g.boxN == 0) return LKS_OK;
    if (c->fused2d) {
        CU(launch_set_int(c->nbase, n, c->st));
        CU(launch_t_design_pos(c->plan, 0, c->st));
        CU(launch_t_transfer2d(c->plan, 0, -1, false, c->st));
        c->stats[4] += 3;
        return LKS_OK;
    }
    if (!c->pf_on) return transfer_into<T>(c, n, c->xs[c->xcur], c->st);
    {
        lks_status s = ensure_streams(c);
        if (s != LKS_OK) return s;
    }
    if (c->pf_step == n) {
        CU(cudaStreamWaitEvent(c->st, c->ev_pf, 0));
        use_set(c, 1 - c->xcur);
        c->pf_step = -1;
    } else if (c->cur_step != n) {
        // the current set may still be read by a sensitivity gather on the side stream (a run
        // that changed direction or jumped): wait for the side stream before overwriting it
        CU(cudaEventRecord(c->ev_join, c->side));
        CU(cudaStreamWaitEvent(c->st, c->ev_join, 0));
        lks_status s = transfer_into<T>(c, n, c->xs[c->xcur], c->st);
        if (s != LKS_OK) return s;
    }
    c->cur_step = n;
    // direction of the run: one step on from the previous request, or the same step again (a
    // tape segment's last step, then the adjoint of that segment: the run turns around)
    int dir = 0;
    if (c->pf_last >= 0 && std::abs(n - c->pf_last) == 1) dir = n - c->pf_last;
    else if (c->pf_last == n) dir = -c->pf_dir;
    c->pf_dir = dir;
    c->pf_last = n;
    const int next = n + dir;
    if (dir != 0 && next >= 1 && next <= c->cfg.max_steps && c->pf_step != next) {
        // a stale prefetch still in flight is overwritten after it, in side-stream order
        // the other set was last read by work already on the context's stream
        CU(cudaEventRecord(c->ev_main, c->st));
        CU(cudaStreamWaitEvent(c->side, c->ev_main, 0));
        lks_status s = transfer_into<T>(c, next, c->xs[1 - c->xcur], c->side);
        if (s != LKS_OK) return s;
        CU(cudaEventRecord(c->ev_pf, c->side));
        c->pf_step = next;
    }
    return LKS_OK;
}

// Variant of the fused 3D step for this context: the requested one, else each variant timed on
// the step src -> dst (three launches after one warm-up, CUDA events) and the fastest kept.
// Every variant writes the same dst, so the timing launches leave the step done.
lks_status choose_step3d(lks_ctx* c, const void* src, void* dst) {
    if (c->step3d_req >= 0) {
        c->step3d_var = c->step3d_req;
        return LKS_OK;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(c->st, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        c->step3d_var = 1;
        return LKS_OK;
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = 1;
    cudaError_t err = cudaSuccess;
    for (int v = 0; v < kStep3dVariants && err == cudaSuccess; ++v) {
        for (int r = 0; r < 4 && err == cudaSuccess; ++r) {
            if (r == 1) err = cudaEventRecord(e0, c->st);
            if (err == cudaSuccess)
                err = launch_fused_step3d(c->g, (const V4<float>*)src, (const V4<float>*)c->kus,
                                          (V4<float>*)dst, c->flags + 3, c->st, v);
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, c->st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            bv = v;
        }
        c->stats[4] += 4;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return fail(c, LKS_ERR_CUDA, "step variant timing: %s", cudaGetErrorString(err));
    c->step3d_var = bv;
    return LKS_OK;
}

// One forward step n: src -> dst (3D / FP64 / plain paths).
template <class T>
lks_status forward_step(lks_ctx* c, int n, const void* src, void* dst) {
    lks_status s = transfer_at<T>(c, n);
    if (s != LKS_OK) return s;
    const bool tm = timing_begin(c, n, 0);
    if (sizeof(T) == 4 && c->fused3d && !c->g.ks) {
        if (c->step3d_var < 0) {
            s = choose_step3d(c, src, dst);
            if (s != LKS_OK) return s;
        }
        cudaError_t e = launch_fused_step3d(c->g, (const V4<float>*)src, (const V4<float>*)c->kus,
                                            (V4<float>*)dst, c->flags + 3, c->st, c->step3d_var);
        if (e != cudaSuccess) return fail(c, LKS_ERR_CUDA, "fused step: %s", cudaGetErrorString(e));
        ++c->stats[4];
    } else {
        launch_feq<T>(c->g, (const V4<T>*)src, (T*)c->F, c->st);
        LAUNCHED();
        launch_gather<T>(c->g, (const T*)c->F, (const V4<T>*)c->kus, (V4<T>*)dst, c->st);
        LAUNCHED();
    }
    if (tm) timing_end(c, 0);
    return LKS_OK;
}

char* slot_ptr(lks_ctx* c, int slot) { return c->pool + (size_t)slot * c->snap_bytes; }

lks_status copy_state(lks_ctx* c, void* dst, const void* src, cudaStream_t st) {
    CU(cudaMemcpyAsync(dst, src, (size_t)c->g.nodes * 4 * c->tsz, cudaMemcpyDeviceToDevice, st));
    return LKS_OK;
}

// One adjoint step n on the per-context kernels: lambda^n (lam[lam_par]) -> lambda^{n-1}.
template <class T>
lks_status adjoint_step(lks_ctx* c, int n, const void* sn, const void* sp) {
    const double h = 1.0 / (double)(c->cfg.win_end - c->cfg.win_begin + 1);
    const double hn = (n >= c->cfg.win_begin && n <= c->cfg.win_end) ? h : 0.0;
    lks_status s = transfer_at<T>(c, n);
    if (s != LKS_OK) return s;
    V4<T>* lc = st4<T>(c->lam[c->lam_par]);
    V4<T>* ln = st4<T>(c->lam[1 - c->lam_par]);
    const bool side_sens = c->pf_on && c->side && c->d.nd > 0 && c->g.boxN > 0;
    if (side_sens) {   // e alternates between two buffers; wait for the gather that read this one
        c->e = c->ebuf[c->epar];
        CU(cudaStreamWaitEvent(c->st, c->ev_sens[c->epar], 0));
    }
    const bool tm = timing_begin(c, n, 1);
    launch_adj_bcT<T>(c->g, lc, hn, c->st);
    LAUNCHED();
    if (sizeof(T) == 4 && c->fused3d && !c->g.ks) {
        cudaError_t e = launch_fused_adj3d(c->g, (const V4<float>*)lc, (V4<float>*)ln,
                                           (const V4<float>*)c->kus, (const V4<float>*)sn,
                                           (const V4<float>*)sp, (float*)c->e, c->face, hn,
                                           c->flags + 3, c->st, c->adj3d_var);
        if (e != cudaSuccess) return fail(c, LKS_ERR_CUDA, "fused adjoint: %s", cudaGetErrorString(e));
        c->stats[4] += 2;
    } else {
        launch_adj_mu<T>(c->g, lc, (const V4<T>*)c->kus, (const V4<T>*)sn, st4<T>(c->mu),
                         (T*)c->e, hn, c->st, (const V4<T>*)c->u3);
        LAUNCHED();
        launch_adj_moments<T>(c->g, st4<T>(c->mu), (const V4<T>*)sp, ln, (T*)c->phi, c->st,
                              (V4<T>*)c->u3);
        LAUNCHED();
        launch_adj_divT<T>(c->g, (const T*)c->phi, ln, c->st);
        LAUNCHED();
    }
    if (tm) timing_end(c, 1);
    if (c->d.nd > 0 && c->g.boxN > 0) {
        // on the side stream (3D): after this step's adjoint kernels, before the prefetch that
        // will next overwrite this step's transfer set; dJ/dgamma sums stay in step order
        cudaStream_t ss = c->st;
        if (side_sens) {
            CU(cudaEventRecord(c->ev_adj, c->st));
            CU(cudaStreamWaitEvent(c->side, c->ev_adj, 0));
            ss = c->side;
        }
        if (c->gaxis)
            launch_sens_axis<T>(c->d, c->g, c->as, (const T*)c->e, (const T*)c->kprime, c->gacc,
                                ss);
        else
            launch_sens<T>(c->d, c->g, c->ts, (const T*)c->e, (const T*)c->kprime, c->gacc, ss);
        LAUNCHED();
        if (side_sens) {
            CU(cudaEventRecord(c->ev_sens[c->epar], c->side));
            c->epar ^= 1;
        }
    }
    c->lam_par ^= 1;
    return LKS_OK;
}

int seg_start(const lks_ctx* c, int a) { return a * c->K; }
int seg_end(const lks_ctx* c, int a) { return std::min((a + 1) * c->K, c->n_fwd); }
// ---------------------------------------------------------------- groups of contexts
// A group runs one checkpoint schedule for contexts of identical step count and snapshot pool:
// the single-context calls use a group of one, lks_batch_* a group over all its contexts.  On
// the instance-table path (D2Q9 FP32) every phase of a step is one launch over the whole group,
// and a run of steps can be captured once into a CUDA graph and replayed.


lks_status gfail(Group& G, lks_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    for (int i = 0; i < G.count; ++i) G.cs[i]->err = buf;
    return s;
}

#define GCU(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return gfail(G, LKS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

Group self_group(lks_ctx*& c) {
    Group G;
    G.cs = &c;
    G.count = 1;
    G.table = c->fused2d;
    G.plan = &c->plan;
    G.nbase = c->nbase;
    G.tile_fwd = c->tile_fwd;
    G.tile_adj = c->tile_adj;
    G.st = c->st;
    return G;
}

// Every context of the group keeps the transfers of a whole tape segment (2D table path).
bool tape_transfers(const Group& G) {
    if (!G.table) return false;
    for (int i = 0; i < G.count; ++i)
        if (!G.cs[i]->ktape || G.cs[i]->K + 1 > G.cs[i]->ktape_slots) return false;
    return true;
}

// Table-path launch sequences of one forward / adjoint step at offset k from *nbase.  kslot >= 0:
// the step's transfer goes to (forward) or comes from (adjoint) slot kslot of the transfer tape.
// The design positions of a run's first step come from their own launch, those of the later
// steps from the previous step's transfer (first, next).
cudaError_t table_fwd_launches(const Group& G, int k, int src, int dst, bool with_obj, int kslot,
                               bool first, bool next, lks_ctx* timed, int n, int& nl) {
    cudaError_t e;
    if (first) {
        if ((e = launch_t_design_pos(*G.plan, k, G.st)) != cudaSuccess) return e;
        ++nl;
    }
    if ((e = launch_t_transfer2d(*G.plan, k, kslot, next, G.st)) != cudaSuccess) return e;
    const bool tm = timed && timing_begin(timed, n, 0);
    if ((e = launch_t_step2d(*G.plan, G.tile_fwd, src, dst, kslot, G.st)) != cudaSuccess)
        return e;
    if (tm) timing_end(timed, 0);
    nl += 2;
    if (with_obj) {
        if ((e = launch_t_objective(*G.plan, k, dst, G.st)) != cudaSuccess) return e;
        ++nl;
    }
    return cudaSuccess;
}

// The adjoint step gathers the transpose of the boundary copies itself, and the sensitivity
// gather forms the design positions of its step.
cudaError_t table_adj_launches(const Group& G, int k, int lam_in, int lam_out, int sn, int sp,
                               int kslot, lks_ctx* timed, int n, int& nl) {
    cudaError_t e;
    if (kslot < 0) {
        if ((e = launch_t_design_pos(*G.plan, k, G.st)) != cudaSuccess) return e;
        if ((e = launch_t_transfer2d(*G.plan, k, -1, false, G.st)) != cudaSuccess) return e;
        nl += 2;
    }
    const bool tm = timed && timing_begin(timed, n, 1);
    if ((e = launch_t_adj2d(*G.plan, G.tile_adj, k, lam_in, lam_out, sn, sp, kslot, G.st)) !=
        cudaSuccess)
        return e;
    if (tm) timing_end(timed, 1);
    if ((e = launch_t_sens(*G.plan, k, G.st)) != cudaSuccess) return e;
    nl += 2;
    return cudaSuccess;
}

// Run `len` table-path steps from base: fn(k, nl) issues step k (1..len) and counts launches.
// With a graph cache the sequence is captured once per key and replayed.
template <class Fn>
lks_status table_run(Group& G, std::tuple<int, int, int, int, int, int> key, int base, int len,
                     Fn fn) {
    GCU(launch_set_int(G.nbase, base, G.st));
    ++G.launches;
    if (!G.graphs) {
        int nl = 0;
        for (int k = 1; k <= len; ++k) {
            cudaError_t e = fn(k, nl, true);
            if (e != cudaSuccess)
                return gfail(G, LKS_ERR_CUDA, "table kernel launch: %s", cudaGetErrorString(e));
        }
        G.launches += nl;
        return LKS_OK;
    }
    auto it = G.graphs->execs.find(key);
    if (it == G.graphs->execs.end()) {
        GCU(cudaStreamBeginCapture(G.st, cudaStreamCaptureModeThreadLocal));
        int nl = 0;
        cudaError_t e = cudaSuccess;
        for (int k = 1; k <= len && e == cudaSuccess; ++k) e = fn(k, nl, false);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(G.st, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return gfail(G, LKS_ERR_CUDA, "graph capture: %s",
                         cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return gfail(G, LKS_ERR_CUDA, "graph instantiate: %s",
                                           cudaGetErrorString(e));
        it = G.graphs->execs.emplace(key, exec).first;
        G.graphs->nodes[key] = nl;
    }
    GCU(cudaGraphLaunch(it->second, G.st));
    G.launches += G.graphs->nodes[key];
    return LKS_OK;
}

// ---------------------------------------------------------------- schedule over a group

// Advance every context of the group from from_level to to_level.  Without a tape the two
// working buffers alternate; with a tape (segment tape_seg, whose start level sits in tape slot
// 0) every level is written straight into its own tape slot and the working buffer keeps
// from_level.
template <class T>
lks_status run_steps(Group& G, int from_level, int to_level, bool with_obj, int tape_seg) {
    lks_ctx* c0 = G.cs[0];
    const int len = to_level - from_level;
    if (len > 0 && G.table) {
        const int w0 = c0->work;
        const int toff = tape_seg >= 0 ? from_level - tape_seg * c0->K : 0;
        // the objective kernel only where some instance's window meets these steps
        bool obj = false;
        for (int i = 0; i < G.count && with_obj; ++i)
            obj = obj || (G.cs[i]->cfg.win_begin <= to_level &&
                          G.cs[i]->cfg.win_end > from_level);
        // a taped step leaves its transfer in the transfer tape slot of its level
        const bool kt = tape_seg >= 0 && tape_transfers(G);
        auto fn = [&](int k, int& nl, bool direct) -> cudaError_t {
            int src, dst;
            if (tape_seg >= 0) {
                src = BUF_POOL + toff + k - 1;
                dst = BUF_POOL + toff + k;
            } else {
                const int w = (w0 + k - 1) & 1;
                src = BUF_S0 + w;
                dst = BUF_S0 + 1 - w;
            }
            return table_fwd_launches(G, k, src, dst, obj, kt ? toff + k : -1, k == 1, k < len,
                                      (direct && G.count == 1) ? c0 : nullptr, from_level + k, nl);
        };
        const auto key = std::make_tuple(tape_seg >= 0 ? 1 : 0, obj ? 1 : 0, len,
                                         tape_seg >= 0 ? toff : w0, G.tile_fwd, kt ? 1 : 0);
        lks_status s = table_run(G, key, from_level, len, fn);
        if (s != LKS_OK) return s;
        for (int i = 0; i < G.count; ++i) {
            lks_ctx* c = G.cs[i];
            if (tape_seg >= 0) {
                c->last = slot_ptr(c, toff + len);
            } else {
                c->work = (w0 + len) & 1;
                c->last = c->s[c->work];
            }
            c->stats[with_obj ? 0 : 1] += len;
        }
    } else if (len > 0) {
        lks_ctx* c = c0;
        for (int n = from_level + 1; n <= to_level; ++n) {
            const void* src;
            void* dst;
            if (tape_seg >= 0) {
                src = slot_ptr(c, n - 1 - tape_seg * c->K);
                dst = slot_ptr(c, n - tape_seg * c->K);
            } else {
                src = c->s[c->work];
                dst = c->s[1 - c->work];
            }
            lks_status s = forward_step<T>(c, n, src, dst);
            if (s != LKS_OK) return s;
            if (tape_seg < 0) c->work = 1 - c->work;
            c->last = dst;
            if (with_obj && n >= c->cfg.win_begin && n <= c->cfg.win_end) {
                launch_objective<T>(c->g, (const V4<T>*)dst, c->jstep + n, c->st);
                LAUNCHED();
            }
            if (with_obj) ++c->stats[0];
            else ++c->stats[1];
        }
    }
    for (int i = 0; i < G.count; ++i)
        G.cs[i]->work_level = (tape_seg >= 0) ? from_level : to_level;
    return LKS_OK;
}

lks_status restore_level(Group& G, int seg) {
    for (int i = 0; i < G.count; ++i) {
        lks_ctx* c = G.cs[i];
        const int lev = seg_start(c, seg);
        if (c->work_level == lev) continue;
        if (seg != 0 && c->slot_of[seg] < 0) return fail(c, LKS_ERR_ARG, "schedule: no snapshot");
        const void* src = (seg == 0) ? c->s0 : (const void*)slot_ptr(c, c->slot_of[seg]);
        lks_status s = copy_state(c, c->s[c->work], src, G.st);
        if (s != LKS_OK) return s;
        c->work_level = lev;
    }
    return LKS_OK;
}

template <class T>
lks_status exec_forward_action(Group& G, const Act& a, bool with_obj) {
    lks_ctx* c0 = G.cs[0];
    switch (a.kind) {
        case A_RESTORE:
            return restore_level(G, a.a);
        case A_ADVANCE:
            return run_steps<T>(G, seg_start(c0, a.a), seg_start(c0, a.b), with_obj, -1);
        case A_STORE:
            for (int i = 0; i < G.count; ++i) {
                lks_ctx* c = G.cs[i];
                if (c->free_slots.empty()) return fail(c, LKS_ERR_NOMEM, "schedule: out of slots");
                const int sl = c->free_slots.back();
                c->free_slots.pop_back();
                c->slot_of[a.a] = sl;
                lks_status s = copy_state(c, slot_ptr(c, sl), c->s[c->work], G.st);
                if (s != LKS_OK) return s;
            }
            return LKS_OK;
        case A_FREE:
            for (int i = 0; i < G.count; ++i) {
                lks_ctx* c = G.cs[i];
                c->free_slots.push_back(c->slot_of[a.a]);
                c->slot_of[a.a] = -1;
            }
            return LKS_OK;
        case A_TAPE:
            for (int i = 0; i < G.count; ++i) {
                lks_ctx* c = G.cs[i];
                lks_status s = copy_state(c, slot_ptr(c, 0), c->s[c->work], G.st);
                if (s != LKS_OK) return s;
            }
            return run_steps<T>(G, seg_start(c0, a.a), seg_end(c0, a.a), with_obj, a.a);
        default:
            return gfail(G, LKS_ERR_ARG, "schedule: unexpected action");
    }
}

template <class T>
lks_status exec_adj(Group& G, int seg) {
    lks_ctx* c0 = G.cs[0];
    const int a = seg_start(c0, seg), b = seg_end(c0, seg), len = b - a;
    if (len <= 0) return LKS_OK;
    if (!G.table) {
        for (int n = b; n > a; --n) {
            lks_status s = adjoint_step<T>(c0, n, slot_ptr(c0, n - a), slot_ptr(c0, n - 1 - a));
            if (s != LKS_OK) return s;
        }
        return LKS_OK;
    }
    const int par0 = c0->lam_par;
    // the tape of this segment (levels 0..len) holds the transfer of step a + kk in slot kk
    const bool kt = tape_transfers(G);
    auto fn = [&](int k, int& nl, bool direct) -> cudaError_t {
        const int kk = len - k + 1;                 // step n = a + kk, from b down to a + 1
        const int par = par0 ^ ((k - 1) & 1);
        return table_adj_launches(G, kk, BUF_LAM0 + par, BUF_LAM0 + 1 - par, BUF_POOL + kk,
                                  BUF_POOL + kk - 1, kt ? kk : -1,
                                  (direct && G.count == 1) ? c0 : nullptr, a + kk, nl);
    };
    const auto key = std::make_tuple(2, kt ? 1 : 0, len, par0, 0, G.tile_adj);
    lks_status s = table_run(G, key, a, len, fn);
    if (s != LKS_OK) return s;
    for (int i = 0; i < G.count; ++i) G.cs[i]->lam_par = par0 ^ (len & 1);
    return LKS_OK;
}

template <class T>
lks_status do_forward(Group& G, int N) {
    for (int i = 0; i < G.count; ++i) {
        lks_ctx* c = G.cs[i];
        c->n_fwd = N;
        plan_tape(N, c->pool_slots, c->K, c->M, c->S);
        c->acts.clear();
        gen_schedule(0, c->M, c->S, c->acts);
        c->slot_of.assign(c->M + 1, -1);
        c->free_slots.clear();
        for (int k = c->pool_slots - 1; k >= c->K + 1; --k) c->free_slots.push_back(k);
        c->stats[0] = c->stats[1] = 0;
        c->stats[2] = c->S;
        c->stats[3] = c->K;
        c->stats[4] = 0;
        c->work = 0;
        c->work_level = -1;
        c->last = nullptr;
        c->fwd_valid = false;
        {
            lks_status s = transfer_join(c);
            if (s != LKS_OK) return s;
        }
        CU(cudaMemsetAsync(c->jstep, 0, (size_t)(c->cfg.max_steps + 2) * 8, G.st));
        CU(cudaMemsetAsync(c->flags, 0, 64, G.st));
    }
    const std::vector<Act>& acts = G.cs[0]->acts;
    size_t i = 0;
    for (; i < acts.size(); ++i) {
        lks_status s = exec_forward_action<T>(G, acts[i], true);
        if (s != LKS_OK) return s;
        if (acts[i].kind == A_TAPE) break;
    }
    std::vector<std::vector<double>> js(G.count);
    std::vector<int> fl(4 * (size_t)G.count);
    for (int k = 0; k < G.count; ++k) {
        lks_ctx* c = G.cs[k];
        lks_status st = transfer_settle(c);   // the adjoint may reuse the last step's transfer
        if (st != LKS_OK) return st;
        c->adj_begin = i + 1;
        js[k].assign(c->cfg.max_steps + 2, 0.0);
        CU(cudaMemcpyAsync(js[k].data(), c->jstep, js[k].size() * 8, cudaMemcpyDeviceToHost, G.st));
        launch_check_state<T>(c->g, (const V4<T>*)c->last, c->flags + 2, G.st);
        LAUNCHED();
        CU(cudaMemcpyAsync(c->s_end, c->last, c->snap_bytes, cudaMemcpyDeviceToDevice, G.st));
        CU(cudaMemcpyAsync(fl.data() + 4 * k, c->flags, 16, cudaMemcpyDeviceToHost, G.st));
    }
    GCU(cudaStreamSynchronize(G.st));
    lks_status worst = LKS_OK;
    for (int k = 0; k < G.count; ++k) {
        lks_ctx* c = G.cs[k];
        const int* f = fl.data() + 4 * k;
        lks_status s = LKS_OK;
        if (f[1]) s = fail(c, LKS_ERR_ARG, "transfer tap list overflow");
        else if (f[3] & 8) s = fail(c, LKS_ERR_TIMEOUT, "a tensor-copy wait timed out in the fused step");
        else if (f[3]) s = fail(c, LKS_ERR_CUDA, "fused step reported error %d", f[3]);
        else if (f[2]) s = fail(c, LKS_ERR_DIVERGED, "state diverged (non-finite or |u| >= 0.5)");
        if (s != LKS_OK) {
            if (worst == LKS_OK) worst = s;
            continue;
        }
        const int w0 = c->cfg.win_begin, w1 = std::min(c->cfg.win_end, N);
        const double h = 1.0 / (double)(c->cfg.win_end - c->cfg.win_begin + 1);
        c->have_end = true;
        double J = 0.0;
        for (int n = w0; n <= w1; ++n) J += h * js[k][n];   // J = h sum_n j_n in step order
        c->J = J;
        c->fwd_valid = true;
    }
    return worst;
}

template <class T>
lks_status do_adjoint(Group& G) {
    for (int i = 0; i < G.count; ++i) {
        lks_ctx* c = G.cs[i];
        c->lam_par = 0;
        CU(cudaMemsetAsync(c->flags, 0, 64, G.st));
        if (c->adj_warm && c->have_lend)   // warm start: lambda^N from the last lambda^0
            CU(cudaMemcpyAsync(c->lam[0], c->l_end, c->snap_bytes, cudaMemcpyDeviceToDevice, G.st));
        else
            CU(cudaMemsetAsync(c->lam[0], 0, c->snap_bytes, G.st));
        if (c->u3) CU(cudaMemsetAsync(c->u3, 0, c->snap_bytes, G.st));
        if (c->d.nd > 0) CU(cudaMemsetAsync(c->gacc, 0, (size_t)c->d.nd * 8, G.st));
    }
    lks_ctx* c0 = G.cs[0];
    for (size_t i = c0->adj_begin - 1; i < c0->acts.size(); ++i) {
        const Act& a = c0->acts[i];
        if (a.kind == A_TAPE && i == c0->adj_begin - 1) continue;  // recorded by the forward
        lks_status s = (a.kind == A_ADJ) ? exec_adj<T>(G, a.a) : exec_forward_action<T>(G, a, false);
        if (s != LKS_OK) return s;
    }
    // the tape of the last segment has been overwritten: a second adjoint needs a new forward
    std::vector<int> fl(4 * (size_t)G.count);
    for (int k = 0; k < G.count; ++k) {
        lks_ctx* c = G.cs[k];
        c->fwd_valid = false;
        {
            lks_status st = transfer_join(c);
            if (st != LKS_OK) return st;
        }
        CU(cudaMemcpyAsync(c->l_end, c->lam[c->lam_par], c->snap_bytes, cudaMemcpyDeviceToDevice,
                           G.st));
        c->have_lend = true;
        CU(cudaMemcpyAsync(fl.data() + 4 * k, c->flags, 16, cudaMemcpyDeviceToHost, G.st));
    }
    GCU(cudaStreamSynchronize(G.st));
    lks_status worst = LKS_OK;
    for (int k = 0; k < G.count; ++k) {
        lks_ctx* c = G.cs[k];
        const int* f = fl.data() + 4 * k;
        lks_status s = LKS_OK;
        if (f[1]) s = fail(c, LKS_ERR_ARG, "transfer tap list overflow");
        else if (f[3] & 8) s = fail(c, LKS_ERR_TIMEOUT, "a tensor-copy wait timed out in the fused step");
        else if (f[3]) s = fail(c, LKS_ERR_CUDA, "fused step reported error %d", f[3]);
        if (s != LKS_OK && worst == LKS_OK) worst = s;
    }
    return worst;
}

template <class T>
lks_status reset_initial(lks_ctx* c) {
    launch_fill_uniform<T>(c->g, st4<T>(c->s0), c->cfg.u_init, c->st);
    LAUNCHED();
    launch_apply_bc<T>(c->g, st4<T>(c->s0), c->st);
    LAUNCHED();
    return LKS_OK;
}

// Host record of a context's instance-table entry (valid once design and motion are set).
Inst make_inst(const lks_ctx* c) {
    Inst I;
    std::memset(&I, 0, sizeof(I));
    I.g = c->g;
    I.d = c->d;
    I.pos_b[0] = reinterpret_cast<int2*>(c->ts.col_base);
    I.pos_sc[0] = c->ts.col_sc;
    I.pos_b[1] = reinterpret_cast<int2*>(c->pos2_b);
    I.pos_sc[1] = c->pos2_sc;
    I.motion = c->dmotion;
    I.bufs = c->dbufs;
    I.kref = (const float*)c->kref;
    I.kprime = (const float*)c->kprime;
    I.kus = (V4<float>*)c->kus;
    I.kus_tape = (V4<float>*)c->ktape;
    I.e = (float*)c->e;
    I.gacc = c->gacc;
    I.jstep = c->jstep;
    I.win_begin = c->cfg.win_begin;
    I.win_end = c->cfg.win_end;
    // the same FP64 expressions as the per-node source of the plain kernels, rounded once
    const double h = 1.0 / (double)(c->cfg.win_end - c->cfg.win_begin + 1);
    const Geom& g = c->g;
    I.hwin = h;
    I.Af = (float)g.A;
    I.bf[0] = (float)g.body[0];
    I.bf[1] = (float)g.body[1];
    I.src_r = g.okind == 0 ? (float)(-h / (3.0 * g.ocount)) : 0.f;
    I.src_x = g.okind == 0 ? 0.f : (float)(-h * g.odir[0] / g.ocount);
    I.src_y = g.okind == 0 ? 0.f : (float)(-h * g.odir[1] / g.ocount);
    for (int f = 0; f < 4; ++f) {
        I.bcf[f] = make_float4((float)g.bcv[f][0], (float)g.bcv[f][1], 0.f,
                               (float)(g.bcv[f][3] - g.rho0));
        I.bckeep[f] = g.bc[f] == BC_WALL || g.bc[f] == BC_INLET;
    }
    return I;
}

// Work units of one instance per unit kind (lks_table.h).
void inst_units(const lks_ctx* c, int out[U_COUNT]) {
    const Geom& g = c->g;
    const bool body = c->d.nd > 0 && g.boxN > 0;
    out[U_DCOL] = body ? (int)((c->d.ncol + kUnitThreads - 1) / kUnitThreads) : 0;
    // footprint box in tiles of kBoxTile x kBoxTile nodes (the 2D transfer stages the design
    // nodes a tile reads in shared memory)
    out[U_BOX] = body ? ((g.bn[0] + kBoxTile - 1) / kBoxTile) * ((g.bn[1] + kBoxTile - 1) / kBoxTile)
                      : 0;
    out[U_INST] = 1;
    for (int k = 0; k < kTileCfgs; ++k)
        out[U_TILE0 + k] = tile_count(g.n[0], tile_tx(k), g.periodic[0]) *
                           tile_count(g.n[1], tile_ty(k), g.periodic[1]);
}

// Build a plan over contexts: the table and prefix arrays go to dinst / dpre (device, with
// room for cs.size() entries), the host plan gets the totals and the persistent grids.
cudaError_t build_plan(const std::vector<lks_ctx*>& cs, Inst* dinst, int* dpre, int* nbase,
                       cudaStream_t st, Plan& p) {
    const int B = (int)cs.size();
    std::vector<Inst> tab(B);
    std::vector<int> pre((size_t)U_COUNT * (B + 1), 0);
    for (int i = 0; i < B; ++i) {
        tab[i] = make_inst(cs[i]);
        int u[U_COUNT];
        inst_units(cs[i], u);
        for (int k = 0; k < U_COUNT; ++k)
            pre[(size_t)k * (B + 1) + i + 1] = pre[(size_t)k * (B + 1) + i] + u[k];
    }
    cudaError_t e = cudaMemcpyAsync(dinst, tab.data(), sizeof(Inst) * B, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dpre, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host vectors go out of scope
    if (e != cudaSuccess) return e;
    std::memset(&p, 0, sizeof(p));
    p.tab = dinst;
    p.pre = dpre;
    p.count = B;
    p.nbase = nbase;
    for (int k = 0; k < U_COUNT; ++k) p.total[k] = pre[(size_t)k * (B + 1) + B];
    plan_grids(p);
    return cudaGetLastError();
}

// kappa_ref and kappa' from the stored gamma, through the filter chain when it is on (the
// [0,1] check of gamma sets flags[0]).
lks_status design_prep(lks_ctx* c) {
    const double* src = c->gamma;
    if (c->fR > 0.0) {
        launch_filter(c->d, c->fR, c->fbeta, c->feta, c->gamma, c->gbar, c->hp, c->fws, c->st);
        LAUNCHED();
        src = c->gbar;
    }
    if (c->prec == LKS_FP64)
        launch_design_prep<double>(c->d, src, c->cfg.kappa_max, c->cfg.q, (double*)c->kref,
                                   (double*)c->kref_t, (double*)c->kprime, c->flags, c->st);
    else
        launch_design_prep<float>(c->d, src, c->cfg.kappa_max, c->cfg.q, (float*)c->kref,
                                  (float*)c->kref_t, (float*)c->kprime, c->flags, c->st);
    LAUNCHED();
    return LKS_OK;
}

// dJ/dgamma of the last adjoint: the accumulator, or its pull-back through the filter chain.
const double* design_gradient(lks_ctx* c, cudaStream_t st) {
    if (c->fR <= 0.0) return c->gacc;
    launch_filter_T(c->d, c->fR, c->gacc, c->hp, c->fws, c->gout, st);
    ++c->stats[4];
    return c->gout;
}

// After a new motion table: rows with cos/sin evaluated on the host go to the device (the
// instance-table kernels read them there), and a table context rebuilds its one-entry plan.
lks_status finish_motion(lks_ctx* c) {
    const int rows = c->cfg.max_steps + 1;
    std::vector<Motion> mr(rows);
    for (int n = 0; n < rows; ++n) mr[n] = motion_row(c, n);
    CU(cudaMemcpyAsync(c->dmotion, mr.data(), sizeof(Motion) * rows, cudaMemcpyHostToDevice, c->st));
    CU(cudaStreamSynchronize(c->st));
    ++c->geo_gen;
    if (c->fused2d) {
        std::vector<lks_ctx*> one(1, c);
        CU(build_plan(one, c->dinst, c->dpre, c->nbase, c->st, c->plan));
    }
    c->have_motion = true;
    return LKS_OK;
}

template lks_status transfer_at<float>(lks_ctx*, int);
template lks_status transfer_at<double>(lks_ctx*, int);
template lks_status reset_initial<float>(lks_ctx*);
template lks_status reset_initial<double>(lks_ctx*);
template lks_status do_forward<float>(Group&, int);
template lks_status do_forward<double>(Group&, int);
template lks_status do_adjoint<float>(Group&);
template lks_status do_adjoint<double>(Group&);

}  // namespace eng
}  // namespace lks
