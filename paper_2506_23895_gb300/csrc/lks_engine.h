// Internal declarations of the host engine, shared by its translation units (not part of the
// public ABI, which is include/lks.h): the context record, the checkpoint-schedule actions,
// groups of contexts and the run machinery.
//   lks_schedule.cu  binomial checkpoint schedule over tape segments (host only)
//   lks_run.cu       transfers, forward and adjoint steps, runs of steps over a group of
//                    contexts, CUDA graphs of the instance-table path, the schedule's execution
//   lks_engine.cu    validation, workspace layout and the per-context C ABI
//   lks_batch.cu     batches of contexts (lks_batch_*)
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "lks.h"
#include "lks_internal.h"
#include "lks_table.h"

namespace lks {
namespace eng {

enum ActKind { A_RESTORE = 0, A_ADVANCE = 1, A_STORE = 2, A_FREE = 3, A_TAPE = 4, A_ADJ = 5 };
struct Act {
    int kind, a, b;
};

// Reverse segments [a, b) with s free snapshot slots into `out` (lks_schedule.cu).
void gen_schedule(int a, int b, int s, std::vector<Act>& out);
// Tape length K, segment count M and checkpoint slots S for N steps and P pool slots.
void plan_tape(int N, int P, int& K, int& M, int& S);

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace eng
}  // namespace lks

// the engine's translation units all work in the library namespace
using namespace lks;

struct lks_ctx {
    lks_config cfg;
    Geom g;
    Design d;
    int prec;
    size_t tsz;
    cudaStream_t st;
    // workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    void* s[2];
    void* s0;
    void* lam[2];       // the two adjoint buffers; lam[lam_par] holds lambda^n
    int lam_par = 0;
    void* F;
    void* mu;
    void* phi;
    void* kus;
    void* e;
    double* gamma;
    void* kref;
    void* kprime;
    void* kref_t;
    void* k2;
    float* face;
    void* u3;           // 3 U~ of the previous adjoint step (printed-ALKS variant only)
    double* gacc;
    double* jstep;
    TransferScratch ts;
    int* flags;
    char* pool;
    int pool_slots;
    size_t snap_bytes;
    void* ktape = nullptr;       // transfer tape of the 2D table path (ktape_slots box records)
    int ktape_slots = 0;
    void* pos2_b = nullptr;      // 2D table path: design positions of odd steps (int2 per column)
    float4* pos2_sc = nullptr;   // and their sin, cos table
    // host state
    std::vector<double> motion;
    bool have_design = false, have_motion = false, fwd_valid = false;
    int n_fwd = 0;
    int K = 0, M = 0, S = 0;
    std::vector<lks::eng::Act> acts;
    size_t adj_begin = 0;
    std::vector<int> slot_of;   // segment -> pool slot (-1 none)
    std::vector<int> free_slots;
    int work = 0;               // index of the working state buffer
    int work_level = -1;        // step level held by the working buffer (-1 unknown)
    double J = 0.0;
    long long stats[5] = {0, 0, 0, 0, 0};
    const void* last = nullptr;  // buffer holding the newest forward level
    bool fused3d = false;        // FP32 3D non-periodic: one fused kernel per forward step
    // instance table of this context (D2Q9 FP32: the table kernels of lks_fused2d.cu)
    bool fused2d = false;
    Motion* dmotion = nullptr;   // device motion rows
    void** dbufs = nullptr;      // device buffer table (BUF_*)
    std::vector<void*> hbufs;    // its host copy
    Inst* dinst = nullptr;
    int* dpre = nullptr;         // device prefix arrays, U_COUNT x 2
    int* nbase = nullptr;        // device step base of this context's own runs
    Plan plan;
    int geo_gen = 0;             // bumped when the footprint box changes
    int tile_fwd = 0, tile_adj = 0;   // tile shapes of the fused 2D kernels
    bool gaxis = false;          // 3D rotation about an axis other than z
    int step3d_req = 1;          // fused 3D step variant requested (-1: time them once)
    int step3d_var = -1;         // variant in use (-1: not chosen yet)
    int adj3d_var = 1;           // fused 3D adjoint variant (kAdj3dVariants)
    double axis[3] = {0.0, 0.0, 1.0};
    AxisScratch as;
    // 3D transfers in two buffer sets: the current one (kus, k2, ts, as above point into it)
    // and one the next step's transfer is prefetched into on a side stream
    struct XSlot {
        void* kus;
        void* k2;
        TransferScratch ts;
        AxisScratch as;
    } xs[2];
    int xcur = 0;
    bool pf_on = false;          // prefetching enabled (3D with a design grid)
    int cur_step = -1;           // step whose transfer the current set holds (-1: none)
    int pf_step = -1;            // step being prefetched into the other set (-1: none)
    int pf_last = -1;            // step of the previous transfer request
    int pf_dir = 0;              // direction of the run at that request (+1, -1, 0)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_main = nullptr, ev_pf = nullptr, ev_join = nullptr;
    // the sensitivity gather of a 3D adjoint step runs on the side stream too, reading e from
    // one of two buffers while the next step writes the other
    void* ebuf[2] = {nullptr, nullptr};
    int epar = 0;
    cudaEvent_t ev_adj = nullptr, ev_sens[2] = {nullptr, nullptr};
    // forward and adjoint runs of a 3D context execute on an internal stream of the highest
    // priority, forked from and joined back to the caller's stream, so that the stencil blocks
    // win the block scheduler and the side-stream work fills the gaps
    cudaStream_t run_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_back = nullptr;
    cudaStream_t user_st = nullptr;
    // design chain: density filter radius (0 = off), projection steepness and threshold
    double fR = 0.0, fbeta = 1.0, feta = 0.5;
    double* gbar = nullptr;      // projected field the solver sees
    double* hp = nullptr;        // H'(filtered gamma)
    double* fws = nullptr;       // filter normaliser per design node
    double* gout = nullptr;      // dJ/dgamma through the chain
    double* gtmp = nullptr;      // design-grid scratch
    double* scal = nullptr;      // device scalars
    // static solids and warm starts
    void* ks = nullptr;          // static Brinkman field storage (g.ks points here when set)
    void* s_end = nullptr;       // final state of the last forward run
    void* l_end = nullptr;       // lambda^0 of the last adjoint run
    bool have_end = false, have_lend = false, adj_warm = false;
    // optional event timing of the stencil kernels, sampled every timing_stride steps
    int timing_stride = 0;
    std::vector<cudaEvent_t> tev[2];
    size_t tused[2] = {0, 0};
    std::string err;
};

namespace lks {
namespace eng {

// Record the message of a failed call on the context and return its status.
lks_status fail(lks_ctx* c, lks_status s, const char* fmt, ...);
// cudaMalloc behind the host-side fault injection of lks_inject_alloc_failure.
cudaError_t dev_alloc(void** p, size_t bytes);

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, LKS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

// A device allocation inside an entry point: LKS_ERR_NOMEM with a message on failure.
#define ALLOC(pp, bytes)                                                                  \
    do {                                                                                  \
        if (dev_alloc((void**)(pp), (bytes)) != cudaSuccess) {                            \
            cudaGetLastError();                                                           \
            return fail(c, LKS_ERR_NOMEM, "device allocation of %zu bytes failed",        \
                        (size_t)(bytes));                                                 \
        }                                                                                 \
    } while (0)

#define LAUNCHED()                                                                        \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, LKS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_));    \
        ++c->stats[4];                                                                    \
    } while (0)

template <class T>
inline V4<T>* st4(void* p) {
    return (V4<T>*)p;
}

struct GraphCache {
    std::map<std::tuple<int, int, int, int, int, int>, cudaGraphExec_t> execs;
    std::map<std::tuple<int, int, int, int, int, int>, int> nodes;
    ~GraphCache() {
        for (auto& kv : execs) cudaGraphExecDestroy(kv.second);
    }
    void clear() {
        for (auto& kv : execs) cudaGraphExecDestroy(kv.second);
        execs.clear();
        nodes.clear();
    }
};

struct Group {
    lks_ctx* const* cs = nullptr;
    int count = 0;
    bool table = false;          // instance-table kernels
    const Plan* plan = nullptr;
    int* nbase = nullptr;
    int tile_fwd = 0, tile_adj = 0;
    GraphCache* graphs = nullptr;   // null: launch directly
    cudaStream_t st = nullptr;
    long long launches = 0;      // kernels launched (graph nodes included)
};

Group self_group(lks_ctx*& c);
char* slot_ptr(lks_ctx* c, int slot);
Motion motion_row(const lks_ctx* c, int n);
lks_status run_fork(lks_ctx* c);
lks_status run_join(lks_ctx* c, lks_status s);
lks_status transfer_join(lks_ctx* c);
lks_status finish_motion(lks_ctx* c);
lks_status design_prep(lks_ctx* c);
const double* design_gradient(lks_ctx* c, cudaStream_t st);
cudaError_t build_plan(const std::vector<lks_ctx*>& cs, Inst* dinst, int* dpre, int* nbase,
                       cudaStream_t st, Plan& p);
template <class T>
lks_status transfer_at(lks_ctx* c, int n);
template <class T>
lks_status reset_initial(lks_ctx* c);
template <class T>
lks_status do_forward(Group& G, int N);
template <class T>
lks_status do_adjoint(Group& G);

}  // namespace eng
}  // namespace lks
