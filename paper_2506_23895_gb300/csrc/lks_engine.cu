// Host engine behind the C ABI of include/lks.h: validates the problem, carves the device
// workspace, runs Algorithm 1 (forward with the objective of Sec. 2.5) and the reverse adjoint
// sweep (Algorithm 2 structure, exact discrete adjoint) under a binomial checkpoint schedule
// over tape segments, so that the stored history fits the given device memory.
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

using namespace lks;

namespace {

enum ActKind { A_RESTORE = 0, A_ADVANCE = 1, A_STORE = 2, A_FREE = 3, A_TAPE = 4, A_ADJ = 5 };
struct Act {
    int kind, a, b;
};

// Number of segments reversible with s free snapshot slots when every segment is advanced at
// most r times: C(s + r, s) (Griewank & Walther's binomial bound), capped.
double binom_beta(int s, int r) {
    double v = 1.0;
    for (int i = 1; i <= s; ++i) {
        v = v * (double)(r + i) / (double)i;
        if (v > 1e15) return 1e15;
    }
    return v;
}

// Reverse segments [a, b) given the state at segment a's start (snapshot or initial state)
// and s free snapshot slots.  The right part is reversed first with one slot fewer; the split
// makes the right part as long as the binomial bound allows, which minimises re-advancing.
void gen_schedule(int a, int b, int s, std::vector<Act>& out) {
    if (b - a == 1) {
        out.push_back({A_RESTORE, a, 0});
        out.push_back({A_TAPE, a, 0});
        out.push_back({A_ADJ, a, 0});
        return;
    }
    if (s <= 0) {
        for (int j = b - 1; j >= a; --j) {
            out.push_back({A_RESTORE, a, 0});
            if (j > a) out.push_back({A_ADVANCE, a, j});
            out.push_back({A_TAPE, j, 0});
            out.push_back({A_ADJ, j, 0});
        }
        return;
    }
    const int L = b - a;
    int r = 1;
    while (binom_beta(s, r) < (double)L) ++r;
    const double right = binom_beta(s - 1, r);
    long long left = (long long)L - (long long)std::min(right, (double)L);
    int m = a + (int)std::max(1LL, left);
    if (m >= b) m = b - 1;
    out.push_back({A_RESTORE, a, 0});
    out.push_back({A_ADVANCE, a, m});
    out.push_back({A_STORE, m, 0});
    gen_schedule(m, b, s - 1, out);
    out.push_back({A_FREE, m, 0});
    gen_schedule(a, m, s, out);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

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
    // host state
    std::vector<double> motion;
    bool have_design = false, have_motion = false, fwd_valid = false;
    int n_fwd = 0;
    int K = 0, M = 0, S = 0;
    std::vector<Act> acts;
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

namespace {

lks_status fail(lks_ctx* c, lks_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, LKS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

// Host-side fault injection (lks_inject_alloc_failure): a countdown of device allocations; the
// allocation that brings it to zero reports failure without calling the allocator.
std::atomic<int> g_fail_alloc{0};

cudaError_t dev_alloc(void** p, size_t bytes) {
    int k = g_fail_alloc.load();
    while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

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

// True when a 3D configuration rotates about an axis other than z.
bool general_axis(const lks_config* cfg) {
    const double* a = cfg->rot_axis;
    return cfg->dim == 3 && !(a[0] == 0.0 && a[1] == 0.0 && (a[2] == 0.0 || a[2] == 1.0));
}

bool validate(const lks_config* cfg, std::string& why) {
    if (!cfg) {
        why = "null config";
        return false;
    }
    if (cfg->dim != 2 && cfg->dim != 3) {
        why = "dim must be 2 or 3";
        return false;
    }
    const int n[3] = {cfg->nx, cfg->ny, cfg->dim == 3 ? cfg->nz : 1};
    for (int a = 0; a < cfg->dim; ++a)
        if (n[a] < 3) {
            why = "every active axis needs at least 3 nodes";
            return false;
        }
    if ((double)n[0] * n[1] * n[2] >= 2147483648.0) {
        why = "grids of 2^31 nodes or more are not supported";
        return false;
    }
    if (cfg->dim == 2 && cfg->nz != 1) {
        why = "nz must be 1 in 2D";
        return false;
    }
    if (cfg->lx < 0 || (cfg->lx > 0 && (cfg->ly < 1 || cfg->lz < 1))) {
        why = "bad design grid size";
        return false;
    }
    if (cfg->dim == 2 && cfg->lx > 0 && cfg->lz != 1) {
        why = "lz must be 1 in 2D";
        return false;
    }
    if (cfg->precision != LKS_FP32 && cfg->precision != LKS_FP64) {
        why = "precision must be LKS_FP32 or LKS_FP64";
        return false;
    }
    if (cfg->max_steps < 1) {
        why = "max_steps must be >= 1";
        return false;
    }
    if (!(cfg->A < 0.75) || !(cfg->A > -10.0)) {
        why = "A must give a positive viscosity (A < 0.75)";
        return false;
    }
    for (int a = 0; a < cfg->dim; ++a) {
        const bool p0 = cfg->bc[2 * a] == LKS_BC_PERIODIC, p1 = cfg->bc[2 * a + 1] == LKS_BC_PERIODIC;
        if (p0 != p1) {
            why = "PERIODIC must be set on both faces of an axis";
            return false;
        }
        for (int sd = 0; sd < 2; ++sd)
            if (cfg->bc[2 * a + sd] < 0 || cfg->bc[2 * a + sd] > 3) {
                why = "unknown boundary type";
                return false;
            }
    }
    if (cfg->win_begin < 1 || cfg->win_end < cfg->win_begin) {
        why = "objective window must satisfy 1 <= win_begin <= win_end";
        return false;
    }
    if (general_axis(cfg)) {
        const double* a = cfg->rot_axis;
        const double n2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
        if (!(std::fabs(n2 - 1.0) < 1e-9)) {
            why = "rot_axis must be a unit vector";
            return false;
        }
    }
    if (cfg->obj_kind != LKS_OBJ_PRESSURE && cfg->obj_kind != LKS_OBJ_VELOCITY) {
        why = "unknown objective kind";
        return false;
    }
    return true;
}

// Node indices of the objective's target region in ascending order (box, then cylinder).
std::vector<int> target_list(const lks_config* c) {
    std::vector<int> out;
    const int* b = c->obj_box;
    const int nz = c->dim == 3 ? c->nz : 1;
    const int z0 = c->dim == 3 ? b[4] : 0, z1 = c->dim == 3 ? b[5] : 0;
    for (int z = std::max(0, z0); z <= std::min(z1, nz - 1); ++z)
        for (int y = std::max(0, b[2]); y <= std::min(b[3], c->ny - 1); ++y)
            for (int x = std::max(0, b[0]); x <= std::min(b[1], c->nx - 1); ++x) {
                if (c->obj_cyl_r > 0.0) {
                    const double dx = x - c->obj_cyl_c[0], dy = y - c->obj_cyl_c[1];
                    if (dx * dx + dy * dy > c->obj_cyl_r * c->obj_cyl_r) continue;
                }
                out.push_back((int)(((long long)z * c->ny + y) * c->nx + x));
            }
    return out;
}

// Count target nodes on the host (the same membership test the kernels use).
double count_target(const lks_config* c) {
    const int* b = c->obj_box;
    double cnt = 0;
    const int z0 = c->dim == 3 ? b[4] : 0, z1 = c->dim == 3 ? b[5] : 0;
    for (int z = std::max(0, z0); z <= std::min(z1, (c->dim == 3 ? c->nz : 1) - 1); ++z)
        for (int y = std::max(0, b[2]); y <= std::min(b[3], c->ny - 1); ++y)
            for (int x = std::max(0, b[0]); x <= std::min(b[1], c->nx - 1); ++x) {
                if (c->obj_cyl_r > 0.0) {
                    const double dx = x - c->obj_cyl_c[0], dy = y - c->obj_cyl_c[1];
                    if (dx * dx + dy * dy > c->obj_cyl_r * c->obj_cyl_r) continue;
                }
                cnt += 1;
            }
    return cnt;
}

struct Layout {
    size_t off[96];
    size_t total;
    int pool_slots;
    size_t snap;
};

enum {
    L_S0, L_S1, L_SINIT, L_L0, L_L1, L_F, L_MU, L_PHI, L_KUS, L_E, L_GAMMA, L_KREF, L_KPRIME,
    L_GACC, L_JSTEP, L_CBASE, L_CFRAC, L_ZTI, L_ZTW, L_TCNT, L_TIDX, L_TW, L_CM, L_DZB, L_DZF,
    L_FLAGS, L_KREFT, L_K2, L_FACE, L_TGT, L_U3, L_MOTION, L_BUFS, L_INST, L_PRE, L_GBAR,
    L_HP, L_FWS, L_GOUT, L_GTMP, L_SCAL, L_CSC, L_KS, L_SEND, L_LEND, L_GBASE, L_GFRAC,
    L_GCNT, L_GIDX,
    // the second transfer buffer set (3D): same sizes as L_KUS, L_K2, L_CBASE, ...
    L_KUS2, L_K22, L_CBASE2, L_CFRAC2, L_CSC2, L_ZTI2, L_ZTW2, L_TCNT2, L_TIDX2, L_TW2, L_CM2,
    L_DZB2, L_DZF2, L_GBASE2, L_GFRAC2, L_GCNT2, L_GIDX2, L_E2,
    L_POOL,
    L_COUNT
};
static_assert(L_COUNT <= 96, "Layout::off holds 96 regions");

Layout make_layout(const lks_config* cfg) {
    Layout L;
    const size_t T = cfg->precision == LKS_FP64 ? 8 : 4;
    const int dim = cfg->dim;
    const long long nodes = (long long)cfg->nx * cfg->ny * (dim == 3 ? cfg->nz : 1);
    const int Q = dim == 3 ? 15 : 9;
    const long long nd = cfg->lx > 0 ? (long long)cfg->lx * cfg->ly * (dim == 3 ? cfg->lz : 1) : 0;
    const long long ncol = cfg->lx > 0 ? (long long)cfg->lx * cfg->ly : 0;
    const long long cols = (long long)cfg->nx * cfg->ny;   // box columns, worst case
    const int nzb = dim == 3 ? cfg->nz : 1;
    const size_t state = align256((size_t)nodes * 4 * T);
    size_t sz[L_COUNT];
    sz[L_S0] = sz[L_S1] = sz[L_SINIT] = sz[L_L0] = sz[L_L1] = state;
    sz[L_F] = (size_t)Q * nodes * T;
    sz[L_MU] = state;
    sz[L_PHI] = (size_t)6 * nodes * T;
    sz[L_KUS] = nd ? state : 0;
    sz[L_E] = nd ? (size_t)nodes * T : 0;
    sz[L_GAMMA] = (size_t)std::max(nd, 1LL) * 8;
    sz[L_KREF] = sz[L_KPRIME] = (size_t)std::max(nd, 1LL) * T;
    sz[L_GACC] = (size_t)std::max(nd, 1LL) * 8;
    sz[L_JSTEP] = (size_t)(cfg->max_steps + 2) * 8;
    sz[L_CBASE] = (size_t)std::max(ncol, 1LL) * 2 * 4;
    sz[L_CFRAC] = (size_t)std::max(ncol, 1LL) * 2 * T;
    sz[L_ZTI] = (size_t)nzb * 4 * 4;
    sz[L_ZTW] = (size_t)nzb * 4 * T;
    sz[L_TCNT] = nd ? (size_t)cols * 4 : 0;
    sz[L_TIDX] = nd ? (size_t)cols * kMaxTaps * 4 : 0;
    sz[L_TW] = nd ? (size_t)cols * kMaxTaps * T : 0;
    sz[L_CM] = nd ? (size_t)cols * 3 * T : 0;
    sz[L_DZB] = (size_t)std::max(cfg->lz, 1) * 4;
    sz[L_DZF] = (size_t)std::max(cfg->lz, 1) * T;
    // snapshot pool
    const long long N = cfg->max_steps;
    long long P;
    if (cfg->ckpt_bytes == 0) {
        const double full = (double)(N + 1) * (double)state;
        if (full <= 8.0 * (1ull << 30)) {
            P = N + 1;
        } else {
            const long long K = (long long)std::ceil(std::sqrt((double)N));
            const long long Mseg = (N + K - 1) / K;
            P = (K + 1) + (Mseg - 1);
        }
    } else {
        P = std::max(3LL, (long long)(cfg->ckpt_bytes / state));
        P = std::min(P, N + 1);
    }
    sz[L_FLAGS] = 64;
    sz[L_MOTION] = (size_t)(cfg->max_steps + 1) * sizeof(Motion);
    sz[L_BUFS] = (size_t)(BUF_POOL + P) * sizeof(void*);
    sz[L_INST] = sizeof(Inst);
    sz[L_PRE] = (size_t)U_COUNT * 2 * sizeof(int);
    sz[L_GBAR] = sz[L_HP] = sz[L_FWS] = sz[L_GOUT] = sz[L_GTMP] = (size_t)std::max(nd, 1LL) * 8;
    sz[L_SCAL] = 64;
    sz[L_CSC] = (size_t)std::max(ncol, 1LL) * 16;
    sz[L_KS] = (size_t)nodes * T;
    sz[L_SEND] = sz[L_LEND] = state;
    {   // general-axis transfer: per design node and per box cell (worst case: every node)
        const bool ga = general_axis(cfg) && nd > 0;
        sz[L_GBASE] = ga ? (size_t)nd * 16 : 0;
        sz[L_GFRAC] = ga ? (size_t)nd * 4 * T : 0;
        sz[L_GCNT] = ga ? (size_t)nodes * 4 : 0;
        sz[L_GIDX] = ga ? (size_t)nodes * kCellMax * 4 : 0;
    }
    sz[L_TGT] = (size_t)std::max(1.0, count_target(cfg)) * 4;
    sz[L_U3] = (cfg->flags & LKS_FLAG_PAPER_ALKS) ? state : 0;
    sz[L_KREFT] = (size_t)std::max(nd, 1LL) * T;
    sz[L_K2] = nd ? (size_t)cols * std::max(cfg->lz, 1) * T : 0;
    {
        const long long n0 = cfg->nx, n1 = cfg->ny, n2 = dim == 3 ? cfg->nz : 1;
        sz[L_FACE] = (size_t)6 * (n1 * n2 + n0 * n2 + n0 * n1) * 4;
    }
    {   // second transfer set for the prefetch of the next step's transfer (3D only)
        const bool two = dim == 3 && nd > 0;
        const int first[17] = {L_KUS, L_K2, L_CBASE, L_CFRAC, L_CSC, L_ZTI, L_ZTW, L_TCNT,
                               L_TIDX, L_TW, L_CM, L_DZB, L_DZF, L_GBASE, L_GFRAC, L_GCNT, L_GIDX};
        for (int i = 0; i < 17; ++i) sz[L_KUS2 + i] = two ? sz[first[i]] : 0;
        sz[L_E2] = two ? sz[L_E] : 0;
    }
    sz[L_POOL] = (size_t)P * state;
    size_t off = 0;
    for (int i = 0; i < L_COUNT; ++i) {
        L.off[i] = off;
        off += align256(sz[i]);
    }
    L.total = off;
    L.pool_slots = (int)P;
    L.snap = state;
    return L;
}

// Pick the tape length K and the number of checkpoint slots S for N steps and P pool slots.
void plan_tape(int N, int P, int& K, int& M, int& S) {
    if (P >= N + 1) {
        K = N;
        M = 1;
        S = 0;
        return;
    }
    K = (int)std::ceil(std::sqrt((double)N));
    if (K + 1 > P - 1) K = std::max(1, P / 2 - 1);
    M = (N + K - 1) / K;
    S = P - (K + 1);
    if (S < 0) S = 0;
}

template <class T>
V4<T>* st4(void* p) {
    return (V4<T>*)p;
}

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
        CU(launch_t_transfer2d(c->plan, 0, c->st));
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
                                           c->flags + 3, c->st);
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

// Table-path launch sequences of one forward / adjoint step at offset k from *nbase.
cudaError_t table_fwd_launches(const Group& G, int k, int src, int dst, bool with_obj,
                               lks_ctx* timed, int n, int& nl) {
    cudaError_t e;
    if ((e = launch_t_design_pos(*G.plan, k, G.st)) != cudaSuccess) return e;
    if ((e = launch_t_transfer2d(*G.plan, k, G.st)) != cudaSuccess) return e;
    const bool tm = timed && timing_begin(timed, n, 0);
    if ((e = launch_t_step2d(*G.plan, G.tile_fwd, src, dst, G.st)) != cudaSuccess) return e;
    if (tm) timing_end(timed, 0);
    nl += 3;
    if (with_obj) {
        if ((e = launch_t_objective(*G.plan, k, dst, G.st)) != cudaSuccess) return e;
        ++nl;
    }
    return cudaSuccess;
}

cudaError_t table_adj_launches(const Group& G, int k, int lam_in, int lam_out, int sn, int sp,
                               lks_ctx* timed, int n, int& nl) {
    cudaError_t e;
    if ((e = launch_t_design_pos(*G.plan, k, G.st)) != cudaSuccess) return e;
    if ((e = launch_t_transfer2d(*G.plan, k, G.st)) != cudaSuccess) return e;
    const bool tm = timed && timing_begin(timed, n, 1);
    if ((e = launch_t_bcT2d(*G.plan, k, lam_in, G.st)) != cudaSuccess) return e;
    if ((e = launch_t_adj2d(*G.plan, G.tile_adj, k, lam_in, lam_out, sn, sp, G.st)) !=
        cudaSuccess)
        return e;
    if (tm) timing_end(timed, 1);
    if ((e = launch_t_sens(*G.plan, G.st)) != cudaSuccess) return e;
    nl += 5;
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
            return table_fwd_launches(G, k, src, dst, obj,
                                      (direct && G.count == 1) ? c0 : nullptr, from_level + k, nl);
        };
        const auto key = std::make_tuple(tape_seg >= 0 ? 1 : 0, obj ? 1 : 0, len,
                                         tape_seg >= 0 ? toff : w0, G.tile_fwd, 0);
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
    auto fn = [&](int k, int& nl, bool direct) -> cudaError_t {
        const int kk = len - k + 1;                 // step n = a + kk, from b down to a + 1
        const int par = par0 ^ ((k - 1) & 1);
        return table_adj_launches(G, kk, BUF_LAM0 + par, BUF_LAM0 + 1 - par, BUF_POOL + kk,
                                  BUF_POOL + kk - 1, (direct && G.count == 1) ? c0 : nullptr,
                                  a + kk, nl);
    };
    const auto key = std::make_tuple(2, 0, len, par0, 0, G.tile_adj);
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
    I.ts = c->ts;
    I.motion = c->dmotion;
    I.bufs = c->dbufs;
    I.kref = (const float*)c->kref;
    I.kprime = (const float*)c->kprime;
    I.kus = (V4<float>*)c->kus;
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
    out[U_SHELL] = (2 * (g.n[0] + g.n[1]) + kUnitThreads - 1) / kUnitThreads;
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

}  // namespace

extern "C" {

size_t lks_workspace_bytes(const lks_config* cfg) {
    std::string why;
    if (!validate(cfg, why)) return 0;
    return make_layout(cfg).total;
}

lks_status lks_create(const lks_config* cfg, void* workspace, size_t ws_bytes, lks_ctx** out) {
    if (!out) return LKS_ERR_ARG;
    *out = nullptr;
    std::string why;
    if (!validate(cfg, why)) {
        fprintf(stderr, "lks_create: %s\n", why.c_str());
        return LKS_ERR_ARG;
    }
    const double cnt = count_target(cfg);
    if (cnt <= 0) {
        fprintf(stderr, "lks_create: objective region is empty\n");
        return LKS_ERR_ARG;
    }
    lks_ctx* c = new lks_ctx();
    c->cfg = *cfg;
    c->prec = cfg->precision;
    c->tsz = c->prec == LKS_FP64 ? 8 : 4;
    c->st = (cudaStream_t)cfg->stream;
    Geom& g = c->g;
    std::memset(&g, 0, sizeof(g));
    g.dim = cfg->dim;
    g.n[0] = cfg->nx;
    g.n[1] = cfg->ny;
    g.n[2] = cfg->dim == 3 ? cfg->nz : 1;
    for (int a = 0; a < 3; ++a) g.periodic[a] = (a >= cfg->dim) || cfg->bc[2 * a] == LKS_BC_PERIODIC;
    g.nodes = (long long)g.n[0] * g.n[1] * g.n[2];
    for (int f = 0; f < 6; ++f) {
        g.bc[f] = cfg->bc[f];
        for (int k = 0; k < 4; ++k) g.bcv[f][k] = cfg->bc_val[f][k];
    }
    g.rho0 = cfg->rho0;
    g.A = cfg->A;
    for (int a = 0; a < 3; ++a) g.body[a] = cfg->body_force[a];
    g.okind = cfg->obj_kind;
    for (int a = 0; a < 3; ++a) {  // clip the target box to the grid (2D: z = 0)
        g.obox[2 * a] = std::max(0, a < cfg->dim ? cfg->obj_box[2 * a] : 0);
        g.obox[2 * a + 1] = std::min(g.n[a] - 1, a < cfg->dim ? cfg->obj_box[2 * a + 1] : 0);
    }
    for (int a = 0; a < 3; ++a) g.odir[a] = cfg->obj_dir[a];
    g.ocyl_r = cfg->obj_cyl_r;
    g.ocyl_c[0] = cfg->obj_cyl_c[0];
    g.ocyl_c[1] = cfg->obj_cyl_c[1];
    g.ocount = cnt;
    g.boxN = 0;
    Design& d = c->d;
    d.L[0] = cfg->lx;
    d.L[1] = cfg->lx > 0 ? cfg->ly : 0;
    d.L[2] = cfg->lx > 0 ? (cfg->dim == 3 ? cfg->lz : 1) : 0;
    for (int a = 0; a < 3; ++a) {
        d.xiG[a] = cfg->xi_G[a];
        d.xiGf[a] = (float)cfg->xi_G[a];
    }
    d.nd = (long long)d.L[0] * d.L[1] * d.L[2];
    d.ncol = (long long)d.L[0] * d.L[1];

    const Layout L = make_layout(cfg);
    if (workspace) {
        if (ws_bytes < L.total || ((uintptr_t)workspace & 255)) {
            delete c;
            fprintf(stderr, "lks_create: workspace too small or misaligned\n");
            return LKS_ERR_NOMEM;
        }
        c->ws = (char*)workspace;
        c->own_ws = false;
    } else {
        if (dev_alloc((void**)&c->ws, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return LKS_ERR_NOMEM;
        }
        c->own_ws = true;
    }
    c->ws_bytes = L.total;
    char* w = c->ws;
    c->s[0] = w + L.off[L_S0];
    c->s[1] = w + L.off[L_S1];
    c->s0 = w + L.off[L_SINIT];
    c->lam[0] = w + L.off[L_L0];
    c->lam[1] = w + L.off[L_L1];
    c->F = w + L.off[L_F];
    c->mu = w + L.off[L_MU];
    c->phi = w + L.off[L_PHI];
    c->kus = w + L.off[L_KUS];
    c->e = w + L.off[L_E];
    c->gamma = (double*)(w + L.off[L_GAMMA]);
    c->kref = w + L.off[L_KREF];
    c->kprime = w + L.off[L_KPRIME];
    c->kref_t = w + L.off[L_KREFT];
    c->k2 = w + L.off[L_K2];
    c->face = (float*)(w + L.off[L_FACE]);
    c->u3 = (cfg->flags & LKS_FLAG_PAPER_ALKS) ? (void*)(w + L.off[L_U3]) : nullptr;
    c->gacc = (double*)(w + L.off[L_GACC]);
    c->jstep = (double*)(w + L.off[L_JSTEP]);
    c->ts.col_base = (int*)(w + L.off[L_CBASE]);
    c->ts.col_frac = w + L.off[L_CFRAC];
    c->ts.col_sc = (float4*)(w + L.off[L_CSC]);
    c->ts.zt_idx = (int*)(w + L.off[L_ZTI]);
    c->ts.zt_w = w + L.off[L_ZTW];
    c->ts.tap_cnt = (int*)(w + L.off[L_TCNT]);
    c->ts.tap_idx = (int*)(w + L.off[L_TIDX]);
    c->ts.tap_w = w + L.off[L_TW];
    c->ts.col_m = w + L.off[L_CM];
    c->ts.dz_base = (int*)(w + L.off[L_DZB]);
    c->ts.dz_frac = w + L.off[L_DZF];
    c->flags = (int*)(w + L.off[L_FLAGS]);
    {
        const std::vector<int> tl = target_list(cfg);
        int* dt = (int*)(w + L.off[L_TGT]);
        if (cudaMemcpy(dt, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            cudaGetLastError();
            if (c->own_ws) cudaFree(c->ws);
            delete c;
            return LKS_ERR_CUDA;
        }
        c->g.otarget = dt;
    }
    c->ts.err = c->flags + 1;
    c->fused3d = (c->prec == LKS_FP32) &&
                 !(cfg->flags & (LKS_FLAG_PLAIN_KERNELS | LKS_FLAG_PAPER_ALKS)) &&
                 fused3d_eligible(g);
    c->pool = w + L.off[L_POOL];
    c->pool_slots = L.pool_slots;
    c->snap_bytes = L.snap;
    c->fused2d = (c->prec == LKS_FP32) && g.dim == 2 &&
                 !(cfg->flags & (LKS_FLAG_PLAIN_KERNELS | LKS_FLAG_PAPER_ALKS));
    c->dmotion = (Motion*)(w + L.off[L_MOTION]);
    c->dbufs = (void**)(w + L.off[L_BUFS]);
    c->dinst = (Inst*)(w + L.off[L_INST]);
    c->dpre = (int*)(w + L.off[L_PRE]);
    c->gbar = (double*)(w + L.off[L_GBAR]);
    c->hp = (double*)(w + L.off[L_HP]);
    c->fws = (double*)(w + L.off[L_FWS]);
    c->gout = (double*)(w + L.off[L_GOUT]);
    c->gtmp = (double*)(w + L.off[L_GTMP]);
    c->scal = (double*)(w + L.off[L_SCAL]);
    c->ks = w + L.off[L_KS];
    c->gaxis = general_axis(cfg) && c->d.nd > 0;
    if (general_axis(cfg))
        for (int a = 0; a < 3; ++a) c->axis[a] = cfg->rot_axis[a];
    c->as.base = (int4*)(w + L.off[L_GBASE]);
    c->as.frac = w + L.off[L_GFRAC];
    c->as.cnt = (int*)(w + L.off[L_GCNT]);
    c->as.idx = (int*)(w + L.off[L_GIDX]);
    {   // the two transfer sets
        lks_ctx::XSlot& a = c->xs[0];
        a.kus = c->kus;
        a.k2 = c->k2;
        a.ts = c->ts;
        a.as = c->as;
        lks_ctx::XSlot& b = c->xs[1];
        b.kus = w + L.off[L_KUS2];
        b.k2 = w + L.off[L_K22];
        b.ts = c->ts;
        b.ts.col_base = (int*)(w + L.off[L_CBASE2]);
        b.ts.col_frac = w + L.off[L_CFRAC2];
        b.ts.col_sc = (float4*)(w + L.off[L_CSC2]);
        b.ts.zt_idx = (int*)(w + L.off[L_ZTI2]);
        b.ts.zt_w = w + L.off[L_ZTW2];
        b.ts.tap_cnt = (int*)(w + L.off[L_TCNT2]);
        b.ts.tap_idx = (int*)(w + L.off[L_TIDX2]);
        b.ts.tap_w = w + L.off[L_TW2];
        b.ts.col_m = w + L.off[L_CM2];
        b.ts.dz_base = (int*)(w + L.off[L_DZB2]);
        b.ts.dz_frac = w + L.off[L_DZF2];
        b.as.base = (int4*)(w + L.off[L_GBASE2]);
        b.as.frac = w + L.off[L_GFRAC2];
        b.as.cnt = (int*)(w + L.off[L_GCNT2]);
        b.as.idx = (int*)(w + L.off[L_GIDX2]);
        c->pf_on = cfg->dim == 3 && c->d.nd > 0;
        c->ebuf[0] = c->e;
        c->ebuf[1] = w + L.off[L_E2];
    }
    c->s_end = w + L.off[L_SEND];
    c->l_end = w + L.off[L_LEND];
    c->nbase = c->flags + 8;
    c->hbufs.assign(BUF_POOL + c->pool_slots, nullptr);
    c->hbufs[BUF_S0] = c->s[0];
    c->hbufs[BUF_S1] = c->s[1];
    c->hbufs[BUF_INIT] = c->s0;
    c->hbufs[BUF_LAM0] = c->lam[0];
    c->hbufs[BUF_LAM1] = c->lam[1];
    for (int k = 0; k < c->pool_slots; ++k) c->hbufs[BUF_POOL + k] = slot_ptr(c, k);
    lks_status s = LKS_OK;
    if (cudaMemcpy(c->dbufs, c->hbufs.data(), c->hbufs.size() * sizeof(void*),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        s = LKS_ERR_CUDA;
    if (s == LKS_OK && cudaMemsetAsync(c->flags, 0, 64, c->st) != cudaSuccess) s = LKS_ERR_CUDA;
    if (s == LKS_OK) s = c->prec == LKS_FP64 ? reset_initial<double>(c) : reset_initial<float>(c);
    if (s != LKS_OK) {
        lks_destroy(c);
        return s;
    }
    *out = c;
    return LKS_OK;
}

lks_status lks_set_design(lks_ctx* c, const double* gamma, int on_device) {
    if (!c) return LKS_ERR_ARG;
    c->fwd_valid = false;
    if (c->d.nd == 0) {
        c->have_design = true;
        return LKS_OK;
    }
    if (!gamma) return fail(c, LKS_ERR_ARG, "gamma is NULL");
    if (!on_device) {
        for (long long k = 0; k < c->d.nd; ++k)
            if (!(gamma[k] >= 0.0 && gamma[k] <= 1.0))
                return fail(c, LKS_ERR_ARG, "gamma[%lld] = %g outside [0,1]", k, gamma[k]);
    }
    CU(cudaMemcpyAsync(c->gamma, gamma, (size_t)c->d.nd * 8,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
    CU(cudaMemsetAsync(c->flags, 0, 4, c->st));
    lks_status s = design_prep(c);
    if (s != LKS_OK) return s;
    if (on_device) {
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, c->flags, 4, cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
        if (bad) return fail(c, LKS_ERR_ARG, "gamma outside [0,1]");
    }
    c->have_design = true;
    return LKS_OK;
}

lks_status lks_set_filter(lks_ctx* c, double R, double beta, double eta) {
    if (!c) return LKS_ERR_ARG;
    if (!(R >= 0.0) || (R > 0.0 && (!(beta > 0.0) || !(eta > 0.0 && eta < 1.0))))
        return fail(c, LKS_ERR_ARG, "filter needs R >= 0, and beta > 0, 0 < eta < 1 when R > 0");
    c->fR = R;
    c->fbeta = beta;
    c->feta = eta;
    c->fwd_valid = false;
    if (c->have_design && c->d.nd > 0) {
        lks_status s = design_prep(c);
        if (s != LKS_OK) return s;
    }
    return LKS_OK;
}

lks_status lks_volume(lks_ctx* c, double vmax, double* G_out, double* dGdgamma, int on_device) {
    if (!c || !G_out) return LKS_ERR_ARG;
    if (!(vmax > 0.0)) return fail(c, LKS_ERR_ARG, "vmax must be positive");
    if (!c->have_design || c->d.nd == 0) return fail(c, LKS_ERR_ORDER, "no design set");
    const long long nd = c->d.nd;
    launch_design_sum(nd, c->fR > 0.0 ? c->gbar : c->gamma, c->scal, c->st);
    LAUNCHED();
    double sum = 0.0;
    CU(cudaMemcpyAsync(&sum, c->scal, 8, cudaMemcpyDeviceToHost, c->st));
    const double dv = 1.0 / (vmax * (double)nd);
    if (dGdgamma) {
        launch_fill_f64(c->gtmp, nd, dv, c->st);
        LAUNCHED();
        const double* src = c->gtmp;
        if (c->fR > 0.0) {
            launch_filter_T(c->d, c->fR, c->gtmp, c->hp, c->fws, c->gout, c->st);
            LAUNCHED();
            src = c->gout;
        }
        CU(cudaMemcpyAsync(dGdgamma, src, (size_t)nd * 8,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
    }
    CU(cudaStreamSynchronize(c->st));
    *G_out = sum * dv - 1.0;
    return LKS_OK;
}

lks_status lks_set_static(lks_ctx* c, const double* kappa_s) {
    if (!c) return LKS_ERR_ARG;
    c->fwd_valid = false;
    if (!kappa_s) {
        c->g.ks = nullptr;
    } else {
        const size_t n = (size_t)c->g.nodes;
        for (size_t m = 0; m < n; ++m)
            if (!(kappa_s[m] >= 0.0) || !std::isfinite(kappa_s[m]))
                return fail(c, LKS_ERR_ARG, "kappa_s[%zu] = %g is not a finite value >= 0", m,
                            kappa_s[m]);
        if (c->prec == LKS_FP64) {
            CU(cudaMemcpy(c->ks, kappa_s, n * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> f(kappa_s, kappa_s + n);
            CU(cudaMemcpy(c->ks, f.data(), n * 4, cudaMemcpyHostToDevice));
        }
        c->g.ks = c->ks;
    }
    if (c->fused2d && c->have_motion) {
        std::vector<lks_ctx*> one(1, c);
        CU(build_plan(one, c->dinst, c->dpre, c->nbase, c->st, c->plan));
    }
    ++c->geo_gen;
    return LKS_OK;
}

lks_status lks_warm_start(lks_ctx* c) {
    if (!c) return LKS_ERR_ARG;
    if (!c->have_end) return fail(c, LKS_ERR_ORDER, "warm start needs a completed forward run");
    CU(cudaMemcpyAsync(c->s0, c->s_end, c->snap_bytes, cudaMemcpyDeviceToDevice, c->st));
    c->fwd_valid = false;
    return LKS_OK;
}

lks_status lks_set_adjoint_start(lks_ctx* c, int warm) {
    if (!c) return LKS_ERR_ARG;
    c->adj_warm = warm != 0;
    return LKS_OK;
}

lks_status lks_get_adjoint_state(const lks_ctx* cc, double* out) {
    lks_ctx* c = const_cast<lks_ctx*>(cc);
    if (!c || !out) return LKS_ERR_ARG;
    if (!c->have_lend) return fail(c, LKS_ERR_ORDER, "no adjoint run yet");
    double* tmp = nullptr;
    const size_t bytes = (size_t)c->g.nodes * 4 * 8;
    ALLOC(&tmp, bytes);
    if (c->prec == LKS_FP64)
        launch_state_to_f64<double>(c->g, (const V4<double>*)c->l_end, tmp, c->st, false);
    else
        launch_state_to_f64<float>(c->g, (const V4<float>*)c->l_end, tmp, c->st, false);
    cudaError_t e1 = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, c->st);
    cudaError_t e2 = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(c, LKS_ERR_CUDA, "get_adjoint_state: %s",
                    cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return LKS_OK;
}

lks_status lks_set_motion(lks_ctx* c, const lks_motion* m) {
    if (!c || !m || !m->rows) return c ? fail(c, LKS_ERR_ARG, "motion is NULL") : LKS_ERR_ARG;
    c->fwd_valid = false;
    if (m->n_rows < c->cfg.max_steps + 1)
        return fail(c, LKS_ERR_ARG, "motion has %d rows, need max_steps + 1 = %d", m->n_rows,
                    c->cfg.max_steps + 1);
    c->motion.assign(m->rows, m->rows + 8 * (size_t)m->n_rows);
    Geom& g = c->g;
    if (c->d.nd == 0) {
        g.boxN = 0;
        return finish_motion(c);
    }
    // union over steps of the analysis nodes strictly within two cells of a moved design node
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    const double cx[2] = {0.0, (double)(c->d.L[0] - 1)}, cy[2] = {0.0, (double)(c->d.L[1] - 1)};
    for (int n = 1; n <= c->cfg.max_steps; ++n) {
        const Motion mo = motion_row(c, n);
        if (c->gaxis) {   // images of the design box's eight corners bound its image
            for (int cidx = 0; cidx < 8; ++cidx) {
                double dv[3];
                for (int a = 0; a < 3; ++a)
                    dv[a] = ((cidx >> a) & 1 ? (double)(c->d.L[a] - 1) : 0.0) - c->d.xiG[a];
                for (int a = 0; a < 3; ++a) {
                    const double xr = mo.R[3 * a] * dv[0] + mo.R[3 * a + 1] * dv[1] +
                                      mo.R[3 * a + 2] * dv[2] + mo.xG[a];
                    lo[a] = std::min(lo[a], xr);
                    hi[a] = std::max(hi[a], xr);
                }
            }
            continue;
        }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const double dx = cx[a] - c->d.xiG[0], dy = cy[b] - c->d.xiG[1];
                const double xr = mo.c * dx - mo.s * dy + mo.xG[0];
                const double yr = mo.s * dx + mo.c * dy + mo.xG[1];
                lo[0] = std::min(lo[0], xr);
                hi[0] = std::max(hi[0], xr);
                lo[1] = std::min(lo[1], yr);
                hi[1] = std::max(hi[1], yr);
            }
        if (g.dim == 3) {
            const double z0 = 0.0 - c->d.xiG[2] + mo.xG[2];
            const double z1 = (double)(c->d.L[2] - 1) - c->d.xiG[2] + mo.xG[2];
            lo[2] = std::min(lo[2], z0);
            hi[2] = std::max(hi[2], z1);
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (a >= g.dim) {
            g.blo[a] = 0;
            g.bn[a] = 1;
            continue;
        }
        const int l = (int)std::floor(lo[a] - 2.0) + 1;
        const int h = (int)std::ceil(hi[a] + 2.0) - 1;
        const int minok = g.periodic[a] ? 0 : 1;
        const int maxok = g.periodic[a] ? g.n[a] - 1 : g.n[a] - 2;
        if (l < minok || h > maxok)
            return fail(c, LKS_ERR_ARG,
                        "design footprint [%d,%d] on axis %d leaves the interior [%d,%d]", l, h, a,
                        minok, maxok);
        g.blo[a] = l;
        g.bn[a] = h - l + 1;
    }
    g.boxN = (long long)g.bn[0] * g.bn[1] * g.bn[2];
    return finish_motion(c);
}

lks_status lks_set_initial_state(lks_ctx* c, const double* state) {
    if (!c) return LKS_ERR_ARG;
    c->fwd_valid = false;
    if (!state) return c->prec == LKS_FP64 ? reset_initial<double>(c) : reset_initial<float>(c);
    double* tmp = nullptr;
    const size_t bytes = (size_t)c->g.nodes * 4 * 8;
    ALLOC(&tmp, bytes);
    cudaError_t e1 = cudaMemcpyAsync(tmp, state, bytes, cudaMemcpyHostToDevice, c->st);
    if (c->prec == LKS_FP64) launch_state_from_f64<double>(c->g, tmp, st4<double>(c->s0), c->st);
    else launch_state_from_f64<float>(c->g, tmp, st4<float>(c->s0), c->st);
    cudaError_t e2 = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(c, LKS_ERR_CUDA, "set_initial_state: %s",
                    cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return LKS_OK;
}

lks_status lks_forward(lks_ctx* c, int n_steps, double* J_out) {
    if (!c) return LKS_ERR_ARG;
    if (!c->have_design || !c->have_motion)
        return fail(c, LKS_ERR_ORDER, "set_design and set_motion must precede forward");
    if (n_steps < 1 || n_steps > c->cfg.max_steps)
        return fail(c, LKS_ERR_ARG, "n_steps must be in [1, max_steps]");
    c->fwd_valid = false;
    lks_status s = run_fork(c);
    if (s != LKS_OK) return run_join(c, s);
    Group G = self_group(c);
    s = c->prec == LKS_FP64 ? do_forward<double>(G, n_steps) : do_forward<float>(G, n_steps);
    c->stats[4] += G.launches;
    s = run_join(c, s);
    if (s != LKS_OK) return s;
    if (J_out) *J_out = c->J;
    return LKS_OK;
}

lks_status lks_adjoint(lks_ctx* c, double* dJdgamma, int on_device) {
    if (!c) return LKS_ERR_ARG;
    if (!c->fwd_valid) return fail(c, LKS_ERR_ORDER, "adjoint needs a preceding forward run");
    lks_status s = run_fork(c);
    if (s != LKS_OK) return run_join(c, s);
    Group G = self_group(c);
    s = c->prec == LKS_FP64 ? do_adjoint<double>(G) : do_adjoint<float>(G);
    c->stats[4] += G.launches;
    s = run_join(c, s);
    if (s != LKS_OK) return s;
    if (c->d.nd > 0 && dJdgamma) {
        CU(cudaMemcpyAsync(dJdgamma, design_gradient(c, c->st), (size_t)c->d.nd * 8,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
    }
    return LKS_OK;
}

lks_status lks_get_state(const lks_ctx* cc, double* out) {
    lks_ctx* c = const_cast<lks_ctx*>(cc);
    if (!c || !out) return LKS_ERR_ARG;
    double* tmp = nullptr;
    const size_t bytes = (size_t)c->g.nodes * 4 * 8;
    ALLOC(&tmp, bytes);
    const void* src = c->last ? c->last : c->s0;
    if (c->prec == LKS_FP64)
        launch_state_to_f64<double>(c->g, (const V4<double>*)src, tmp, c->st);
    else
        launch_state_to_f64<float>(c->g, (const V4<float>*)src, tmp, c->st);
    cudaError_t e1 = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, c->st);
    cudaError_t e2 = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
        return fail(c, LKS_ERR_CUDA, "get_state: %s",
                    cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return LKS_OK;
}

lks_status lks_transfer(lks_ctx* c, int step, double* kappa_out, double* us_out) {
    if (!c || !kappa_out || !us_out) return LKS_ERR_ARG;
    if (!c->have_design || !c->have_motion) return fail(c, LKS_ERR_ORDER, "design/motion unset");
    if (step < 0 || (size_t)step >= c->motion.size() / 8) return fail(c, LKS_ERR_ARG, "bad step");
    const size_t nodes = (size_t)c->g.nodes;
    if (c->d.nd == 0 || c->g.boxN == 0) {
        std::fill(kappa_out, kappa_out + nodes, 0.0);
        std::fill(us_out, us_out + 3 * nodes, 0.0);
        return LKS_OK;
    }
    {   // a fresh transfer into the current set, with nothing left in flight afterwards
        lks_status sj = transfer_join(c);
        if (sj != LKS_OK) return sj;
    }
    lks_status s = c->prec == LKS_FP64 ? transfer_at<double>(c, step) : transfer_at<float>(c, step);
    if (s == LKS_OK) s = transfer_join(c);
    if (s != LKS_OK) return s;
    double* tmp = nullptr;
    ALLOC(&tmp, nodes * 4 * 8);
    if (c->prec == LKS_FP64)
        launch_box_to_grid<double>(c->g, (const V4<double>*)c->kus, tmp, tmp + nodes, c->st);
    else
        launch_box_to_grid<float>(c->g, (const V4<float>*)c->kus, tmp, tmp + nodes, c->st);
    cudaError_t e1 = cudaMemcpyAsync(kappa_out, tmp, nodes * 8, cudaMemcpyDeviceToHost, c->st);
    cudaError_t e2 = cudaMemcpyAsync(us_out, tmp + nodes, 3 * nodes * 8, cudaMemcpyDeviceToHost, c->st);
    cudaError_t e3 = cudaStreamSynchronize(c->st);
    cudaFree(tmp);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
        return fail(c, LKS_ERR_CUDA, "transfer copy failed");
    return LKS_OK;
}

int lks_uses_fused(const lks_ctx* c) {
    return !c ? 0 : ((c->fused3d && !c->g.ks) ? 1 : (c->fused2d ? 2 : 0));
}

lks_status lks_step_variant(lks_ctx* c, int request, int* chosen) {
    if (!c || request < -2 || request >= kStep3dVariants)
        return c ? fail(c, LKS_ERR_ARG, "step variant must be in [-2, %d]", kStep3dVariants - 1)
                 : LKS_ERR_ARG;
    if (request >= -1) {
        c->step3d_req = request;
        c->step3d_var = -1;
    }
    if (chosen) *chosen = c->step3d_var;
    return LKS_OK;
}

lks_status lks_get_stats(const lks_ctx* c, long long* st5) {
    if (!c || !st5) return LKS_ERR_ARG;
    for (int i = 0; i < 5; ++i) st5[i] = c->stats[i];
    return LKS_OK;
}

int lks_checkpoint_schedule(int n_segments, int free_slots, int* triples, int cap) {
    if (n_segments < 1 || free_slots < 0 || (!triples && cap > 0)) return -1;
    std::vector<Act> acts;
    gen_schedule(0, n_segments, free_slots, acts);
    const int n = (int)std::min<size_t>(acts.size(), (size_t)std::max(cap, 0));
    for (int i = 0; i < n; ++i) {
        triples[3 * i] = acts[i].kind;
        triples[3 * i + 1] = acts[i].a;
        triples[3 * i + 2] = acts[i].b;
    }
    return (int)acts.size();
}

lks_status lks_set_timing(lks_ctx* c, int stride) {
    if (!c || stride < 0) return LKS_ERR_ARG;
    c->timing_stride = stride;
    c->tused[0] = c->tused[1] = 0;
    return LKS_OK;
}

lks_status lks_read_timing(lks_ctx* c, double* out4) {
    if (!c || !out4) return LKS_ERR_ARG;
    CU(cudaStreamSynchronize(c->st));
    for (int w = 0; w < 2; ++w) {
        double tot = 0.0;
        for (size_t i = 0; i + 1 < c->tused[w]; i += 2) {
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, c->tev[w][i], c->tev[w][i + 1]));
            tot += ms;
        }
        out4[2 * w] = tot;
        out4[2 * w + 1] = (double)(c->tused[w] / 2);
        c->tused[w] = 0;
    }
    return LKS_OK;
}

const char* lks_last_error(const lks_ctx* c) { return c ? c->err.c_str() : "null context"; }

int lks_inject_alloc_failure(int nth) { return g_fail_alloc.exchange(nth > 0 ? nth : 0); }

void lks_destroy(lks_ctx* c) {
    if (!c) return;
    for (int w = 0; w < 2; ++w)
        for (cudaEvent_t e : c->tev[w]) cudaEventDestroy(e);
    if (c->run_st) {
        cudaStreamSynchronize(c->run_st);
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->run_st);
        cudaStreamDestroy(c->side);
        for (cudaEvent_t e : {c->ev_main, c->ev_pf, c->ev_join, c->ev_adj, c->ev_sens[0],
                              c->ev_sens[1], c->ev_fork, c->ev_back})
            cudaEventDestroy(e);
    }
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
}

}  // extern "C"

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
            BCU(launch_t_transfer2d(b->plan, 1, b->st));
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
                    return w == 0 ? launch_t_step2d(b->plan, k, BUF_INIT, BUF_S1, b->st)
                                  : launch_t_adj2d(b->plan, k, 1, BUF_LAM0, BUF_LAM1, BUF_INIT,
                                                   BUF_INIT, b->st);
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
