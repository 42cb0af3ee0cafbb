// Host engine behind the C ABI of include/lks.h: validates the problem, carves the device
// workspace, runs Algorithm 1 (forward with the objective of Sec. 2.5) and the reverse adjoint
// sweep (Algorithm 2 structure, exact discrete adjoint) under a binomial checkpoint schedule
// over tape segments, so that the stored history fits the given device memory.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lks.h"
#include "lks_internal.h"

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
    void* lam[2];
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

#define LAUNCHED()                                                                        \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, LKS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e_));    \
        ++c->stats[4];                                                                    \
    } while (0)

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
    size_t off[32];
    size_t total;
    int pool_slots;
    size_t snap;
};

enum {
    L_S0, L_S1, L_SINIT, L_L0, L_L1, L_F, L_MU, L_PHI, L_KUS, L_E, L_GAMMA, L_KREF, L_KPRIME,
    L_GACC, L_JSTEP, L_CBASE, L_CFRAC, L_ZTI, L_ZTW, L_TCNT, L_TIDX, L_TW, L_CM, L_DZB, L_DZF,
    L_FLAGS, L_KREFT, L_K2, L_FACE, L_TGT, L_U3, L_POOL, L_COUNT
};

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
    sz[L_FLAGS] = 64;
    sz[L_TGT] = (size_t)std::max(1.0, count_target(cfg)) * 4;
    sz[L_U3] = (cfg->flags & LKS_FLAG_PAPER_ALKS) ? state : 0;
    sz[L_KREFT] = (size_t)std::max(nd, 1LL) * T;
    sz[L_K2] = nd ? (size_t)cols * std::max(cfg->lz, 1) * T : 0;
    {
        const long long n0 = cfg->nx, n1 = cfg->ny, n2 = dim == 3 ? cfg->nz : 1;
        sz[L_FACE] = (size_t)6 * (n1 * n2 + n0 * n2 + n0 * n1) * 4;
    }
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
    }
    return m;
}

template <class T>
lks_status transfer_at(lks_ctx* c, int n) {
    if (c->d.nd == 0 || c->g.boxN == 0) return LKS_OK;
    const Motion m = motion_row(c, n);
    launch_design_pos<T>(c->d, c->g, m, c->ts, c->st);
    LAUNCHED();
    launch_transfer<T>(c->d, c->g, m, c->ts, (const T*)c->kref_t, (T*)c->k2, st4<T>(c->kus),
                       c->st);
    LAUNCHED();
    return LKS_OK;
}

// One forward step n: s[src] -> s[dst].
template <class T>
lks_status forward_step(lks_ctx* c, int n, const void* src, void* dst) {
    lks_status s = transfer_at<T>(c, n);
    if (s != LKS_OK) return s;
    const bool tm = timing_begin(c, n, 0);
    if (sizeof(T) == 4 && c->fused3d) {
        cudaError_t e = launch_fused_step3d(c->g, (const V4<float>*)src, (const V4<float>*)c->kus,
                                            (V4<float>*)dst, c->flags + 3, c->st);
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

// Tape slots are the first K+1 of the pool: slot t holds level seg*K + t.
int tape_slot(const lks_ctx* c, int t) { return t; }

lks_status copy_state(lks_ctx* c, void* dst, const void* src) {
    CU(cudaMemcpyAsync(dst, src, (size_t)c->g.nodes * 4 * c->tsz, cudaMemcpyDeviceToDevice, c->st));
    return LKS_OK;
}

template <class T>
lks_status run_steps(lks_ctx* c, int from_level, int to_level, bool with_obj, int tape_seg) {
    // Advance from from_level to to_level.  Without a tape the two working buffers alternate;
    // with a tape (segment tape_seg, whose start level sits in tape slot 0) every level is
    // written straight into its own tape slot and the working buffer keeps from_level.
    for (int n = from_level + 1; n <= to_level; ++n) {
        const void* src;
        void* dst;
        if (tape_seg >= 0) {
            src = slot_ptr(c, tape_slot(c, n - 1 - tape_seg * c->K));
            dst = slot_ptr(c, tape_slot(c, n - tape_seg * c->K));
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
    c->work_level = (tape_seg >= 0) ? from_level : to_level;
    return LKS_OK;
}

int seg_start(const lks_ctx* c, int a) { return a * c->K; }
int seg_end(const lks_ctx* c, int a) { return std::min((a + 1) * c->K, c->n_fwd); }

template <class T>
lks_status restore_level(lks_ctx* c, int seg) {
    const int lev = seg_start(c, seg);
    if (c->work_level == lev) return LKS_OK;
    const void* src = (seg == 0) ? c->s0 : (const void*)slot_ptr(c, c->slot_of[seg]);
    if (seg != 0 && c->slot_of[seg] < 0) return fail(c, LKS_ERR_ARG, "schedule: no snapshot");
    lks_status s = copy_state(c, c->s[c->work], src);
    c->work_level = lev;
    return s;
}

template <class T>
lks_status exec_forward_action(lks_ctx* c, const Act& a, bool with_obj) {
    switch (a.kind) {
        case A_RESTORE:
            return restore_level<T>(c, a.a);
        case A_ADVANCE:
            return run_steps<T>(c, seg_start(c, a.a), seg_start(c, a.b), with_obj, -1);
        case A_STORE: {
            if (c->free_slots.empty()) return fail(c, LKS_ERR_NOMEM, "schedule: out of slots");
            int sl = c->free_slots.back();
            c->free_slots.pop_back();
            c->slot_of[a.a] = sl;
            return copy_state(c, slot_ptr(c, sl), c->s[c->work]);
        }
        case A_FREE:
            c->free_slots.push_back(c->slot_of[a.a]);
            c->slot_of[a.a] = -1;
            return LKS_OK;
        case A_TAPE: {
            lks_status s = copy_state(c, slot_ptr(c, tape_slot(c, 0)), c->s[c->work]);
            if (s != LKS_OK) return s;
            return run_steps<T>(c, seg_start(c, a.a), seg_end(c, a.a), with_obj, a.a);
        }
        default:
            return fail(c, LKS_ERR_ARG, "schedule: unexpected action");
    }
}

template <class T>
lks_status adjoint_step(lks_ctx* c, int n, const void* sn, const void* sp) {
    const double h = 1.0 / (double)(c->cfg.win_end - c->cfg.win_begin + 1);
    const double hn = (n >= c->cfg.win_begin && n <= c->cfg.win_end) ? h : 0.0;
    lks_status s = transfer_at<T>(c, n);
    if (s != LKS_OK) return s;
    V4<T>* lc = st4<T>(c->lam[0]);
    V4<T>* ln = st4<T>(c->lam[1]);
    const bool tm = timing_begin(c, n, 1);
    launch_adj_bcT<T>(c->g, lc, hn, c->st);
    LAUNCHED();
    if (sizeof(T) == 4 && c->fused3d) {
        cudaError_t e = launch_fused_adj3d(c->g, (const V4<float>*)lc, (V4<float>*)ln,
                                           (const V4<float>*)c->kus, (const V4<float>*)sn,
                                           (const V4<float>*)sp, (float*)c->e, c->face, hn,
                                           c->flags + 3, c->st);
        if (e != cudaSuccess) return fail(c, LKS_ERR_CUDA, "fused adjoint: %s", cudaGetErrorString(e));
        c->stats[4] += 2;
        if (tm) timing_end(c, 1);
        if (c->d.nd > 0 && c->g.boxN > 0) {
            launch_sens<T>(c->d, c->g, c->ts, (const T*)c->e, (const T*)c->kprime, c->gacc, c->st);
            LAUNCHED();
        }
        std::swap(c->lam[0], c->lam[1]);
        return LKS_OK;
    }
    launch_adj_mu<T>(c->g, lc, (const V4<T>*)c->kus, (const V4<T>*)sn, st4<T>(c->mu),
                     (T*)c->e, hn, c->st, (const V4<T>*)c->u3);
    LAUNCHED();
    launch_adj_moments<T>(c->g, st4<T>(c->mu), (const V4<T>*)sp, ln, (T*)c->phi, c->st,
                          (V4<T>*)c->u3);
    LAUNCHED();
    launch_adj_divT<T>(c->g, (const T*)c->phi, ln, c->st);
    LAUNCHED();
    if (tm) timing_end(c, 1);
    if (c->d.nd > 0 && c->g.boxN > 0) {
        launch_sens<T>(c->d, c->g, c->ts, (const T*)c->e, (const T*)c->kprime, c->gacc, c->st);
        LAUNCHED();
    }
    std::swap(c->lam[0], c->lam[1]);
    return LKS_OK;
}

template <class T>
lks_status exec_adj(lks_ctx* c, int seg) {
    const int a = seg_start(c, seg), b = seg_end(c, seg);
    for (int n = b; n > a; --n) {
        const void* sn = slot_ptr(c, tape_slot(c, n - a));
        const void* sp = slot_ptr(c, tape_slot(c, n - 1 - a));
        lks_status s = adjoint_step<T>(c, n, sn, sp);
        if (s != LKS_OK) return s;
    }
    return LKS_OK;
}

template <class T>
lks_status do_forward(lks_ctx* c, int N) {
    c->n_fwd = N;
    plan_tape(N, c->pool_slots, c->K, c->M, c->S);
    c->acts.clear();
    gen_schedule(0, c->M, c->S, c->acts);
    c->slot_of.assign(c->M + 1, -1);
    c->free_slots.clear();
    for (int i = c->pool_slots - 1; i >= c->K + 1; --i) c->free_slots.push_back(i);
    c->stats[0] = c->stats[1] = 0;
    c->stats[2] = c->S;
    c->stats[3] = c->K;
    c->stats[4] = 0;
    c->work = 0;
    c->work_level = -1;
    c->last = nullptr;
    CU(cudaMemsetAsync(c->jstep, 0, (size_t)(c->cfg.max_steps + 2) * 8, c->st));
    CU(cudaMemsetAsync(c->flags, 0, 64, c->st));
    size_t i = 0;
    for (; i < c->acts.size(); ++i) {
        const Act& a = c->acts[i];
        lks_status s = exec_forward_action<T>(c, a, true);
        if (s != LKS_OK) return s;
        if (a.kind == A_TAPE) break;
    }
    c->adj_begin = i + 1;
    // J = h sum_n j_n in step order
    const int w0 = c->cfg.win_begin, w1 = std::min(c->cfg.win_end, N);
    std::vector<double> js(c->cfg.max_steps + 2, 0.0);
    CU(cudaMemcpyAsync(js.data(), c->jstep, js.size() * 8, cudaMemcpyDeviceToHost, c->st));
    launch_check_state<T>(c->g, (const V4<T>*)c->last, c->flags + 2, c->st);
    LAUNCHED();
    int fl[4];
    CU(cudaMemcpyAsync(fl, c->flags, sizeof(fl), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (fl[1]) return fail(c, LKS_ERR_ARG, "transfer tap list overflow");
    if (fl[3] & 8) return fail(c, LKS_ERR_TIMEOUT, "a tensor-copy wait timed out in the fused step");
    if (fl[3]) return fail(c, LKS_ERR_CUDA, "fused step reported error %d", fl[3]);
    if (fl[2]) return fail(c, LKS_ERR_DIVERGED, "state diverged (non-finite or |u| >= 0.5)");
    const double h = 1.0 / (double)(c->cfg.win_end - c->cfg.win_begin + 1);
    double J = 0.0;
    for (int n = w0; n <= w1; ++n) J += h * js[n];
    c->J = J;
    c->fwd_valid = true;
    return LKS_OK;
}

template <class T>
lks_status do_adjoint(lks_ctx* c) {
    CU(cudaMemsetAsync(c->flags, 0, 64, c->st));
    CU(cudaMemsetAsync(c->lam[0], 0, c->snap_bytes, c->st));
    if (c->u3) CU(cudaMemsetAsync(c->u3, 0, c->snap_bytes, c->st));
    if (c->d.nd > 0) CU(cudaMemsetAsync(c->gacc, 0, (size_t)c->d.nd * 8, c->st));
    for (size_t i = c->adj_begin - 1; i < c->acts.size(); ++i) {
        const Act& a = c->acts[i];
        if (a.kind == A_TAPE && i == c->adj_begin - 1) continue;  // recorded by the forward
        lks_status s = (a.kind == A_ADJ) ? exec_adj<T>(c, a.a) : exec_forward_action<T>(c, a, false);
        if (s != LKS_OK) return s;
    }
    // the schedule may be replayed by another adjoint call of the same forward: the tape of
    // the last segment has been overwritten, so a second adjoint needs a new forward
    c->fwd_valid = false;
    int fl[4];
    CU(cudaMemcpyAsync(fl, c->flags, sizeof(fl), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (fl[1]) return fail(c, LKS_ERR_ARG, "transfer tap list overflow");
    if (fl[3] & 8) return fail(c, LKS_ERR_TIMEOUT, "a tensor-copy wait timed out in the fused step");
    if (fl[3]) return fail(c, LKS_ERR_CUDA, "fused step reported error %d", fl[3]);
    return LKS_OK;
}

template <class T>
lks_status reset_initial(lks_ctx* c) {
    launch_fill_uniform<T>(c->g, st4<T>(c->s0), c->cfg.u_init, c->st);
    LAUNCHED();
    launch_apply_bc<T>(c->g, st4<T>(c->s0), c->st);
    LAUNCHED();
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
    for (int a = 0; a < 3; ++a) d.xiG[a] = cfg->xi_G[a];
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
        if (cudaMalloc((void**)&c->ws, L.total) != cudaSuccess) {
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
    lks_status s = LKS_OK;
    if (cudaMemsetAsync(c->flags, 0, 64, c->st) != cudaSuccess) s = LKS_ERR_CUDA;
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
    if (c->prec == LKS_FP64)
        launch_design_prep<double>(c->d, c->gamma, c->cfg.kappa_max, c->cfg.q, (double*)c->kref,
                                   (double*)c->kref_t, (double*)c->kprime, c->flags, c->st);
    else
        launch_design_prep<float>(c->d, c->gamma, c->cfg.kappa_max, c->cfg.q, (float*)c->kref,
                                  (float*)c->kref_t, (float*)c->kprime, c->flags, c->st);
    LAUNCHED();
    if (on_device) {
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, c->flags, 4, cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
        if (bad) return fail(c, LKS_ERR_ARG, "gamma outside [0,1]");
    }
    c->have_design = true;
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
        c->have_motion = true;
        return LKS_OK;
    }
    // union over steps of the analysis nodes strictly within two cells of a moved design node
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    const double cx[2] = {0.0, (double)(c->d.L[0] - 1)}, cy[2] = {0.0, (double)(c->d.L[1] - 1)};
    for (int n = 1; n <= c->cfg.max_steps; ++n) {
        const Motion mo = motion_row(c, n);
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
    c->have_motion = true;
    return LKS_OK;
}

lks_status lks_set_initial_state(lks_ctx* c, const double* state) {
    if (!c) return LKS_ERR_ARG;
    c->fwd_valid = false;
    if (!state) return c->prec == LKS_FP64 ? reset_initial<double>(c) : reset_initial<float>(c);
    double* tmp = nullptr;
    const size_t bytes = (size_t)c->g.nodes * 4 * 8;
    CU(cudaMalloc(&tmp, bytes));
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
    lks_status s = c->prec == LKS_FP64 ? do_forward<double>(c, n_steps) : do_forward<float>(c, n_steps);
    if (s != LKS_OK) return s;
    if (J_out) *J_out = c->J;
    return LKS_OK;
}

lks_status lks_adjoint(lks_ctx* c, double* dJdgamma, int on_device) {
    if (!c) return LKS_ERR_ARG;
    if (!c->fwd_valid) return fail(c, LKS_ERR_ORDER, "adjoint needs a preceding forward run");
    lks_status s = c->prec == LKS_FP64 ? do_adjoint<double>(c) : do_adjoint<float>(c);
    if (s != LKS_OK) return s;
    if (c->d.nd > 0 && dJdgamma) {
        CU(cudaMemcpyAsync(dJdgamma, c->gacc, (size_t)c->d.nd * 8,
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
    CU(cudaMalloc(&tmp, bytes));
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
    lks_status s = c->prec == LKS_FP64 ? transfer_at<double>(c, step) : transfer_at<float>(c, step);
    if (s != LKS_OK) return s;
    double* tmp = nullptr;
    CU(cudaMalloc(&tmp, nodes * 4 * 8));
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

int lks_uses_fused(const lks_ctx* c) { return c && c->fused3d ? 1 : 0; }

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

void lks_destroy(lks_ctx* c) {
    if (!c) return;
    for (int w = 0; w < 2; ++w)
        for (cudaEvent_t e : c->tev[w]) cudaEventDestroy(e);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
}

}  // extern "C"
