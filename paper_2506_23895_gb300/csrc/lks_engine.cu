// Host engine behind the C ABI of include/lks.h: validates the problem, carves the device
// workspace, runs Algorithm 1 (forward with the objective of Sec. 2.5) and the reverse adjoint
// sweep (Algorithm 2 structure, exact discrete adjoint) under a binomial checkpoint schedule
// over tape segments, so that the stored history fits the given device memory.
#include "lks_engine.h"

using namespace lks;
using namespace lks::eng;

namespace lks {
namespace eng {

lks_status fail(lks_ctx* c, lks_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

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

}  // namespace eng
}  // namespace lks

namespace {

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
    int ktape_slots;   // slots of the transfer tape (0: none)
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
    L_KTAPE, L_PB2, L_PSC2, L_POOL,
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
    // FP32 2D contexts with a design keep the transfer (kappa, u_S on the footprint box) of each
    // taped step, so that the adjoint of the step reads it instead of transferring again; a tape
    // of up to max(ceil(sqrt(N)) + 2, 64) steps (the checkpointed schedules' tape length, and
    // short full-history runs), each slot sized for the whole grid (the box is known only once
    // the motion is set)
    {
        const bool t2d = cfg->precision == LKS_FP32 && dim == 2 && nd > 0 &&
                         !(cfg->flags & (LKS_FLAG_PLAIN_KERNELS | LKS_FLAG_PAPER_ALKS));
        const long long kt = std::max((long long)std::ceil(std::sqrt((double)N)) + 2, 64LL);
        L.ktape_slots = t2d ? (int)std::min(P, kt) : 0;
        sz[L_KTAPE] = (size_t)L.ktape_slots * state;
        // design positions of the steps of odd parity (even: L_CBASE, L_CSC)
        sz[L_PB2] = t2d ? (size_t)ncol * 8 : 0;
        sz[L_PSC2] = t2d ? (size_t)ncol * 16 : 0;
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
    c->ktape_slots = c->fused2d ? L.ktape_slots : 0;
    c->ktape = c->ktape_slots > 0 ? (void*)(w + L.off[L_KTAPE]) : nullptr;
    c->pos2_b = w + L.off[L_PB2];
    c->pos2_sc = (float4*)(w + L.off[L_PSC2]);
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

lks_status lks_adjoint_variant(lks_ctx* c, int request, int* chosen) {
    if (!c || request < -2 || request == -1 || request >= kAdj3dVariants)
        return c ? fail(c, LKS_ERR_ARG, "adjoint variant must be -2 or in [0, %d]",
                        kAdj3dVariants - 1)
                 : LKS_ERR_ARG;
    if (request >= 0) c->adj3d_var = request;
    if (chosen) *chosen = c->adj3d_var;
    return LKS_OK;
}

lks_status lks_get_stats(const lks_ctx* c, long long* st5) {
    if (!c || !st5) return LKS_ERR_ARG;
    for (int i = 0; i < 5; ++i) st5[i] = c->stats[i];
    return LKS_OK;
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
