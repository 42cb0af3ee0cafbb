// D2Q9 FP32 kernels over instance tables (lks_table.h): every launch covers all instances of a
// plan with a persistent grid that walks the concatenated work units.
//
//   k_t_design_pos  x_ref, y_ref of every design column (col_pos_sc), for a run's first step;
//   k_t_transfer2d  kappa and u_S on every footprint-box node (transfer2d_node, Sec. 2.3), into
//                   the box buffer or the transfer tape, and the next step's design positions;
//   k_t_step2d      fused LKS step (Alg. 1; Sec. 2.2 f^eq with the viscosity term, Eqs. rho,
//                   u, u_ex_2, bc_rho, bc_u) on TX x TY tiles: the state tile with a two-cell
//                   halo goes to shared memory, f^eq of the tile and a one-cell rim is
//                   evaluated once per node and direction, then gathered;
//   k_t_objective   one block per instance inside the objective window (Sec. 2.5);
//   k_t_adj2d       fused exact adjoint step (structure of Alg. 2, Eqs. arho, au, as): lambda
//                   plus the transpose of the boundary copies, to mu (Brinkman transpose and
//                   the kappa sensitivity density e), moments
//                   of F~ on the tile and a one-cell rim, adjoint equilibrium and the full
//                   transposed velocity gradient including the one-sided boundary rows;
//   k_t_sens        dJ/dgamma gather per design node (sens2d_node, Sec. 2.4).
#include <cuda_runtime.h>

#include "lks_table.h"
#include "lks_units.cuh"

namespace lks {

namespace {

constexpr int NT = 256;

// Instance of work unit u: the last i with pre[i] <= u (pre has count + 1 entries).
__device__ __forceinline__ int find_inst(const int* __restrict__ pre, int count, int u) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int wrap_any(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

__device__ __forceinline__ int step_of(const Plan& p, int noff) { return __ldg(p.nbase) + noff; }

// Stage instance i's record in shared memory when the block moves to it: kernels then read the
// geometry from shared memory, which their global stores cannot alias, instead of reloading it
// from global memory after every store.  Called by all threads; ends with a barrier when it
// copies.
// kslot >= 0 points the staged record's kus at slot kslot of the instance's transfer tape.
__device__ __forceinline__ void stage_inst(const Plan& p, int i, int& cur, Inst& sI,
                                          int kslot = -1) {
    if (i == cur) return;
    __syncthreads();
    const int* src = reinterpret_cast<const int*>(p.tab + i);
    int* dst = reinterpret_cast<int*>(&sI);
    for (int k = threadIdx.x; k < (int)(sizeof(Inst) / 4); k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
    if (kslot >= 0) {
        if (threadIdx.x == 0) sI.kus = sI.kus_tape + (long long)kslot * sI.g.boxN;
        __syncthreads();
    }
    cur = i;
}

// kappa, u_S records of a launch: the box buffer or slot kslot of the transfer tape (a taped
// forward step writes its transfer there; the adjoint of that step reads it back).
__device__ __forceinline__ V4<float>* kus_slot(const Inst& I, int kslot) {
    return kslot < 0 ? I.kus : I.kus_tape + (long long)kslot * I.g.boxN;
}

// ---------------------------------------------------------------- element-wise phases

// Design positions of step n (unit u of the design-column units) into the set of n's parity.
__device__ __forceinline__ void design_pos_unit(const Plan& p, int u, int n) {
    const int* pre = p.pre + U_DCOL * (p.count + 1);
    const int i = find_inst(pre, p.count, u);
    const Inst& I = p.tab[i];
    const long long k = (long long)(u - pre[i]) * kUnitThreads + threadIdx.x;
    if (k >= I.d.ncol) return;
    int2 b;
    float4 sc;
    col_pos_sc(I.d, I.motion[n], k, b, sc);
    I.pos_b[n & 1][k] = b;
    I.pos_sc[n & 1][k] = sc;
}

__global__ void __launch_bounds__(NT) k_t_design_pos(Plan p, int noff) {
    const int n = step_of(p, noff);
    for (int u = blockIdx.x; u < p.total[U_DCOL]; u += gridDim.x) design_pos_unit(p, u, n);
}

// One 16 x 16 tile of the footprint box per work unit.  The design nodes any node of the tile can
// reach (the tile's inverse rigid image widened by the kernel radius: at most 30 x 30 nodes) are
// staged in shared memory with contiguous reads and binned by their integer base into a table of
// cells; every node then visits the 4 x 4 cells whose taps cover it, so that it touches only the
// design nodes in its support (about 16, against some 36 window candidates).  A tile whose table
// overflows runs the candidate loop of transfer2d_node on the staged copy instead.
constexpr int kTrWin = 32;   // staged window side (design nodes)
static_assert(kBoxTile * kBoxTile == NT, "one box tile per block of NT threads");
// Cells of the tile's design-node table: the integer bases b that can reach a node of the tile
// (b in [x - 2, x + 1] per axis), kTrCells per axis; a unit-spaced rotated lattice puts at most
// two design nodes in one unit cell, kTrCap leaves room (a fuller cell sends the tile back to the
// candidate loop).
constexpr int kTrCells = kBoxTile + 3, kTrCap = 4;

// With next, the units past the box tiles form the design positions of step n + 1 (the next
// transfer's), into the other parity's set.
__global__ void __launch_bounds__(NT, 5) k_t_transfer2d(Plan p, int noff, int kslot, int next) {
    __shared__ int2 sb[kTrWin * kTrWin];
    __shared__ float4 ssc[kTrWin * kTrWin];
    __shared__ float skr[kTrWin * kTrWin];
    __shared__ int swin[4];
    __shared__ int scnt[kTrCells * kTrCells];
    __shared__ unsigned short sent[kTrCells * kTrCells * kTrCap];
    __shared__ int sfull;
    const int* pre = p.pre + U_BOX * (p.count + 1);
    const int n = step_of(p, noff);
    const int nbox = p.total[U_BOX];
    const int nall = nbox + (next ? p.total[U_DCOL] : 0);
    for (int u = blockIdx.x; u < nall; u += gridDim.x) {
        if (u >= nbox) {   // block-uniform: no barrier follows in this iteration
            design_pos_unit(p, u - nbox, n + 1);
            continue;
        }
        const int i = find_inst(pre, p.count, u);
        const Inst& I = p.tab[i];
        const Design& d = I.d;
        const Geom& g = I.g;
        const Motion& m = I.motion[n];
        const int ntx = (g.bn[0] + kBoxTile - 1) / kBoxTile;
        const int t = u - pre[i];
        const int bx0 = (t % ntx) * kBoxTile, by0 = (t / ntx) * kBoxTile;
        const int lx = threadIdx.x % kBoxTile, ly = threadIdx.x / kBoxTile;
        const int bx = bx0 + lx, by = by0 + ly;
        const bool node = bx < g.bn[0] && by < g.bn[1];
        const int x = g.blo[0] + bx, y = g.blo[1] + by;
        const float c = m.cf, s = m.sf;
        const float R = 2.f * (fabsf(c) + fabsf(s)) + 0.01f;
        // this node's candidate window (the same expressions as transfer2d_node)
        const float px = (float)x - m.xgf[0], py = (float)y - m.xgf[1];
        const float ic = c * px + s * py + d.xiGf[0];
        const float jc = -s * px + c * py + d.xiGf[1];
        const int i0 = max(0, (int)ceilf(ic - R)), i1 = min(d.L[0] - 1, (int)floorf(ic + R));
        const int j0 = max(0, (int)ceilf(jc - R)), j1 = min(d.L[1] - 1, (int)floorf(jc + R));
        __syncthreads();   // the previous unit's staged window is no longer read
        if (threadIdx.x == 0) {
            swin[0] = 1 << 30;
            swin[1] = -(1 << 30);
            swin[2] = 1 << 30;
            swin[3] = -(1 << 30);
            sfull = 0;
        }
        for (int e = threadIdx.x; e < kTrCells * kTrCells; e += NT) scnt[e] = 0;
        __syncthreads();
        if (node && i0 <= i1 && j0 <= j1) {
            atomicMin(&swin[0], i0);
            atomicMax(&swin[1], i1);
            atomicMin(&swin[2], j0);
            atomicMax(&swin[3], j1);
        }
        __syncthreads();
        const int wi0 = swin[0], wj0 = swin[2];
        const int wni = swin[1] - wi0 + 1, wnj = swin[3] - wj0 + 1;
        const bool staged = wni <= kTrWin && wnj <= kTrWin;
        // the tile's first analysis node less 2: the lowest base whose taps reach the tile
        const int cx0 = g.blo[0] + bx0 - 2, cy0 = g.blo[1] + by0 - 2;
        if (staged && wni > 0 && wnj > 0) {
            const int2* base = I.pos_b[n & 1];
            for (int e = threadIdx.x; e < wni * wnj; e += NT) {
                const int jj = e / wni, ii = e - jj * wni;
                const int k = (wj0 + jj) * d.L[0] + wi0 + ii;
                const int2 bk = __ldg(base + k);
                sb[jj * kTrWin + ii] = bk;
                ssc[jj * kTrWin + ii] = __ldg(I.pos_sc[n & 1] + k);
                skr[jj * kTrWin + ii] = __ldg(I.kref + k);
                const int cx = bk.x - cx0, cy = bk.y - cy0;
                if ((unsigned)cx < (unsigned)kTrCells && (unsigned)cy < (unsigned)kTrCells) {
                    const int cell = cy * kTrCells + cx;
                    const int slot = atomicAdd(&scnt[cell], 1);
                    if (slot < kTrCap) sent[cell * kTrCap + slot] = (unsigned short)(jj * kTrWin + ii);
                    else sfull = 1;
                }
            }
        }
        __syncthreads();
        // each cell's design nodes in design index order (the staging order of the slots is not
        // fixed)
        if (staged && !sfull) {
            for (int cell = threadIdx.x; cell < kTrCells * kTrCells; cell += NT) {
                const int cnt = scnt[cell];
                unsigned short* ent = sent + cell * kTrCap;
                for (int a1 = 1; a1 < cnt; ++a1)
                    for (int a2 = a1; a2 > 0 && ent[a2 - 1] > ent[a2]; --a2) {
                        const unsigned short tmp = ent[a2];
                        ent[a2] = ent[a2 - 1];
                        ent[a2 - 1] = tmp;
                    }
            }
        }
        __syncthreads();
        if (!node) continue;
        const long long bi = (long long)by * g.bn[0] + bx;
        if (!staged) {   // a window wider than the staging area: the global-memory path
            transfer2d_node(d, g, m, I.pos_b[n & 1], I.pos_sc[n & 1], I.kref, kus_slot(I, kslot),
                            bi);
            continue;
        }
        const float gx0 = d.xiGf[0], gy0 = d.xiGf[1];
        float kap = 0.f, m0 = 0.f, m1x = 0.f, m1y = 0.f;
        if (!sfull) {
            // the design nodes whose base b reaches (x, y): b = (x, y) + 1 - (qx, qy), qx, qy in
            // 0..3, visited by tap (qy, qx) and then in design index order within a cell
            const int ccx = x - cx0 + 1, ccy = y - cy0 + 1;
#pragma unroll
            for (int qy = 0; qy < 4; ++qy)
#pragma unroll
                for (int qx = 0; qx < 4; ++qx) {
                    const int cell = (ccy - qy) * kTrCells + (ccx - qx);
                    const int cnt = scnt[cell];
                    for (int a1 = 0; a1 < cnt; ++a1) {
                        const int sk = sent[cell * kTrCap + a1];
                        const float4 sc = ssc[sk];
                        const float W = tap_weight(qx, sc.x, sc.y) * tap_weight(qy, sc.z, sc.w);
                        kap += W * skr[sk];
                        m0 += W;
                        m1x += W * ((float)(wi0 + (sk & (kTrWin - 1))) - gx0);
                        m1y += W * ((float)(wj0 + (sk / kTrWin)) - gy0);
                    }
                }
        } else {
            for (int j = j0; j <= j1; ++j)
                for (int ii = i0; ii <= i1; ++ii) {
                    const int sk = (j - wj0) * kTrWin + (ii - wi0);
                    const int2 b = sb[sk];
                    const int qx = x - b.x + 1, qy = y - b.y + 1;
                    if ((unsigned)qx > 3u || (unsigned)qy > 3u) continue;
                    const float4 sc = ssc[sk];
                    const float W = tap_weight(qx, sc.x, sc.y) * tap_weight(qy, sc.z, sc.w);
                    kap += W * skr[sk];
                    m0 += W;
                    m1x += W * ((float)ii - gx0);
                    m1y += W * ((float)j - gy0);
                }
        }
        const float om = m.omf;
        V4<float> o;
        o.r = kap;
        o.x = (-s * m1x - c * m1y) * om + m.ugf[0] * m0;
        o.y = (c * m1x - s * m1y) * om + m.ugf[1] * m0;
        o.z = 0.f;
        kus_slot(I, kslot)[bi] = o;
    }
}

__global__ void __launch_bounds__(kObjThreads) k_t_objective(Plan p, int noff, int src) {
    const int n = step_of(p, noff);
    for (int i = blockIdx.x; i < p.count; i += gridDim.x) {
        const Inst& I = p.tab[i];
        if (n < I.win_begin || n > I.win_end) continue;   // uniform over the block
        objective_block<float>(I.g, (const V4<float>*)I.bufs[src], I.jstep + n);
    }
}

__global__ void __launch_bounds__(NT) k_t_sens(Plan p, int noff) {
    const int* pre = p.pre + U_DCOL * (p.count + 1);
    const int n = step_of(p, noff);
    for (int u = blockIdx.x; u < p.total[U_DCOL]; u += gridDim.x) {
        const int i = find_inst(pre, p.count, u);
        const Inst& I = p.tab[i];
        const long long k = (long long)(u - pre[i]) * kUnitThreads + threadIdx.x;
        if (k < I.d.ncol) sens2d_node(I.d, I.g, I.motion[n], I.e, I.kprime, I.gacc, k);
    }
}

__global__ void k_set_int(int* dst, int v) { *dst = v; }

// deriv_coef in single precision (same rows: central, periodic, one-sided on boundary nodes).
__device__ __forceinline__ float deriv_coef_f(int i, int n, int periodic, int off) {
    if (periodic || (i > 0 && i < n - 1)) return off == 1 ? 0.5f : (off == -1 ? -0.5f : 0.f);
    if (i == 0) return off == 0 ? -1.5f : (off == 1 ? 2.f : (off == 2 ? -0.5f : 0.f));
    return off == 0 ? 1.5f : (off == -1 ? -2.f : (off == -2 ? 0.5f : 0.f));
}

// ---------------------------------------------------------------- fused forward step

// Tile position of unit `local` of an instance for tiles TX x TY.
template <int TX, int TY>
__device__ __forceinline__ void tile_xy(const Geom& g, int local, int& x0, int& y0) {
    const int ntx = tile_count(g.n[0], TX, g.periodic[0]);
    const int ky = local / ntx, kx = local - ky * ntx;
    x0 = kx * TX - tile_origin(g.n[0], TX, g.periodic[0]);
    y0 = ky * TY - tile_origin(g.n[1], TY, g.periodic[1]);
}

// Load a (TY+4) x (TX+4) tile of float4 node records starting at (x0-2, y0-2): periodic axes
// wrap, positions outside a non-periodic axis read as zero.
template <int TX, int TY>
__device__ __forceinline__ void load_tile(const Geom& g, const float4* __restrict__ src, int x0,
                                          int y0, float4* S) {
    constexpr int HX = TX + 4, HY = TY + 4;
    const int n0 = g.n[0], n1 = g.n[1];
    const bool p0 = g.periodic[0], p1 = g.periodic[1];
    for (int k = threadIdx.x; k < HX * HY; k += NT) {
        const int ly = k / HX, lx = k - ly * HX;
        int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        if (p0) gx = wrap_any(gx, n0);
        if (p1) gy = wrap_any(gy, n1);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gx >= 0 && gx < n0 && gy >= 0 && gy < n1) v = __ldg(src + (long long)gy * n0 + gx);
        S[k] = v;
    }
}

// The arithmetic of the helpers below is written with explicitly rounded operations
// (__fmaf_rn, __fmul_rn, __fadd_rn, __fsub_rn), which the compiler neither contracts nor
// reorders: the tile and the row-marching forward kernels then compute bitwise the same state.
#define FMA_ __fmaf_rn
#define MUL_ __fmul_rn
#define ADD_ __fadd_rn
#define SUB_ __fsub_rn

// First derivative of the velocity along one axis from a node's record v and its neighbours at
// +-1 (p1, m1) and +-2 (p2, m2): central, or the second-order one-sided difference on a
// non-periodic boundary node (side -1: low face, +1: high face).
__device__ __forceinline__ void dvel_v(int side, const float4& v, const float4& p1,
                                       const float4& m1, const float4& p2, const float4& m2,
                                       float& dux, float& duy) {
    if (side == 0) {
        dux = FMA_(0.5f, p1.y, MUL_(-0.5f, m1.y));
        duy = FMA_(0.5f, p1.z, MUL_(-0.5f, m1.z));
    } else if (side < 0) {
        dux = FMA_(-1.5f, v.y, FMA_(2.f, p1.y, MUL_(-0.5f, p2.y)));
        duy = FMA_(-1.5f, v.z, FMA_(2.f, p1.z, MUL_(-0.5f, p2.z)));
    } else {
        dux = FMA_(1.5f, v.y, FMA_(-2.f, m1.y, MUL_(0.5f, m2.y)));
        duy = FMA_(1.5f, v.z, FMA_(-2.f, m1.z, MUL_(0.5f, m2.z)));
    }
}

// The same at the node whose record sits at S[s] (neighbours at +-step); reads only the
// values the side uses.
__device__ __forceinline__ void dvel(const float4* S, int s, int step, int side, float& dux,
                                     float& duy) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (side == 0) dvel_v(0, z, S[s + step], S[s - step], z, z, dux, duy);
    else if (side < 0) dvel_v(-1, S[s], S[s + step], z, S[s + 2 * step], z, dux, duy);
    else dvel_v(1, S[s], z, S[s - step], z, S[s - 2 * step], dux, duy);
}

__device__ __forceinline__ int face_side(int c, int n, int periodic) {
    if (periodic) return 0;
    return c == 0 ? -1 : (c == n - 1 ? 1 : 0);
}

// A tile is interior when its two-cell halo lies inside the grid at least one node away from
// every non-periodic boundary: then no index wraps, no node of the halo is a boundary node and
// no boundary node is sourced from the tile, and the kernels take a path without those tests.
template <int TX, int TY>
__device__ __forceinline__ bool interior_tile(const Geom& g, int x0, int y0) {
    return x0 - 3 >= 0 && x0 + TX + 2 <= g.n[0] - 1 && y0 - 3 >= 0 && y0 + TY + 2 <= g.n[1] - 1;
}

// f^eq of the eight moving directions (D2Q9 order 1..8) at a node with record v and velocity
// gradient g_ab = d u_a / d x_b: w_i (rho - rho0 - 1.5 u^2 + 4.5 (c.u)^2 + A c.S.c + 3 c.u),
// opposite directions sharing their symmetric part.
__device__ __forceinline__ void feq8_v(const float4& v, float A, float gxx, float gyx, float gxy,
                                       float gyy, float f[8]) {
    // the weight products w1, 4.5 w1, 3 w1, ... are those of Wts<float, 2>, which keep the
    // lattice identities exact in single precision
    using W = Wts<float, 2>;
    const float ux = v.y, uy = v.z;
    const float base = FMA_(-1.5f, FMA_(ux, ux, MUL_(uy, uy)), v.x);
    const float ax = MUL_(A, MUL_(2.f, gxx)), ay = MUL_(A, MUL_(2.f, gyy));
    const float sd = ADD_(MUL_(2.f, gxx), MUL_(2.f, gyy)), so = MUL_(2.f, ADD_(gxy, gyx));
    const float ad = MUL_(A, ADD_(sd, so)), ae = MUL_(A, SUB_(sd, so));
    const float cpp = ADD_(ux, uy), cmp = SUB_(uy, ux);
    const float sx = FMA_(MUL_(W::h_1, ux), ux, MUL_(W::w1, ADD_(base, ax)));
    const float sy = FMA_(MUL_(W::h_1, uy), uy, MUL_(W::w1, ADD_(base, ay)));
    const float spp = FMA_(MUL_(W::h_2, cpp), cpp, MUL_(W::w2, ADD_(base, ad)));
    const float smp = FMA_(MUL_(W::h_2, cmp), cmp, MUL_(W::w2, ADD_(base, ae)));
    f[0] = FMA_(W::w3_1, ux, sx);
    f[1] = FMA_(W::w3_1, uy, sy);
    f[2] = FMA_(-W::w3_1, ux, sx);
    f[3] = FMA_(-W::w3_1, uy, sy);
    f[4] = FMA_(W::w3_2, cpp, spp);
    f[5] = FMA_(W::w3_2, cmp, smp);
    f[6] = FMA_(-W::w3_2, cpp, spp);
    f[7] = FMA_(-W::w3_2, cmp, smp);
}

// Rest direction: f_0 = w0 (rho - rho0 - 1.5 u^2).
__device__ __forceinline__ float feq0_v(const float4& v) {
    return MUL_(Wts<float, 2>::w0, FMA_(-1.5f, FMA_(v.y, v.y, MUL_(v.z, v.z)), v.x));
}

// Output node from its nine gathered values: rho* = sum f_i, u* = sum c_i f_i (Eqs. rho, u),
// the body force and the Brinkman update (Eq. u_ex_2) with kappa, u_S (ks, zero outside the
// footprint box) and a static solid's kappa_s.
__device__ __forceinline__ V4<float> gather_out(float f0, float f1, float f2, float f3, float f4,
                                                float f5, float f6, float f7, float f8,
                                                const float4& ks, float kst, float bfx,
                                                float bfy) {
    V4<float> o;
    o.r = ADD_(ADD_(ADD_(ADD_(f0, f1), ADD_(f2, f3)), ADD_(ADD_(f4, f5), ADD_(f6, f7))), f8);
    const float usx = ADD_(ADD_(ADD_(SUB_(f1, f3), SUB_(f5, f6)), SUB_(f8, f7)), bfx);
    const float usy = ADD_(SUB_(ADD_(SUB_(f2, f4), ADD_(f5, f6)), ADD_(f7, f8)), bfy);
    if (ks.x != 0.f || ks.y != 0.f || ks.z != 0.f) {
        const float inv = __fdiv_rn(1.f, ADD_(ADD_(1.f, ks.x), kst));
        o.x = MUL_(FMA_(ks.x, ks.y, usx), inv);
        o.y = MUL_(FMA_(ks.x, ks.z, usy), inv);
    } else if (kst != 0.f) {
        const float inv = __fdiv_rn(1.f, ADD_(1.f, kst));
        o.x = MUL_(usx, inv);
        o.y = MUL_(usy, inv);
    } else {
        o.x = usx;
        o.y = usy;
    }
    o.z = 0.f;
    return o;
}

// Does the node rectangle [xa, xb] x [ya, yb] meet the footprint box (the target box)?  Tested
// once per tile, so that tiles away from the moving body or the objective skip the per-node
// tests.  Periodic wraps are not taken into account: callers pass the flag only where no node
// of the rectangle wraps.
__device__ __forceinline__ bool meets_box(const Geom& g, int xa, int xb, int ya, int yb) {
    return g.boxN > 0 && xb >= g.blo[0] && xa < g.blo[0] + g.bn[0] && yb >= g.blo[1] &&
           ya < g.blo[1] + g.bn[1];
}
__device__ __forceinline__ bool meets_target(const Geom& g, int xa, int xb, int ya, int yb) {
    return xb >= g.obox[0] && xa <= g.obox[1] && yb >= g.obox[2] && ya <= g.obox[3];
}

// Boundary copies sourced by interior node (x, y) of value o (Eqs. bc_rho, bc_u): a node next to
// one face writes that face's boundary node with the face's single-precision values (the values
// bc_value gives); a node next to two faces (a corner's source) takes the general rule.
__device__ __forceinline__ void write_bc2(const Inst& I, int x, int y, const V4<float>& o,
                                          V4<float>* out) {
    const Geom& g = I.g;
    const int n0 = g.n[0], n1 = g.n[1];
    const bool xl = !g.periodic[0] && x == 1, xh = !g.periodic[0] && x == n0 - 2;
    const bool yl = !g.periodic[1] && y == 1, yh = !g.periodic[1] && y == n1 - 2;
    const int nf = (int)xl + (int)xh + (int)yl + (int)yh;
    if (nf == 0) return;
    if (nf > 1) {
        write_bc_from(g, x, y, 0, o, out);
        return;
    }
    const int f = xl ? 0 : (xh ? 1 : (yl ? 2 : 3));
    const int bx = xl ? 0 : (xh ? n0 - 1 : x), by = yl ? 0 : (yh ? n1 - 1 : y);
    const float4 p = I.bcf[f];
    V4<float> b;
    if (I.bckeep[f]) {
        b.r = o.r;
        b.x = p.x;
        b.y = p.y;
    } else {
        b.r = p.w;
        b.x = f < 2 ? o.x : p.x;
        b.y = f < 2 ? p.y : o.y;
    }
    b.z = 0.f;
    out[(long long)by * n0 + bx] = b;
}

// kappa, u_S at node (x, y) of the footprint box, else zero.
__device__ __forceinline__ float4 kus_at(const Inst& I, int x, int y) {
    long long bi;
    return in_box(I.g, x, y, 0, bi) ? __ldg((const float4*)I.kus + bi)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
}

// One tile of the forward step.  EDGE: the general path (wraps, grid edges, boundary nodes).
template <int TX, int TY, bool EDGE>
__device__ __forceinline__ void step_tile(const Inst& I, int x0, int y0, int src, int dst,
                                          float4* S, float* F) {
    constexpr int HX = TX + 4, FX = TX + 2, FY = TY + 2, FN = FX * FY;
    const Geom& g = I.g;
    const int n0 = g.n[0], n1 = g.n[1];
    const float4* sp = (const float4*)I.bufs[src];
    if (EDGE) {
        load_tile<TX, TY>(g, sp, x0, y0, S);
    } else {
        const float4* base = sp + (long long)(y0 - 2) * n0 + (x0 - 2);
        for (int k = threadIdx.x; k < HX * (TY + 4); k += NT) {
            const int ly = k / HX, lx = k - ly * HX;
            S[k] = __ldg(base + (long long)ly * n0 + lx);
        }
    }
    __syncthreads();
    const bool tbox = EDGE || meets_box(g, x0, x0 + TX - 1, y0, y0 + TY - 1);
    const float A = I.Af, bfx = I.bf[0], bfy = I.bf[1];
    // f^eq of every direction at the tile and its one-cell rim
    for (int k = threadIdx.x; k < FN; k += NT) {
        const int fy = k / FX, fx = k - fy * FX;
        const int s = (fy + 1) * HX + fx + 1;
        float gxx, gyx, gxy, gyy;   // g_ab = d u_a / d x_b
        if (EDGE) {
            int gx = x0 - 1 + fx, gy = y0 - 1 + fy;
            if (g.periodic[0]) gx = wrap_any(gx, n0);
            else if (gx < 0 || gx >= n0) continue;
            if (g.periodic[1]) gy = wrap_any(gy, n1);
            else if (gy < 0 || gy >= n1) continue;
            dvel(S, s, 1, face_side(gx, n0, g.periodic[0]), gxx, gyx);
            dvel(S, s, HX, face_side(gy, n1, g.periodic[1]), gxy, gyy);
        } else {
            dvel(S, s, 1, 0, gxx, gyx);
            dvel(S, s, HX, 0, gxy, gyy);
        }
        float fv[8];
        feq8_v(S[s], A, gxx, gyx, gxy, gyy, fv);
#pragma unroll
        for (int q = 0; q < 8; ++q) F[q * FN + k] = fv[q];
    }
    __syncthreads();
    // gather rho* = sum f_i(x - c_i), u* = sum c_i f_i(x - c_i); Brinkman update; BCs
    V4<float>* out = (V4<float>*)I.bufs[dst];
    for (int k = threadIdx.x; k < TX * TY; k += NT) {
        const int ty = k / TX, tx = k - ty * TX;
        const int x = x0 + tx, y = y0 + ty;
        if (EDGE && (x < 0 || x >= n0 || y < 0 || y >= n1 || is_boundary(g, x, y, 0))) continue;
        const int f = (ty + 1) * FX + tx + 1;
        const float f0 = feq0_v(S[(ty + 2) * HX + tx + 2]);
        const float f1 = F[0 * FN + f - 1];        // from x - (1, 0)
        const float f2 = F[1 * FN + f - FX];       // from x - (0, 1)
        const float f3 = F[2 * FN + f + 1];        // from x + (1, 0)
        const float f4 = F[3 * FN + f + FX];       // from x + (0, 1)
        const float f5 = F[4 * FN + f - FX - 1];   // from x - (1, 1)
        const float f6 = F[5 * FN + f - FX + 1];   // from x - (-1, 1)
        const float f7 = F[6 * FN + f + FX + 1];   // from x + (1, 1)
        const float f8 = F[7 * FN + f + FX - 1];   // from x - (1, -1)
        const long long m = (long long)y * n0 + x;
        const float kst = g.ks ? ((const float*)g.ks)[m] : 0.f;
        const V4<float> o = gather_out(f0, f1, f2, f3, f4, f5, f6, f7, f8,
                                       tbox ? kus_at(I, x, y) : make_float4(0.f, 0.f, 0.f, 0.f),
                                       kst, bfx, bfy);
        out[m] = o;
        if (EDGE) write_bc2(I, x, y, o, out);
    }
    __syncthreads();
}

template <int TX, int TY>
__global__ void __launch_bounds__(NT) k_t_step2d(Plan p, const int* __restrict__ pre, int total,
                                                 int src, int dst, int kslot) {
    constexpr int HX = TX + 4, HY = TY + 4;
    extern __shared__ float4 smem[];
    float4* S = smem;                          // HY x HX state records
    float* F = (float*)(smem + HX * HY);       // 8 planes of FY x FX: f_1..f_8
    __shared__ Inst sI;
    int cur = -1;
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        const int i = find_inst(pre, p.count, u);
        stage_inst(p, i, cur, sI, kslot);
        int x0, y0;
        tile_xy<TX, TY>(sI.g, u - pre[i], x0, y0);
        if (interior_tile<TX, TY>(sI.g, x0, y0))
            step_tile<TX, TY, false>(sI, x0, y0, src, dst, S, F);
        else
            step_tile<TX, TY, true>(sI, x0, y0, src, dst, S, F);
    }
}

// cp.async: 16-byte copies global -> shared (src_bytes 0 fills zeros), commit, wait.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// ---------------------------------------------------------------- row-marching forward step
// A block owns a strip of SW = NTH - 2 output columns and a chunk of YC output rows and marches
// up the rows.  State rows stream through a six-row cp.async ring two rows ahead of use; per
// F-row f every thread evaluates f^eq at column x0 - 1 + t (the strip and one rim column on
// each side: 2 / SW extra work where a tile recomputes its whole rim), the six directions that
// leave the column go through shared memory, and each output node collects its nine values
// over three consecutive F-rows in registers.  With the helpers above the values are those of
// the tile kernel, bit for bit.
template <int NTH, int YC>
__global__ void __launch_bounds__(NTH) k_t_step2d_rows(Plan p, const int* __restrict__ pre,
                                                        int total, int src, int dst, int kslot) {
    // ring of state rows: 8 slots (6 in use: two rows below the f^eq row to three above), so
    // that the slot of a row is its index & 7, negative indices included
    constexpr int SW = NTH - 2, RW = NTH + 2, NR = 8;
    __shared__ float4 R[NR][RW];     // state rows, columns x0 - 2 .. x0 + SW + 1
    __shared__ float Fs[6][NTH];     // f_1, f_3, f_5, f_6, f_7, f_8 of the current F-row
    __shared__ Inst sI;
    int cur = -1;
    const int t = threadIdx.x;
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        const int i = find_inst(pre, p.count, u);
        stage_inst(p, i, cur, sI, kslot);
        const Geom& g = sI.g;
        const int n0 = g.n[0], n1 = g.n[1], p0 = g.periodic[0], p1 = g.periodic[1];
        const int ns = tile_count(n0, SW, p0);
        const int loc = u - pre[i];
        const int kc = loc / ns, kx = loc - kc * ns;
        const int x0 = kx * SW - tile_origin(n0, SW, p0);
        const int y0 = kc * YC - tile_origin(n1, YC, p1), y1 = y0 + YC;
        const float4* sp = (const float4*)sI.bufs[src];
        V4<float>* out = (V4<float>*)sI.bufs[dst];
        const float A = sI.Af, bfx = sI.bf[0], bfy = sI.bf[1];
        const bool tbox = p0 || p1 || meets_box(g, x0, x0 + SW, y0, y1 - 1);
        auto slot = [](int r) { return r & (NR - 1); };
        auto issue_row = [&](int r) {   // state row r (unwrapped index) into its ring slot
            float4* row = R[slot(r)];
            int gy = r;
            bool rin = true;
            if (p1) gy = wrap_any(gy, n1);
            else rin = gy >= 0 && gy < n1;
            for (int k = t; k < RW; k += NTH) {
                int gx = x0 - 2 + k;
                bool in = rin;
                if (p0) gx = wrap_any(gx, n0);
                else in = in && gx >= 0 && gx < n0;
                cp_async16(row + k, in ? sp + (long long)gy * n0 + gx : sp, in ? 16 : 0);
            }
        };
        __syncthreads();   // the ring and Fs of the previous unit are no longer read
        for (int r = y0 - 3; r <= y0 + 1; ++r) issue_row(r);
        cp_async_commit();
        // this thread's f^eq column and, for 1 <= t <= SW, output column
        const int xr = x0 - 1 + t;
        int xc = xr;
        bool cin = true;
        if (p0) xc = wrap_any(xc, n0);
        else cin = xc >= 0 && xc < n0;
        const int sx = face_side(xc, n0, p0);
        const bool ocol = t >= 1 && t <= SW &&
                          (p0 ? (xr >= 0 && xr < n0) : (xr >= 1 && xr <= n0 - 2));
        float a2 = 0.f, a5 = 0.f, a6 = 0.f;   // f2, f5, f6 collected for the next row
        float b2 = 0.f, b5 = 0.f, b6 = 0.f;   // the same for the row after that
        float c0 = 0.f, c1 = 0.f, c3 = 0.f;   // f0, f1, f3 collected for the next row
        for (int f = y0 - 1; f <= y1; ++f) {
            if (f + 3 <= y1 + 2) issue_row(f + 3);
            cp_async_commit();
            cp_async_wait1();
            __syncthreads();
            float fv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float f0 = 0.f;
            int fy = f;
            bool rin = true;
            if (p1) fy = wrap_any(fy, n1);
            else rin = fy >= 0 && fy < n1;
            if (cin && rin) {   // f^eq at (xc, f)
                const float4* r0 = R[slot(f)];
                const float4* rp = R[slot(f + 1)];
                const float4* rm = R[slot(f - 1)];
                const int c = t + 1;
                const float4 v = r0[c], z = make_float4(0.f, 0.f, 0.f, 0.f);
                float gxx, gyx, gxy, gyy;
                if (sx == 0) dvel_v(0, z, r0[c + 1], r0[c - 1], z, z, gxx, gyx);
                else if (sx < 0) dvel_v(-1, v, r0[c + 1], z, r0[c + 2], z, gxx, gyx);
                else dvel_v(1, v, z, r0[c - 1], z, r0[c - 2], gxx, gyx);
                const int sy = face_side(fy, n1, p1);
                if (sy == 0) dvel_v(0, z, rp[c], rm[c], z, z, gxy, gyy);
                else if (sy < 0) dvel_v(-1, v, rp[c], z, R[slot(f + 2)][c], z, gxy, gyy);
                else dvel_v(1, v, z, rm[c], z, R[slot(f - 2)][c], gxy, gyy);
                feq8_v(v, A, gxx, gyx, gxy, gyy, fv);
                f0 = feq0_v(v);
            }
            Fs[0][t] = fv[0];   // f_1
            Fs[1][t] = fv[2];   // f_3
            Fs[2][t] = fv[4];   // f_5
            Fs[3][t] = fv[5];   // f_6
            Fs[4][t] = fv[6];   // f_7
            Fs[5][t] = fv[7];   // f_8
            __syncthreads();
            if (t >= 1 && t <= SW) {
                // values the nodes (x, f - 1), (x, f), (x, f + 1) receive from F-row f
                const float g4 = fv[3], g7 = Fs[4][t + 1], g8 = Fs[5][t - 1];
                const float g1 = Fs[0][t - 1], g3 = Fs[1][t + 1];
                const float g2 = fv[1], g5 = Fs[2][t - 1], g6 = Fs[3][t + 1];
                const int y = f - 1;   // output row completed by this F-row
                bool orow = y >= y0 && y < y1;
                orow = orow && (p1 ? (y >= 0 && y < n1) : (y >= 1 && y <= n1 - 2));
                if (ocol && orow) {
                    const long long m = (long long)y * n0 + xc;
                    const float kst = g.ks ? ((const float*)g.ks)[m] : 0.f;
                    const V4<float> o = gather_out(
                        c0, c1, b2, c3, g4, b5, b6, g7, g8,
                        tbox ? kus_at(sI, xc, y) : make_float4(0.f, 0.f, 0.f, 0.f), kst, bfx,
                        bfy);
                    out[m] = o;
                    write_bc2(sI, xc, y, o, out);
                }
                b2 = a2;
                b5 = a5;
                b6 = a6;
                a2 = g2;
                a5 = g5;
                a6 = g6;
                c0 = f0;
                c1 = g1;
                c3 = g3;
            }
        }
    }
}

// ---------------------------------------------------------------- fused adjoint step

// Objective source of the adjoint step in single precision, fixed per tile.
struct ObjSrc {
    bool on;                  // inside the objective window
    float r, x, y;            // d j / d (rho, ux, uy) at a target node, times h_n
    bool cyl;
};

__device__ __forceinline__ ObjSrc obj_src(const Inst& I, int n) {
    ObjSrc o;
    o.on = n >= I.win_begin && n <= I.win_end;
    o.r = I.src_r;
    o.x = I.src_x;
    o.y = I.src_y;
    o.cyl = I.g.ocyl_r > 0.0;
    return o;
}

__device__ __forceinline__ bool in_target2(const Geom& g, const ObjSrc& o, int x, int y) {
    if (x < g.obox[0] || x > g.obox[1] || y < g.obox[2] || y > g.obox[3]) return false;
    if (o.cyl) {   // the same FP64 test as the host's target list
        const double dx = x - g.ocyl_c[0], dy = y - g.ocyl_c[1];
        if (dx * dx + dy * dy > g.ocyl_r * g.ocyl_r) return false;
    }
    return true;
}

// lambda at a node next to a face plus the transpose of the boundary copies it sources (out of
// line: few nodes take it, and the tile loop keeps its registers).
__device__ __noinline__ float4 bcT_fold(const Geom& g, const float4* lam, const ObjAdd<float>& h,
                                        int x, int y, float4 lv) {
    V4<float> acc;
    acc.r = lv.x;
    acc.x = lv.y;
    acc.y = lv.z;
    acc.z = lv.w;
    bcT_gather<float>(g, (const V4<float>*)lam, h, x, y, 0, acc);
    return make_float4(acc.r, acc.x, acc.y, acc.z);
}

// The same for a node next to a single face (most of them): its one boundary node inline, with
// the arithmetic of bcT_gather; nodes next to two faces take bcT_fold.
__device__ __forceinline__ float4 bcT_fold2(const Inst& I, const float4* lam,
                                            const ObjAdd<float>& h, int x, int y, float4 lv) {
    const Geom& g = I.g;
    const int n0 = g.n[0], n1 = g.n[1];
    const bool xl = !g.periodic[0] && x == 1, xh = !g.periodic[0] && x == n0 - 2;
    const bool yl = !g.periodic[1] && y == 1, yh = !g.periodic[1] && y == n1 - 2;
    if ((int)xl + (int)xh + (int)yl + (int)yh != 1) return bcT_fold(g, lam, h, x, y, lv);
    const int f = xl ? 0 : (xh ? 1 : (yl ? 2 : 3));
    const int bx = xl ? 0 : (xh ? n0 - 1 : x), by = yl ? 0 : (yh ? n1 - 1 : y);
    V4<float> lb;
    {
        const float4 t = lam[(long long)by * n0 + bx];
        lb.r = t.x;
        lb.x = t.y;
        lb.y = t.z;
        lb.z = t.w;
    }
    obj_source(g, bx, by, 0, h, lb);
    if (I.bckeep[f]) lv.x += lb.r;
    else if (f < 2) lv.y += lb.x;
    else lv.z += lb.y;
    return lv;
}

// One tile of the adjoint step.  EDGE: the general path (wraps, grid edges, boundary nodes,
// one-sided boundary rows of the transposed gradient).
template <int TX, int TY, bool EDGE>
__device__ __forceinline__ void adj_tile(const Inst& I, int x0, int y0, const ObjSrc& os,
                                         int lam_in, int lam_out, int sn, int sp, float4* M,
                                         float* Q) {
    constexpr int HX = TX + 4, HY = TY + 4, FX = TX + 2, FY = TY + 2, FN = FX * FY;
    using W = Wts<float, 2>;
    const Geom& g = I.g;
    const int n0 = g.n[0], n1 = g.n[1];
    const float4* lam = (const float4*)I.bufs[lam_in];
    const V4<float>* su = (const V4<float>*)I.bufs[sn];
    // tiles whose halo misses the footprint box (the target) skip those per-node tests
    const bool tbox = EDGE || meets_box(g, x0 - 2, x0 + TX + 1, y0 - 2, y0 + TY + 1);
    const bool ttgt = os.on && (EDGE || meets_target(g, x0 - 2, x0 + TX + 1, y0 - 2, y0 + TY + 1));
    // tiles whose halo holds a node next to a face: such a node first collects the transpose of
    // the boundary copies it sources (Eqs. bc_rho, bc_u; boundary nodes are read only)
    const bool tbc = EDGE || x0 - 2 <= 1 || x0 + TX + 1 >= n0 - 2 || y0 - 2 <= 1 ||
                     y0 + TY + 1 >= n1 - 2;
    ObjAdd<float> bsrc;   // the objective source of the boundary nodes inside the target
    bsrc.on = os.on;
    bsrc.r = os.r;
    bsrc.x = os.x;
    bsrc.y = os.y;
    bsrc.z = 0.f;
    // 1. mu on the tile and a two-cell halo; e on the tile's own box nodes
    for (int k = threadIdx.x; k < HX * HY; k += NT) {
        const int ly = k / HX, lx = k - ly * HX;
        int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        if (EDGE) {
            if (g.periodic[0]) gx = wrap_any(gx, n0);
            if (g.periodic[1]) gy = wrap_any(gy, n1);
        }
        float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!EDGE || (gx >= 0 && gx < n0 && gy >= 0 && gy < n1 && !is_boundary(g, gx, gy, 0))) {
            const long long gm = (long long)gy * n0 + gx;
            float4 lv = __ldg(lam + gm);
            if (tbc && sources_boundary(g, gx, gy, 0)) lv = bcT_fold2(I, lam, bsrc, gx, gy, lv);
            float lr = lv.x, lux = lv.y, luy = lv.z;
            if (ttgt && in_target2(g, os, gx, gy)) {
                lr += os.r;
                lux += os.x;
                luy += os.y;
            }
            long long bi;
            const float kst = g.ks ? ((const float*)g.ks)[gm] : 0.f;
            if (tbox && in_box(g, gx, gy, 0, bi)) {
                const V4<float> ks = I.kus[bi];
                const float inv = 1.f / (1.f + ks.r + kst);
                lux *= inv;
                luy *= inv;
                const bool own = lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2;
                if (own) {
                    const V4<float> un = su[gm];
                    I.e[bi] = lux * (ks.x - un.x) + luy * (ks.y - un.y);
                }
            } else if (kst != 0.f) {
                const float inv = 1.f / (1.f + kst);
                lux *= inv;
                luy *= inv;
            }
            m = make_float4(lr, lux, luy, 0.f);
        }
        M[k] = m;
    }
    __syncthreads();
    // 2. moments of F~_i(y) = mu_rho(y + c_i) + c_i . mu_u(y + c_i) on the tile and rim
    for (int k = threadIdx.x; k < FN; k += NT) {
        const int fy = k / FX, fx = k - fy * FX;
        const int s = (fy + 1) * HX + fx + 1;
        const float4 c0 = M[s];
        const float4 xp = M[s + 1], xm = M[s - 1], yp = M[s + HX], ym = M[s - HX];
        const float4 pp = M[s + HX + 1], mp = M[s + HX - 1], mm = M[s - HX - 1],
                     pm = M[s - HX + 1];
        // F~ of the eight moving directions, then R~, 3 U~ and 9 S~ with the weight products
        // of Wts<float, 2>
        const float fxp = xp.x + xp.y, fxm = xm.x - xm.y, fyp = yp.x + yp.z, fym = ym.x - ym.z;
        const float fpp = pp.x + pp.y + pp.z, fmp = mp.x - mp.y + mp.z;
        const float fmm = mm.x - mm.y - mm.z, fpm = pm.x + pm.y - pm.z;
        const float dsum = (fpp + fmp) + (fmm + fpm);
        Q[k] = W::w0 * c0.x + W::w1 * ((fxp + fxm) + (fyp + fym)) + W::w2 * dsum;
        Q[FN + k] = W::w3_1 * (fxp - fxm) + W::w3_2 * ((fpp - fmp) + (fpm - fmm));
        Q[2 * FN + k] = W::w3_1 * (fyp - fym) + W::w3_2 * ((fpp + fmp) - (fmm + fpm));
        Q[3 * FN + k] = W::s_1 * (fxp + fxm) + W::s_2 * dsum;
        Q[4 * FN + k] = W::s_2 * ((fpp - fmp) + (fmm - fpm));
        Q[5 * FN + k] = W::s_1 * (fyp + fym) + W::s_2 * dsum;
    }
    __syncthreads();
    // 3. lambda^{n-1} = (R~, 3 U~ - 3 R~ u + 9 S~ u + D^T (2 A S~)) on the tile; Q holds
    //    R~, 3 U~ and 9 S~, so the transposed gradient takes 2 A / 9 times the stored values
    const V4<float>* sprev = (const V4<float>*)I.bufs[sp];
    V4<float>* out = (V4<float>*)I.bufs[lam_out];
    const float twoA = (float)(2.0 * g.A / 9.0);
    for (int k = threadIdx.x; k < TX * TY; k += NT) {
        const int ty = k / TX, tx = k - ty * TX;
        const int x = x0 + tx, y = y0 + ty;
        if (EDGE && (x < 0 || x >= n0 || y < 0 || y >= n1)) continue;
        const int q = (ty + 1) * FX + tx + 1;
        const V4<float> v = sprev[(long long)y * n0 + x];
        const float R = Q[q], Ux = Q[FN + q], Uy = Q[2 * FN + q];
        const float Sxx = Q[3 * FN + q], Sxy = Q[4 * FN + q], Syy = Q[5 * FN + q];
        const float R3 = 3.f * R;
        float lx = Ux - R3 * v.x;
        float ly = Uy - R3 * v.y;
        lx += Sxx * v.x;
        lx += Sxy * v.y;
        ly += Sxy * v.x;
        ly += Syy * v.y;
        // transposed gradient: rows y' = x - kk e_b whose stencil reaches x; phi_ab = 2 A S~_ab,
        // b = x uses (Sxx, Sxy), b = y uses (Sxy, Syy)
        float ax = 0.f, ay = 0.f;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int c = b == 0 ? x : y, nn = b == 0 ? n0 : n1, per = g.periodic[b];
            const int step = b == 0 ? 1 : FX;
#pragma unroll
            for (int kk = -2; kk <= 2; ++kk) {
                float cf;
                if (EDGE) {
                    int yi = c - kk;
                    if (per) yi = wrap_any(yi, nn);
                    else if (yi < 0 || yi >= nn) continue;
                    cf = deriv_coef_f(yi, nn, per, kk);
                    if (cf == 0.f) continue;
                } else {
                    if (kk != 1 && kk != -1) continue;
                    cf = kk == 1 ? 0.5f : -0.5f;
                }
                const int qq = q - kk * step;
                // rows two nodes away are boundary rows, which the tile origin keeps inside
                // the tile; the test only keeps a shared-memory read in bounds regardless
                if (EDGE && (qq < 0 || qq >= FN)) continue;
                const float pa = twoA * Q[(b == 0 ? 3 : 4) * FN + qq];
                const float pb = twoA * Q[(b == 0 ? 4 : 5) * FN + qq];
                ax += cf * pa;
                ay += cf * pb;
            }
        }
        V4<float> o;
        o.r = R;
        o.x = lx + ax;
        o.y = ly + ay;
        o.z = 0.f;
        out[(long long)y * n0 + x] = o;
    }
    __syncthreads();
}

template <int TX, int TY>
__global__ void __launch_bounds__(NT) k_t_adj2d(Plan p, const int* __restrict__ pre, int total,
                                                int noff, int lam_in, int lam_out, int sn,
                                                int sp, int kslot) {
    constexpr int HX = TX + 4, HY = TY + 4;
    extern __shared__ float4 smem[];
    float4* M = smem;                          // HY x HX: mu (rho, x, y, -)
    float* Q = (float*)(smem + HX * HY);       // 6 planes of FY x FX: R~, 3 U~, 9 S~ (xx, xy, yy)
    const int n = step_of(p, noff);
    __shared__ Inst sI;
    int cur = -1;
    ObjSrc os;
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
        const int i = find_inst(pre, p.count, u);
        if (i != cur) {
            stage_inst(p, i, cur, sI, kslot);
            os = obj_src(sI, n);
        }
        int x0, y0;
        tile_xy<TX, TY>(sI.g, u - pre[i], x0, y0);
        if (interior_tile<TX, TY>(sI.g, x0, y0))
            adj_tile<TX, TY, false>(sI, x0, y0, os, lam_in, lam_out, sn, sp, M, Q);
        else
            adj_tile<TX, TY, true>(sI, x0, y0, os, lam_in, lam_out, sn, sp, M, Q);
    }
}

// Row-marching step configurations 5..8: threads per strip and rows per chunk.
template <int C>
struct RowCfg {
    static constexpr int NTH = tile_tx(C) + 2, YC = tile_ty(C);
};

template <int C>
int occ_rows() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_t_step2d_rows<RowCfg<C>::NTH, RowCfg<C>::YC>, RowCfg<C>::NTH, 0);
    return b;
}

template <int C>
cudaError_t rows_cfg(const Plan& p, int src, int dst, int kslot, cudaStream_t st) {
    const int unit = U_TILE0 + C;
    if (p.total[unit] == 0) return cudaSuccess;
    k_t_step2d_rows<RowCfg<C>::NTH, RowCfg<C>::YC><<<p.grid[unit], RowCfg<C>::NTH, 0, st>>>(
        p, p.pre + unit * (p.count + 1), p.total[unit], src, dst, kslot);
    return cudaGetLastError();
}

template <int C>
struct Cfg {
    static constexpr int TX = tile_tx(C), TY = tile_ty(C);
    static constexpr size_t step_smem = (size_t)(TX + 4) * (TY + 4) * 16 + (size_t)8 * (TX + 2) * (TY + 2) * 4;
    static constexpr size_t adj_smem = (size_t)(TX + 4) * (TY + 4) * 16 + (size_t)6 * (TX + 2) * (TY + 2) * 4;
};

template <int C>
int occ_step() {
    int b = 0;
    cudaFuncSetAttribute(k_t_step2d<Cfg<C>::TX, Cfg<C>::TY>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<C>::step_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t_step2d<Cfg<C>::TX, Cfg<C>::TY>, NT,
                                                  Cfg<C>::step_smem);
    return b;
}
template <int C>
int occ_adj() {
    int b = 0;
    cudaFuncSetAttribute(k_t_adj2d<Cfg<C>::TX, Cfg<C>::TY>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<C>::adj_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t_adj2d<Cfg<C>::TX, Cfg<C>::TY>, NT,
                                                  Cfg<C>::adj_smem);
    return b;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int cap_grid(long long units, int per_sm) {
    const long long g = (long long)sm_count() * std::max(per_sm, 1);
    return (int)std::max(1LL, std::min(units, g));
}

template <int C>
cudaError_t step_cfg(const Plan& p, int src, int dst, int kslot, cudaStream_t st) {
    const int unit = U_TILE0 + C;
    if (p.total[unit] == 0) return cudaSuccess;
    k_t_step2d<Cfg<C>::TX, Cfg<C>::TY><<<p.grid[unit], NT, Cfg<C>::step_smem, st>>>(
        p, p.pre + unit * (p.count + 1), p.total[unit], src, dst, kslot);
    return cudaGetLastError();
}

template <int C>
cudaError_t adj_cfg(const Plan& p, int noff, int li, int lo, int sn, int sp, int kslot,
                    cudaStream_t st) {
    const int unit = U_TILE0 + C;
    if (p.total[unit] == 0) return cudaSuccess;
    k_t_adj2d<Cfg<C>::TX, Cfg<C>::TY><<<p.grid[U_COUNT + C], NT, Cfg<C>::adj_smem, st>>>(
        p, p.pre + unit * (p.count + 1), p.total[unit], noff, li, lo, sn, sp, kslot);
    return cudaGetLastError();
}

}  // namespace

void plan_grids(Plan& p) {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t_transfer2d, NT, 0);
    p.grid[U_BOX] = cap_grid(p.total[U_BOX], b);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t_design_pos, NT, 0);
    p.grid[U_DCOL] = cap_grid(p.total[U_DCOL], b);
    p.grid[U_INST] = std::max(1, p.count);
    const int os[kTileCfgs] = {occ_step<0>(), occ_step<1>(), occ_step<2>(), occ_step<3>(),
                               occ_step<4>(), occ_rows<5>(),  occ_rows<6>(),  occ_rows<7>(),
                               occ_rows<8>()};
    const int oa[kAdjCfgs] = {occ_adj<0>(), occ_adj<1>(), occ_adj<2>(), occ_adj<3>(),
                              occ_adj<4>()};
    for (int c = 0; c < kTileCfgs; ++c) p.grid[U_TILE0 + c] = cap_grid(p.total[U_TILE0 + c], os[c]);
    for (int c = 0; c < kAdjCfgs; ++c) p.grid[U_COUNT + c] = cap_grid(p.total[U_TILE0 + c], oa[c]);
    cudaGetLastError();
}

cudaError_t launch_t_design_pos(const Plan& p, int noff, cudaStream_t st) {
    if (p.total[U_DCOL] == 0) return cudaSuccess;
    k_t_design_pos<<<p.grid[U_DCOL], NT, 0, st>>>(p, noff);
    return cudaGetLastError();
}

cudaError_t launch_t_transfer2d(const Plan& p, int noff, int kslot, bool next, cudaStream_t st) {
    if (p.total[U_BOX] == 0) return cudaSuccess;
    k_t_transfer2d<<<p.grid[U_BOX], NT, 0, st>>>(p, noff, kslot, next ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_t_step2d(const Plan& p, int cfg, int src, int dst, int kslot,
                            cudaStream_t st) {
    switch (cfg) {
        case 0: return step_cfg<0>(p, src, dst, kslot, st);
        case 1: return step_cfg<1>(p, src, dst, kslot, st);
        case 2: return step_cfg<2>(p, src, dst, kslot, st);
        case 3: return step_cfg<3>(p, src, dst, kslot, st);
        case 4: return step_cfg<4>(p, src, dst, kslot, st);
        case 5: return rows_cfg<5>(p, src, dst, kslot, st);
        case 6: return rows_cfg<6>(p, src, dst, kslot, st);
        case 7: return rows_cfg<7>(p, src, dst, kslot, st);
        case 8: return rows_cfg<8>(p, src, dst, kslot, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_t_objective(const Plan& p, int noff, int src, cudaStream_t st) {
    k_t_objective<<<p.grid[U_INST], kObjThreads, 0, st>>>(p, noff, src);
    return cudaGetLastError();
}

cudaError_t launch_t_adj2d(const Plan& p, int cfg, int noff, int lam_in, int lam_out, int sn,
                           int sp, int kslot, cudaStream_t st) {
    switch (cfg) {
        case 0: return adj_cfg<0>(p, noff, lam_in, lam_out, sn, sp, kslot, st);
        case 1: return adj_cfg<1>(p, noff, lam_in, lam_out, sn, sp, kslot, st);
        case 2: return adj_cfg<2>(p, noff, lam_in, lam_out, sn, sp, kslot, st);
        case 3: return adj_cfg<3>(p, noff, lam_in, lam_out, sn, sp, kslot, st);
        case 4: return adj_cfg<4>(p, noff, lam_in, lam_out, sn, sp, kslot, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_t_sens(const Plan& p, int noff, cudaStream_t st) {
    if (p.total[U_DCOL] == 0) return cudaSuccess;
    k_t_sens<<<p.grid[U_DCOL], NT, 0, st>>>(p, noff);
    return cudaGetLastError();
}

cudaError_t launch_set_int(int* dst, int v, cudaStream_t st) {
    k_set_int<<<1, 1, 0, st>>>(dst, v);
    return cudaGetLastError();
}

}  // namespace lks
