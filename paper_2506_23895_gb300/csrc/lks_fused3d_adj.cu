// Fused D3Q15 adjoint step for the FP32 path on non-periodic grids (exact discrete adjoint of
// the fused forward step; structure of Alg. 2, Eqs. arho, au, as and the adjoint equilibrium).
//
// Input lambda^n has already received the boundary copies (transpose of Eqs. bc_rho, bc_u) on
// its interior nodes.  Per z plane, a block of 32 x 16 columns:
//   1. receives lambda^n (float4 per node, two-cell halo) by TMA into a five-slot ring and
//      converts it in place to mu: 0 on boundary nodes and outside the grid, otherwise
//      (lambda_rho + d j/d rho, (lambda_u + d j/d u) / (1 + kappa)) -- the transpose of the
//      Brinkman update (Eq. u_ex_2) -- and, on the tile's nodes inside the footprint box,
//      e = mu_u . (u_S - u^n), the sensitivity density dJ/dkappa;
//   2. gathers F~_i(y) = mu_rho(y + c_i) + c_i . mu_u(y + c_i) on the tile
//      into R~ = sum w F~, U~ = sum w c F~, S~ = sum w c c F~ (corner sums by a butterfly), and
//      on a one-cell rim (corners excepted) the three S~ components its tile neighbour needs;
//   3. writes lambda^{n-1} = (R~, 3 U~ + 9 S~ u^{n-1} - 3 R~ u^{n-1} + D^T(2 A S~)) for the
//      tile, with the transposed gradient in its central form; boundary rows' one-sided parts
//      are added afterwards by k_adj_bcorr from the 2 A S~ values this kernel stores for
//      boundary nodes.
// HBM traffic per node: lambda^n in, u^{n-1} in, lambda^{n-1} out (and u^n, kappa, e on the box).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "lks_device.cuh"
#include "lks_tma.cuh"

namespace lks {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int HX = TX + 4, HY = TY + 4;     // lambda tile with a two-cell halo
constexpr int PX = HX + 1;                  // row pitch of a ring plane (odd: columns hit all banks)
constexpr int FX = TX + 2, FY = TY + 2;     // moment region with a one-cell halo
constexpr int PF = FX + 1;                  // row pitch of the S~ planes (odd)
constexpr int NSLOT = 5;
constexpr int NTHR = TX * TY;
// rim nodes of the moment region whose S~ the transposed gradient reads: the two y-rim rows
// (warps 0 and 1, one row each) and the two x-rim columns (lanes 0..15 of warp 2); the four
// corners of the region are never read
constexpr int NRIM1 = 2 * TX + 2 * TY;
static_assert(TX == 32 && 2 * TY <= 32, "rim rows map to whole warps");
constexpr int NRIM2 = HX * HY - TX * TY;    // 176 halo nodes to convert
constexpr int NS = 5;                       // S~ components shared in-plane: xx xy xz yy yz
constexpr unsigned PLANE_BYTES = PX * HY * 16;   // bytes one TMA box delivers
constexpr int SLOT = (PLANE_BYTES + 127) / 128 * 128 / 16;   // float4 per ring slot (128 B aligned)
constexpr size_t OFF_RAW = 0;
constexpr size_t OFF_S = OFF_RAW + (size_t)NSLOT * SLOT * 16;
constexpr size_t OFF_BAR = OFF_S + (size_t)2 * NS * PF * FY * 4;
constexpr size_t SMEM_BYTES = OFF_BAR + NSLOT * 8;

struct AdjArgs {
    Geom g;
    float4* lam_out;
    const float4* kus;
    const float4* sn;      // state at level n (u^n for e)
    const float4* sp;      // state at level n-1
    float* e;              // footprint box
    float* face;           // 2 A S~_{.beta} on the six faces
    long long face_off[6];
    int* err;
    int zchunk;
    float A9;              // A / 9
    float obj_r, obj_u[3]; // d j / d s at target nodes, times the window weight
    int has_obj;           // any of them non-zero
};

// Per-column facts of a node column (x, y), evaluated once per thread so that the per-plane
// conversion tests z only: bit 0 interior in x and y (not on an x or y face, inside the grid),
// bit 1 inside the footprint box in x and y, bit 2 inside the objective target in x and y.
constexpr int COL_IN = 1, COL_BOX = 2, COL_TGT = 4;
__device__ __forceinline__ int col_flags(const Geom& g, int gx, int gy) {
    int f = 0;
    if (gx >= 1 && gy >= 1 && gx <= g.n[0] - 2 && gy <= g.n[1] - 2) f |= COL_IN;
    const int bx = gx - g.blo[0], by = gy - g.blo[1];
    if (g.boxN > 0 && bx >= 0 && by >= 0 && bx < g.bn[0] && by < g.bn[1]) f |= COL_BOX;
    bool t = gx >= g.obox[0] && gx <= g.obox[1] && gy >= g.obox[2] && gy <= g.obox[3];
    if (t && g.ocyl_r > 0.0) {
        const double dx = gx - g.ocyl_c[0], dy = gy - g.ocyl_c[1];
        t = dx * dx + dy * dy <= g.ocyl_r * g.ocyl_r;
    }
    if (t) f |= COL_TGT;
    return f;
}

// Convert lambda to mu at raw-tile slot position v (node gx, gy, gz with column flags cf): 0 on
// boundary nodes and outside the grid; otherwise the objective source (target nodes, has_obj)
// and the Brinkman transpose (footprint box).  `own` marks a node of the tile: only those write e.
__device__ __forceinline__ void to_mu(const AdjArgs& a, float4& v, int cf, int gx, int gy, int gz,
                                      bool own, bool has_obj) {
    const Geom& g = a.g;
    if (!(cf & COL_IN) || gz <= 0 || gz >= g.n[2] - 1) {
        v = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float4 l = v;
    if (has_obj && (cf & COL_TGT) && gz >= g.obox[4] && gz <= g.obox[5]) {
        l.x += a.obj_r;
        l.y += a.obj_u[0];
        l.z += a.obj_u[1];
        l.w += a.obj_u[2];
    }
    const int bz = gz - g.blo[2];
    if ((cf & COL_BOX) && bz >= 0 && bz < g.bn[2]) {
        const long long bi =
            ((long long)bz * g.bn[1] + (gy - g.blo[1])) * g.bn[0] + (gx - g.blo[0]);
        const float4 ks = a.kus[bi];
        const float inv = 1.f / (1.f + ks.x);
        l.y *= inv;
        l.z *= inv;
        l.w *= inv;
        if (own) {
            const float4 un = a.sn[((long long)gz * g.n[1] + gy) * g.n[0] + gx];
            a.e[bi] = l.y * (ks.y - un.y) + l.z * (ks.z - un.z) + l.w * (ks.w - un.w);
        }
    }
    v = l;
}

// R = R~, U = 3 U~, S = 9 S~ (the multiples the adjoint equilibrium uses, each formed with the
// weight products of Wts<float, 3> so that the lattice identities hold exactly).
struct Mom {
    float R, Ux, Uy, Uz, Sxx, Sxy, Sxz, Syy, Syz, Szz;
};

// Corner neighbours (sx, sy, sz) of a node: F~ = mu_rho + sx mu_x + sy mu_y + sz mu_z there.
// For one sy and one sz, from the records np (sx = +1) and nm (sx = -1) of the corner plane:
// a = F~(+1) + F~(-1), b = F~(+1) - F~(-1).
__device__ __forceinline__ void corner_pair(const float4 np, const float4 nm, float sy, float sz,
                                            float& a, float& b) {
    const float base_p = np.x + sy * np.z + sz * np.w;
    const float base_m = nm.x + sy * nm.z + sz * nm.w;
    const float gp = base_p + np.y;   // sx = +1
    const float gm = base_m - nm.y;   // sx = -1
    a = gp + gm;
    b = gp - gm;
}

// Sums of F~ over the eight corner neighbours, from a_, b_ indexed [sy > 0 ? 0 : 1][sz > 0 ?
// 0 : 1]: G = sum F~, and the sums weighted by sx, sy, sz, sx sy, sx sz, sy sz.
struct Corners {
    float G, xG, yG, zG, xyG, xzG, yzG;
};

__device__ __forceinline__ Corners corner_sums(const float (&a_)[2][2], const float (&b_)[2][2]) {
    const float Ap = a_[0][0] + a_[1][0], Am = a_[0][1] + a_[1][1];
    const float Adp = a_[0][0] - a_[1][0], Adm = a_[0][1] - a_[1][1];
    const float Bp = b_[0][0] + b_[1][0], Bm = b_[0][1] + b_[1][1];
    const float Bdp = b_[0][0] - b_[1][0], Bdm = b_[0][1] - b_[1][1];
    Corners c;
    c.G = Ap + Am;
    c.zG = Ap - Am;
    c.yG = Adp + Adm;
    c.yzG = Adp - Adm;
    c.xG = Bp + Bm;
    c.xzG = Bp - Bm;
    c.xyG = Bdp + Bdm;
    return c;
}

// The corner sums of a node from mu in planes p-1 (cm) and p+1 (cp); pointers at the node.
__device__ __forceinline__ Corners corners(const float4* __restrict__ cm,
                                           const float4* __restrict__ cp) {
    float a_[2][2], b_[2][2];
#pragma unroll
    for (int jz = 0; jz < 2; ++jz) {
        const float4* pl = jz == 0 ? cp : cm;
#pragma unroll
        for (int jy = 0; jy < 2; ++jy) {
            const int oy = jy == 0 ? PX : -PX;
            corner_pair(pl[oy + 1], pl[oy - 1], jy == 0 ? 1.f : -1.f, jz == 0 ? 1.f : -1.f,
                        a_[jy][jz], b_[jy][jz]);
        }
    }
    return corner_sums(a_, b_);
}

// The sz = -1 corner terms of plane pl seen from the node one plane above: c = (a[sy = +1],
// a[sy = -1], b[sy = +1], b[sy = -1]).
__device__ __forceinline__ void corner_below(const float4* __restrict__ pl, float (&c)[4]) {
#pragma unroll
    for (int jy = 0; jy < 2; ++jy) {
        const int oy = jy == 0 ? PX : -PX;
        corner_pair(pl[oy + 1], pl[oy - 1], jy == 0 ? 1.f : -1.f, -1.f, c[jy], c[2 + jy]);
    }
}

// Moments from the in-plane face sums g(p|m)(x|y), the z-face sums gpz, gmz, mu_rho of the node
// (s_rho) and the corner sums.
__device__ __forceinline__ Mom assemble(float s_rho, float gpx, float gmx, float gpy, float gmy,
                                        float gpz, float gmz, const Corners& k) {
    using Wf = Wts<float, 3>;
    Mom m;
    const float ax = gpx + gmx, ay = gpy + gmy, az = gpz + gmz;
    const float s2G = Wf::s_2 * k.G;
    m.R = Wf::w0 * s_rho + Wf::w1 * (ax + ay + az) + Wf::w2 * k.G;
    m.Ux = Wf::w3_1 * (gpx - gmx) + Wf::w3_2 * k.xG;
    m.Uy = Wf::w3_1 * (gpy - gmy) + Wf::w3_2 * k.yG;
    m.Uz = Wf::w3_1 * (gpz - gmz) + Wf::w3_2 * k.zG;
    m.Sxx = Wf::s_1 * ax + s2G;
    m.Syy = Wf::s_1 * ay + s2G;
    m.Szz = Wf::s_1 * az + s2G;
    m.Sxy = Wf::s_2 * k.xyG;
    m.Sxz = Wf::s_2 * k.xzG;
    m.Syz = Wf::s_2 * k.yzG;
    return m;
}

// Moments of F~ at one node from mu in planes p-1 (cm), p (c0), p+1 (cp); pointers at the node.
__device__ __forceinline__ Mom moments(const float4* __restrict__ c0,
                                       const float4* __restrict__ cm,
                                       const float4* __restrict__ cp) {
    const float4 s = c0[0], xp = c0[1], xm = c0[-1], yp = c0[PX], ym = c0[-PX];
    const float4 zp = cp[0], zm = cm[0];
    const float gpx = xp.x + xp.y, gmx = xm.x - xm.y;
    const float gpy = yp.x + yp.z, gmy = ym.x - ym.z;
    const float gpz = zp.x + zp.w, gmz = zm.x - zm.w;
    const Corners k = corners(cm, cp);
    return assemble(s.x, gpx, gmx, gpy, gmy, gpz, gmz, k);
}

// moments() for a thread that marches one column in z and keeps in registers what the next
// planes reuse: the node's own mu in planes p-1, p, p+1 (own_m, own_0, own_p: mu_rho and mu_z)
// and the sz = -1 corner terms of plane p-1 (below, formed two planes earlier from the same
// records); it reads only the four in-plane faces and the four corners of plane p+1 (c0, cp:
// pointers at the node) and returns plane p+1's sz = -1 terms for node p+2 in next_below.
__device__ __forceinline__ Mom moments_marched(const float4* __restrict__ c0,
                                               const float4* __restrict__ cp, float2 own_m,
                                               float own_0, float2 own_p,
                                               const float (&below)[4],
                                               float (&next_below)[4]) {
    const float4 xp = c0[1], xm = c0[-1], yp = c0[PX], ym = c0[-PX];
    const float gpx = xp.x + xp.y, gmx = xm.x - xm.y;
    const float gpy = yp.x + yp.z, gmy = ym.x - ym.z;
    const float gpz = own_p.x + own_p.y, gmz = own_m.x - own_m.y;
    float a_[2][2], b_[2][2];
#pragma unroll
    for (int jy = 0; jy < 2; ++jy) {
        const int oy = jy == 0 ? PX : -PX;
        const float sy = jy == 0 ? 1.f : -1.f;
        const float4 np = cp[oy + 1], nm = cp[oy - 1];
        corner_pair(np, nm, sy, 1.f, a_[jy][0], b_[jy][0]);
        corner_pair(np, nm, sy, -1.f, next_below[jy], next_below[2 + jy]);
        a_[jy][1] = below[jy];
        b_[jy][1] = below[2 + jy];
    }
    const Corners k = corner_sums(a_, b_);
    return assemble(own_0, gpx, gmx, gpy, gmy, gpz, gmz, k);
}

// The in-plane S~ components (9 S~) that the transposed gradient takes from a rim node: x-rim
// nodes (XRIM) give xx, xy, xz from the +-x faces and the corners, y-rim nodes give xy, yy, yz
// from the +-y faces and the corners; the same expressions as moments().
template <bool XRIM>
__device__ __forceinline__ void rim_moments(const float4* __restrict__ c0,
                                            const float4* __restrict__ cm,
                                            const float4* __restrict__ cp, float& s0, float& s1,
                                            float& s2) {
    using Wf = Wts<float, 3>;
    const Corners k = corners(cm, cp);
    const float s2G = Wf::s_2 * k.G;
    if (XRIM) {
        const float4 xp = c0[1], xm = c0[-1];
        const float gpx = xp.x + xp.y, gmx = xm.x - xm.y;
        s0 = Wf::s_1 * (gpx + gmx) + s2G;
        s1 = Wf::s_2 * k.xyG;
        s2 = Wf::s_2 * k.xzG;
    } else {
        const float4 yp = c0[PX], ym = c0[-PX];
        const float gpy = yp.x + yp.z, gmy = ym.x - ym.z;
        s0 = Wf::s_2 * k.xyG;
        s1 = Wf::s_1 * (gpy + gmy) + s2G;
        s2 = Wf::s_2 * k.yzG;
    }
}

// ONEBAR = false: per plane a barrier after the TMA wait and one after the conversion.
// ONEBAR = true: every thread waits on the plane it converts and the conversion runs one plane
// further ahead, so a single barrier per plane orders everything; each thread keeps its own
// column's mu and the corner terms of the plane below in registers (moments_marched), which
// takes three blocks per SM (80 registers) instead of four.
template <bool ONEBAR>
constexpr int adj_minb() {
    return ONEBAR ? 3 : 4;
}

template <bool ONEBAR>
__global__ void __launch_bounds__(NTHR, adj_minb<ONEBAR>())
    k_fused_adj3d(const __grid_constant__ CUtensorMap tmap, const AdjArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    float4* raw = reinterpret_cast<float4*>(smem + OFF_RAW);
    float* sS = reinterpret_cast<float*>(smem + OFF_S);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    const Geom& g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int q0 = blockIdx.z * a.zchunk;
    const int q1 = min(nz, q0 + a.zchunk);
    const int nplanes = q1 - q0 + 4;   // lambda planes q0-2 .. q1+1
    if ((smem_addr(smem) & 127u) != 0u) {
        if (tid == 0) atomicOr(a.err, 16);
        return;
    }
    // halo node to convert (tid < NRIM2), in raw-tile coordinates
    int cx = 0, cy = 0;
    if (tid < NRIM2) {
        if (tid < 2 * HX) {
            cx = tid % HX;
            cy = tid / HX;
        } else if (tid < 4 * HX) {
            cx = (tid - 2 * HX) % HX;
            cy = HY - 2 + (tid - 2 * HX) / HX;
        } else {
            const int t = tid - 4 * HX;   // 32 nodes: columns 0, 1, HX-2, HX-1 of rows 2..HY-3
            const int col = t / TY, row = t % TY;
            cx = col < 2 ? col : HX - 4 + col;
            cy = 2 + row;
        }
    }
    // rim node of the moment region (tid < NRIM1), in moment-region coordinates
    int rfx = 0, rfy = 0;
    if (tid < TX) {
        rfx = 1 + tid;
        rfy = 0;
    } else if (tid < 2 * TX) {
        rfx = 1 + tid - TX;
        rfy = FY - 1;
    } else if (tid < 2 * TX + TY) {
        rfx = 0;
        rfy = 1 + (tid - 2 * TX);
    } else if (tid < NRIM1) {
        rfx = FX - 1;
        rfy = 1 + (tid - 2 * TX - TY);
    }
    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(smem_addr(&bars[s]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < (ONEBAR ? NSLOT : 2) && k < nplanes; ++k)
            tma_load_box(smem_addr(raw + (size_t)k * SLOT), &tmap, x0 - 2, y0 - 2,
                         q0 - 2 + k, smem_addr(&bars[k]), PLANE_BYTES);
    }
    __syncthreads();

    const int gx = x0 + tx, gy = y0 + ty;
    const bool own_in = gx < nx && gy < ny;
    const int cf_own = col_flags(g, gx, gy);
    const int cf_halo = col_flags(g, x0 - 2 + cx, y0 - 2 + cy);
    const bool has_obj = a.has_obj != 0;
    const int hp = (ty + 2) * PX + (tx + 2);       // own node in the raw tile
    const int hc = cy * PX + cx;                   // halo node to convert
    const int hr = (rfy + 1) * PX + (rfx + 1);     // rim node of the moment region
    constexpr int FS = PF * FY;
    const int fo = (ty + 1) * PF + (tx + 1);
    const int fr = rfy * PF + rfx;
    const long long zstride = (long long)nx * ny;
    const long long col = (long long)gy * nx + gx;
    const float A9 = a.A9;   // A / 9: the stored moments are 9 S~

    Mom prev = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    float szm_x = 0.f, szm_y = 0.f, szm_z = 0.f;   // S~_{.z} of plane p-2
    // ONEBAR: the own node's (mu_rho, mu_z) in planes p-1, p, p+1 and the sz = -1 corner terms
    // of plane p-1 (below) and of plane p (below_next)
    float2 own_m = make_float2(0.f, 0.f), own_0 = own_m, own_p = own_m;
    float below[4] = {0.f, 0.f, 0.f, 0.f}, below_next[4] = {0.f, 0.f, 0.f, 0.f};
    bool ok = true;
    // moments of plane p from the converted planes p-1 (rm), p (r0), p+1 (rp) on the tile and
    // its rim, then lambda^{n-1} of plane p-1 (u: u^{n-1} there)
    auto plane = [&](int p, const float4* rm, const float4* r0, const float4* rp,
                     const float4& u, bool write_out) {
        const int q = p - 1;
        float* sw = sS + (size_t)(p & 1) * NS * FS;
        Mom m;
        if constexpr (ONEBAR) {
            // the terms of plane p-1 come from plane p-3's pass, but not for the first two planes
            if (p < q0 + 1) corner_below(rm + hp, below);
            float nb[4];
            m = moments_marched(r0 + hp, rp + hp, own_m, own_0.x, own_p, below, nb);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                below[k] = below_next[k];
                below_next[k] = nb[k];
            }
        } else {
            m = moments(r0 + hp, rm + hp, rp + hp);
        }
        sw[0 * FS + fo] = m.Sxx;
        sw[1 * FS + fo] = m.Sxy;
        sw[2 * FS + fo] = m.Sxz;
        sw[3 * FS + fo] = m.Syy;
        sw[4 * FS + fo] = m.Syz;
        if (tid < 2 * TX) {
            float s0, s1, s2;
            rim_moments<false>(r0 + hr, rm + hr, rp + hr, s0, s1, s2);
            sw[1 * FS + fr] = s0;
            sw[3 * FS + fr] = s1;
            sw[4 * FS + fr] = s2;
        } else if (tid < NRIM1) {
            float s0, s1, s2;
            rim_moments<true>(r0 + hr, rm + hr, rp + hr, s0, s1, s2);
            sw[0 * FS + fr] = s0;
            sw[1 * FS + fr] = s1;
            sw[2 * FS + fr] = s2;
        }
        // 3. lambda^{n-1} of plane q = p - 1 (its in-plane S~ was stored last iteration)
        if (write_out) {
            const float* sr = sS + (size_t)(q & 1) * NS * FS;
            // D^T (2 A S~) in central form: A [S~_a.(x-1) - S~_a.(x+1) + ... ]
            const float tx_x = sr[0 * FS + fo - 1] - sr[0 * FS + fo + 1];
            const float tx_y = sr[1 * FS + fo - 1] - sr[1 * FS + fo + 1];
            const float tx_z = sr[2 * FS + fo - 1] - sr[2 * FS + fo + 1];
            const float ty_x = sr[1 * FS + fo - PF] - sr[1 * FS + fo + PF];
            const float ty_y = sr[3 * FS + fo - PF] - sr[3 * FS + fo + PF];
            const float ty_z = sr[4 * FS + fo - PF] - sr[4 * FS + fo + PF];
            const float tz_x = szm_x - m.Sxz, tz_y = szm_y - m.Syz, tz_z = szm_z - m.Szz;
            const Mom& c = prev;
            const float R3 = 3.f * c.R;
            float4 o;
            o.x = c.R;
            o.y = (c.Ux - R3 * u.y) + (c.Sxx * u.y + c.Sxy * u.z + c.Sxz * u.w) +
                  A9 * (tx_x + ty_x + tz_x);
            o.z = (c.Uy - R3 * u.z) + (c.Sxy * u.y + c.Syy * u.z + c.Syz * u.w) +
                  A9 * (tx_y + ty_y + tz_y);
            o.w = (c.Uz - R3 * u.w) + (c.Sxz * u.y + c.Syz * u.z + c.Szz * u.w) +
                  A9 * (tx_z + ty_z + tz_z);
            a.lam_out[q * zstride + col] = o;
            // boundary nodes keep 2 A S~_{.beta} for the one-sided parts of D^T
            const float A2 = 2.f * A9;
            if (gx == 0 || gx == nx - 1) {
                float* f = a.face + a.face_off[gx == 0 ? 0 : 1] + 3 * ((long long)q * ny + gy);
                f[0] = A2 * c.Sxx;
                f[1] = A2 * c.Sxy;
                f[2] = A2 * c.Sxz;
            }
            if (gy == 0 || gy == ny - 1) {
                float* f = a.face + a.face_off[gy == 0 ? 2 : 3] + 3 * ((long long)q * nx + gx);
                f[0] = A2 * c.Sxy;
                f[1] = A2 * c.Syy;
                f[2] = A2 * c.Syz;
            }
            if (q == 0 || q == nz - 1) {
                float* f = a.face + a.face_off[q == 0 ? 4 : 5] + 3 * col;
                f[0] = A2 * c.Sxz;
                f[1] = A2 * c.Syz;
                f[2] = A2 * c.Szz;
            }
        }
        szm_x = prev.Sxz;
        szm_y = prev.Syz;
        szm_z = prev.Szz;
        prev = m;
    };

    if (!ONEBAR) {
        int cslot = 0;                 // slot of the plane being converted (k = p - q0 + 3)
        int wpar = 0;                  // parity of the load in cslot
        int ik = 2, islot = 2;         // next load to issue
        for (int p = q0 - 3; p <= q1; ++p) {
            bool good = true;
            if (tid == 0) good = mbar_wait(smem_addr(&bars[cslot]), wpar);
            if (__syncthreads_or(!good)) {
                ok = false;
                break;
            }
            if (tid == 0 && ik < nplanes) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_box(smem_addr(raw + (size_t)islot * SLOT), &tmap, x0 - 2, y0 - 2,
                             q0 - 2 + ik, smem_addr(&bars[islot]), PLANE_BYTES);
            }
            ++ik;
            if (++islot == NSLOT) islot = 0;
            // u^{n-1} of this column's output plane p - 1, fetched before the stencil work
            const int q = p - 1;
            const bool write_out = q >= q0 && own_in;
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            if (write_out) u = a.sp[q * zstride + col];
            // 1. lambda -> mu for plane p + 1
            {
                float4* pl = raw + (size_t)cslot * SLOT;
                const int gz = p + 1;
                to_mu(a, pl[hp], cf_own, gx, gy, gz, own_in, has_obj);
                if (tid < NRIM2)
                    to_mu(a, pl[hc], cf_halo, x0 - 2 + cx, y0 - 2 + cy, gz, false, has_obj);
            }
            const int sl_p = cslot;                                   // plane p + 1
            const int sl_0 = cslot == 0 ? NSLOT - 1 : cslot - 1;      // plane p
            const int sl_m = sl_0 == 0 ? NSLOT - 1 : sl_0 - 1;        // plane p - 1
            if (++cslot == NSLOT) {
                cslot = 0;
                wpar ^= 1;
            }
            __syncthreads();
            if (p < q0 - 1) continue;
            plane(p, raw + (size_t)sl_m * SLOT, raw + (size_t)sl_0 * SLOT,
                  raw + (size_t)sl_p * SLOT, u, write_out);
        }
    } else {
        // one barrier per plane: iteration p converts plane p + 2 (load kc) while it forms the
        // moments of plane p from planes converted before the previous barrier
        int kc = 0;
        for (int p = q0 - 4; p <= q1; ++p, ++kc) {
            bool good = true;
            const int q = p - 1;
            const bool write_out = q >= q0 && own_in;
            float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
            if (write_out) u = a.sp[q * zstride + col];
            float4 nv = make_float4(0.f, 0.f, 0.f, 0.f);   // own mu of plane p + 2
            if (kc < nplanes) {
                good = mbar_wait_once(smem_addr(&bars[kc % NSLOT]), (kc / NSLOT) & 1);
                float4* pl = raw + (size_t)(kc % NSLOT) * SLOT;
                const int gz = p + 2;
                nv = pl[hp];
                to_mu(a, nv, cf_own, gx, gy, gz, own_in, has_obj);
                pl[hp] = nv;
                if (tid < NRIM2)
                    to_mu(a, pl[hc], cf_halo, x0 - 2 + cx, y0 - 2 + cy, gz, false, has_obj);
            }
            if (p >= q0 - 1)
                plane(p, raw + (size_t)((kc - 3) % NSLOT) * SLOT,
                      raw + (size_t)((kc - 2) % NSLOT) * SLOT,
                      raw + (size_t)((kc - 1) % NSLOT) * SLOT, u, write_out);
            own_m = own_0;
            own_0 = own_p;
            own_p = make_float2(nv.x, nv.w);
            if (__syncthreads_or(!good)) {
                ok = false;
                break;
            }
            // the slot of plane p - 1 (load kc - 3) is free: it takes load kc + 2
            const int kn = kc + 2;
            if (tid == 0 && kn >= NSLOT && kn < nplanes) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_box(smem_addr(raw + (size_t)(kn % NSLOT) * SLOT), &tmap, x0 - 2,
                             y0 - 2, q0 - 2 + kn, smem_addr(&bars[kn % NSLOT]), PLANE_BYTES);
            }
        }
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(a.err, 8);
            const long long t0 = clock64();
            while (clock64() - t0 < (1LL << 28)) {
            }
        }
        __syncthreads();
    }
}

// One-sided parts of the transposed gradient on non-periodic axes: node z within two rows of
// a face gets delta * (2 A S~_{.beta}) of the face node it projects to, with delta = -3/2,
// +3/2, -1/2 at rows 0, 1, 2 (low face) and +3/2, -3/2, +1/2 at rows n-1, n-2, n-3 (high face):
// the exact one-sided stencil minus the central one the fused kernel applied.
__global__ void k_adj_bcorr(Geom g, const float* __restrict__ face, FaceOffsets fo,
                            float4* __restrict__ lam) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // enumerate slabs of thickness 3 next to each face; a node near several faces is owned by
    // the first slab containing it
    const long long per[3] = {3LL * g.n[1] * g.n[2], 3LL * g.n[0] * g.n[2], 3LL * g.n[0] * g.n[1]};
    long long r = t;
    int slab = 0;
    while (slab < 6 && r >= per[slab / 2]) {
        r -= per[slab / 2];
        ++slab;
    }
    if (slab >= 6) return;
    const int ax = slab / 2;
    int c[3];
    const int b0 = (ax == 0) ? 1 : 0, b1 = (ax == 2) ? 1 : 2;
    const int layer = (int)((unsigned)r % 3u);
    const unsigned rr = (unsigned)r / 3u;
    c[ax] = (slab & 1) ? g.n[ax] - 1 - layer : layer;
    c[b0] = (int)(rr % (unsigned)g.n[b0]);
    c[b1] = (int)(rr / (unsigned)g.n[b0]);
    for (int e = 0; e < slab; ++e) {
        const int ae = e / 2;
        const int d = (e & 1) ? g.n[ae] - 1 - c[ae] : c[ae];
        if (d >= 0 && d <= 2) return;
    }
    float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int a = f / 2;
        const int d = (f & 1) ? g.n[a] - 1 - c[a] : c[a];
        if (d > 2) continue;
        const float lo[3] = {-1.5f, 1.5f, -0.5f};
        const float delta = (f & 1) ? -lo[d] : lo[d];
        const int e0 = (a == 0) ? 1 : 0, e1 = (a == 2) ? 1 : 2;
        const float* fp = face + fo.off[f] + 3 * ((long long)c[e1] * g.n[e0] + c[e0]);
        sx += delta * fp[0];
        sy += delta * fp[1];
        sz += delta * fp[2];
    }
    const long long m = ((long long)c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
    float4 v = lam[m];
    v.y += sx;
    v.z += sy;
    v.w += sz;
    lam[m] = v;
}

}  // namespace

void face_offsets(const Geom& g, FaceOffsets& fo, long long& total) {
    long long off = 0;
    for (int f = 0; f < 6; ++f) {
        const int a = f / 2;
        const int e0 = (a == 0) ? 1 : 0, e1 = (a == 2) ? 1 : 2;
        fo.off[f] = off;
        off += 3LL * g.n[e0] * g.n[e1];
    }
    total = off;
}

cudaError_t launch_fused_adj3d(const Geom& g, const V4<float>* lam_in, V4<float>* lam_out,
                               const V4<float>* kus, const V4<float>* sn, const V4<float>* sp,
                               float* e, float* face, double h, int* err, cudaStream_t st,
                               int variant) {
    CUtensorMap map;
    // a box one column wider than the tile: the unused last column pads the row pitch
    if (!encode_state_map(&map, lam_in, g, PX, HY)) return cudaErrorInvalidValue;
    static std::atomic<unsigned> attr{0};   // devices whose shared-memory limit is raised
    if (!device_done(attr)) {
        cudaError_t r = cudaFuncSetAttribute(k_fused_adj3d<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM_BYTES);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_fused_adj3d<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (r != cudaSuccess) return r;
        device_mark(attr);
    }
    AdjArgs a;
    a.g = g;
    a.lam_out = reinterpret_cast<float4*>(lam_out);
    a.kus = reinterpret_cast<const float4*>(kus);
    a.sn = reinterpret_cast<const float4*>(sn);
    a.sp = reinterpret_cast<const float4*>(sp);
    a.e = e;
    a.face = face;
    FaceOffsets fo;
    long long tot;
    face_offsets(g, fo, tot);
    for (int f = 0; f < 6; ++f) a.face_off[f] = fo.off[f];
    a.err = err;
    a.A9 = (float)(g.A / 9.0);
    a.obj_r = 0.f;
    a.obj_u[0] = a.obj_u[1] = a.obj_u[2] = 0.f;
    if (h != 0.0) {
        if (g.okind == 0) a.obj_r = (float)(-h / (3.0 * g.ocount));
        else
            for (int k = 0; k < 3; ++k) a.obj_u[k] = (float)(-h * g.odir[k] / g.ocount);
    }
    a.has_obj = (a.obj_r != 0.f || a.obj_u[0] != 0.f || a.obj_u[1] != 0.f || a.obj_u[2] != 0.f);
    const int tiles_x = (g.n[0] + TX - 1) / TX, tiles_y = (g.n[1] + TY - 1) / TY;
    a.zchunk = fused_zchunk_waves(g, (long long)tiles_x * tiles_y,
                                  variant == 1 ? adj_minb<true>() : adj_minb<false>());
    const int chunks = (g.n[2] + a.zchunk - 1) / a.zchunk;
    if (variant == 1)
        k_fused_adj3d<true><<<dim3(tiles_x, tiles_y, chunks), NTHR, SMEM_BYTES, st>>>(map, a);
    else
        k_fused_adj3d<false><<<dim3(tiles_x, tiles_y, chunks), NTHR, SMEM_BYTES, st>>>(map, a);
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    const long long shell = 6LL * ((long long)g.n[1] * g.n[2] + (long long)g.n[0] * g.n[2] +
                                   (long long)g.n[0] * g.n[1]);
    k_adj_bcorr<<<(unsigned)((shell + 255) / 256), 256, 0, st>>>(g, face, fo,
                                                                reinterpret_cast<float4*>(lam_out));
    return cudaGetLastError();
}

}  // namespace lks
