// Device-side helpers: lattice velocity sets, node classification, boundary rules and the
// velocity-gradient stencil.  Used by every kernel file of the library.
#pragma once

#include "lks_internal.h"

namespace lks {

// ------------------------------------------------------------------ lattices (Sec. 2.2)
// D2Q9: rest, 4 axes, 4 diagonals.  D3Q15: rest, 6 axes, 8 cube corners.  Standard weights
// (4/9, 1/9, 1/36) and (2/9, 1/9, 1/72).
template <int D>
struct Lat;

template <>
struct Lat<2> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int c(int i, int a) {
        // order: 0 | +x +y -x -y | (+,+) (-,+) (-,-) (+,-)
        return a == 0 ? ((i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0))
             : a == 1 ? ((i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0))
                      : 0;
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <>
struct Lat<3> {
    static constexpr int Q = 15;
    // order: 0 | +x -x +y -y +z -z | corners (sx,sy,sz) for k = 7..14 enumerated below
    __host__ __device__ static constexpr int corner(int k, int a) {
        // k = 0..7 -> signs of the 8 corners: bit a set -> -1
        return ((k >> a) & 1) ? -1 : 1;
    }
    __host__ __device__ static constexpr int c(int i, int a) {
        return i == 0 ? 0
             : i < 7 ? ((i - 1) / 2 == a ? ((i - 1) % 2 == 0 ? 1 : -1) : 0)
                     : corner(i - 7, a);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
};

// ------------------------------------------------------------------ weights as used
// The constants the kernels multiply by, per number type.  The scheme keeps a uniform state
// uniform only through exact identities of the lattice weights:
//   mass        w0 + 2D w1 + 2^D w2 = 1                (coefficient of rho - rho0 in rho*)
//   velocity    2 (3 w1) + 2^D (3 w2) = 1              (coefficient of u in u*, and of mu_u in
//                                                       3 U~ in the adjoint)
//   kinetic     2 (4.5 w1) + 2^D (4.5 w2) = 1.5         (the (c.u)^2 terms against -1.5 u^2)
//   adjoint     2 (9 w1) + 2^D (9 w2) = 3              (9 S~ against 3 R~)
// In double the nominal fractions satisfy them to rounding.  In single precision 1/9, 1/72 and
// 1/3 round so that, e.g., 2 fl(3 fl(1/9)) + 8 fl(3 fl(1/72)) = 1 + 3e-8: every step would
// multiply the velocity by that factor, a drift that grows over a flow-through time.  So the
// single-precision kernels multiply by separate constants w3_1 = "3 w1", w3_2 = "3 w2",
// h_1 = "4.5 w1", h_2 = "4.5 w2", s_1 = "9 w1", s_2 = "9 w2", chosen so that every identity
// above holds exactly for the stored values: h_1 = 1/2, h_2 = 4.5 w2 and s_1 = 1, s_2 = 9 w2
// are exact binary fractions; w3_1 = fl(1/3) and w3_2 = (1 - 2 w3_1) / 2^D, which is exact in
// binary; w1 = fl(1/9) and w2 one ulp below fl(w2 nominal), so that w0 = 1 - 2D w1 - 2^D w2 is
// a single-precision number.  Each differs from its nominal value by less than 1e-7 relative.
template <class T, int D>
struct Wts;

template <>
struct Wts<double, 3> {
    static constexpr double w0 = 2.0 / 9.0, w1 = 1.0 / 9.0, w2 = 1.0 / 72.0;
    static constexpr double w3_1 = 1.0 / 3.0, w3_2 = 1.0 / 24.0;
    static constexpr double h_1 = 0.5, h_2 = 0.0625, s_1 = 1.0, s_2 = 0.125;
};
template <>
struct Wts<double, 2> {
    static constexpr double w0 = 4.0 / 9.0, w1 = 1.0 / 9.0, w2 = 1.0 / 36.0;
    static constexpr double w3_1 = 1.0 / 3.0, w3_2 = 1.0 / 12.0;
    static constexpr double h_1 = 0.5, h_2 = 0.125, s_1 = 1.0, s_2 = 0.25;
};
template <>
struct Wts<float, 3> {
    static constexpr float w0 = 0x1.c71c72p-3f, w1 = 0x1.c71c72p-4f, w2 = 0x1.c71c70p-7f;
    static constexpr float w3_1 = 0x1.555556p-2f, w3_2 = 0x1.555554p-5f;
    static constexpr float h_1 = 0.5f, h_2 = 0.0625f, s_1 = 1.0f, s_2 = 0.125f;
};
template <>
struct Wts<float, 2> {
    static constexpr float w0 = 0x1.c71c72p-2f, w1 = 0x1.c71c72p-4f, w2 = 0x1.c71c70p-6f;
    static constexpr float w3_1 = 0x1.555556p-2f, w3_2 = 0x1.555554p-4f;
    static constexpr float h_1 = 0.5f, h_2 = 0.125f, s_1 = 1.0f, s_2 = 0.25f;
};

// The identities, checked at compile time (each sum is exact in double).
template <class W, int D>
constexpr bool weights_consistent() {
    return (double)W::w0 + 2.0 * D * (double)W::w1 + (double)(1 << D) * (double)W::w2 == 1.0 &&
           2.0 * (double)W::w3_1 + (double)(1 << D) * (double)W::w3_2 == 1.0 &&
           2.0 * (double)W::h_1 + (double)(1 << D) * (double)W::h_2 == 1.5 &&
           2.0 * (double)W::s_1 + (double)(1 << D) * (double)W::s_2 == 3.0;
}
static_assert(weights_consistent<Wts<float, 3>, 3>(), "D3Q15 single-precision weights");
static_assert(weights_consistent<Wts<float, 2>, 2>(), "D2Q9 single-precision weights");

// ------------------------------------------------------------------ indexing

__device__ __forceinline__ long long node_index(const Geom& g, int x, int y, int z) {
    return ((long long)z * g.n[1] + y) * g.n[0] + x;
}

__device__ __forceinline__ int wrapi(int i, int n) {
    i = (i < 0) ? i + n : i;
    return (i >= n) ? i - n : i;
}

__device__ __forceinline__ bool is_boundary(const Geom& g, int x, int y, int z) {
    const int c[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a < g.dim && !g.periodic[a] && (c[a] == 0 || c[a] == g.n[a] - 1)) return true;
    return false;
}

__device__ __forceinline__ bool in_box(const Geom& g, int x, int y, int z, long long& bi) {
    int bx = x - g.blo[0], by = y - g.blo[1], bz = z - g.blo[2];
    if (g.boxN == 0 || bx < 0 || by < 0 || bz < 0 || bx >= g.bn[0] || by >= g.bn[1] ||
        bz >= g.bn[2])
        return false;
    bi = ((long long)bz * g.bn[1] + by) * g.bn[0] + bx;
    return true;
}

__device__ __forceinline__ bool in_target(const Geom& g, int x, int y, int z) {
    if (x < g.obox[0] || x > g.obox[1] || y < g.obox[2] || y > g.obox[3]) return false;
    if (g.dim == 3 && (z < g.obox[4] || z > g.obox[5])) return false;
    if (g.ocyl_r > 0.0) {
        double dx = x - g.ocyl_c[0], dy = y - g.ocyl_c[1];
        if (dx * dx + dy * dy > g.ocyl_r * g.ocyl_r) return false;
    }
    return true;
}

// ------------------------------------------------------------------ boundary rules
// Boundary node b copies the unprescribed quantities from the interior node one step inward
// along each boundary normal it lies on.  The face that decides b's type is the one with the
// highest precedence (WALL > INLET > OUTLET), ties to the lower face index.

__device__ __forceinline__ int bc_prec(int t) {
    return t == BC_WALL ? 3 : (t == BC_INLET ? 2 : (t == BC_OUTLET ? 1 : 0));
}

// Winning face of a boundary node given which faces it lies on (side[a]: -1 none, 0 low, 1 high).
__device__ __forceinline__ int winning_face(const Geom& g, const int side[3]) {
    int best = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (side[a] < 0) continue;
        int f = 2 * a + side[a];
        if (best < 0 || bc_prec(g.bc[f]) > bc_prec(g.bc[best])) best = f;
    }
    return best;
}

// Value of boundary node (winning face f) given its source node's value v.
template <class T>
__device__ __forceinline__ V4<T> bc_value(const Geom& g, int f, const V4<T>& v) {
    V4<T> b;
    int t = g.bc[f];
    if (t == BC_WALL || t == BC_INLET) {
        b.r = v.r;
        b.x = (T)g.bcv[f][0];
        b.y = (T)g.bcv[f][1];
        b.z = (g.dim == 3) ? (T)g.bcv[f][2] : (T)0;
    } else {
        int na = f / 2;
        b.r = (T)(g.bcv[f][3] - g.rho0);
        b.x = (na == 0) ? v.x : (T)g.bcv[f][0];
        b.y = (na == 1) ? v.y : (T)g.bcv[f][1];
        b.z = (g.dim == 3) ? ((na == 2) ? v.z : (T)g.bcv[f][2]) : (T)0;
    }
    return b;
}

// Visit every boundary node whose copy source is interior node (x, y, z): fn(bx, by, bz, face)
// with the winning face of that boundary node.  Along each non-periodic axis the node can step
// out to the low face (coordinate 1) and/or the high face (coordinate n-2); every non-empty
// combination of such steps is one boundary node.  Fully unrolled, so no local arrays.
template <class F>
__device__ __forceinline__ void for_each_sourced_boundary(const Geom& g, int x, int y, int z,
                                                          F&& fn) {
    const int c[3] = {x, y, z};
#pragma unroll
    for (int mx = 0; mx < 3; ++mx)
#pragma unroll
        for (int my = 0; my < 3; ++my)
#pragma unroll
            for (int mz = 0; mz < 3; ++mz) {
                if (mx == 0 && my == 0 && mz == 0) continue;
                const int m[3] = {mx, my, mz};
                bool ok = true;
                int b[3], side[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    b[a] = c[a];
                    side[a] = -1;
                    if (m[a] == 0) continue;
                    const bool active = a < g.dim && !g.periodic[a];
                    if (m[a] == 1) {
                        ok = ok && active && c[a] == 1;
                        b[a] = 0;
                        side[a] = 0;
                    } else {
                        ok = ok && active && c[a] == g.n[a] - 2;
                        b[a] = g.n[a] - 1;
                        side[a] = 1;
                    }
                }
                if (!ok) continue;
                fn(b[0], b[1], b[2], winning_face(g, side));
            }
}

// True if interior node (x, y, z) is the copy source of some boundary node.
__device__ __forceinline__ bool sources_boundary(const Geom& g, int x, int y, int z) {
    const int c[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a < g.dim && !g.periodic[a] && (c[a] == 1 || c[a] == g.n[a] - 2)) return true;
    return false;
}

// Write every boundary node whose copy source is interior node (x,y,z) holding value v.
template <class T>
__device__ __forceinline__ void write_bc_from(const Geom& g, int x, int y, int z,
                                              const V4<T>& v, V4<T>* s) {
    if (!sources_boundary(g, x, y, z)) return;
    for_each_sourced_boundary(g, x, y, z, [&](int bx, int by, int bz, int f) {
        s[node_index(g, bx, by, bz)] = bc_value(g, f, v);
    });
}

// ------------------------------------------------------------------ gradient stencil
// First derivative along an axis: central difference, periodic wrap, and the second-order
// one-sided difference on a non-periodic boundary node (the reading taken for the velocity
// gradient of f^eq).  coef(i, off): weight of row i's stencil at offset off (0 if none).
__device__ __forceinline__ double deriv_coef(int i, int n, int periodic, int off) {
    if (periodic) return off == 1 ? 0.5 : (off == -1 ? -0.5 : 0.0);
    if (i == 0) return off == 0 ? -1.5 : (off == 1 ? 2.0 : (off == 2 ? -0.5 : 0.0));
    if (i == n - 1) return off == 0 ? 1.5 : (off == -1 ? -2.0 : (off == -2 ? 0.5 : 0.0));
    return off == 1 ? 0.5 : (off == -1 ? -0.5 : 0.0);
}

// Peskin four-point cosine kernel w(r) = (1 + cos(pi r / 2)) / 4 for |r| < 2 (Sec. 2.3).
__device__ __forceinline__ double peskin(double r) {
    return fabs(r) < 2.0 ? 0.25 * (1.0 + cospi(0.5 * r)) : 0.0;
}
__device__ __forceinline__ float peskin(float r) {
    return fabsf(r) < 2.0f ? 0.25f * (1.0f + cospif(0.5f * r)) : 0.0f;
}

}  // namespace lks
