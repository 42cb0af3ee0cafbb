// Per-unit device bodies shared by the single-context kernels and the instance-table kernels
// (one launch over many contexts), so both run exactly the same arithmetic per node, design
// column or boundary node.
#pragma once

#include "lks_device.cuh"

namespace lks {

// ---------------------------------------------------------------- design positions (Sec. 2.3)
// x_ref, y_ref of design column k (FP64) as integer base + fraction in [0,1).
template <class T>
__device__ __forceinline__ void design_col_pos(const Design& d, const Motion& m,
                                               const TransferScratch& ts, long long k) {
    T* frac = (T*)ts.col_frac;
    const int i = (int)((unsigned)k % (unsigned)d.L[0]), j = (int)((unsigned)k / (unsigned)d.L[0]);
    const double dx = i - d.xiG[0], dy = j - d.xiG[1];
    const double xr = m.c * dx - m.s * dy + m.xG[0];   // Eq. rigid_body_position
    const double yr = m.s * dx + m.c * dy + m.xG[1];
    const double bx = floor(xr), by = floor(yr);
    ts.col_base[2 * k] = (int)bx;
    ts.col_base[2 * k + 1] = (int)by;
    frac[2 * k] = (T)(xr - bx);
    frac[2 * k + 1] = (T)(yr - by);
}

// ---------------------------------------------------------------- 2D transfer (table path)
// Design column k for the D2Q9 instance-table kernels: integer base of x_ref, y_ref (FP64, as
// design_col_pos) and, per axis, S = sin(pi f/2), C = cos(pi f/2) of the fraction f.  The four
// taps of the cosine kernel then follow without further trigonometry: for an analysis node at
// base + q, q = -1, 0, 1, 2, w = (1 - S)/4, (1 + C)/4, (1 + S)/4, (1 - C)/4 (w(r) =
// (1 + cos(pi r/2))/4 at r = q - f).
// x_ref = x_G + a da - b db of one axis in single precision without losing the fraction:
// Dekker's exact product split (with fma) and Knuth's two-sum carry the rounding errors, so
// base + frac equals x_ref to about 1e-12 although every operation is FP32 (GB300's FP64 rate is
// a small fraction of its FP32 rate).  Returns the integer base; frac in [0, 1).
__device__ __forceinline__ int ref_coord(float ah, float al, float da, float bh, float bl,
                                         float db, int gi, float gh, float gl, float& frac) {
    const float p = ah * da, pe = fmaf(ah, da, -p);     // a_hi da = p + pe exactly
    const float q = bh * db, qe = fmaf(bh, db, -q);     // b_hi db = q + qe exactly
    const float r = p - q, rb = r - p;
    const float re = (p - (r - rb)) + (-q - rb);        // p - q = r + re exactly
    const float t = r + gh, tb = t - r;
    const float te = (r - (t - tb)) + (gh - tb);        // r + gh = t + te exactly
    const float lo = ((te + re) + (pe - qe)) + (fmaf(al, da, -bl * db) + gl);
    float fl = floorf(t);
    float f = (t - fl) + lo;                            // t - floor(t) is exact
    if (f < 0.f) {
        f += 1.f;
        fl -= 1.f;
    } else if (f >= 1.f) {
        f -= 1.f;
        fl += 1.f;
    }
    frac = f;
    return gi + (int)fl;
}

__device__ __forceinline__ void col_pos_sc(const Design& d, const Motion& m, long long k, int2& b,
                                           float4& sc) {
    const int i = (int)((unsigned)k % (unsigned)d.L[0]), j = (int)((unsigned)k / (unsigned)d.L[0]);
    const float dx = (float)i - d.xiGf[0], dy = (float)j - d.xiGf[1];
    float fx, fy;   // Eq. rigid_body_position: x_ref = c dx - s dy + x_G, y_ref = s dx + c dy + y_G
    b.x = ref_coord(m.ch, m.cl, dx, m.sh, m.sl, dy, m.xgi[0], m.xgh[0], m.xgl[0], fx);
    b.y = ref_coord(m.sh, m.sl, dx, -m.ch, -m.cl, dy, m.xgi[1], m.xgh[1], m.xgl[1], fy);
    sincospif(0.5f * fx, &sc.x, &sc.y);
    sincospif(0.5f * fy, &sc.z, &sc.w);
}


__device__ __forceinline__ float tap_weight(int q1, float S, float C) {
    // q1 = q + 1 in 0..3
    const float t = q1 == 0 ? -S : (q1 == 1 ? C : (q1 == 2 ? S : -C));
    return 0.25f * (1.f + t);
}

// kappa(x) = sum_xi W(x - x_ref(xi)) kappa_ref(xi) and u_S = omega R'(theta) m1 + u_G m0 with
// m0 = sum W, m1 = sum W (xi - xi_G) at box node bi (Eqs. brinkman_ref, velocity_ref; u_ref is
// affine in xi).  The design nodes whose taps cover x are found through the inverse rigid map
// (a window widened against rounding) and summed in design index order.
__device__ __forceinline__ void transfer2d_node(const Design& d, const Geom& g, const Motion& m,
                                                const int2* __restrict__ pb,
                                                const float4* __restrict__ psc,
                                                const float* __restrict__ kref,
                                                V4<float>* kus, long long bi) {
    const int x = g.blo[0] + (int)((unsigned)bi % (unsigned)g.bn[0]);
    const int y = g.blo[1] + (int)((unsigned)bi / (unsigned)g.bn[0]);
    const float c = m.cf, s = m.sf;
    const float px = (float)x - m.xgf[0], py = (float)y - m.xgf[1];
    const float ic = c * px + s * py + d.xiGf[0];
    const float jc = -s * px + c * py + d.xiGf[1];
    const float R = 2.f * (fabsf(c) + fabsf(s)) + 0.01f;
    const int i0 = max(0, (int)ceilf(ic - R)), i1 = min(d.L[0] - 1, (int)floorf(ic + R));
    const int j0 = max(0, (int)ceilf(jc - R)), j1 = min(d.L[1] - 1, (int)floorf(jc + R));
    const float gx0 = d.xiGf[0], gy0 = d.xiGf[1];
    float kap = 0.f, m0 = 0.f, m1x = 0.f, m1y = 0.f;
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
            const int k = j * d.L[0] + i;
            const int2 b = __ldg(pb + k);
            const int qx = x - b.x + 1, qy = y - b.y + 1;
            if ((unsigned)qx > 3u || (unsigned)qy > 3u) continue;
            const float4 sc = __ldg(psc + k);
            const float W = tap_weight(qx, sc.x, sc.y) * tap_weight(qy, sc.z, sc.w);
            kap += W * __ldg(kref + k);
            m0 += W;
            m1x += W * ((float)i - gx0);
            m1y += W * ((float)j - gy0);
        }
    const float om = m.omf;
    V4<float> o;
    o.r = kap;
    o.x = (-s * m1x - c * m1y) * om + m.ugf[0] * m0;
    o.y = (c * m1x - s * m1y) * om + m.ugf[1] * m0;
    o.z = 0.f;
    kus[bi] = o;
}

// Sensitivity gather for design node k on the table path: sum over its 4 x 4 taps of
// W e(x) with the same tap weights as transfer2d_node (the node's position at the step formed
// here, by the same function), times kappa', added to dJ/dgamma (FP64).
__device__ __forceinline__ void sens2d_node(const Design& d, const Geom& g, const Motion& m,
                                            const float* __restrict__ e,
                                            const float* __restrict__ kprime,
                                            double* __restrict__ gacc, long long k) {
    int2 b;
    float4 sc;
    col_pos_sc(d, m, k, b, sc);
    const int ex0 = b.x - 1 - g.blo[0], ey0 = b.y - 1 - g.blo[1];
    float acc = 0.f;
#pragma unroll
    for (int ty = 0; ty < 4; ++ty) {
        const int ey = ey0 + ty;
        if (ey < 0 || ey >= g.bn[1]) continue;
        const float wy = tap_weight(ty, sc.z, sc.w);
#pragma unroll
        for (int tx = 0; tx < 4; ++tx) {
            const int ex = ex0 + tx;
            if (ex < 0 || ex >= g.bn[0]) continue;
            acc += (tap_weight(tx, sc.x, sc.y) * wy) * e[(long long)ey * g.bn[0] + ex];
        }
    }
    gacc[k] += (double)kprime[k] * (double)acc;
}

// ---------------------------------------------------------------- sensitivity gather (Sec. 2.4)
// For design column k and kSensRun planes from z0: sum_x W(x - x_ref) e(x) over the support (the
// transpose of the kappa transfer), times kappa', added to dJ/dgamma in FP64.  The z shift is
// the same for every design plane, so each analysis plane's 4 x 4 x-y tap sum is formed once
// and the four z weights slide over them.
constexpr int kSensRun = 4;

template <class T>
__device__ __forceinline__ void sens_run(const Design& d, const Geom& g, const TransferScratch& ts,
                                         const T* __restrict__ e, const T* __restrict__ kprime,
                                         double* __restrict__ gacc, long long t) {
    const unsigned k = (unsigned)t % (unsigned)d.ncol;   // design column
    const int z0 = (int)((unsigned)t / (unsigned)d.ncol) * kSensRun;
    const int z1 = min(d.L[2], z0 + kSensRun);
    const T* frac = (const T*)ts.col_frac;
    const int bx = ts.col_base[2 * k], by = ts.col_base[2 * k + 1];
    const T fx = frac[2 * k], fy = frac[2 * k + 1];
    T wx[4], wy[4], wz[4];
    const T fz = ((const T*)ts.dz_frac)[0];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        wx[q] = peskin((T)(q - 1) - fx);
        wy[q] = peskin((T)(q - 1) - fy);
        wz[q] = (g.dim == 3) ? peskin((T)(q - 1) - fz) : (q == 1 ? (T)1 : (T)0);
    }
    const int ex0 = bx - 1 - g.blo[0], ey0 = by - 1 - g.blo[1];
    // x-y tap sum of analysis plane z (0 outside the box, where W vanishes)
    auto plane_sum = [&](int z) -> T {
        const int ez = z - g.blo[2];
        if (ez < 0 || ez >= g.bn[2]) return (T)0;
        const T* ep = e + (long long)ez * g.bn[1] * g.bn[0];
        T acc = (T)0;
#pragma unroll
        for (int ty = 0; ty < 4; ++ty) {
            const int ey = ey0 + ty;
            if (ey < 0 || ey >= g.bn[1] || wy[ty] == (T)0) continue;
#pragma unroll
            for (int tx = 0; tx < 4; ++tx) {
                const int ex = ex0 + tx;
                const T W = wx[tx] * wy[ty];
                if (ex < 0 || ex >= g.bn[0] || W == (T)0) continue;
                acc += W * ep[(long long)ey * g.bn[0] + ex];
            }
        }
        return acc;
    };
    const int zb0 = (g.dim == 3) ? ts.dz_base[z0] : 0;   // analysis base plane of design plane z0
    T s0 = plane_sum(zb0 - 1), s1 = plane_sum(zb0), s2 = plane_sum(zb0 + 1);
    for (int zeta = z0; zeta < z1; ++zeta) {
        const int zb = zb0 + (zeta - z0);
        const T s3 = (g.dim == 3) ? plane_sum(zb + 2) : (T)0;
        const T acc = wz[0] * s0 + wz[1] * s1 + wz[2] * s2 + wz[3] * s3;
        const long long dn = (long long)zeta * d.ncol + k;
        gacc[dn] += (double)kprime[dn] * (double)acc;
        s0 = s1;
        s1 = s2;
        s2 = s3;
    }
}

// ---------------------------------------------------------------- objective (Sec. 2.5)
// j = -(rho0 + mean(rho - rho0))/3 (J1) or -mean(n.u) (J2) over the target list, one block of
// kObjThreads threads, fixed-order FP64 reduction.
constexpr int kObjThreads = 256;

template <class T>
__device__ __forceinline__ void objective_block(const Geom& g, const V4<T>* __restrict__ s,
                                                double* jstep) {
    __shared__ double red[kObjThreads];
    const int tot = (int)g.ocount;
    double acc = 0.0;
    for (int k = threadIdx.x; k < tot; k += kObjThreads) {
        const V4<T> v = s[g.otarget[k]];
        if (g.okind == 0)
            acc += (double)v.r;
        else
            acc += g.odir[0] * (double)v.x + g.odir[1] * (double)v.y + g.odir[2] * (double)v.z;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kObjThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double sum = red[0];
        jstep[0] = (g.okind == 0) ? -(g.rho0 + sum / g.ocount) / 3.0 : -sum / g.ocount;
    }
    __syncthreads();
}

// Objective's direct adjoint source at one node (h = window weight or 0 outside the window).
// Objective source h_n dj/ds at a target node (Sec. 2.5) in the precision T of the state, formed
// on the host in FP64 and rounded once: the device never divides in FP64.
template <class T>
struct ObjAdd {
    T r, x, y, z;
    int on;   // h_n != 0
};
template <class T>
inline ObjAdd<T> obj_add(const Geom& g, double h) {
    ObjAdd<T> o;
    o.on = h != 0.0;
    o.r = o.x = o.y = o.z = (T)0;
    if (h == 0.0) return o;
    if (g.okind == 0) {
        o.r = (T)(-h / (3.0 * g.ocount));
    } else {
        o.x = (T)(-h * g.odir[0] / g.ocount);
        o.y = (T)(-h * g.odir[1] / g.ocount);
        o.z = (T)(-h * g.odir[2] / g.ocount);
    }
    return o;
}

template <class T>
__device__ __forceinline__ void obj_source(const Geom& g, int x, int y, int z, const ObjAdd<T>& o,
                                           V4<T>& l) {
    if (!o.on || !in_target(g, x, y, z)) return;
    if (g.okind == 0) {
        l.r += o.r;
    } else {
        l.x += o.x;
        l.y += o.y;
        l.z += o.z;
    }
}

// ---------------------------------------------------------------- boundary transpose
// Transpose of the boundary copies at interior node (x, y, z): it collects the copied
// components of the boundary nodes it sources (WALL/INLET copy rho, OUTLET copies the normal
// velocity), after their objective source.  Boundary nodes are read only; later kernels treat
// them as zero.
// bcT_gather adds those components to acc (the node's own value); bcT_node stores the sum.
template <class T>
__device__ __forceinline__ void bcT_gather(const Geom& g, const V4<T>* lam, const ObjAdd<T>& h,
                                           int x, int y, int z, V4<T>& acc) {
    for_each_sourced_boundary(g, x, y, z, [&](int bx, int by, int bz, int f) {
        V4<T> lb = lam[node_index(g, bx, by, bz)];
        obj_source(g, bx, by, bz, h, lb);
        const int t = g.bc[f];
        if (t == BC_WALL || t == BC_INLET) {
            acc.r += lb.r;
        } else {
            const int na = f / 2;
            if (na == 0) acc.x += lb.x;
            if (na == 1) acc.y += lb.y;
            if (na == 2) acc.z += lb.z;
        }
    });
}

template <class T>
__device__ __forceinline__ void bcT_node(const Geom& g, V4<T>* lam, const ObjAdd<T>& h, int x,
                                         int y, int z) {
    if (!sources_boundary(g, x, y, z)) return;
    const long long m = node_index(g, x, y, z);
    V4<T> acc = lam[m];
    bcT_gather<T>(g, lam, h, x, y, z, acc);
    lam[m] = acc;
}

}  // namespace lks
