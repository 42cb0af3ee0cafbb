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

// ---------------------------------------------------------------- 2D transfer, one box node
// kappa(x) = sum_xi W(x - x_ref(xi)) kappa_ref(xi) and u_S = omega R'(theta) m1 + u_G m0 with
// m0 = sum W, m1 = sum W (xi - xi_G) (Eqs. brinkman_ref, velocity_ref; u_ref is affine in xi).
// The design nodes whose support covers x are found through the inverse rigid map and summed
// in design index order.
template <class T>
__device__ __forceinline__ void transfer2d_node(const Design& d, const Geom& g, const Motion& m,
                                                const TransferScratch& ts,
                                                const T* __restrict__ kref, V4<T>* kus,
                                                long long bi) {
    const int x = g.blo[0] + (int)((unsigned)bi % (unsigned)g.bn[0]);
    const int y = g.blo[1] + (int)((unsigned)bi / (unsigned)g.bn[0]);
    const double px = x - m.xG[0], py = y - m.xG[1];
    const double ic = m.c * px + m.s * py + d.xiG[0];
    const double jc = -m.s * px + m.c * py + d.xiG[1];
    const double R = 2.0 * (fabs(m.c) + fabs(m.s)) + 1e-6;
    const int i0 = max(0, (int)ceil(ic - R)), i1 = min(d.L[0] - 1, (int)floor(ic + R));
    const int j0 = max(0, (int)ceil(jc - R)), j1 = min(d.L[1] - 1, (int)floor(jc + R));
    const T* frac = (const T*)ts.col_frac;
    T kap = (T)0, m0 = (T)0, m1x = (T)0, m1y = (T)0;
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
            const long long k = (long long)j * d.L[0] + i;
            const T rx = (T)(x - ts.col_base[2 * k]) - frac[2 * k];
            const T ry = (T)(y - ts.col_base[2 * k + 1]) - frac[2 * k + 1];
            if (!(fabs((double)rx) < 2.0 && fabs((double)ry) < 2.0)) continue;
            const T W = peskin(rx) * peskin(ry);
            if (W == (T)0) continue;
            kap += W * kref[k];
            m0 += W;
            m1x += W * (T)(i - d.xiG[0]);
            m1y += W * (T)(j - d.xiG[1]);
        }
    const T om = (T)m.om, c = (T)m.c, s = (T)m.s;
    V4<T> o;
    o.r = kap;
    o.x = (-s * m1x - c * m1y) * om + (T)m.uG[0] * m0;
    o.y = (c * m1x - s * m1y) * om + (T)m.uG[1] * m0;
    o.z = (T)0;
    kus[bi] = o;
}

// ---------------------------------------------------------------- sensitivity gather (Sec. 2.4)
// For design column k and kSensRun planes from z0: sum_x W(x - x_ref) e(x) over the support (the
// transpose of the kappa transfer), times kappa', added to dJ/dgamma in FP64.  The z shift is
// the same for every design plane, so each analysis plane's 4 x 4 x-y tap sum is formed once
// and the four z weights slide over them.
constexpr int kSensRun = 8;

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
template <class T>
__device__ __forceinline__ void obj_source(const Geom& g, int x, int y, int z, double h,
                                           V4<T>& l) {
    if (h == 0.0 || !in_target(g, x, y, z)) return;
    if (g.okind == 0) {
        l.r += (T)(-h / (3.0 * g.ocount));
    } else {
        l.x += (T)(-h * g.odir[0] / g.ocount);
        l.y += (T)(-h * g.odir[1] / g.ocount);
        l.z += (T)(-h * g.odir[2] / g.ocount);
    }
}

// Window weight h_n of step n: 1/(window length) inside the window, else 0.
__host__ __device__ __forceinline__ double window_weight(int n, int wb, int we) {
    const double h = 1.0 / (double)(we - wb + 1);
    return (n >= wb && n <= we) ? h : 0.0;
}

// ---------------------------------------------------------------- boundary transpose
// Transpose of the boundary copies at interior node (x, y, z): it collects the copied
// components of the boundary nodes it sources (WALL/INLET copy rho, OUTLET copies the normal
// velocity), after their objective source.  Boundary nodes are read only; later kernels treat
// them as zero.
template <class T>
__device__ __forceinline__ void bcT_node(const Geom& g, V4<T>* lam, double h, int x, int y,
                                         int z) {
    if (!sources_boundary(g, x, y, z)) return;
    const long long m = node_index(g, x, y, z);
    V4<T> acc = lam[m];
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
    lam[m] = acc;
}

}  // namespace lks
