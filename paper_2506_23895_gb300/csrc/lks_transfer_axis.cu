// Transfer and sensitivity gather for a design grid rotating about a general 3D axis (Sec. 2.3,
// Eqs. brinkman_ref, velocity_ref with R(theta) from Rodrigues' formula).  The kernel weight
// no longer separates into a column part and a z part, so the gather goes through cell lists:
//   k_ga_pos    x_ref of every design node (FP64) as integer base + fraction;
//   k_ga_cells  for every cell of the footprint box, the design nodes whose base is that cell,
//               found through the inverse rigid map (at most 8: the preimage of a unit cell
//               is a unit cube, which holds at most 8 points at mutual distance >= 1) and
//               listed in design index order;
//   k_ga_fill   kappa = sum W kappa_ref and u_S = omega a x (R m1) + u_G m0 on every box node,
//               gathered from the cells base in [x - 2, x + 1]^3 whose taps cover it;
//   k_ga_sens   per design node, sum of W e(x) over its 4^3 taps, times kappa' (FP64).
// Deterministic gathers throughout; no atomics.
#include "lks_units.cuh"

namespace lks {

namespace {

constexpr int kThreads = 256;
inline unsigned grid_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ void design_coords(const Design& d, long long k, int& i, int& j,
                                              int& l) {
    i = (int)(k % d.L[0]);
    j = (int)((k / d.L[0]) % d.L[1]);
    l = (int)(k / d.ncol);
}

template <class T>
__global__ void k_ga_pos(Design d, Motion m, int4* __restrict__ base, V4<T>* __restrict__ frac) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= d.nd) return;
    int i, j, l;
    design_coords(d, k, i, j, l);
    const double dv[3] = {i - d.xiG[0], j - d.xiG[1], l - d.xiG[2]};
    int b[3];
    T f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double xr = m.R[3 * a] * dv[0] + m.R[3 * a + 1] * dv[1] + m.R[3 * a + 2] * dv[2] +
                          m.xG[a];   // Eq. rigid_body_position
        const double fl = floor(xr);
        b[a] = (int)fl;
        f[a] = (T)(xr - fl);
    }
    base[k] = make_int4(b[0], b[1], b[2], 0);
    V4<T> o;
    o.r = f[0];
    o.x = f[1];
    o.y = f[2];
    o.z = (T)0;
    frac[k] = o;
}

// Cell lists over the footprint box: cnt[c], idx[c][kCellMax].
template <class T>
__global__ void k_ga_cells(Design d, Geom g, Motion m, const int4* __restrict__ base,
                           int* __restrict__ cnt, int* __restrict__ idx) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= g.boxN) return;
    const int cx = g.blo[0] + (int)(c % g.bn[0]);
    const int cy = g.blo[1] + (int)((c / g.bn[0]) % g.bn[1]);
    const int cz = g.blo[2] + (int)(c / ((long long)g.bn[0] * g.bn[1]));
    // preimage of the cell's centre: xi = R^T (x + 1/2 - x_G) + xi_G
    const double p[3] = {cx + 0.5 - m.xG[0], cy + 0.5 - m.xG[1], cz + 0.5 - m.xG[2]};
    int lo[3], hi[3];
    const double h = 0.8660254037844387 + 1e-6;   // half the diagonal of a unit cube
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double xi = m.R[a] * p[0] + m.R[3 + a] * p[1] + m.R[6 + a] * p[2] + d.xiG[a];
        lo[a] = max(0, (int)ceil(xi - h));
        hi[a] = min(d.L[a] - 1, (int)floor(xi + h));
    }
    int n = 0;
    int* out = idx + c * kCellMax;
    for (int l = lo[2]; l <= hi[2]; ++l)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                const long long k = ((long long)l * d.L[1] + j) * d.L[0] + i;
                const int4 b = base[k];
                if (b.x == cx && b.y == cy && b.z == cz && n < kCellMax) out[n++] = (int)k;
            }
    cnt[c] = n;
}

template <class T>
__global__ void k_ga_fill(Design d, Geom g, Motion m, const int* __restrict__ cnt,
                          const int* __restrict__ idx, const int4* __restrict__ base,
                          const V4<T>* __restrict__ frac, const T* __restrict__ kref,
                          V4<T>* __restrict__ kus) {
    const long long bi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (bi >= g.boxN) return;
    const long long plane = (long long)g.bn[0] * g.bn[1];
    const int bx = (int)(bi % g.bn[0]), by = (int)((bi / g.bn[0]) % g.bn[1]),
              bz = (int)(bi / plane);
    const int x = g.blo[0] + bx, y = g.blo[1] + by, z = g.blo[2] + bz;
    T kap = (T)0, m0 = (T)0, m1[3] = {(T)0, (T)0, (T)0};
    for (int qz = -2; qz <= 1; ++qz) {
        const int ez = bz + qz;
        if (ez < 0 || ez >= g.bn[2]) continue;
        for (int qy = -2; qy <= 1; ++qy) {
            const int ey = by + qy;
            if (ey < 0 || ey >= g.bn[1]) continue;
            for (int qx = -2; qx <= 1; ++qx) {
                const int ex = bx + qx;
                if (ex < 0 || ex >= g.bn[0]) continue;
                const long long c = ez * plane + (long long)ey * g.bn[0] + ex;
                const int nc = cnt[c];
                for (int e = 0; e < nc; ++e) {
                    const int k = idx[c * kCellMax + e];
                    const int4 b = base[k];
                    const V4<T> f = frac[k];
                    const T W = peskin((T)(x - b.x) - f.r) * peskin((T)(y - b.y) - f.x) *
                                peskin((T)(z - b.z) - f.y);
                    int i, j, l;
                    design_coords(d, k, i, j, l);
                    kap += W * kref[k];
                    m0 += W;
                    m1[0] += W * (T)(i - d.xiG[0]);
                    m1[1] += W * (T)(j - d.xiG[1]);
                    m1[2] += W * (T)(l - d.xiG[2]);
                }
            }
        }
    }
    // u_S = omega a x (R m1) + u_G m0 (u_ref is affine in xi, Eq. rigid_body_velocity)
    T rm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        rm[a] = (T)m.R[3 * a] * m1[0] + (T)m.R[3 * a + 1] * m1[1] + (T)m.R[3 * a + 2] * m1[2];
    const T ax = (T)m.ax[0], ay = (T)m.ax[1], az = (T)m.ax[2], om = (T)m.om;
    V4<T> o;
    o.r = kap;
    o.x = om * (ay * rm[2] - az * rm[1]) + (T)m.uG[0] * m0;
    o.y = om * (az * rm[0] - ax * rm[2]) + (T)m.uG[1] * m0;
    o.z = om * (ax * rm[1] - ay * rm[0]) + (T)m.uG[2] * m0;
    kus[bi] = o;
}

template <class T>
__global__ void k_ga_sens(Design d, Geom g, const int4* __restrict__ base,
                          const V4<T>* __restrict__ frac, const T* __restrict__ e,
                          const T* __restrict__ kprime, double* __restrict__ gacc) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= d.nd) return;
    const int4 b = base[k];
    const V4<T> f = frac[k];
    T wx[4], wy[4], wz[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        wx[q] = peskin((T)(q - 1) - f.r);
        wy[q] = peskin((T)(q - 1) - f.x);
        wz[q] = peskin((T)(q - 1) - f.y);
    }
    const long long plane = (long long)g.bn[0] * g.bn[1];
    T acc = (T)0;
    for (int tz = 0; tz < 4; ++tz) {
        const int ez = b.z - 1 + tz - g.blo[2];
        if (ez < 0 || ez >= g.bn[2]) continue;
        for (int ty = 0; ty < 4; ++ty) {
            const int ey = b.y - 1 + ty - g.blo[1];
            if (ey < 0 || ey >= g.bn[1]) continue;
            for (int tx = 0; tx < 4; ++tx) {
                const int ex = b.x - 1 + tx - g.blo[0];
                if (ex < 0 || ex >= g.bn[0]) continue;
                acc += (wx[tx] * wy[ty] * wz[tz]) * e[ez * plane + (long long)ey * g.bn[0] + ex];
            }
        }
    }
    gacc[k] += (double)kprime[k] * (double)acc;
}

}  // namespace

template <class T>
void launch_transfer_axis(const Design& d, const Geom& g, const Motion& m, AxisScratch as,
                          const T* kref, V4<T>* kus, cudaStream_t st) {
    if (d.nd == 0 || g.boxN == 0) return;
    k_ga_pos<T><<<grid_for(d.nd), kThreads, 0, st>>>(d, m, as.base, (V4<T>*)as.frac);
    k_ga_cells<T><<<grid_for(g.boxN), kThreads, 0, st>>>(d, g, m, as.base, as.cnt, as.idx);
    k_ga_fill<T><<<grid_for(g.boxN), kThreads, 0, st>>>(d, g, m, as.cnt, as.idx, as.base,
                                                        (const V4<T>*)as.frac, kref, kus);
}

template <class T>
void launch_sens_axis(const Design& d, const Geom& g, AxisScratch as, const T* e,
                      const T* kprime, double* gacc, cudaStream_t st) {
    if (d.nd == 0 || g.boxN == 0) return;
    k_ga_sens<T><<<grid_for(d.nd), kThreads, 0, st>>>(d, g, as.base, (const V4<T>*)as.frac, e,
                                                      kprime, gacc);
}

template void launch_transfer_axis<float>(const Design&, const Geom&, const Motion&, AxisScratch,
                                          const float*, V4<float>*, cudaStream_t);
template void launch_transfer_axis<double>(const Design&, const Geom&, const Motion&,
                                           AxisScratch, const double*, V4<double>*, cudaStream_t);
template void launch_sens_axis<float>(const Design&, const Geom&, AxisScratch, const float*,
                                      const float*, double*, cudaStream_t);
template void launch_sens_axis<double>(const Design&, const Geom&, AxisScratch, const double*,
                                       const double*, double*, cudaStream_t);

}  // namespace lks
