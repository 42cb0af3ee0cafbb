// Design-grid kernels: the Brinkman interpolation kappa_ref(gamma) (Sec. 2.3), the per-step
// transfer of kappa and u_S from the rigidly moved design grid onto the analysis grid
// (Eqs. brinkman_ref, velocity_ref with Peskin's cosine kernel) and its transpose, the design
// sensitivity gather (Sec. 2.4).
//
// The rotation is in the x-y plane (about z in 3D, as in Sec. 3.3), so the kernel weight
// W = w(dx) w(dy) w(dz) separates into an x-y part that is the same for every design plane and
// a z part that is the same for every design column.  Per step:
//   k_design_pos  x_ref, y_ref of every design column (FP64) as integer base + fraction, and
//                 the z taps of every analysis plane of the footprint box;
//   k_tap_lists   for each analysis column of the box, the design columns whose support covers
//                 it (found through the inverse rigid map) with their x-y weights, in design
//                 index order, the moments m0 = sum W, m1 = sum W (xi - xi_G), and for every
//                 design plane the x-y transfer of kappa_ref;
//   k_fill        kappa = sum over the z taps of that, u_S = omega R'(theta) m1 + u_G m0, on
//                 the box: deterministic gathers, no atomics;
//   k_sens        for each design node, sum_x W(x - x_ref) e(x) over its 4^d support (the
//                 transpose of the kappa transfer), accumulated into dJ/dgamma in FP64.
#include "lks_units.cuh"

namespace lks {

namespace {

constexpr int kThreads = 256;
constexpr int kSmallThreads = 64;
inline unsigned grid_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__global__ void k_design_prep_check(long long nd, const double* gamma, int* bad) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= nd) return;
    const double gm = gamma[k];
    if (!(gm >= 0.0 && gm <= 1.0)) atomicOr(bad, 1);
}

template <class T>
__global__ void k_design_prep(long long nd, long long ncol, int lz,
                              const double* __restrict__ gamma, double kmax, double q,
                              T* __restrict__ kref, T* __restrict__ kref_t,
                              T* __restrict__ kprime) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= nd) return;
    const double gm = gamma[k];
    const double d = (1.0 - gm) + q;
    const T kr = (T)(kmax * q * gm / d);             // kappa_ref (Sec. 2.3)
    kref[k] = kr;
    kref_t[(k % ncol) * lz + k / ncol] = kr;         // [column][zeta] copy for the transfer
    kprime[k] = (T)(kmax * q * (1.0 + q) / (d * d));   // d kappa_ref / d gamma
}

template <class T>
__global__ void k_design_pos(Design d, Geom g, Motion m, TransferScratch ts) {
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < d.ncol) {
        design_col_pos<T>(d, m, ts, k);
        return;
    }
    k -= d.ncol;
    const int lz = d.L[2];
    if (k < lz) {  // moved z of design plane k (3D: pure shift; 2D: the single plane at 0)
        T* dzf = (T*)ts.dz_frac;
        if (g.dim == 3) {
            const double zr = (double)k - d.xiG[2] + m.xG[2];
            const double bz = floor(zr);
            ts.dz_base[k] = (int)bz;
            dzf[k] = (T)(zr - bz);
        } else {
            ts.dz_base[k] = 0;
            dzf[k] = (T)0;
        }
        return;
    }
    k -= lz;
    if (k < g.bn[2]) {  // z taps of analysis plane blo_z + k
        int* zi = ts.zt_idx + 4 * k;
        T* zw = (T*)ts.zt_w + 4 * k;
        for (int t = 0; t < 4; ++t) {
            zi[t] = -1;
            zw[t] = (T)0;
        }
        if (g.dim == 2) {
            zi[0] = 0;
            zw[0] = (T)1;
            return;
        }
        const int z = g.blo[2] + (int)k;
        const double shift = m.xG[2] - d.xiG[2];       // z_ref(zeta) = zeta + shift
        const int z0 = (int)floor((double)z - shift) - 1;
        int cnt = 0;
        for (int t = 0; t < 4; ++t) {
            const int zeta = z0 + t;
            if (zeta < 0 || zeta >= lz) continue;
            const double zr = (double)zeta + shift;
            const double bz = floor(zr);
            const T r = (T)(z - (int)bz) - (T)(zr - bz);
            if (!(fabs((double)r) < 2.0)) continue;
            const T w = peskin(r);
            if (w == (T)0) continue;
            zi[cnt] = zeta;
            zw[cnt] = w;
            ++cnt;
        }
    }
}

// One warp per box column.  The lanes test the candidate design columns of a window around the
// inverse rigid map (j outer, i inner, 32 at a time); a ballot keeps the accepted ones in that
// order, and every lane sums the moments over them in the same order, so the lists and sums are
// those of a sequential scan.  The window is found in single precision with a margin far above
// its rounding: it only has to contain the support, each candidate is tested exactly.  The warp
// then forms K2[col][zeta] = sum over the taps of W_xy kappa_ref(zeta, tap), the x-y transfer of
// every design plane, lanes running along zeta (coalesced in kref_t), taps in list order.
constexpr int kTapWarps = kThreads / 32;

template <class T>
__global__ void __launch_bounds__(kThreads)
    k_tap_lists(Design d, Geom g, Motion m, TransferScratch ts, const T* __restrict__ kref_t,
                T* __restrict__ k2) {
    __shared__ T s_w[kTapWarps][kMaxTaps];
    __shared__ int s_k[kTapWarps][kMaxTaps];
    const long long ncols = (long long)g.bn[0] * g.bn[1];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long col = (long long)blockIdx.x * kTapWarps + wid;
    if (col >= ncols) return;   // whole warps
    const int x = g.blo[0] + (int)(col % g.bn[0]);
    const int y = g.blo[1] + (int)(col / g.bn[0]);
    // inverse rigid map: design coordinates of this analysis column
    const float px = (float)x - m.xgf[0], py = (float)y - m.xgf[1];
    const float ic = fmaf(m.cf, px, fmaf(m.sf, py, d.xiGf[0]));
    const float jc = fmaf(-m.sf, px, fmaf(m.cf, py, d.xiGf[1]));
    const float R = 2.f * (fabsf(m.cf) + fabsf(m.sf)) + 0.01f;
    const int i0 = max(0, (int)ceilf(ic - R)), i1 = min(d.L[0] - 1, (int)floorf(ic + R));
    const int j0 = max(0, (int)ceilf(jc - R)), j1 = min(d.L[1] - 1, (int)floorf(jc + R));
    const int wi = i1 - i0 + 1;
    const int nc = (wi > 0 && j1 >= j0) ? wi * (j1 - j0 + 1) : 0;
    // xi - xi_G in T: from the single-precision centre where that is exact
    const bool fxi = sizeof(T) == 4 && (double)d.xiGf[0] == d.xiG[0] &&
                     (double)d.xiGf[1] == d.xiG[1];
    const T* frac = (const T*)ts.col_frac;
    int* tidx = ts.tap_idx + col * kMaxTaps;
    T* tw = (T*)ts.tap_w + col * kMaxTaps;
    int cnt = 0;
    bool over = false;
    T m0 = (T)0, m1x = (T)0, m1y = (T)0;
    for (int b = 0; b < nc && !over; b += 32) {
        const int c = b + lane;
        int k = 0;
        T W = (T)0, di = (T)0, dj = (T)0;
        if (c < nc) {
            const int j = j0 + c / wi, i = i0 + c % wi;
            k = j * d.L[0] + i;
            const T rx = (T)(x - ts.col_base[2 * k]) - frac[2 * k];
            const T ry = (T)(y - ts.col_base[2 * k + 1]) - frac[2 * k + 1];
            if (fabs(rx) < (T)2 && fabs(ry) < (T)2) W = peskin(rx) * peskin(ry);   // exact in T
            di = fxi ? (T)((float)i - d.xiGf[0]) : (T)(i - d.xiG[0]);
            dj = fxi ? (T)((float)j - d.xiGf[1]) : (T)(j - d.xiG[1]);
        }
        const unsigned acc = __ballot_sync(0xffffffffu, W != (T)0);
        const int pos = cnt + __popc(acc & ((1u << lane) - 1u));
        if (W != (T)0 && pos < kMaxTaps) {
            tidx[pos] = k;
            tw[pos] = W;
            s_k[wid][pos] = k;
            s_w[wid][pos] = W;
        }
        for (unsigned r = acc; r != 0u; r &= r - 1u) {   // warp-uniform: taps in window order
            if (cnt == kMaxTaps) {
                over = true;
                break;
            }
            const int src = __ffs(r) - 1;
            const T Ws = __shfl_sync(0xffffffffu, W, src);
            m0 += Ws;
            m1x += Ws * __shfl_sync(0xffffffffu, di, src);
            m1y += Ws * __shfl_sync(0xffffffffu, dj, src);
            ++cnt;
        }
    }
    if (lane == 0) {
        if (over) atomicOr(ts.err, 1);
        ts.tap_cnt[col] = cnt;
        T* cm = (T*)ts.col_m + 3 * col;
        cm[0] = m0;
        cm[1] = m1x;
        cm[2] = m1y;
    }
    __syncwarp();
    const int lz = d.L[2];
    const T* sw = s_w[wid];
    const int* sk = s_k[wid];
    for (int z = lane; z < lz; z += 32) {
        T a = (T)0;
#pragma unroll 4
        for (int e = 0; e < cnt; ++e) a += sw[e] * kref_t[(long long)sk[e] * lz + z];
        k2[col * lz + z] = a;
    }
}

// The same lists, moments and plane sums with one thread per box column, for transfers with few
// design planes over many columns (large 2D boxes): there a box column is a single node, and a
// warp per column would leave its lanes idle over the plane sums.
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_tap_lists_col(Design d, Geom g, Motion m, TransferScratch ts, const T* __restrict__ kref_t,
                    T* __restrict__ k2) {
    const long long ncols = (long long)g.bn[0] * g.bn[1];
    const long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    const int x = g.blo[0] + (int)(col % g.bn[0]);
    const int y = g.blo[1] + (int)(col / g.bn[0]);
    const float px = (float)x - m.xgf[0], py = (float)y - m.xgf[1];
    const float ic = fmaf(m.cf, px, fmaf(m.sf, py, d.xiGf[0]));
    const float jc = fmaf(-m.sf, px, fmaf(m.cf, py, d.xiGf[1]));
    const float R = 2.f * (fabsf(m.cf) + fabsf(m.sf)) + 0.01f;
    const int i0 = max(0, (int)ceilf(ic - R)), i1 = min(d.L[0] - 1, (int)floorf(ic + R));
    const int j0 = max(0, (int)ceilf(jc - R)), j1 = min(d.L[1] - 1, (int)floorf(jc + R));
    const T* frac = (const T*)ts.col_frac;
    int* tidx = ts.tap_idx + col * kMaxTaps;
    T* tw = (T*)ts.tap_w + col * kMaxTaps;
    int cnt = 0;
    T m0 = (T)0, m1x = (T)0, m1y = (T)0;
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
            const int k = j * d.L[0] + i;
            const T rx = (T)(x - ts.col_base[2 * k]) - frac[2 * k];
            const T ry = (T)(y - ts.col_base[2 * k + 1]) - frac[2 * k + 1];
            if (!(fabs(rx) < (T)2 && fabs(ry) < (T)2)) continue;   // exact in T
            const T W = peskin(rx) * peskin(ry);
            if (W == (T)0) continue;
            if (cnt == kMaxTaps) {
                atomicOr(ts.err, 1);
                i = i1;
                j = j1;
                break;
            }
            tidx[cnt] = k;
            tw[cnt] = W;
            ++cnt;
            m0 += W;
            m1x += W * (T)(i - d.xiG[0]);
            m1y += W * (T)(j - d.xiG[1]);
        }
    ts.tap_cnt[col] = cnt;
    T* cm = (T*)ts.col_m + 3 * col;
    cm[0] = m0;
    cm[1] = m1x;
    cm[2] = m1y;
    const int lz = d.L[2];
    for (int z = 0; z < lz; ++z) {
        T a = (T)0;
        for (int e = 0; e < cnt; ++e) a += tw[e] * kref_t[(long long)tidx[e] * lz + z];
        k2[col * lz + z] = a;
    }
}

// The fill: kappa = sum over the z taps of w_z K2 and u_S = m_z (omega R'(theta) m1 + u_G m0)
// on every node of the footprint box (u_ref is affine in xi, Eq. rigid_body_velocity).  A block
// covers 32 box columns x 8 box planes; the K2 values those planes need (a window of at most
// 11 consecutive zeta, the z map being a translation) are staged in shared memory with
// contiguous reads along zeta, so that the node loop reads no strided global data.
constexpr int kFillCols = 32, kFillPlanes = 8, kFillSpan = kFillPlanes + 3;

template <class T>
__global__ void __launch_bounds__(kFillCols * kFillPlanes)
    k_fill(Design d, Geom g, Motion m, TransferScratch ts, const T* __restrict__ k2,
           V4<T>* __restrict__ kus) {
    __shared__ T sk[kFillCols][kFillSpan + 1];
    __shared__ int zlo_s;
    const long long ncols = (long long)g.bn[0] * g.bn[1];
    const int lc = threadIdx.x % kFillCols, lb = threadIdx.x / kFillCols;
    const long long col0 = (long long)blockIdx.x * kFillCols;
    const int bz0 = blockIdx.y * kFillPlanes;
    if (threadIdx.x == 0) {   // lowest design plane any of the block's box planes reads
        int lo = 1 << 30;
        for (int b = bz0; b < min(bz0 + kFillPlanes, g.bn[2]); ++b)
            for (int t = 0; t < 4; ++t) {
                const int z = ts.zt_idx[4 * b + t];
                if (z >= 0) lo = min(lo, z);
            }
        zlo_s = lo;
    }
    __syncthreads();
    const int zlo = zlo_s;
    for (int i = threadIdx.x; i < kFillCols * kFillSpan; i += blockDim.x) {
        const int c = i / kFillSpan, z = i % kFillSpan;
        const long long col = col0 + c;
        T v = (T)0;
        if (col < ncols && zlo + z < d.L[2]) v = k2[col * d.L[2] + zlo + z];
        sk[c][z] = v;
    }
    __syncthreads();
    const long long col = col0 + lc;
    const int bz = bz0 + lb;
    if (col >= ncols || bz >= g.bn[2]) return;
    const int* zi = ts.zt_idx + 4 * bz;
    const T* zw = (const T*)ts.zt_w + 4 * bz;
    T kap = (T)0, mz = (T)0;
    for (int t = 0; t < 4; ++t) {
        const int zeta = zi[t];
        if (zeta < 0) continue;
        mz += zw[t];
        const int r = zeta - zlo;
        const T kz = (r < kFillSpan) ? sk[lc][r] : k2[col * d.L[2] + zeta];
        kap += zw[t] * kz;
    }
    const T* cm = (const T*)ts.col_m + 3 * col;
    // single-precision motion fields for T = float (the same roundings as converting here)
    const bool f32 = sizeof(T) == 4;
    const T om = f32 ? (T)m.omf : (T)m.om, c = f32 ? (T)m.cf : (T)m.c, s = f32 ? (T)m.sf : (T)m.s;
    const T ug0 = f32 ? (T)m.ugf[0] : (T)m.uG[0], ug1 = f32 ? (T)m.ugf[1] : (T)m.uG[1];
    const T ug2 = f32 ? (T)m.ugf[2] : (T)m.uG[2];
    V4<T> o;
    o.r = kap;
    o.x = mz * ((-s * cm[1] - c * cm[2]) * om + ug0 * cm[0]);
    o.y = mz * ((c * cm[1] - s * cm[2]) * om + ug1 * cm[0]);
    o.z = (g.dim == 3) ? mz * (ug2 * cm[0]) : (T)0;
    kus[(long long)bz * ncols + col] = o;
}

// Sensitivity gather: one thread per design column and kSensRun planes (sens_run).
template <class T>
__global__ void k_sens(Design d, Geom g, TransferScratch ts, const T* __restrict__ e,
                       const T* __restrict__ kprime, double* __restrict__ gacc) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const unsigned runs = (unsigned)((d.L[2] + kSensRun - 1) / kSensRun);
    if (t >= (long long)d.ncol * runs) return;
    sens_run<T>(d, g, ts, e, kprime, gacc, t);
}

template <class T>
__global__ void k_box_to_grid(Geom g, const V4<T>* __restrict__ kus, double* kappa, double* us) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    const unsigned t = (unsigned)m / (unsigned)g.n[0];
    const int x = (int)((unsigned)m - t * (unsigned)g.n[0]);
    const int y = (int)(t % (unsigned)g.n[1]), z = (int)(t / (unsigned)g.n[1]);
    long long bi;
    double k = 0, a = 0, b = 0, c = 0;
    if (in_box(g, x, y, z, bi)) {
        const V4<T> v = kus[bi];
        k = v.r;
        a = v.x;
        b = v.y;
        c = v.z;
    }
    kappa[m] = k;
    us[m] = a;
    us[g.nodes + m] = b;
    us[2 * g.nodes + m] = c;
}

// ---------------------------------------------------------------- design chain
// Density filter with linear weights w = max(0, R - |xi_i - xi_j|) over the design grid and the
// tanh Heaviside projection (the projection filter the paper cites, Secs. 1 and 3.1), in FP64:
// gb = H(F gamma), hp = H'(F gamma), wsum = sum_j w_ij.  One thread per design node, offsets
// visited in (z, y, x) order.
__global__ void k_filter(Design d, double R, int rr, double beta, double eta,
                         const double* __restrict__ gamma, double* __restrict__ gb,
                         double* __restrict__ hp, double* __restrict__ wsum) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= d.nd) return;
    const int x = (int)(k % d.L[0]), y = (int)((k / d.L[0]) % d.L[1]), z = (int)(k / d.ncol);
    const int rz = d.L[2] > 1 ? rr : 0;
    double acc = 0.0, W = 0.0;
    for (int dz = -rz; dz <= rz; ++dz)
        for (int dy = -rr; dy <= rr; ++dy)
            for (int dx = -rr; dx <= rr; ++dx) {
                const double w = R - sqrt((double)(dx * dx + dy * dy + dz * dz));
                if (!(w > 0.0)) continue;
                const int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx < 0 || yy < 0 || zz < 0 || xx >= d.L[0] || yy >= d.L[1] || zz >= d.L[2])
                    continue;
                acc += w * gamma[((long long)zz * d.L[1] + yy) * d.L[0] + xx];
                W += w;
            }
    const double gt = acc / W;
    const double den = tanh(beta * eta) + tanh(beta * (1.0 - eta));
    const double t = tanh(beta * (gt - eta));
    gb[k] = (tanh(beta * eta) + t) / den;
    hp[k] = beta * (1.0 - t * t) / den;
    wsum[k] = W;
}

// Transposed chain: out_j = sum_i w_ij hp_i g_i / wsum_i (a gather over the same offsets).
__global__ void k_filter_T(Design d, double R, int rr, const double* __restrict__ g,
                           const double* __restrict__ hp, const double* __restrict__ wsum,
                           double* __restrict__ out) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= d.nd) return;
    const int x = (int)(k % d.L[0]), y = (int)((k / d.L[0]) % d.L[1]), z = (int)(k / d.ncol);
    const int rz = d.L[2] > 1 ? rr : 0;
    double acc = 0.0;
    for (int dz = -rz; dz <= rz; ++dz)
        for (int dy = -rr; dy <= rr; ++dy)
            for (int dx = -rr; dx <= rr; ++dx) {
                const double w = R - sqrt((double)(dx * dx + dy * dy + dz * dz));
                if (!(w > 0.0)) continue;
                const int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx < 0 || yy < 0 || zz < 0 || xx >= d.L[0] || yy >= d.L[1] || zz >= d.L[2])
                    continue;
                const long long i = ((long long)zz * d.L[1] + yy) * d.L[0] + xx;
                acc += w * (hp ? hp[i] * g[i] : g[i]) / wsum[i];
            }
    out[k] = acc;
}

// sum of a design field in a fixed order (one block, FP64 tree), for the volume constraint.
__global__ void k_design_sum(long long nd, const double* __restrict__ a, double* out) {
    __shared__ double red[kThreads];
    double acc = 0.0;
    for (long long k = threadIdx.x; k < nd; k += kThreads) acc += a[k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_fill_f64(long long n, double v, double* a) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) a[k] = v;
}

}  // namespace

void launch_fill_f64(double* a, long long n, double v, cudaStream_t st) {
    if (n > 0) k_fill_f64<<<grid_for(n), kThreads, 0, st>>>(n, v, a);
}

void launch_filter(const Design& d, double R, double beta, double eta, const double* gamma,
                   double* gb, double* hp, double* wsum, cudaStream_t st) {
    if (d.nd == 0) return;
    k_filter<<<grid_for(d.nd), kThreads, 0, st>>>(d, R, (int)ceil(R), beta, eta, gamma, gb, hp,
                                                  wsum);
}

void launch_filter_T(const Design& d, double R, const double* g, const double* hp,
                     const double* wsum, double* out, cudaStream_t st) {
    if (d.nd == 0) return;
    k_filter_T<<<grid_for(d.nd), kThreads, 0, st>>>(d, R, (int)ceil(R), g, hp, wsum, out);
}

void launch_design_sum(long long nd, const double* a, double* out, cudaStream_t st) {
    k_design_sum<<<1, kThreads, 0, st>>>(nd, a, out);
}

template <class T>
void launch_design_prep(const Design& d, const double* gamma, double kappa_max, double q,
                        T* kref, T* kref_t, T* kprime, int* bad, cudaStream_t st) {
    if (d.nd == 0) return;
    k_design_prep_check<<<grid_for(d.nd), kThreads, 0, st>>>(d.nd, gamma, bad);
    k_design_prep<T><<<grid_for(d.nd), kThreads, 0, st>>>(d.nd, d.ncol, d.L[2], gamma, kappa_max,
                                                          q, kref, kref_t, kprime);
}

template <class T>
void launch_design_pos(const Design& d, const Geom& g, const Motion& m, TransferScratch ts,
                       cudaStream_t st) {
    if (d.nd == 0 || g.boxN == 0) return;
    const long long n = d.ncol + d.L[2] + g.bn[2];
    // small blocks: these grids are a few hundred to a few thousand threads, and their
    // dependent scattered reads want as many SMs as possible
    k_design_pos<T><<<(unsigned)((n + kSmallThreads - 1) / kSmallThreads), kSmallThreads, 0, st>>>(
        d, g, m, ts);
}

template <class T>
void launch_transfer(const Design& d, const Geom& g, const Motion& m, TransferScratch ts,
                     const T* kref_t, T* k2, V4<T>* kus, cudaStream_t st) {
    if (d.nd == 0 || g.boxN == 0) return;
    const long long ncols = (long long)g.bn[0] * g.bn[1];
    // a warp per column while the warps stay few or the planes many; one thread per column for
    // the large single-plane boxes of 2D transfers
    if (d.L[2] >= 8 || ncols <= 16384)
        k_tap_lists<T><<<(unsigned)((ncols + kTapWarps - 1) / kTapWarps), kThreads, 0, st>>>(
            d, g, m, ts, kref_t, k2);
    else
        k_tap_lists_col<T><<<(unsigned)((ncols + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            d, g, m, ts, kref_t, k2);
    const dim3 fgrd((unsigned)((ncols + kFillCols - 1) / kFillCols),
                    (unsigned)((g.bn[2] + kFillPlanes - 1) / kFillPlanes));
    k_fill<T><<<fgrd, kFillCols * kFillPlanes, 0, st>>>(d, g, m, ts, k2, kus);
}

template <class T>
void launch_sens(const Design& d, const Geom& g, TransferScratch ts, const T* e,
                 const T* kprime, double* gacc, cudaStream_t st) {
    if (d.nd == 0 || g.boxN == 0) return;
    const long long n = d.ncol * ((d.L[2] + kSensRun - 1) / kSensRun);
    k_sens<T><<<grid_for(n), kThreads, 0, st>>>(d, g, ts, e, kprime, gacc);
}

template <class T>
void launch_box_to_grid(const Geom& g, const V4<T>* kus, double* kappa, double* us,
                        cudaStream_t st) {
    k_box_to_grid<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, kus, kappa, us);
}

#define LKS_INST_T(T)                                                                        \
    template void launch_design_prep<T>(const Design&, const double*, double, double, T*, T*, \
                                        T*, int*, cudaStream_t);                             \
    template void launch_design_pos<T>(const Design&, const Geom&, const Motion&,             \
                                       TransferScratch, cudaStream_t);                       \
    template void launch_transfer<T>(const Design&, const Geom&, const Motion&,               \
                                     TransferScratch, const T*, T*, V4<T>*, cudaStream_t);   \
    template void launch_sens<T>(const Design&, const Geom&, TransferScratch, const T*,       \
                                 const T*, double*, cudaStream_t);                           \
    template void launch_box_to_grid<T>(const Geom&, const V4<T>*, double*, double*,          \
                                        cudaStream_t);

LKS_INST_T(float)
LKS_INST_T(double)

}  // namespace lks
