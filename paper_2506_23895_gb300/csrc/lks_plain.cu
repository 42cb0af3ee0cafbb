// Plain per-node kernels of the LKS step and its exact discrete adjoint.
//
// Forward step (Alg. 1): k_feq evaluates f_i^eq at every node from the old state (Sec. 2.2,
// equilibrium with the viscosity term) into a Q-plane scratch, k_gather sums f_i^eq(x - c_i)
// into rho*, u* (Eqs. rho, u), applies the Brinkman update u = (u* + kappa u_S)/(1 + kappa)
// (Eq. u_ex_2) and writes the boundary nodes sourced from each interior node (Eqs. bc_rho,
// bc_u).  Adjoint step (Alg. 2 structure, exact transpose of the above): k_adj_bcT pushes
// boundary adjoints onto their copy sources, k_adj_mu divides by (1 + kappa) and forms the
// kappa sensitivity density e, k_adj_moments gathers F~_i(y) = mu_rho(y+c_i) + c_i.mu_u(y+c_i)
// into the moments of Eqs. arho, au, as and the adjoint equilibrium, k_adj_divT adds the
// transposed velocity-gradient term.  These kernels are templated on the scalar type; the
// double instantiation is the plain FP64 path.
#include "lks_units.cuh"

namespace lks {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ void node_coords(const Geom& g, long long m, int& x, int& y, int& z) {
    // node counts are below 2^31 (checked at create): 32-bit division
    const unsigned mu = (unsigned)m, nx = (unsigned)g.n[0], ny = (unsigned)g.n[1];
    const unsigned t = mu / nx;
    x = (int)(mu - t * nx);
    y = (int)(t % ny);
    z = (int)(t / ny);
}

template <class T>
__global__ void k_init_state(Geom g, V4<T>* s) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    V4<T> v;
    v.r = (T)0;
    v.x = (T)0;
    v.y = (T)0;
    v.z = (T)0;
    s[m] = v;
}

template <class T>
__global__ void k_fill_uniform(Geom g, V4<T>* s, T ux, T uy, T uz) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    V4<T> v;
    v.r = (T)0;
    v.x = ux;
    v.y = uy;
    v.z = uz;
    s[m] = v;
}

// Every boundary node takes its value from its copy source (used for initial states).
template <class T>
__global__ void k_apply_bc(Geom g, V4<T>* s) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    int x, y, z;
    node_coords(g, m, x, y, z);
    if (is_boundary(g, x, y, z)) return;
    write_bc_from(g, x, y, z, s[m], s);
}

// f_i^eq of one node (Sec. 2.2) from rho - rho0, u and S = G + G^T (G_ab = d u_a / d x_b):
// the symmetric part of each opposite-direction pair (c, -c) is formed once and the pair
// differs only in the sign of 3 c.u; the weight products are those of Wts<T, D>.  Writes the
// Q values in the order of Lat<D>.
template <class T>
__device__ __forceinline__ void feq_pairs3(const V4<T>& v, const T S[3][3], T A, T* __restrict__ F,
                                           long long stride) {
    using W = Wts<T, 3>;
    const T ux = v.x, uy = v.y, uz = v.z;
    const T P = v.r - (T)1.5 * (ux * ux + uy * uy + uz * uz);
    F[0] = W::w0 * P;
    const T u[3] = {ux, uy, uz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {   // axes: directions 1 + 2a (+) and 2 + 2a (-)
        const T sym = W::w1 * (P + A * S[a][a]) + W::h_1 * u[a] * u[a];
        F[(1 + 2 * a) * stride] = sym + W::w3_1 * u[a];
        F[(2 + 2 * a) * stride] = sym - W::w3_1 * u[a];
    }
    const T tr = S[0][0] + S[1][1] + S[2][2];
    // corners k = 0..3 have sz = +1 (directions 7..10), their opposites are 14..11:
    // c.S.c = tr S + 2 (sx sy S_xy + sx S_xz + sy S_yz)
    const T base = W::w2 * (P + A * tr), A2w = (T)2 * A * W::w2;
    const T xy = A2w * S[0][1], xz = A2w * S[0][2], yz = A2w * S[1][2];
    const T cross[4] = {xy + xz + yz, -xy - xz + yz, -xy + xz - yz, xy - xz - yz};
    const T cuv[4] = {ux + uy + uz, -ux + uy + uz, ux - uy + uz, -ux - uy + uz};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T cu = cuv[k];
        const T sym = (base + cross[k]) + W::h_2 * cu * cu;
        F[(7 + k) * stride] = sym + W::w3_2 * cu;
        F[(14 - k) * stride] = sym - W::w3_2 * cu;
    }
}

template <class T>
__device__ __forceinline__ void feq_pairs2(const V4<T>& v, const T S[3][3], T A, T* __restrict__ F,
                                           long long stride) {
    using W = Wts<T, 2>;
    const T ux = v.x, uy = v.y;
    const T P = v.r - (T)1.5 * (ux * ux + uy * uy);
    F[0] = W::w0 * P;
    const T u[2] = {ux, uy};
#pragma unroll
    for (int a = 0; a < 2; ++a) {   // axes: +a is direction 1 + a, -a is 3 + a
        const T sym = W::w1 * (P + A * S[a][a]) + W::h_1 * u[a] * u[a];
        F[(1 + a) * stride] = sym + W::w3_1 * u[a];
        F[(3 + a) * stride] = sym - W::w3_1 * u[a];
    }
    const T tr = S[0][0] + S[1][1];
    // diagonals (+,+) = 5 with (-,-) = 7, (-,+) = 6 with (+,-) = 8
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const T sx = k ? (T)-1 : (T)1;
        const T cu = sx * ux + uy;
        const T sym = W::w2 * (P + A * (tr + (T)2 * sx * S[0][1])) + W::h_2 * cu * cu;
        F[(5 + k) * stride] = sym + W::w3_2 * cu;
        F[(7 + k) * stride] = sym - W::w3_2 * cu;
    }
}

template <class T, int D>
__global__ void k_feq(Geom g, const V4<T>* __restrict__ s, T* __restrict__ F) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    int c[3];
    node_coords(g, m, c[0], c[1], c[2]);
    const V4<T> v = s[m];
    T G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[a][b] = (T)0;
    bool inner = true;   // central differences along every axis without a wrap
#pragma unroll
    for (int b = 0; b < D; ++b) inner = inner && c[b] >= 1 && c[b] <= g.n[b] - 2;
    if (inner) {
        long long st = 1;
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const V4<T> wp = s[m + st], wm = s[m - st];
            G[0][b] = (T)0.5 * (wp.x - wm.x);
            G[1][b] = (T)0.5 * (wp.y - wm.y);
            if (D == 3) G[2][b] = (T)0.5 * (wp.z - wm.z);
            st *= g.n[b];
        }
    } else {
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const int i = c[b], n = g.n[b], per = g.periodic[b];
#pragma unroll
            for (int off = -2; off <= 2; ++off) {
                const T cf = (T)deriv_coef(i, n, per, off);
                if (cf == (T)0) continue;
                int q[3] = {c[0], c[1], c[2]};
                q[b] = wrapi(i + off, n);
                const V4<T> w = s[node_index(g, q[0], q[1], q[2])];
                G[0][b] += cf * w.x;
                G[1][b] += cf * w.y;
                if (D == 3) G[2][b] += cf * w.z;
            }
        }
    }
    T S[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) S[a][b] = G[a][b] + G[b][a];
    if (D == 3) feq_pairs3<T>(v, S, (T)g.A, F + m, g.nodes);
    else feq_pairs2<T>(v, S, (T)g.A, F + m, g.nodes);
}

template <class T, int D>
__global__ void k_gather(Geom g, const T* __restrict__ F, const V4<T>* __restrict__ kus,
                         V4<T>* __restrict__ out) {
    using L = Lat<D>;
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    int x, y, z;
    node_coords(g, m, x, y, z);
    if (is_boundary(g, x, y, z)) return;
    T rs = (T)0, us[3] = {(T)0, (T)0, (T)0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int xs = wrapi(x - L::c(i, 0), g.n[0]);
        const int ys = wrapi(y - L::c(i, 1), g.n[1]);
        const int zs = (D == 3) ? wrapi(z - L::c(i, 2), g.n[2]) : 0;
        const T f = F[(long long)i * g.nodes + node_index(g, xs, ys, zs)];
        rs += f;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (L::c(i, a) != 0) us[a] += (T)L::c(i, a) * f;
    }
    V4<T> o;
    o.r = rs;
    long long bi;
    // a static solid adds kappa_s (solid velocity 0) to the Brinkman denominator
    const T kst = g.ks ? ((const T*)g.ks)[m] : (T)0;
    if (in_box(g, x, y, z, bi)) {
        const V4<T> ks = kus[bi];
        const T k = ks.r, inv = (T)1 / ((T)1 + k + kst);
        o.x = (us[0] + (T)g.body[0] + k * ks.x) * inv;
        o.y = (us[1] + (T)g.body[1] + k * ks.y) * inv;
        o.z = (D == 3) ? (us[2] + (T)g.body[2] + k * ks.z) * inv : (T)0;
    } else if (kst != (T)0) {
        const T inv = (T)1 / ((T)1 + kst);
        o.x = (us[0] + (T)g.body[0]) * inv;
        o.y = (us[1] + (T)g.body[1]) * inv;
        o.z = (D == 3) ? (us[2] + (T)g.body[2]) * inv : (T)0;
    } else {
        o.x = us[0] + (T)g.body[0];
        o.y = us[1] + (T)g.body[1];
        o.z = (D == 3) ? us[2] + (T)g.body[2] : (T)0;
    }
    out[m] = o;
    write_bc_from(g, x, y, z, o, out);
}

// Objective at one level (Sec. 2.5): one block (objective_block).
template <class T>
__global__ void k_objective(Geom g, const V4<T>* __restrict__ s, double* jstep) {
    objective_block<T>(g, s, jstep);
}

// Transpose of the boundary copies: each interior node adjacent to the boundary collects the
// copied components of the boundary nodes it sources (WALL/INLET copy rho, OUTLET copies the
// normal velocity).  Boundary nodes are read only; later kernels treat them as zero.
// Shell enumeration: slab s (0..5) is the interior layer next to face s (axis s/2, low or
// high side); a node next to several faces is handled by the first slab that contains it.
__device__ __forceinline__ bool shell_node(const Geom& g, long long t, int& x, int& y, int& z) {
    const unsigned per0 = (unsigned)g.n[1] * g.n[2], per1 = (unsigned)g.n[0] * g.n[2],
                   per2 = (unsigned)g.n[0] * g.n[1];
    unsigned r = (unsigned)t;
    int slab = 0;
    while (slab < 6) {
        const unsigned pa = slab < 2 ? per0 : (slab < 4 ? per1 : per2);
        if (r < pa) break;
        r -= pa;
        ++slab;
    }
    t = r;
    if (slab >= 6) return false;
    const int a = slab / 2;
    if (a >= g.dim || g.periodic[a]) return false;
    const int fixed = (slab & 1) ? g.n[a] - 2 : 1;
    int c[3];
    const int b0 = (a == 0) ? 1 : 0, b1 = (a == 2) ? 1 : 2;
    c[a] = fixed;
    c[b0] = (int)((unsigned)t % (unsigned)g.n[b0]);
    c[b1] = (int)((unsigned)t / (unsigned)g.n[b0]);
    // owned by an earlier slab?
    for (int e = 0; e < slab; ++e) {
        const int ae = e / 2;
        if (ae >= g.dim || g.periodic[ae]) continue;
        if (c[ae] == ((e & 1) ? g.n[ae] - 2 : 1)) return false;
    }
    x = c[0];
    y = c[1];
    z = c[2];
    return !is_boundary(g, x, y, z);
}

template <class T>
__global__ void k_adj_bcT(Geom g, V4<T>* lam, ObjAdd<T> h) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int x, y, z;
    if (!shell_node(g, t, x, y, z)) return;
    bcT_node<T>(g, lam, h, x, y, z);
}

// mu = (lam_rho, lam_u / (1 + kappa + kappa_s)) on interior nodes, 0 on boundary nodes; in
// the footprint box also e = mu_u . (u_S - u^n) = dJ/dkappa(x, t_n).
template <class T>
__global__ void k_adj_mu(Geom g, const V4<T>* __restrict__ lam, const V4<T>* __restrict__ kus,
                         const V4<T>* __restrict__ sn, V4<T>* __restrict__ mu,
                         T* __restrict__ e, ObjAdd<T> h, const V4<T>* __restrict__ u3) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    int x, y, z;
    node_coords(g, m, x, y, z);
    V4<T> o;
    if (is_boundary(g, x, y, z)) {
        o.r = o.x = o.y = o.z = (T)0;
        mu[m] = o;
        return;
    }
    V4<T> l = lam[m];
    obj_source(g, x, y, z, h, l);
    o.r = l.r;
    long long bi;
    const T kst = g.ks ? ((const T*)g.ks)[m] : (T)0;
    const bool box = in_box(g, x, y, z, bi);
    if (box || kst != (T)0) {
        V4<T> ks;
        ks.r = ks.x = ks.y = ks.z = (T)0;
        if (box) ks = kus[bi];
        const T kt = ks.r + kst;   // moving and static Brinkman coefficients
        const T inv = (T)1 / ((T)1 + kt);
        if (u3) {
            // printed ALKS (Eqs. au, au_ex): only the gathered first moment 3 U~ and the
            // objective source take the (1 + kappa)^-1 of the Brinkman term
            const V4<T> a3 = u3[m];
            V4<T> src = l;
            src.x = l.x - lam[m].x;
            src.y = l.y - lam[m].y;
            src.z = l.z - lam[m].z;
            const T fac = kt * inv;
            o.x = l.x - (a3.x + src.x) * fac;
            o.y = l.y - (a3.y + src.y) * fac;
            o.z = l.z - (a3.z + src.z) * fac;
        } else {
            o.x = l.x * inv;
            o.y = l.y * inv;
            o.z = l.z * inv;
        }
        if (box) {
            const V4<T> v = sn[m];
            e[bi] = o.x * (ks.x - v.x) + o.y * (ks.y - v.y) + o.z * (ks.z - v.z);
        }
    } else {
        o.x = l.x;
        o.y = l.y;
        o.z = l.z;
    }
    mu[m] = o;
}

__device__ __forceinline__ int sym6(int a, int b) {
    return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
}

// mu at y + d (0 outside a non-periodic grid).
template <class T>
__device__ __forceinline__ V4<T> mu_at(const Geom& g, const V4<T>* __restrict__ mu, const int c[3],
                                       int dx, int dy, int dz) {
    int q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
    const int d[3] = {dx, dy, dz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0) continue;
        if (g.periodic[a]) q[a] = wrapi(q[a], g.n[a]);
        else if (q[a] < 0 || q[a] >= g.n[a]) {
            V4<T> z;
            z.r = z.x = z.y = z.z = (T)0;
            return z;
        }
    }
    return mu[node_index(g, q[0], q[1], q[2])];
}

// Moments of F~_i(y) = mu_rho(y+c_i) + c_i.mu_u(y+c_i) and the adjoint of f^eq's dependence on
// rho and u at level n-1; phi = 2 A s~ is kept for the transposed gradient.  The sums over the
// lattice run as butterflies over opposite directions and over the sign pattern of the corners:
//   R~ = sum w F~, U~_a = sum w c_a F~, S~_ab = sum w c_a c_b F~.
template <class T, int D>
__global__ void k_adj_moments(Geom g, const V4<T>* __restrict__ mu,
                              const V4<T>* __restrict__ sp, V4<T>* __restrict__ lo,
                              T* __restrict__ phi, V4<T>* __restrict__ u3) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    int c[3];
    node_coords(g, m, c[0], c[1], c[2]);
    T R, U[3] = {(T)0, (T)0, (T)0}, S[6] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0};
    const V4<T> s0 = mu[m];
    // R = R~, U = 3 U~, S = 9 S~, each with the weight products of Wts<T, D>
    if (D == 3) {
        using W = Wts<T, 3>;
        // axes: F~(+a) = mu_rho + mu_a at y + e_a, F~(-a) = mu_rho - mu_a at y - e_a
        T ax_sum = (T)0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const V4<T> p = mu_at<T>(g, mu, c, a == 0, a == 1, a == 2);
            const V4<T> q = mu_at<T>(g, mu, c, -(a == 0), -(a == 1), -(a == 2));
            const T pa = a == 0 ? p.x : (a == 1 ? p.y : p.z);
            const T qa = a == 0 ? q.x : (a == 1 ? q.y : q.z);
            const T fp = p.r + pa, fm = q.r - qa;
            ax_sum += fp + fm;
            U[a] = W::w3_1 * (fp - fm);
            S[a] = W::s_1 * (fp + fm);   // 9 S~_aa, corners added below
        }
        // corners: sums of F~ over the 8 sign patterns weighted by 1, sx, sy, sz, sx sy, sx sz,
        // sy sz, as butterflies over sx, then sy, then sz
        T f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int sx = (k & 1) ? -1 : 1, sy = (k & 2) ? -1 : 1, sz = (k & 4) ? -1 : 1;
            const V4<T> n = mu_at<T>(g, mu, c, sx, sy, sz);
            const T bx = sx > 0 ? n.r + n.x : n.r - n.x;
            const T by = sy > 0 ? bx + n.y : bx - n.y;
            f[k] = sz > 0 ? by + n.z : by - n.z;
        }
        T a[4], b[4];   // over sx: index (sy, sz) = k >> 1
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a[j] = f[2 * j] + f[2 * j + 1];
            b[j] = f[2 * j] - f[2 * j + 1];
        }
        // over sy: index sz
        const T A0 = a[0] + a[1], A1 = a[2] + a[3], Ay0 = a[0] - a[1], Ay1 = a[2] - a[3];
        const T B0 = b[0] + b[1], B1 = b[2] + b[3], By0 = b[0] - b[1], By1 = b[2] - b[3];
        const T c1 = A0 + A1, cz = A0 - A1, cy = Ay0 + Ay1, cyz = Ay0 - Ay1;
        const T cx = B0 + B1, cxz = B0 - B1, cxy = By0 + By1;
        R = W::w0 * s0.r + W::w1 * ax_sum + W::w2 * c1;
        U[0] += W::w3_2 * cx;
        U[1] += W::w3_2 * cy;
        U[2] += W::w3_2 * cz;
        S[0] += W::s_2 * c1;
        S[1] += W::s_2 * c1;
        S[2] += W::s_2 * c1;
        S[3] = W::s_2 * cxy;
        S[4] = W::s_2 * cxz;
        S[5] = W::s_2 * cyz;
    } else {
        using W = Wts<T, 2>;
        T ax_sum = (T)0;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const V4<T> p = mu_at<T>(g, mu, c, a == 0, a == 1, 0);
            const V4<T> q = mu_at<T>(g, mu, c, -(a == 0), -(a == 1), 0);
            const T pa = a == 0 ? p.x : p.y, qa = a == 0 ? q.x : q.y;
            const T fp = p.r + pa, fm = q.r - qa;
            ax_sum += fp + fm;
            U[a] = W::w3_1 * (fp - fm);
            S[a] = W::s_1 * (fp + fm);
        }
        T f[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int sx = (k & 1) ? -1 : 1, sy = (k & 2) ? -1 : 1;
            const V4<T> n = mu_at<T>(g, mu, c, sx, sy, 0);
            const T bx = sx > 0 ? n.r + n.x : n.r - n.x;
            f[k] = sy > 0 ? bx + n.y : bx - n.y;
        }
        const T a0 = f[0] + f[1], a1 = f[2] + f[3], b0 = f[0] - f[1], b1 = f[2] - f[3];
        const T c1 = a0 + a1, cy = a0 - a1, cx = b0 + b1, cxy = b0 - b1;
        R = W::w0 * s0.r + W::w1 * ax_sum + W::w2 * c1;
        U[0] += W::w3_2 * cx;
        U[1] += W::w3_2 * cy;
        S[0] += W::s_2 * c1;
        S[1] += W::s_2 * c1;
        S[3] = W::s_2 * cxy;
    }
    const V4<T> v = sp[m];
    const T u[3] = {v.x, v.y, D == 3 ? v.z : (T)0};
    V4<T> o;
    o.r = R;
    T lu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lu[a] = (T)0;
        if (a < D) {
            lu[a] = U[a] - (T)3 * R * u[a];
#pragma unroll
            for (int b = 0; b < D; ++b) lu[a] += S[sym6(a, b)] * u[b];
        }
    }
    o.x = lu[0];
    o.y = lu[1];
    o.z = lu[2];
    lo[m] = o;
    if (u3) {
        V4<T> a;
        a.r = (T)0;
        a.x = U[0];
        a.y = U[1];
        a.z = (D == 3) ? U[2] : (T)0;
        u3[m] = a;
    }
    const T twoA = (T)(2.0 * g.A / 9.0);   // phi = 2 A S~ from the stored 9 S~
#pragma unroll
    for (int k = 0; k < 6; ++k) phi[(long long)k * g.nodes + m] = twoA * S[k];
}

// lam_u,alpha(z) += sum_beta (D_beta^T phi_alpha,beta)(z): the transpose of the velocity-gradient
// stencil, gathered per node from the rows whose stencil reaches z.
template <class T, int D>
__global__ void k_adj_divT(Geom g, const T* __restrict__ phi, V4<T>* __restrict__ lo) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    int c[3];
    node_coords(g, m, c[0], c[1], c[2]);
    T acc[3] = {(T)0, (T)0, (T)0};
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const int n = g.n[b], per = g.periodic[b];
#pragma unroll
        for (int k = -2; k <= 2; ++k) {
            int yi = c[b] - k;
            if (per) yi = wrapi(yi, n);
            else if (yi < 0 || yi >= n) continue;
            const T cf = (T)deriv_coef(yi, n, per, k);
            if (cf == (T)0) continue;
            int q[3] = {c[0], c[1], c[2]};
            q[b] = yi;
            const long long mq = node_index(g, q[0], q[1], q[2]);
#pragma unroll
            for (int a = 0; a < D; ++a) acc[a] += cf * phi[(long long)sym6(a, b) * g.nodes + mq];
        }
    }
    V4<T> o = lo[m];
    o.x += acc[0];
    o.y += acc[1];
    if (D == 3) o.z += acc[2];
    lo[m] = o;
}

template <class T>
__global__ void k_check_state(Geom g, const V4<T>* __restrict__ s, int* flag) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    const V4<T> v = s[m];
    const T a = fabs(v.x) + fabs(v.y) + fabs(v.z);
    if (!(a < (T)0.5) || !(fabs(v.r) < (T)1e30)) atomicOr(flag, 1);
}

template <class T>
__global__ void k_state_to_f64(Geom g, const V4<T>* __restrict__ s, double* __restrict__ out,
                               double r0) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    const V4<T> v = s[m];
    out[m] = r0 + (double)v.r;
    out[g.nodes + m] = (double)v.x;
    out[2 * g.nodes + m] = (double)v.y;
    out[3 * g.nodes + m] = (double)v.z;
}

template <class T>
__global__ void k_state_from_f64(Geom g, const double* __restrict__ in, V4<T>* __restrict__ s) {
    long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= g.nodes) return;
    V4<T> v;
    v.r = (T)(in[m] - g.rho0);
    v.x = (T)in[g.nodes + m];
    v.y = (T)in[2 * g.nodes + m];
    v.z = (g.dim == 3) ? (T)in[3 * g.nodes + m] : (T)0;
    s[m] = v;
}

}  // namespace

template <class T>
void launch_init_state(const Geom& g, V4<T>* s, cudaStream_t st) {
    k_fill_uniform<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s, (T)0, (T)0, (T)0);
}

template <class T>
void launch_fill_uniform(const Geom& g, V4<T>* s, const double u[3], cudaStream_t st) {
    k_fill_uniform<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s, (T)u[0], (T)u[1],
                                                              g.dim == 3 ? (T)u[2] : (T)0);
}

template <class T>
void launch_apply_bc(const Geom& g, V4<T>* s, cudaStream_t st) {
    k_apply_bc<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s);
}

template <class T>
void launch_feq(const Geom& g, const V4<T>* s, T* F, cudaStream_t st) {
    if (g.dim == 2) k_feq<T, 2><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s, F);
    else k_feq<T, 3><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s, F);
}

template <class T>
void launch_gather(const Geom& g, const T* F, const V4<T>* kus, V4<T>* out, cudaStream_t st) {
    if (g.dim == 2) k_gather<T, 2><<<grid_for(g.nodes), kThreads, 0, st>>>(g, F, kus, out);
    else k_gather<T, 3><<<grid_for(g.nodes), kThreads, 0, st>>>(g, F, kus, out);
}

template <class T>
void launch_objective(const Geom& g, const V4<T>* s, double* jstep, cudaStream_t st) {
    k_objective<T><<<1, kObjThreads, 0, st>>>(g, s, jstep);
}

template <class T>
void launch_adj_bcT(const Geom& g, V4<T>* lam, double h, cudaStream_t st) {
    const long long shell = 2LL * ((long long)g.n[1] * g.n[2] + (long long)g.n[0] * g.n[2] +
                                   (long long)g.n[0] * g.n[1]);
    k_adj_bcT<T><<<grid_for(shell), kThreads, 0, st>>>(g, lam, obj_add<T>(g, h));
}

template <class T>
void launch_adj_mu(const Geom& g, const V4<T>* lam, const V4<T>* kus, const V4<T>* sn,
                   V4<T>* mu, T* e, double h, cudaStream_t st, const V4<T>* u3) {
    k_adj_mu<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, lam, kus, sn, mu, e, obj_add<T>(g, h),
                                                        u3);
}

template <class T>
void launch_adj_moments(const Geom& g, const V4<T>* mu, const V4<T>* sp, V4<T>* lam_out,
                        T* phi, cudaStream_t st, V4<T>* u3) {
    if (g.dim == 2)
        k_adj_moments<T, 2><<<grid_for(g.nodes), kThreads, 0, st>>>(g, mu, sp, lam_out, phi, u3);
    else
        k_adj_moments<T, 3><<<grid_for(g.nodes), kThreads, 0, st>>>(g, mu, sp, lam_out, phi, u3);
}

template <class T>
void launch_adj_divT(const Geom& g, const T* phi, V4<T>* lam_out, cudaStream_t st) {
    if (g.dim == 2) k_adj_divT<T, 2><<<grid_for(g.nodes), kThreads, 0, st>>>(g, phi, lam_out);
    else k_adj_divT<T, 3><<<grid_for(g.nodes), kThreads, 0, st>>>(g, phi, lam_out);
}

template <class T>
void launch_check_state(const Geom& g, const V4<T>* s, int* flag, cudaStream_t st) {
    k_check_state<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s, flag);
}

template <class T>
void launch_state_to_f64(const Geom& g, const V4<T>* s, double* out, cudaStream_t st,
                         bool add_rho0) {
    k_state_to_f64<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, s, out,
                                                               add_rho0 ? g.rho0 : 0.0);
}

template <class T>
void launch_state_from_f64(const Geom& g, const double* in, V4<T>* s, cudaStream_t st) {
    k_state_from_f64<T><<<grid_for(g.nodes), kThreads, 0, st>>>(g, in, s);
}

#define LKS_INST(T)                                                                          \
    template void launch_init_state<T>(const Geom&, V4<T>*, cudaStream_t);                   \
    template void launch_fill_uniform<T>(const Geom&, V4<T>*, const double*, cudaStream_t);  \
    template void launch_apply_bc<T>(const Geom&, V4<T>*, cudaStream_t);                     \
    template void launch_feq<T>(const Geom&, const V4<T>*, T*, cudaStream_t);                \
    template void launch_gather<T>(const Geom&, const T*, const V4<T>*, V4<T>*, cudaStream_t); \
    template void launch_objective<T>(const Geom&, const V4<T>*, double*, cudaStream_t);     \
    template void launch_adj_bcT<T>(const Geom&, V4<T>*, double, cudaStream_t);              \
    template void launch_adj_mu<T>(const Geom&, const V4<T>*, const V4<T>*, const V4<T>*,    \
                                   V4<T>*, T*, double, cudaStream_t, const V4<T>*);          \
    template void launch_adj_moments<T>(const Geom&, const V4<T>*, const V4<T>*, V4<T>*, T*, \
                                        cudaStream_t, V4<T>*);                               \
    template void launch_adj_divT<T>(const Geom&, const T*, V4<T>*, cudaStream_t);           \
    template void launch_check_state<T>(const Geom&, const V4<T>*, int*, cudaStream_t);      \
    template void launch_state_to_f64<T>(const Geom&, const V4<T>*, double*, cudaStream_t, bool);  \
    template void launch_state_from_f64<T>(const Geom&, const double*, V4<T>*, cudaStream_t);

LKS_INST(float)
LKS_INST(double)

}  // namespace lks
