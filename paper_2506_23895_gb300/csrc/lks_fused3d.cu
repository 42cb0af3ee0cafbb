// Fused D3Q15 LKS step for the FP32 path on non-periodic grids: one kernel per time step.
//
// Algorithm 1's stencil part (Eqs. rho, u with the viscosity term of f^eq, the Brinkman update
// of Eq. u_ex_2 and the boundary rules of Eqs. bc_rho, bc_u) in one pass over the state:
//   * a block owns a 32 x 8 tile of output columns and marches along z over a chunk of planes;
//   * raw state planes (rho - rho0, u as one float4 per node) with a halo of two cells arrive in
//     a five-slot shared-memory ring through cp.async.bulk.tensor (TMA) completing on mbarriers;
//     the waits are bounded and a stalled copy sets an error flag instead of hanging;
//   * every node's f_i^eq is evaluated once, at its source, with the opposite-direction pairs
//     sharing their symmetric part; the 12 directions that leave the column go through shared
//     memory, the rest/+z/-z values stay in registers;
//   * each thread accumulates rho*, u* for its column over three planes (c_z = -1, 0, +1
//     groups), then applies the Brinkman update and writes the boundary nodes it sources.
// HBM traffic per node and step: one float4 read (the halo re-reads hit L2) and one write.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "lks_device.cuh"
#include "lks_tma.cuh"

namespace lks {

namespace {

constexpr int TX = 32, TY = 8;              // output tile
constexpr int HX = TX + 4, HY = TY + 4;     // raw tile with a two-cell halo
constexpr int FX = TX + 2, FY = TY + 2;     // f^eq region with a one-cell halo
constexpr int NSLOT = 5;                    // raw-plane ring depth (3 planes in flight)
constexpr int NTHR = TX * TY;               // 256
constexpr int NHALO = FX * FY - TX * TY;    // 84 extra f^eq nodes on the tile rim
constexpr int NCROSS = 12;                  // directions leaving the column
constexpr unsigned PLANE_BYTES = HX * HY * 16;

// shared-memory layout (bytes)
constexpr size_t OFF_RAW = 0;
constexpr size_t OFF_F = OFF_RAW + (size_t)NSLOT * PLANE_BYTES;
constexpr size_t OFF_BAR = OFF_F + (size_t)NCROSS * FX * FY * 4;
constexpr size_t SMEM_BYTES = OFF_BAR + NSLOT * 8;

// cross-direction slots in sF: 0 +x, 1 -x, 2 +y, 3 -y, 4..7 corners with cz=+1 (sx,sy) =
// (+,+),(-,+),(+,-),(-,-), 8..11 corners with cz=-1 in the same (sx,sy) order.

struct FusedArgs {
    Geom g;
    float4* out;
    const float4* kus;
    const float4* src;    // same buffer the tensor map describes (for rare direct loads)
    int* err;
    int zchunk;
    float A, w0, w1, w2;
    float bf[3];          // body force in single precision
};

// Boundary copies sourced by interior node (gx, gy, z) of value o (Eqs. bc_rho, bc_u): every
// boundary node reached by stepping to the low face (coordinate 1) and/or the high face
// (coordinate n - 2) along the axes, with the value of its winning face.  Loops over scalar
// options (no local arrays), so the common path carries no stack traffic.
__device__ __forceinline__ void write_bc_f(const Geom& g, int gx, int gy, int z, float4 o,
                                           float4* out) {
    V4<float> v;
    v.r = o.x;
    v.x = o.y;
    v.y = o.z;
    v.z = o.w;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int nxo = 1 + (gx == 1) + (gx == nx - 2);
    const int nyo = 1 + (gy == 1) + (gy == ny - 2);
    const int nzo = 1 + (z == 1) + (z == nz - 2);
#pragma unroll 1
    for (int i = 0; i < nxo; ++i) {
        const int mx = i == 0 ? 0 : ((i == 1 && gx == 1) ? 1 : 2);
        const int bx = mx == 0 ? gx : (mx == 1 ? 0 : nx - 1);
#pragma unroll 1
        for (int j = 0; j < nyo; ++j) {
            const int my = j == 0 ? 0 : ((j == 1 && gy == 1) ? 1 : 2);
            const int by = my == 0 ? gy : (my == 1 ? 0 : ny - 1);
#pragma unroll 1
            for (int k = 0; k < nzo; ++k) {
                if ((i | j | k) == 0) continue;
                const int mz = k == 0 ? 0 : ((k == 1 && z == 1) ? 1 : 2);
                const int bz = mz == 0 ? z : (mz == 1 ? 0 : nz - 1);
                const int side[3] = {mx - 1, my - 1, mz - 1};
                const V4<float> b = bc_value(g, winning_face(g, side), v);
                out[((long long)bz * ny + by) * nx + bx] = make_float4(b.r, b.x, b.y, b.z);
            }
        }
    }
}

// 2 x first derivative (D = 2 du/dx) of (ux, uy, uz) along one axis from the node c and its
// neighbours at -1/+1 (and -2/+2 for the one-sided forms).  mode 0: central, 1: one-sided at
// the low boundary node, 2: one-sided at the high boundary node.
__device__ __forceinline__ void deriv2(int mode, const float4& c, const float4& m1,
                                       const float4& p1, const float4& m2, const float4& p2,
                                       float& dx, float& dy, float& dz) {
    if (mode == 0) {
        dx = p1.y - m1.y;
        dy = p1.z - m1.z;
        dz = p1.w - m1.w;
    } else if (mode == 1) {   // -3 c + 4 u(+1) - u(+2)
        dx = -3.f * c.y + 4.f * p1.y - p2.y;
        dy = -3.f * c.z + 4.f * p1.z - p2.z;
        dz = -3.f * c.w + 4.f * p1.w - p2.w;
    } else {                  // 3 c - 4 u(-1) + u(-2)
        dx = 3.f * c.y - 4.f * m1.y + m2.y;
        dy = 3.f * c.z - 4.f * m1.z + m2.z;
        dz = 3.f * c.w - 4.f * m1.w + m2.w;
    }
}

// f^eq at one node of the f^eq region (Sec. 2.2): stores the 12 values that leave the column
// into sF (at sFn = sF + node index, planes FS apart) and returns rest, +z and -z.
// c0/cm/cp point at the node in planes p, p-1, p+1; zfar is the plane two away for the
// one-sided z difference (only read when zm != 0).
template <bool EDGE>
__device__ __forceinline__ void feq_node(const FusedArgs& a, const float4* __restrict__ c0,
                                         const float4* __restrict__ cm,
                                         const float4* __restrict__ cp, float* __restrict__ sFn,
                                         int xm, int ym, int zm, const float4& zfar,
                                         float& f_rest, float& f_pz, float& f_mz) {
    constexpr int FS = FX * FY;
    const float4 c = c0[0];
    // Dab = 2 d u_a / d x_b
    float Dxx, Dyx, Dzx, Dxy, Dyy, Dzy, Dxz, Dyz, Dzz;
    if (EDGE) {
        deriv2(xm, c, c0[-1], c0[1], xm == 2 ? c0[-2] : c, xm == 1 ? c0[2] : c, Dxx, Dyx, Dzx);
        deriv2(ym, c, c0[-HX], c0[HX], ym == 2 ? c0[-2 * HX] : c, ym == 1 ? c0[2 * HX] : c, Dxy,
               Dyy, Dzy);
        deriv2(zm, c, cm[0], cp[0], zfar, zfar, Dxz, Dyz, Dzz);
    } else {
        const float4 e = c0[1], w = c0[-1], n = c0[HX], s = c0[-HX], u = cp[0], d = cm[0];
        Dxx = e.y - w.y;
        Dyx = e.z - w.z;
        Dzx = e.w - w.w;
        Dxy = n.y - s.y;
        Dyy = n.z - s.z;
        Dzy = n.w - s.w;
        Dxz = u.y - d.y;
        Dyz = u.z - d.z;
        Dzz = u.w - d.w;
    }
    const float A = a.A, hA = 0.5f * a.A;
    // A S_ab with S = grad u + grad u^T (D is twice the derivative)
    const float ASxx = A * Dxx, ASyy = A * Dyy, ASzz = A * Dzz;
    const float ASxy = hA * (Dxy + Dyx);
    const float ASxz = hA * (Dxz + Dzx);
    const float ASyz = hA * (Dyz + Dzy);
    const float ux = c.y, uy = c.z, uz = c.w;
    const float P = c.x - 1.5f * (ux * ux + uy * uy + uz * uz);
    using Wf = Wts<float, 3>;
    f_rest = Wf::w0 * P;
    // axes: w1 (P + A S_aa) + 4.5 w1 u_a^2 +- 3 w1 u_a (the weight products as in Wts)
    const float w1 = Wf::w1, w13 = Wf::w3_1;
    {
        const float b = fmaf(Wf::h_1 * ux, ux, w1 * (P + ASxx));
        sFn[0 * FS] = b + w13 * ux;
        sFn[1 * FS] = b - w13 * ux;
    }
    {
        const float b = fmaf(Wf::h_1 * uy, uy, w1 * (P + ASyy));
        sFn[2 * FS] = b + w13 * uy;
        sFn[3 * FS] = b - w13 * uy;
    }
    {
        const float b = fmaf(Wf::h_1 * uz, uz, w1 * (P + ASzz));
        f_pz = b + w13 * uz;
        f_mz = b - w13 * uz;
    }
    // corners (sx, sy, +1) and their opposites (-sx, -sy, -1):
    // w2 [P + A tr S + 2 A (sx sy S_xy + sx S_xz + sy S_yz)] + 4.5 w2 (c.u)^2 +- 3 w2 (c.u)
    const float w2 = Wf::w2, w23 = Wf::w3_2, w245 = Wf::h_2, w2x2 = 2.f * Wf::w2;
    const float T0 = w2 * (P + ASxx + ASyy + ASzz);
    const float s1 = ux + uy, d1 = ux - uy;
    const float q1 = ASxz + ASyz, q2 = ASyz - ASxz;
    {   // (+,+,+) / (-,-,-)
        const float cu = s1 + uz;
        const float sym = T0 + w245 * cu * cu + w2x2 * (ASxy + q1);
        sFn[4 * FS] = sym + w23 * cu;
        sFn[11 * FS] = sym - w23 * cu;
    }
    {   // (-,+,+) / (+,-,-)
        const float cu = uz - d1;
        const float sym = T0 + w245 * cu * cu + w2x2 * (q2 - ASxy);
        sFn[5 * FS] = sym + w23 * cu;
        sFn[10 * FS] = sym - w23 * cu;
    }
    {   // (+,-,+) / (-,+,-)
        const float cu = uz + d1;
        const float sym = T0 + w245 * cu * cu - w2x2 * (ASxy + q2);
        sFn[6 * FS] = sym + w23 * cu;
        sFn[9 * FS] = sym - w23 * cu;
    }
    {   // (-,-,+) / (+,+,-)
        const float cu = uz - s1;
        const float sym = T0 + w245 * cu * cu + w2x2 * (ASxy - q1);
        sFn[7 * FS] = sym + w23 * cu;
        sFn[8 * FS] = sym - w23 * cu;
    }
}

// Single-precision face values for the boundary copies: per face the prescribed (ux, uy, uz,
// rho - rho0), rounded once on the host, and whether the face keeps the source's rho (wall,
// inlet: u prescribed) or prescribes rho and copies the normal velocity (outlet).
struct ShellFaces {
    float4 v[6];
    int keep_rho[6];
};

// The value bc_value gives a boundary node of face f from its source's value o (x: rho - rho0).
__device__ __forceinline__ float4 face_value(const ShellFaces& F, int f, const float4& o) {
    const float4 p = F.v[f];
    if (F.keep_rho[f]) return make_float4(o.x, p.x, p.y, p.z);
    const int na = f >> 1;
    return make_float4(p.w, na == 0 ? o.y : p.x, na == 1 ? o.z : p.y, na == 2 ? o.w : p.z);
}

// Boundary copies of a z-march forward step (Eqs. bc_rho, bc_u), once the step is written: one
// thread per interior node next to a face -- the x layers, then the y layers without the x
// layers' nodes, then the z layers without both -- each writing the boundary nodes it sources
// (one node of one face for most; edges and corners through write_bc_f).
__global__ void __launch_bounds__(256)
    k_bc_shell3d(Geom g, const __grid_constant__ ShellFaces F, float4* __restrict__ s) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long ix = nx - 2, iy = ny - 2, iz = nz - 2;   // interior extents
    long long r = t;
    int a;
    if (r < 2 * iy * iz) {
        a = 0;
    } else if ((r -= 2 * iy * iz) < 2 * ix * iz) {
        a = 1;
    } else if ((r -= 2 * ix * iz) < 2 * ix * iy) {
        a = 2;
    } else {
        return;
    }
    const bool hi = (r & 1) != 0;
    r >>= 1;
    int x, y, z;
    if (a == 0) {
        x = hi ? nx - 2 : 1;
        y = 1 + (int)(r % iy);
        z = 1 + (int)(r / iy);
        if (hi && ix == 1) return;   // a single interior row: the low layer writes
    } else if (a == 1) {
        y = hi ? ny - 2 : 1;
        x = 1 + (int)(r % ix);
        z = 1 + (int)(r / ix);
        if ((hi && iy == 1) || x == 1 || x == nx - 2) return;
    } else {
        z = hi ? nz - 2 : 1;
        x = 1 + (int)(r % ix);
        y = 1 + (int)(r / ix);
        if ((hi && iz == 1) || x == 1 || x == nx - 2 || y == 1 || y == ny - 2) return;
    }
    const long long m = ((long long)z * ny + y) * nx + x;
    const float4 o = s[m];
    const int nfx = (x == 1) + (x == nx - 2), nfy = (y == 1) + (y == ny - 2);
    const int nfz = (z == 1) + (z == nz - 2);
    if (nfx + nfy + nfz == 1) {
        int f, bx = x, by = y, bz = z;
        if (nfx) {
            f = x == 1 ? 0 : 1;
            bx = x == 1 ? 0 : nx - 1;
        } else if (nfy) {
            f = y == 1 ? 2 : 3;
            by = y == 1 ? 0 : ny - 1;
        } else {
            f = z == 1 ? 4 : 5;
            bz = z == 1 ? 0 : nz - 1;
        }
        s[((long long)bz * ny + by) * nx + bx] = face_value(F, f, o);
        return;
    }
    write_bc_f(g, x, y, z, o, s);
}

__device__ __forceinline__ int axis_mode(int gcoord, int n) {
    return gcoord == 0 ? 1 : (gcoord == n - 1 ? 2 : 0);
}

__global__ void __launch_bounds__(NTHR, 4)
    k_fused_step3d(const __grid_constant__ CUtensorMap tmap, const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    float4* raw = reinterpret_cast<float4*>(smem + OFF_RAW);
    float* sF = reinterpret_cast<float*>(smem + OFF_F);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    const Geom& g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int q0 = blockIdx.z * a.zchunk;
    const int q1 = min(nz, q0 + a.zchunk);
    const int nplanes = q1 - q0 + 4;   // raw planes q0-2 .. q1+1
    // rim node handled by this thread (tid < NHALO)
    int hfx = 0, hfy = 0;
    if (tid < NHALO) {
        if (tid < FX) {
            hfx = tid;
            hfy = 0;
        } else if (tid < 2 * FX) {
            hfx = tid - FX;
            hfy = FY - 1;
        } else if (tid < 2 * FX + TY) {
            hfx = 0;
            hfy = 1 + (tid - 2 * FX);
        } else {
            hfx = FX - 1;
            hfy = 1 + (tid - 2 * FX - TY);
        }
    }
    if ((smem_addr(smem) & 127u) != 0u) {  // TMA destinations need 128-byte alignment
        if (tid == 0) atomicOr(a.err, 16);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(smem_addr(&bars[s]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < NSLOT - 1 && k < nplanes; ++k)
            tma_load_box(smem_addr(raw + (size_t)k * HX * HY), &tmap, x0 - 2, y0 - 2,
                         q0 - 2 + k, smem_addr(&bars[k]), PLANE_BYTES);
    }
    __syncthreads();

    // ---- per-thread constants of the column ----
    const int gx = x0 + tx, gy = y0 + ty;
    const int hgx = x0 - 1 + hfx, hgy = y0 - 1 + hfy;
    const bool edge = (x0 - 1 <= 0) || (x0 + TX >= nx - 1) || (y0 - 1 <= 0) || (y0 + TY >= ny - 1);
    const int pxm = axis_mode(gx, nx), pym = axis_mode(gy, ny);
    const int rxm = axis_mode(hgx, nx), rym = axis_mode(hgy, ny);
    const int hp = (ty + 2) * HX + (tx + 2);      // primary node in the raw tile
    const int hr = (hfy + 1) * HX + (hfx + 1);    // rim node in the raw tile
    float* sFp = sF + (ty + 1) * FX + (tx + 1);
    float* sFr = sF + hfy * FX + hfx;
    const bool has_rim = tid < NHALO;
    const bool out_col = gx >= 1 && gx <= nx - 2 && gy >= 1 && gy <= ny - 2;
    const bool bc_col = gx == 1 || gx == nx - 2 || gy == 1 || gy == ny - 2;
    const int bxx = gx - g.blo[0], byy = gy - g.blo[1];
    const bool box_col = g.boxN > 0 && bxx >= 0 && byy >= 0 && bxx < g.bn[0] && byy < g.bn[1];
    const long long box_plane = (long long)g.bn[0] * g.bn[1];
    const float4* kus_col = a.kus + ((long long)byy * g.bn[0] + bxx) - (long long)g.blo[2] * box_plane;
    const long long zstride = (long long)nx * ny;
    const bool in_xy = gx < nx && gy < ny;
    const bool rim_in_xy = hgx >= 0 && hgx < nx && hgy >= 0 && hgy < ny;
    float4* out_col_ptr = a.out + ((long long)gy * nx + gx);
    const int zlo = max(q0, 1), zhi = nz - 2;
    const float bfx = a.bf[0], bfy = a.bf[1], bfz = a.bf[2];

    float acc0[4] = {0.f, 0.f, 0.f, 0.f};  // plane p (c_z = 0 and -1 groups still to come)
    float acc1[4] = {0.f, 0.f, 0.f, 0.f};  // plane p + 1
    constexpr int FS = FX * FY;
    bool ok = true;
    // ring bookkeeping: slot holding plane p-1, p, p+1; next load slot; wait slot/parity
    int sm = 0, s0 = 1, sp = 2;
    int wslot = 0, wpar = 0;              // next load to wait for
    int islot = NSLOT - 1, ik = NSLOT - 1;  // next load to issue: slot and load index

    for (int p = q0 - 1; p <= q1; ++p) {
        bool good = true;
        if (tid == 0) {
            // refill the slot of plane p-2 (last read before the previous iteration's second
            // barrier) with plane p + NSLOT - 2
            if (ik < nplanes) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_box(smem_addr(raw + (size_t)islot * HX * HY), &tmap, x0 - 2, y0 - 2,
                             q0 - 2 + ik, smem_addr(&bars[islot]), PLANE_BYTES);
            }
            // first iteration waits for loads 0..2, later ones for the newest plane
            const int nwait = (p == q0 - 1) ? 3 : 1;
            for (int i = 0; i < nwait && good; ++i) {
                good = mbar_wait(smem_addr(&bars[wslot]), wpar);
                if (++wslot == NSLOT) {
                    wslot = 0;
                    wpar ^= 1;
                }
            }
        }
        if (__syncthreads_or(!good)) {
            ok = false;
            break;
        }
        ++ik;
        if (++islot == NSLOT) islot = 0;
        const float4* rm = raw + (size_t)sm * HX * HY;
        const float4* r0 = raw + (size_t)s0 * HX * HY;
        const float4* rp = raw + (size_t)sp * HX * HY;
        float f_rest, f_pz, f_mz;
        const int zm = (p == 0) ? 1 : (p == nz - 1 ? 2 : 0);
        if (!edge && zm == 0) {
            const float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f);
            feq_node<false>(a, r0 + hp, rm + hp, rp + hp, sFp, 0, 0, 0, z0, f_rest, f_pz, f_mz);
            if (has_rim) {
                float d0, d1, d2;
                feq_node<false>(a, r0 + hr, rm + hr, rp + hr, sFr, 0, 0, 0, z0, d0, d1, d2);
            }
        } else {
            // plane two away for one-sided z differences, straight from global memory
            const int z2 = (zm == 1) ? 2 : nz - 3;
            float4 zf = make_float4(0.f, 0.f, 0.f, 0.f);
            if (zm != 0 && in_xy) zf = a.src[((long long)z2 * ny + gy) * nx + gx];
            feq_node<true>(a, r0 + hp, rm + hp, rp + hp, sFp, pxm, pym, zm, zf, f_rest, f_pz,
                           f_mz);
            if (has_rim) {
                float4 zr = make_float4(0.f, 0.f, 0.f, 0.f);
                if (zm != 0 && rim_in_xy) zr = a.src[((long long)z2 * ny + hgy) * nx + hgx];
                float d0, d1, d2;
                feq_node<true>(a, r0 + hr, rm + hr, rp + hr, sFr, rxm, rym, zm, zr, d0, d1, d2);
            }
        }
        __syncthreads();
        // gather the three z-groups of plane p's f^eq into planes p-1, p, p+1; a value of
        // direction c comes from the node at (x - c_x, y - c_y)
        const float fpx = sFp[0 * FS - 1], fmx = sFp[1 * FS + 1];
        const float fpy = sFp[2 * FS - FX], fmy = sFp[3 * FS + FX];
        const float cpp_p = sFp[4 * FS - 1 - FX], cmp_p = sFp[5 * FS + 1 - FX];
        const float cpm_p = sFp[6 * FS - 1 + FX], cmm_p = sFp[7 * FS + 1 + FX];
        const float cpp_m = sFp[8 * FS - 1 - FX], cmp_m = sFp[9 * FS + 1 - FX];
        const float cpm_m = sFp[10 * FS - 1 + FX], cmm_m = sFp[11 * FS + 1 + FX];
        // c_z = -1 group completes plane p-1
        {
            const float sxp = cpp_m + cpm_m, sxm = cmp_m + cmm_m;
            const float syp = cpp_m + cmp_m, sym = cpm_m + cmm_m;
            const float all = sxp + sxm + f_mz;
            const int qz = p - 1;
            if (out_col && qz >= zlo && qz <= zhi) {
                const float r = acc0[0] + all;
                const float ux = acc0[1] + (sxp - sxm) + bfx;
                const float uy = acc0[2] + (syp - sym) + bfy;
                const float uz = acc0[3] - all + bfz;
                float4 o;
                o.x = r;
                const int bz = qz - g.blo[2];
                if (box_col && bz >= 0 && bz < g.bn[2]) {
                    const float4 ks = kus_col[(long long)qz * box_plane];
                    const float inv = 1.f / (1.f + ks.x);
                    o.y = fmaf(ks.x, ks.y, ux) * inv;
                    o.z = fmaf(ks.x, ks.z, uy) * inv;
                    o.w = fmaf(ks.x, ks.w, uz) * inv;
                } else {
                    o.y = ux;
                    o.z = uy;
                    o.w = uz;
                }
                out_col_ptr[(long long)qz * zstride] = o;
                if (bc_col || qz == 1 || qz == nz - 2) write_bc_f(g, gx, gy, qz, o, a.out);
            }
        }
        // c_z = 0 group into plane p, c_z = +1 group starts plane p+1
        acc0[0] = acc1[0] + (f_rest + fpx + fmx + fpy + fmy);
        acc0[1] = acc1[1] + (fpx - fmx);
        acc0[2] = acc1[2] + (fpy - fmy);
        acc0[3] = acc1[3];
        {
            const float sxp = cpp_p + cpm_p, sxm = cmp_p + cmm_p;
            const float syp = cpp_p + cmp_p, sym = cpm_p + cmm_p;
            const float all = sxp + sxm + f_pz;
            acc1[0] = all;
            acc1[1] = sxp - sxm;
            acc1[2] = syp - sym;
            acc1[3] = all;
        }
        sm = s0;
        s0 = sp;
        if (++sp == NSLOT) sp = 0;
    }
    if (!ok) {
        // a copy did not land in time: record it, then give the copies still in flight a
        // bounded chance to finish before the block's shared memory goes away
        if (tid == 0) {
            atomicOr(a.err, 8);
            const long long t0 = clock64();
            while (clock64() - t0 < (1LL << 28)) {
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- register z-march variant
// The same step with fewer instructions and one block barrier per plane:
//   * every thread keeps its column's u at plane p-1 and the full node at p in registers, so an
//     f^eq evaluation reads the four in-plane neighbours and the next plane's centre only;
//   * every thread waits on the ring's mbarriers itself (no serialising single-thread wait);
//   * the cross-column f^eq values alternate between two shared-memory buffers, so one barrier
//     per plane orders both their writes and their reads;
//   * tiles of 32 x 8 columns; tiles away from the x and y faces take a path without face
//     tests; in the others only the nodes on a face redo f^eq with one-sided derivatives (one
//     lane of a row, or a whole row), and the rim f^eq work fills whole warps.
// The arithmetic is that of feq_node and the gather above, operation for operation.
// Own column of the x face in a tile of TX columns from x0 when the tile holds exactly one of
// the two x faces, else -1.
__host__ __device__ inline int xface_col(int x0, int nx, int TX) {
    const bool lo = x0 == 0, hi = x0 <= nx - 1 && nx - 1 < x0 + TX;
    return lo == hi ? -1 : (lo ? 0 : nx - 1 - x0);
}

// f^eq-region coordinates (hfx, hfy) of the extra node of thread tid: the one-cell rim over whole
// warps.  In a tile holding exactly one x face, every node of that face's column goes to the
// last rim warp -- its rows (one spare lane per row) and its two rim-row nodes (two more spare
// lanes), whose own lanes in the rim rows then repeat their left neighbour -- so that only that
// warp needs the one-sided x derivatives; otherwise the spare lanes repeat earlier rim nodes.
// Repeated nodes store the same values twice.
template <int TX, int TY, int NHALO>
__device__ __forceinline__ void rim_node(int tid, int x0, int nx, int& hfx, int& hfy) {
    constexpr int FW = TX + 2, FY = TY + 2;
    constexpr int RIMW = (NHALO + 31) / 32 * 32;
    static_assert(RIMW - NHALO >= TY + 2, "spare rim lanes for the face column");
    static_assert(NHALO >= RIMW - 32, "the face column in the last rim warp");
    hfx = 0;
    hfy = 0;
    if (tid >= RIMW) return;
    const int xf = xface_col(x0, nx, TX);
    if (xf >= 0 && tid >= NHALO && tid < NHALO + TY + 2) {
        const int r = tid - NHALO;
        hfx = xf + 1;
        hfy = r < TY ? 1 + r : (r == TY ? 0 : FY - 1);
        return;
    }
    const int rr = tid < NHALO ? tid : tid - (RIMW - NHALO);
    if (rr < FW) {
        hfx = rr;
    } else if (rr < 2 * FW) {
        hfx = rr - FW;
        hfy = FY - 1;
    } else if (rr < 2 * FW + TY) {
        hfy = 1 + (rr - 2 * FW);
    } else {
        hfx = FW - 1;
        hfy = 1 + (rr - 2 * FW - TY);
    }
    if (xf >= 0 && tid < NHALO && (hfy == 0 || hfy == FY - 1) && hfx == xf + 1) hfx = xf;
}

template <int TY_>
struct ZCfg {
    static constexpr int TX = 32, TY = TY_;
    // raw planes: TX + 4 columns with a row pitch of HX = TX + 5 (odd, so that column-strided
    // accesses spread over all shared-memory banks; the TMA box is HX wide); f^eq region: FW
    // columns with row pitch FX = FW + 1
    static constexpr int HX = TX + 5, HY = TY + 4, FW = TX + 2, FX = FW + 1, FY = TY + 2;
    static constexpr int NTHR = TX * TY, NHALO = FW * FY - TX * TY, FS = FX * FY;
    static constexpr int NSLOT = 5;
    static constexpr int MINB = 3;     // resident blocks per SM
    static constexpr unsigned PLANE_BYTES = HX * HY * 16;                 // one TMA box
    static constexpr int SLOT = (PLANE_BYTES + 127) / 128 * 128 / 16;     // float4 per slot
    static constexpr size_t OFF_F = (size_t)NSLOT * SLOT * 16;
    static constexpr size_t OFF_BAR = OFF_F + (size_t)2 * NCROSS * FS * 4;
    static constexpr size_t SMEM = OFF_BAR + NSLOT * 8;
};

// f^eq of one node from registers (centre c, u at p-1 and p+1) and its in-plane neighbours in
// the ring plane (c0 points at the node).  Same operations as feq_node.
template <int HXs, int FSs, bool EDGE>
__device__ __forceinline__ void feq_reg(const FusedArgs& a, const float4* __restrict__ c0,
                                        const float4& c, const float3& um, const float3& up,
                                        float* __restrict__ sFn, int xm, int ym, int zm,
                                        const float4& zfar, float& f_rest, float& f_pz,
                                        float& f_mz) {
    float Dxx, Dyx, Dzx, Dxy, Dyy, Dzy, Dxz, Dyz, Dzz;
    if (EDGE) {
        const float4 cm4 = make_float4(0.f, um.x, um.y, um.z);
        const float4 cp4 = make_float4(0.f, up.x, up.y, up.z);
        deriv2(xm, c, c0[-1], c0[1], xm == 2 ? c0[-2] : c, xm == 1 ? c0[2] : c, Dxx, Dyx, Dzx);
        deriv2(ym, c, c0[-HXs], c0[HXs], ym == 2 ? c0[-2 * HXs] : c, ym == 1 ? c0[2 * HXs] : c,
               Dxy, Dyy, Dzy);
        deriv2(zm, c, cm4, cp4, zfar, zfar, Dxz, Dyz, Dzz);
    } else {
        const float4 e = c0[1], w = c0[-1], n = c0[HXs], s = c0[-HXs];
        Dxx = e.y - w.y;
        Dyx = e.z - w.z;
        Dzx = e.w - w.w;
        Dxy = n.y - s.y;
        Dyy = n.z - s.z;
        Dzy = n.w - s.w;
        Dxz = up.x - um.x;
        Dyz = up.y - um.y;
        Dzz = up.z - um.z;
    }
    const float A = a.A, hA = 0.5f * a.A;
    const float ASxx = A * Dxx, ASyy = A * Dyy, ASzz = A * Dzz;
    const float ASxy = hA * (Dxy + Dyx);
    const float ASxz = hA * (Dxz + Dzx);
    const float ASyz = hA * (Dyz + Dzy);
    const float ux = c.y, uy = c.z, uz = c.w;
    const float P = c.x - 1.5f * (ux * ux + uy * uy + uz * uz);
    using Wf = Wts<float, 3>;
    f_rest = Wf::w0 * P;
    const float w1 = Wf::w1, w13 = Wf::w3_1;
    {
        const float b = fmaf(Wf::h_1 * ux, ux, w1 * (P + ASxx));
        sFn[0 * FSs] = b + w13 * ux;
        sFn[1 * FSs] = b - w13 * ux;
    }
    {
        const float b = fmaf(Wf::h_1 * uy, uy, w1 * (P + ASyy));
        sFn[2 * FSs] = b + w13 * uy;
        sFn[3 * FSs] = b - w13 * uy;
    }
    {
        const float b = fmaf(Wf::h_1 * uz, uz, w1 * (P + ASzz));
        f_pz = b + w13 * uz;
        f_mz = b - w13 * uz;
    }
    const float w2 = Wf::w2, w23 = Wf::w3_2, w245 = Wf::h_2, w2x2 = 2.f * Wf::w2;
    const float T0 = w2 * (P + ASxx + ASyy + ASzz);
    const float s1 = ux + uy, d1 = ux - uy;
    const float q1 = ASxz + ASyz, q2 = ASyz - ASxz;
    {
        const float cu = s1 + uz;
        const float sym = T0 + w245 * cu * cu + w2x2 * (ASxy + q1);
        sFn[4 * FSs] = sym + w23 * cu;
        sFn[11 * FSs] = sym - w23 * cu;
    }
    {
        const float cu = uz - d1;
        const float sym = T0 + w245 * cu * cu + w2x2 * (q2 - ASxy);
        sFn[5 * FSs] = sym + w23 * cu;
        sFn[10 * FSs] = sym - w23 * cu;
    }
    {
        const float cu = uz + d1;
        const float sym = T0 + w245 * cu * cu - w2x2 * (ASxy + q2);
        sFn[6 * FSs] = sym + w23 * cu;
        sFn[9 * FSs] = sym - w23 * cu;
    }
    {
        const float cu = uz - s1;
        const float sym = T0 + w245 * cu * cu + w2x2 * (ASxy - q1);
        sFn[7 * FSs] = sym + w23 * cu;
        sFn[8 * FSs] = sym - w23 * cu;
    }
}

template <int TY_, bool IN>
__device__ __forceinline__ void zbody(const CUtensorMap& tmap, const FusedArgs& a,
                                      unsigned char* smem, int hfx, int hfy, int q0, int q1,
                                      int nplanes) {
    using C = ZCfg<TY_>;
    constexpr int TX = C::TX, TY = C::TY, HX = C::HX, FX = C::FX;
    constexpr int FS = C::FS, NSLOT = C::NSLOT;
    float4* raw = reinterpret_cast<float4*>(smem);
    float* sFbase = reinterpret_cast<float*>(smem + C::OFF_F);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    const Geom& g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const int hgx = x0 - 1 + hfx, hgy = y0 - 1 + hfy;
    const int pxm = axis_mode(gx, nx), pym = axis_mode(gy, ny);
    const int rxm = axis_mode(hgx, nx), rym = axis_mode(hgy, ny);
    // a node on the tile's single x face outside a y-face row: a rim lane evaluates its f^eq
    const bool xskip = !IN && pxm != 0 && pym == 0 && xface_col(x0, nx, TX) >= 0;
    const int hp = (ty + 2) * HX + (tx + 2);
    const int hr = (hfy + 1) * HX + (hfx + 1);
    const int fop = (ty + 1) * FX + (tx + 1);
    const int forr = hfy * FX + hfx;
    constexpr int RIMW = (C::NHALO + 31) / 32 * 32;
    const bool has_rim = tid < RIMW;   // whole warps
    // rim warps holding a face node take the one-sided forms (a uniform choice per warp)
    const bool rim_edge = !IN && __any_sync(0xffffffffu, has_rim && (rxm | rym) != 0);
    const bool out_col = IN || (gx >= 1 && gx <= nx - 2 && gy >= 1 && gy <= ny - 2);
    const int bxx = gx - g.blo[0], byy = gy - g.blo[1];
    const bool box_col = g.boxN > 0 && bxx >= 0 && byy >= 0 && bxx < g.bn[0] && byy < g.bn[1];
    const long long box_plane = (long long)g.bn[0] * g.bn[1];
    const float4* kus_col = a.kus + ((long long)byy * g.bn[0] + bxx) - (long long)g.blo[2] * box_plane;
    const long long zstride = (long long)nx * ny;
    const bool in_xy = IN || (gx < nx && gy < ny);
    const bool rim_in_xy = IN || (hgx >= 0 && hgx < nx && hgy >= 0 && hgy < ny);
    float4* out_col_ptr = a.out + ((long long)gy * nx + gx);
    const int zlo = max(q0, 1), zhi = nz - 2;
    const float bfx = a.bf[0], bfy = a.bf[1], bfz = a.bf[2];

    bool ok = true;
    // prologue: planes q0-2 (load 0) and q0-1 (load 1) into registers
    float3 um, rum;
    float4 c0, rc0;
    {
        bool good = mbar_wait(smem_addr(&bars[0]), 0);
        good = mbar_wait(smem_addr(&bars[1]), 0) && good;
        const float4* r0 = raw;
        const float4* r1 = raw + (size_t)C::SLOT;
        const float4 v = r0[hp];
        um = make_float3(v.y, v.z, v.w);
        c0 = r1[hp];
        const float4 rv = r0[hr];
        rum = make_float3(rv.y, rv.z, rv.w);
        rc0 = r1[hr];
        ok = !__syncthreads_or(!good);
    }
    float acc0[4] = {0.f, 0.f, 0.f, 0.f};
    float acc1[4] = {0.f, 0.f, 0.f, 0.f};
    int s0 = 1;                    // slot of plane p
    int wslot = 2, wpar = 0;       // slot / parity of plane p + 1
    int islot = 0, ik = NSLOT;     // next refill: slot and load index
    // the output node of plane p - 1 in the column, advanced one plane per iteration (it is
    // only dereferenced for planes inside the grid)
    float4* outp = out_col_ptr + (long long)(q0 - 3) * zstride;
    // One plane p.  STEADY (planes away from the z faces and from the chunk's first output): no
    // z-face derivative modes, no z output-range and no z boundary-copy tests.  Off the z faces
    // every node takes the central-difference f^eq; in tiles at an x or y face (IN false) the
    // face nodes then evaluate it again with their one-sided derivatives, and the output keeps
    // its column tests and boundary copies.
    auto plane = [&](int p, auto steady) {
        constexpr bool STEADY = decltype(steady)::value;
        const bool good = mbar_wait_once(smem_addr(&bars[wslot]), wpar);
        const float4* r0 = raw + (size_t)s0 * C::SLOT;
        const float4* rp = raw + (size_t)wslot * C::SLOT;
        float* sF = sFbase + (size_t)((p - q0 + 1) & 1) * NCROSS * FS;
        float* sFp = sF + fop;
        const float4 cpn = rp[hp];
        const float3 up = make_float3(cpn.y, cpn.z, cpn.w);
        float4 rcpn = make_float4(0.f, 0.f, 0.f, 0.f);
        if (has_rim) rcpn = rp[hr];
        const float3 rup = make_float3(rcpn.y, rcpn.z, rcpn.w);
        float f_rest = 0.f, f_pz = 0.f, f_mz = 0.f;
        const int zm = STEADY ? 0 : ((p == 0) ? 1 : (p == nz - 1 ? 2 : 0));
        if (STEADY || zm == 0) {
            const float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (IN) {
                feq_reg<HX, FS, false>(a, r0 + hp, c0, um, up, sFp, 0, 0, 0, z0, f_rest, f_pz,
                                       f_mz);
                if (has_rim) {
                    float d0, d1, d2;
                    feq_reg<HX, FS, false>(a, r0 + hr, rc0, rum, rup, sF + forr, 0, 0, 0, z0, d0,
                                           d1, d2);
                }
            } else {
                // one-sided x / y derivatives where the node is on a face: a y-face row as a
                // whole warp; the rim warps for the rim and the column of the tile's x face,
                // whose lanes in the other rows leave their node to them (xskip)
                if (pym != 0) {
                    feq_reg<HX, FS, true>(a, r0 + hp, c0, um, up, sFp, pxm, pym, 0, z0, f_rest,
                                          f_pz, f_mz);
                } else if (!xskip) {
                    feq_reg<HX, FS, false>(a, r0 + hp, c0, um, up, sFp, 0, 0, 0, z0, f_rest,
                                           f_pz, f_mz);
                    if (pxm != 0)   // a tile holding both x faces
                        feq_reg<HX, FS, true>(a, r0 + hp, c0, um, up, sFp, pxm, 0, 0, z0, f_rest,
                                              f_pz, f_mz);
                }
                if (has_rim) {
                    float d0, d1, d2;
                    if (rim_edge)
                        feq_reg<HX, FS, true>(a, r0 + hr, rc0, rum, rup, sF + forr, rxm, rym, 0,
                                              z0, d0, d1, d2);
                    else
                        feq_reg<HX, FS, false>(a, r0 + hr, rc0, rum, rup, sF + forr, 0, 0, 0, z0,
                                               d0, d1, d2);
                }
            }
        } else {
            const int z2 = (zm == 1) ? 2 : nz - 3;
            float4 zf = make_float4(0.f, 0.f, 0.f, 0.f);
            if (zm != 0 && in_xy) zf = a.src[((long long)z2 * ny + gy) * nx + gx];
            feq_reg<HX, FS, true>(a, r0 + hp, c0, um, up, sFp, pxm, pym, zm, zf, f_rest, f_pz,
                                  f_mz);
            if (has_rim) {
                float4 zr = make_float4(0.f, 0.f, 0.f, 0.f);
                if (zm != 0 && rim_in_xy) zr = a.src[((long long)z2 * ny + hgy) * nx + hgx];
                float d0, d1, d2;
                feq_reg<HX, FS, true>(a, r0 + hr, rc0, rum, rup, sF + forr, rxm, rym, zm, zr, d0,
                                      d1, d2);
            }
        }
        um = make_float3(c0.y, c0.z, c0.w);
        c0 = cpn;
        rum = make_float3(rc0.y, rc0.z, rc0.w);
        rc0 = rcpn;
        if (__syncthreads_or(!good)) {
            ok = false;
            return;
        }
        // every thread is past its reads of plane p - 1: its slot takes load k(p) - 1 + NSLOT
        if (tid == 0 && ik < nplanes) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_load_box(smem_addr(raw + (size_t)islot * C::SLOT), &tmap, x0 - 2, y0 - 2,
                         q0 - 2 + ik, smem_addr(&bars[islot]), C::PLANE_BYTES);
        }
        ++ik;
        if (++islot == NSLOT) islot = 0;
        s0 = wslot;
        if (++wslot == NSLOT) {
            wslot = 0;
            wpar ^= 1;
        }
        const float fpx = sFp[0 * FS - 1], fmx = sFp[1 * FS + 1];
        const float fpy = sFp[2 * FS - FX], fmy = sFp[3 * FS + FX];
        const float cpp_p = sFp[4 * FS - 1 - FX], cmp_p = sFp[5 * FS + 1 - FX];
        const float cpm_p = sFp[6 * FS - 1 + FX], cmm_p = sFp[7 * FS + 1 + FX];
        const float cpp_m = sFp[8 * FS - 1 - FX], cmp_m = sFp[9 * FS + 1 - FX];
        const float cpm_m = sFp[10 * FS - 1 + FX], cmm_m = sFp[11 * FS + 1 + FX];
        outp += zstride;   // plane p - 1
        {
            const float sxp = cpp_m + cpm_m, sxm = cmp_m + cmm_m;
            const float syp = cpp_m + cmp_m, sym = cpm_m + cmm_m;
            const float all = sxp + sxm + f_mz;
            const int qz = p - 1;
            if (STEADY ? out_col : (out_col && qz >= zlo && qz <= zhi)) {
                const float r = acc0[0] + all;
                const float ux = acc0[1] + (sxp - sxm) + bfx;
                const float uy = acc0[2] + (syp - sym) + bfy;
                const float uz = acc0[3] - all + bfz;
                float4 o;
                o.x = r;
                const int bz = qz - g.blo[2];
                if (box_col && bz >= 0 && bz < g.bn[2]) {
                    const float4 ks = kus_col[(long long)qz * box_plane];
                    const float inv = 1.f / (1.f + ks.x);
                    o.y = fmaf(ks.x, ks.y, ux) * inv;
                    o.z = fmaf(ks.x, ks.z, uy) * inv;
                    o.w = fmaf(ks.x, ks.w, uz) * inv;
                } else {
                    o.y = ux;
                    o.z = uy;
                    o.w = uz;
                }
                *outp = o;   // the boundary copies follow in k_bc_shell3d
            }
        }
        acc0[0] = acc1[0] + (f_rest + fpx + fmx + fpy + fmy);
        acc0[1] = acc1[1] + (fpx - fmx);
        acc0[2] = acc1[2] + (fpy - fmy);
        acc0[3] = acc1[3];
        {
            const float sxp = cpp_p + cpm_p, sxm = cmp_p + cmm_p;
            const float syp = cpp_p + cmp_p, sym = cpm_p + cmm_p;
            const float all = sxp + sxm + f_pz;
            acc1[0] = all;
            acc1[1] = sxp - sxm;
            acc1[2] = syp - sym;
            acc1[3] = all;
        }
    };
    // steady planes: output plane p - 1 in [max(q0, 2), nz - 3] and f^eq plane p off the faces
    const int ps0 = max(q0 + 1, 3), ps1 = min(q1, nz - 2);
    int p = q0 - 1;
    for (; ok && p <= q1 && p < ps0; ++p) plane(p, std::false_type{});
#pragma unroll 1
    for (; ok && p <= ps1; ++p) plane(p, std::true_type{});
    for (; ok && p <= q1; ++p) plane(p, std::false_type{});
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

template <int TY_>
__global__ void __launch_bounds__(ZCfg<TY_>::NTHR, ZCfg<TY_>::MINB)
    k_zstep3d(const __grid_constant__ CUtensorMap tmap, const FusedArgs a) {
    using C = ZCfg<TY_>;
    constexpr int TX = C::TX, TY = C::TY;
    constexpr int NSLOT = C::NSLOT;
    extern __shared__ __align__(128) unsigned char smem[];
    float4* raw = reinterpret_cast<float4*>(smem);
    float* sFbase = reinterpret_cast<float*>(smem + C::OFF_F);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    const Geom& g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int q0 = blockIdx.z * a.zchunk;
    const int q1 = min(nz, q0 + a.zchunk);
    const int nplanes = q1 - q0 + 4;   // raw planes q0-2 .. q1+1 (load index k = plane - q0 + 2)
    // rim nodes over whole warps: lanes past the last rim node repeat earlier ones (the same
    // values are stored twice), so no warp splits on the rim work
    int hfx, hfy;   // threads past the rim warps keep (0, 0): they read, never store
    rim_node<TX, TY, C::NHALO>(tid, x0, nx, hfx, hfy);
    if ((smem_addr(smem) & 127u) != 0u) {
        if (tid == 0) atomicOr(a.err, 16);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(smem_addr(&bars[s]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int k = 0; k < NSLOT && k < nplanes; ++k)
            tma_load_box(smem_addr(raw + (size_t)k * C::SLOT), &tmap, x0 - 2, y0 - 2,
                         q0 - 2 + k, smem_addr(&bars[k]), C::PLANE_BYTES);
    }
    __syncthreads();
    // a tile whose raw halo lies inside the grid and whose f^eq region and columns keep two
    // nodes away from the x and y faces takes the path without face tests
    const bool interior = x0 >= 3 && x0 + TX + 2 <= nx - 1 && y0 >= 3 && y0 + TY + 2 <= ny - 1;
    if (interior)
        zbody<TY_, true>(tmap, a, smem, hfx, hfy, q0, q1, nplanes);
    else
        zbody<TY_, false>(tmap, a, smem, hfx, hfy, q0, q1, nplanes);
}

// ---------------------------------------------------------------- plane-pair z-march variant
// The same step with two planes per iteration and packed single-precision arithmetic:
//   * a thread owns one column of a 32 x 8 tile and evaluates f^eq at two consecutive planes
//     (a, a + 1) per iteration, with the two planes' values held as float2 pairs, so the f^eq
//     core, the gather sums and the z-accumulation run on paired FP32 instructions
//     (__ffma2_rn, __fadd2_rn, __fmul2_rn: two operations per instruction issue);
//   * the 12 values that leave the column travel through shared memory as (plane a, plane a+1)
//     pairs: an in-plane shift keeps the pairing, so every exchange is one 8-byte store and one
//     8-byte load for two nodes; the exchange buffers alternate, one block barrier per pair;
//   * raw planes arrive through the same TMA boxes into a six-slot ring, two new planes per
//     iteration, every thread waiting on the mbarriers of the planes it reads (bounded waits);
//   * an iteration completes the outputs of planes a - 1 and a: plane a - 1 from the carried
//     cz = 0 and cz = +1 sums of plane a - 1 and a - 2 plus the cz = -1 sums of plane a, plane
//     a from its own cz = 0 sums, the carried cz = +1 sums of plane a - 1 and the cz = -1 sums
//     of plane a + 1.
// Derivatives are formed per plane in single precision as in feq_node; the arithmetic of f^eq,
// the gather and the Brinkman update is that of the other variants, with the sums in a
// different order (results agree to rounding).
struct PCfg {
    static constexpr int TX = 32, TY = 8;
    static constexpr int HX = TX + 5, HY = TY + 4, FW = TX + 2, FX = FW + 1, FY = TY + 2;
    static constexpr int NTHR = TX * TY, NHALO = FW * FY - TX * TY, FS = FX * FY;
    static constexpr int NSLOT = 6;
    static constexpr int MINB = 2;     // resident blocks per SM
    static constexpr unsigned PLANE_BYTES = HX * HY * 16;
    static constexpr int SLOT = (PLANE_BYTES + 127) / 128 * 128 / 16;   // float4 per ring slot
    static constexpr size_t OFF_F = (size_t)NSLOT * SLOT * 16;
    static constexpr size_t OFF_BAR = OFF_F + (size_t)2 * NCROSS * FS * 8;
    static constexpr size_t SMEM = OFF_BAR + NSLOT * 8;
};

// Packed constants of the pair kernel (both lanes equal).
struct PairK {
    float2 A, hA, m15, w0, w1, w13, nw13, h1, w2, w23, nw23, h2, w2x2, nw2x2, mone;
};

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b: b * (-1) is exact, so this rounds once like a subtraction
__device__ __forceinline__ float2 psub(float2 a, float2 b, float2 mone) {
    return __ffma2_rn(b, mone, a);
}

// Dab = 2 d u_a / d x_b of one plane at one column (naming as in feq_node): c0 points at the
// node in its ring plane, c is the node, um / up the velocity one plane below / above.
struct D9 {
    float xx, yx, zx, xy, yy, zy, xz, yz, zz;
};

template <bool EDGE>
__device__ __forceinline__ void deriv_plane(const float4* __restrict__ c0, const float4& c,
                                            const float3& um, const float3& up, int xm, int ym,
                                            int zm, const float4& zfar, D9& d) {
    constexpr int HXs = PCfg::HX;
    if (EDGE) {
        const float4 cm4 = make_float4(0.f, um.x, um.y, um.z);
        const float4 cp4 = make_float4(0.f, up.x, up.y, up.z);
        deriv2(xm, c, c0[-1], c0[1], xm == 2 ? c0[-2] : c, xm == 1 ? c0[2] : c, d.xx, d.yx, d.zx);
        deriv2(ym, c, c0[-HXs], c0[HXs], ym == 2 ? c0[-2 * HXs] : c, ym == 1 ? c0[2 * HXs] : c,
               d.xy, d.yy, d.zy);
        deriv2(zm, c, cm4, cp4, zfar, zfar, d.xz, d.yz, d.zz);
    } else {
        const float4 e = c0[1], w = c0[-1], n = c0[HXs], s = c0[-HXs];
        d.xx = e.y - w.y;
        d.yx = e.z - w.z;
        d.zx = e.w - w.w;
        d.xy = n.y - s.y;
        d.yy = n.z - s.z;
        d.zy = n.w - s.w;
        d.xz = up.x - um.x;
        d.yz = up.y - um.y;
        d.zz = up.z - um.z;
    }
}

// f^eq of one column at two planes (lanes: plane a, plane a + 1) from the node values c* and
// the derivatives of each plane: stores the 12 values that leave the column into the pair
// planes at sFn (FS pairs apart) and returns rest, +z and -z.  The operations are those of
// feq_node on pairs.
__device__ __forceinline__ void feq_pair(const PairK& k, const float4& ca, const float4& cb,
                                         const D9& da, const D9& db, float2* __restrict__ sFn,
                                         float2& f_rest, float2& f_pz, float2& f_mz) {
    constexpr int FS = PCfg::FS;
    const float2 r = make_float2(ca.x, cb.x), ux = make_float2(ca.y, cb.y);
    const float2 uy = make_float2(ca.z, cb.z), uz = make_float2(ca.w, cb.w);
    const float2 ASxx = pmul(k.A, make_float2(da.xx, db.xx));
    const float2 ASyy = pmul(k.A, make_float2(da.yy, db.yy));
    const float2 ASzz = pmul(k.A, make_float2(da.zz, db.zz));
    const float2 ASxy = pmul(k.hA, padd(make_float2(da.xy, db.xy), make_float2(da.yx, db.yx)));
    const float2 ASxz = pmul(k.hA, padd(make_float2(da.xz, db.xz), make_float2(da.zx, db.zx)));
    const float2 ASyz = pmul(k.hA, padd(make_float2(da.yz, db.yz), make_float2(da.zy, db.zy)));
    const float2 uu = pfma(uz, uz, pfma(uy, uy, pmul(ux, ux)));
    const float2 P = pfma(k.m15, uu, r);
    f_rest = pmul(k.w0, P);
    const float2 Px = padd(P, ASxx);
    {
        const float2 b = pfma(pmul(k.h1, ux), ux, pmul(k.w1, Px));
        sFn[0 * FS] = pfma(k.w13, ux, b);
        sFn[1 * FS] = pfma(k.nw13, ux, b);
    }
    {
        const float2 b = pfma(pmul(k.h1, uy), uy, pmul(k.w1, padd(P, ASyy)));
        sFn[2 * FS] = pfma(k.w13, uy, b);
        sFn[3 * FS] = pfma(k.nw13, uy, b);
    }
    {
        const float2 b = pfma(pmul(k.h1, uz), uz, pmul(k.w1, padd(P, ASzz)));
        f_pz = pfma(k.w13, uz, b);
        f_mz = pfma(k.nw13, uz, b);
    }
    const float2 T0 = pmul(k.w2, padd(padd(Px, ASyy), ASzz));
    const float2 s1 = padd(ux, uy), d1 = psub(ux, uy, k.mone);
    const float2 q1 = padd(ASxz, ASyz), q2 = psub(ASyz, ASxz, k.mone);
    {   // (+,+,+) / (-,-,-)
        const float2 cu = padd(s1, uz);
        const float2 sym = pfma(pmul(k.h2, cu), cu, pfma(k.w2x2, padd(ASxy, q1), T0));
        sFn[4 * FS] = pfma(k.w23, cu, sym);
        sFn[11 * FS] = pfma(k.nw23, cu, sym);
    }
    {   // (-,+,+) / (+,-,-)
        const float2 cu = psub(uz, d1, k.mone);
        const float2 sym = pfma(pmul(k.h2, cu), cu, pfma(k.w2x2, psub(q2, ASxy, k.mone), T0));
        sFn[5 * FS] = pfma(k.w23, cu, sym);
        sFn[10 * FS] = pfma(k.nw23, cu, sym);
    }
    {   // (+,-,+) / (-,+,-)
        const float2 cu = padd(uz, d1);
        const float2 sym = pfma(pmul(k.h2, cu), cu, pfma(k.nw2x2, padd(ASxy, q2), T0));
        sFn[6 * FS] = pfma(k.w23, cu, sym);
        sFn[9 * FS] = pfma(k.nw23, cu, sym);
    }
    {   // (-,-,+) / (+,+,-)
        const float2 cu = psub(uz, s1, k.mone);
        const float2 sym = pfma(pmul(k.h2, cu), cu, pfma(k.w2x2, psub(ASxy, q1, k.mone), T0));
        sFn[7 * FS] = pfma(k.w23, cu, sym);
        sFn[8 * FS] = pfma(k.nw23, cu, sym);
    }
}

struct PairArgs {
    FusedArgs f;
    PairK k;
    float2 bf2[3];   // body force, both lanes
    int has_bf;
};

// Write one output node (Brinkman update, store, boundary copies it sources).
__device__ __forceinline__ void pair_out(const Geom& g, const PairArgs& a, int gx, int gy,
                                         int qz, float r, float ux, float uy, float uz,
                                         bool box_col, const float4* kus_col,
                                         long long box_plane, float4* out_col_ptr,
                                         long long zstride, bool bc_col) {
    float4 o;
    o.x = r;
    const int bz = qz - g.blo[2];
    if (box_col && bz >= 0 && bz < g.bn[2]) {
        const float4 ks = kus_col[(long long)qz * box_plane];
        const float inv = 1.f / (1.f + ks.x);
        o.y = fmaf(ks.x, ks.y, ux) * inv;
        o.z = fmaf(ks.x, ks.z, uy) * inv;
        o.w = fmaf(ks.x, ks.w, uz) * inv;
    } else {
        o.y = ux;
        o.z = uy;
        o.w = uz;
    }
    out_col_ptr[(long long)qz * zstride] = o;
    if (bc_col || qz == 1 || qz == g.n[2] - 2) write_bc_f(g, gx, gy, qz, o, a.f.out);
}

// The z derivative at a z-face plane is the one-sided difference; with a ghost value
// g = 3 u(0) - 3 u(1) + u(2) below plane 0 (or 3 u(n-1) - 3 u(n-2) + u(n-3) above plane n-1) the
// central difference u(1) - g (g - u(n-2)) equals it, so the pair path keeps one formula.
__device__ __forceinline__ float3 zghost(const float3& f, const float3& s, const float3& t) {
    return make_float3(fmaf(3.f, f.x - s.x, t.x), fmaf(3.f, f.y - s.y, t.y),
                       fmaf(3.f, f.z - s.z, t.z));
}

__device__ __forceinline__ float3 u3(const float4& v) { return make_float3(v.y, v.z, v.w); }

// z derivatives (2 d u / d z) of the pair's planes a0 (da) and a0 + 1 (db) at a z face, from
// the ghost value: um, ua, ub, uc are u at a0 - 1 .. a0 + 2; col points at the column in the
// source state (for u(2) or u(nz - 3) when the pair does not hold it).
__device__ __forceinline__ void zface_fix(int a0, int nz, const float3& um, const float3& ua,
                                       const float3& ub, const float3& uc,
                                       const float4* __restrict__ col, long long zstride,
                                       D9& da, D9& db) {
    if (a0 == 0) {   // plane 0 first: ghost below it
        const float3 gh = zghost(ua, ub, uc);
        da.xz = ub.x - gh.x;
        da.yz = ub.y - gh.y;
        da.zz = ub.z - gh.z;
    }
    if (a0 == -1) {  // plane 0 second
        const float3 gh = zghost(ub, uc, u3(col[2 * zstride]));
        db.xz = uc.x - gh.x;
        db.yz = uc.y - gh.y;
        db.zz = uc.z - gh.z;
    }
    if (a0 + 1 == nz - 1) {   // plane nz-1 second: ghost above it
        const float3 gh = zghost(ub, ua, um);
        db.xz = gh.x - ua.x;
        db.yz = gh.y - ua.y;
        db.zz = gh.z - ua.z;
    }
    if (a0 == nz - 1) {   // plane nz-1 first
        const float3 gh = zghost(ua, um, u3(col[(long long)(nz - 3) * zstride]));
        da.xz = gh.x - um.x;
        da.yz = gh.y - um.y;
        da.zz = gh.z - um.z;
    }
}

// The plane-pair march of one interior tile (its raw halo inside the grid, no x or y face
// within two nodes): no face tests in x and y; z-face planes through ghost values.
__device__ __forceinline__ void pbody(const CUtensorMap& tmap, const PairArgs& a,
                                      unsigned char* smem, int hfx, int hfy, int q0, int q1) {
    using C = PCfg;
    constexpr int TX = C::TX, HX = C::HX, FX = C::FX;
    constexpr int FS = C::FS, NSLOT = C::NSLOT;
    float4* raw = reinterpret_cast<float4*>(smem);
    float2* sFbase = reinterpret_cast<float2*>(smem + C::OFF_F);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    const Geom& g = a.f.g;
    const PairK& k = a.k;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * C::TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const int hgx = x0 - 1 + hfx, hgy = y0 - 1 + hfy;
    const int hp = (ty + 2) * HX + (tx + 2);
    const int hr = (hfy + 1) * HX + (hfx + 1);
    const int fop = (ty + 1) * FX + (tx + 1);
    const int forr = hfy * FX + hfx;
    constexpr int RIMW = (C::NHALO + 31) / 32 * 32;
    const bool has_rim = tid < RIMW;
    const bool bc_col = false;
    const int bxx = gx - g.blo[0], byy = gy - g.blo[1];
    const bool box_col = g.boxN > 0 && bxx >= 0 && byy >= 0 && bxx < g.bn[0] && byy < g.bn[1];
    const long long box_plane = (long long)g.bn[0] * g.bn[1];
    const float4* kus_col =
        a.f.kus + ((long long)byy * g.bn[0] + bxx) - (long long)g.blo[2] * box_plane;
    const long long zstride = (long long)nx * ny;
    float4* out_col_ptr = a.f.out + ((long long)gy * nx + gx);
    const float4* src_col = a.f.src + ((long long)gy * nx + gx);
    const float4* src_rim = a.f.src + ((long long)hgy * nx + hgx);
    const int zlo = max(q0, 1), zhi = min(q1 - 1, nz - 2);
    const int npairs = ((q1 - q0 + 1) >> 1) + 1;
    const int nplanes = 2 * npairs + 2;

    bool ok = true;
    float3 um, rum;
    float4 ca, rca;
    {
        bool good = true;
        for (int j = 0; j < 4; ++j) good = mbar_wait_once(smem_addr(&bars[j]), 0) && good;
        um = u3(raw[hp]);
        ca = raw[(size_t)C::SLOT + hp];
        rum = u3(raw[hr]);
        rca = raw[(size_t)C::SLOT + hr];
        ok = !__syncthreads_or(!good);
    }
    float pend_r = 0.f, pend_x = 0.f, pend_y = 0.f, pend_z = 0.f;
    float pc_r = 0.f, pc_x = 0.f, pc_y = 0.f, pc_z = 0.f;
    int ik = NSLOT;
    // ring slots and phase parities of the loads of planes a0, a0 + 1, a0 + 2
    int sa = 1, sb = 2, sc = 3, pb = 0, pcp = 0;
    for (int it = 0; ok && it < npairs; ++it) {
        const int a0 = q0 - 1 + 2 * it;
        bool good = true;
        if (it > 0) good = mbar_wait_once(smem_addr(&bars[sb]), pb);
        good = mbar_wait_once(smem_addr(&bars[sc]), pcp) && good;
        const float4* ra = raw + (size_t)sa * C::SLOT;
        const float4* rb = raw + (size_t)sb * C::SLOT;
        const float4* rc = raw + (size_t)sc * C::SLOT;
        float2* sF = sFbase + (size_t)(it & 1) * NCROSS * FS;
        const float4 cb = rb[hp], cc = rc[hp];
        const float3 ub = u3(cb), uc = u3(cc), ua = u3(ca);
        const bool zface = a0 <= 0 || a0 + 1 >= nz - 1;
        float2 f_rest, f_pz, f_mz;
        {
            D9 da, db;
            const float4 z0 = make_float4(0.f, 0.f, 0.f, 0.f);
            deriv_plane<false>(ra + hp, ca, um, ub, 0, 0, 0, z0, da);
            deriv_plane<false>(rb + hp, cb, ua, uc, 0, 0, 0, z0, db);
            if (zface) zface_fix(a0, nz, um, ua, ub, uc, src_col, zstride, da, db);
            feq_pair(k, ca, cb, da, db, sF + fop, f_rest, f_pz, f_mz);
            if (has_rim) {
                const float4 rcb = rb[hr], rcc = rc[hr];
                const float3 rua = u3(rca), rub = u3(rcb), ruc = u3(rcc);
                deriv_plane<false>(ra + hr, rca, rum, rub, 0, 0, 0, z0, da);
                deriv_plane<false>(rb + hr, rcb, rua, ruc, 0, 0, 0, z0, db);
                if (zface) zface_fix(a0, nz, rum, rua, rub, ruc, src_rim, zstride, da, db);
                float2 d0, d1, d2;
                feq_pair(k, rca, rcb, da, db, sF + forr, d0, d1, d2);
                rum = rub;
                rca = rcc;
            }
        }
        um = ub;
        ca = cc;
        if (__syncthreads_or(!good)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            const int jmax = min(2 * it + 9, nplanes);
            if (ik < jmax) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (; ik < jmax; ++ik)
                tma_load_box(smem_addr(raw + (size_t)(ik % NSLOT) * C::SLOT), &tmap, x0 - 2,
                             y0 - 2, q0 - 2 + ik, smem_addr(&bars[ik % NSLOT]), C::PLANE_BYTES);
        }
        // advance the slots by two planes
        sa = sc;
        sb += 2;
        if (sb >= NSLOT) {
            sb -= NSLOT;
            pb ^= 1;
        }
        sc += 2;
        if (sc >= NSLOT) {
            sc -= NSLOT;
            pcp ^= 1;
        }
        const float2* sFp = sF + fop;
        const float2 fpx = sFp[0 * FS - 1], fmx = sFp[1 * FS + 1];
        const float2 fpy = sFp[2 * FS - FX], fmy = sFp[3 * FS + FX];
        const float2 cpp_p = sFp[4 * FS - 1 - FX], cmp_p = sFp[5 * FS + 1 - FX];
        const float2 cpm_p = sFp[6 * FS - 1 + FX], cmm_p = sFp[7 * FS + 1 + FX];
        const float2 cpp_m = sFp[8 * FS - 1 - FX], cmp_m = sFp[9 * FS + 1 - FX];
        const float2 cpm_m = sFp[10 * FS - 1 + FX], cmm_m = sFp[11 * FS + 1 + FX];
        float2 Mr, Mx, My;
        {
            const float2 sxp = padd(cpp_m, cpm_m), sxm = padd(cmp_m, cmm_m);
            const float2 syp = padd(cpp_m, cmp_m), sym = padd(cpm_m, cmm_m);
            Mr = padd(padd(sxp, sxm), f_mz);
            Mx = psub(sxp, sxm, k.mone);
            My = psub(syp, sym, k.mone);
        }
        const float2 Zr = padd(padd(padd(f_rest, fpx), padd(fmx, fpy)), fmy);
        const float2 Zx = psub(fpx, fmx, k.mone), Zy = psub(fpy, fmy, k.mone);
        float2 Pr, Px, Py;
        {
            const float2 sxp = padd(cpp_p, cpm_p), sxm = padd(cmp_p, cmm_p);
            const float2 syp = padd(cpp_p, cmp_p), sym = padd(cpm_p, cmm_p);
            Pr = padd(padd(sxp, sxm), f_pz);
            Px = psub(sxp, sxm, k.mone);
            Py = psub(syp, sym, k.mone);
        }
        float2 orr = padd(make_float2(pend_r, Zr.x + pc_r), Mr);
        float2 oxx = padd(make_float2(pend_x, Zx.x + pc_x), Mx);
        float2 oyy = padd(make_float2(pend_y, Zy.x + pc_y), My);
        float2 ozz = psub(make_float2(pend_z, pc_z), Mr, k.mone);
        if (a.has_bf) {
            oxx = padd(oxx, a.bf2[0]);
            oyy = padd(oyy, a.bf2[1]);
            ozz = padd(ozz, a.bf2[2]);
        }
        pend_r = Zr.y + Pr.x;
        pend_x = Zx.y + Px.x;
        pend_y = Zy.y + Py.x;
        pend_z = Pr.x;
        pc_r = Pr.y;
        pc_x = Px.y;
        pc_y = Py.y;
        pc_z = Pr.y;
        if (a0 - 1 >= zlo && a0 - 1 <= zhi)
            pair_out(g, a, gx, gy, a0 - 1, orr.x, oxx.x, oyy.x, ozz.x, box_col, kus_col,
                     box_plane, out_col_ptr, zstride, bc_col);
        if (a0 >= zlo && a0 <= zhi)
            pair_out(g, a, gx, gy, a0, orr.y, oxx.y, oyy.y, ozz.y, box_col, kus_col, box_plane,
                     out_col_ptr, zstride, bc_col);
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(a.f.err, 8);
            const long long t0 = clock64();
            while (clock64() - t0 < (1LL << 28)) {
            }
        }
        __syncthreads();
    }
}

// Interior tiles march plane pairs; tiles near an x or y face take the register z-march of
// variant 1 (zbody, its own five-slot ring inside the same shared memory) for their face rules.
__global__ void __launch_bounds__(PCfg::NTHR, PCfg::MINB)
    k_zpair3d(const __grid_constant__ CUtensorMap tmap, const PairArgs a) {
    using C = PCfg;
    using Z = ZCfg<8>;
    static_assert(C::TX == Z::TX && C::TY == Z::TY && C::SLOT == Z::SLOT && C::HX == Z::HX &&
                      C::HY == Z::HY && Z::SMEM <= C::SMEM,
                  "edge tiles reuse the register z-march in the same shared memory");
    constexpr int TX = C::TX, TY = C::TY;
    extern __shared__ __align__(128) unsigned char smem[];
    float4* raw = reinterpret_cast<float4*>(smem);
    const Geom& g = a.f.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int q0 = blockIdx.z * a.f.zchunk;
    const int q1 = min(nz, q0 + a.f.zchunk);
    int hfx, hfy;
    rim_node<TX, TY, C::NHALO>(tid, x0, nx, hfx, hfy);
    if ((smem_addr(smem) & 127u) != 0u) {
        if (tid == 0) atomicOr(a.f.err, 16);
        return;
    }
    const bool interior = x0 >= 3 && x0 + TX + 2 <= nx - 1 && y0 >= 3 && y0 + TY + 2 <= ny - 1;
    if (interior) {
        const int npairs = ((q1 - q0 + 1) >> 1) + 1;
        const int nplanes = 2 * npairs + 2;
        uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
        if (tid == 0) {
            for (int s = 0; s < C::NSLOT; ++s) mbar_init(smem_addr(&bars[s]));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int j = 0; j < C::NSLOT && j < nplanes; ++j)
                tma_load_box(smem_addr(raw + (size_t)j * C::SLOT), &tmap, x0 - 2, y0 - 2,
                             q0 - 2 + j, smem_addr(&bars[j]), C::PLANE_BYTES);
        }
        __syncthreads();
        pbody(tmap, a, smem, hfx, hfy, q0, q1);
    } else {
        const int nplanes = q1 - q0 + 4;
        uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Z::OFF_BAR);
        if (tid == 0) {
            for (int s = 0; s < Z::NSLOT; ++s) mbar_init(smem_addr(&bars[s]));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            for (int j = 0; j < Z::NSLOT && j < nplanes; ++j)
                tma_load_box(smem_addr(raw + (size_t)j * Z::SLOT), &tmap, x0 - 2, y0 - 2,
                             q0 - 2 + j, smem_addr(&bars[j]), Z::PLANE_BYTES);
        }
        __syncthreads();
        zbody<8, false>(tmap, a.f, smem, hfx, hfy, q0, q1, nplanes);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

}  // namespace

bool fused3d_eligible(const Geom& g) {
    return g.dim == 3 && !g.periodic[0] && !g.periodic[1] && !g.periodic[2] && g.n[0] >= 3 &&
           g.n[1] >= 3 && g.n[2] >= 4 && get_encode() != nullptr;
}

// Tensor map over a float4-per-node state array {4, nx, ny, nz} with a {4, bx, by, 1} box;
// coordinates outside the grid read as zeros.
bool encode_state_map(CUtensorMap* map, const void* base, const Geom& g, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[4] = {4, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    cuuint64_t strides[3] = {16, (cuuint64_t)g.n[0] * 16, (cuuint64_t)g.n[0] * g.n[1] * 16};
    cuuint32_t box[4] = {4, (cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Planes per z chunk so that the grid fills a whole number of waves of `per_sm` resident
// blocks per SM, weighing each chunk's three warm-up planes: the chunk count with the best
// product of wave fill and useful-plane fraction, chunks of at least 8 planes (small grids need
// many chunks to fill the SMs at all).
int fused_zchunk_waves(const Geom& g, long long tiles, int per_sm) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)nsm * per_sm;
    const int maxc = std::max(1, g.n[2] / 8);
    int best = 1;
    double best_eff = 0.0;
    for (int c = 1; c <= maxc; ++c) {
        const long long blocks = tiles * c;
        const long long waves = (blocks + slots - 1) / slots;
        const int zc = (g.n[2] + c - 1) / c;
        // useful fraction: filled wave slots x planes that are not pipeline warm-up
        const double eff = (double)blocks / (double)(waves * slots) * zc / (zc + 3.0);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = c;
        }
    }
    return (g.n[2] + best - 1) / best;
}

template <int TY_>
cudaError_t launch_zstep(const Geom& g, const CUtensorMap& map, const FusedArgs& a0,
                         cudaStream_t st) {
    using C = ZCfg<TY_>;
    static std::atomic<unsigned> attr{0};   // devices whose shared-memory limit is raised
    if (!device_done(attr)) {
        cudaError_t e = cudaFuncSetAttribute(k_zstep3d<TY_>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        device_mark(attr);
    }
    FusedArgs a = a0;
    const int tiles_x = (g.n[0] + C::TX - 1) / C::TX, tiles_y = (g.n[1] + C::TY - 1) / C::TY;
    a.zchunk = fused_zchunk_waves(g, (long long)tiles_x * tiles_y, C::MINB);
    const int chunks = (g.n[2] + a.zchunk - 1) / a.zchunk;
    k_zstep3d<TY_><<<dim3(tiles_x, tiles_y, chunks), C::NTHR, C::SMEM, st>>>(map, a);
    return cudaGetLastError();
}

cudaError_t launch_zpair(const Geom& g, const CUtensorMap& map, const FusedArgs& f0,
                         cudaStream_t st) {
    using C = PCfg;
    static std::atomic<unsigned> attr{0};   // devices whose shared-memory limit is raised
    if (!device_done(attr)) {
        cudaError_t e = cudaFuncSetAttribute(k_zpair3d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        device_mark(attr);
    }
    PairArgs a;
    a.f = f0;
    const auto two = [](float v) { return make_float2(v, v); };
    a.k.A = two(f0.A);
    a.k.hA = two(0.5f * f0.A);
    a.k.m15 = two(-1.5f);
    using Wf = Wts<float, 3>;
    a.k.w0 = two(Wf::w0);
    a.k.w1 = two(Wf::w1);
    a.k.w13 = two(Wf::w3_1);
    a.k.nw13 = two(-Wf::w3_1);
    a.k.h1 = two(Wf::h_1);
    a.k.w2 = two(Wf::w2);
    a.k.w23 = two(Wf::w3_2);
    a.k.nw23 = two(-Wf::w3_2);
    a.k.h2 = two(Wf::h_2);
    a.k.w2x2 = two(2.f * Wf::w2);
    a.k.nw2x2 = two(-2.f * Wf::w2);
    a.k.mone = two(-1.f);
    for (int d = 0; d < 3; ++d) a.bf2[d] = two(f0.bf[d]);
    a.has_bf = (f0.bf[0] != 0.f || f0.bf[1] != 0.f || f0.bf[2] != 0.f) ? 1 : 0;
    const int tiles_x = (g.n[0] + C::TX - 1) / C::TX, tiles_y = (g.n[1] + C::TY - 1) / C::TY;
    a.f.zchunk = fused_zchunk_waves(g, (long long)tiles_x * tiles_y, C::MINB);
    const int chunks = (g.n[2] + a.f.zchunk - 1) / a.f.zchunk;
    k_zpair3d<<<dim3(tiles_x, tiles_y, chunks), C::NTHR, C::SMEM, st>>>(map, a);
    return cudaGetLastError();
}

// One fused forward step src -> dst in variant v (0: shared-memory z-march with two barriers
// per plane, 1: register z-march, 2: plane-pair z-march with packed arithmetic), all on
// 32 x 8 tiles.  Returns a CUDA error code.
cudaError_t launch_fused_step3d(const Geom& g, const V4<float>* src, const V4<float>* kus,
                                V4<float>* dst, int* err, cudaStream_t st, int v) {
    FusedArgs a;
    a.g = g;
    a.out = reinterpret_cast<float4*>(dst);
    a.kus = reinterpret_cast<const float4*>(kus);
    a.src = reinterpret_cast<const float4*>(src);
    a.err = err;
    a.A = (float)g.A;
    a.w0 = Wts<float, 3>::w0;
    a.w1 = Wts<float, 3>::w1;
    a.w2 = Wts<float, 3>::w2;
    for (int k = 0; k < 3; ++k) a.bf[k] = (float)g.body[k];
    CUtensorMap map;
    if (v == 1 || v == 2) {
        cudaError_t e;
        if (v == 2) {
            if (!encode_state_map(&map, src, g, PCfg::HX, PCfg::HY)) return cudaErrorInvalidValue;
            e = launch_zpair(g, map, a, st);
        } else {
            if (!encode_state_map(&map, src, g, ZCfg<8>::HX, ZCfg<8>::HY))
                return cudaErrorInvalidValue;
            e = launch_zstep<8>(g, map, a, st);
        }
        if (e != cudaSuccess) return e;
        ShellFaces F;
        for (int f = 0; f < 6; ++f) {
            F.v[f] = make_float4((float)g.bcv[f][0], (float)g.bcv[f][1], (float)g.bcv[f][2],
                                 (float)(g.bcv[f][3] - g.rho0));
            F.keep_rho[f] = g.bc[f] == BC_WALL || g.bc[f] == BC_INLET;
        }
        const long long ix = g.n[0] - 2, iy = g.n[1] - 2, iz = g.n[2] - 2;
        const long long shell = 2 * (iy * iz + ix * iz + ix * iy);
        k_bc_shell3d<<<(unsigned)((shell + 255) / 256), 256, 0, st>>>(g, F, a.out);
        return cudaGetLastError();
    }
    if (!encode_state_map(&map, src, g, HX, HY)) return cudaErrorInvalidValue;
    static std::atomic<unsigned> attr{0};   // devices whose shared-memory limit is raised
    if (!device_done(attr)) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_step3d,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        device_mark(attr);
    }
    const int tiles_x = (g.n[0] + TX - 1) / TX, tiles_y = (g.n[1] + TY - 1) / TY;
    a.zchunk = fused_zchunk_waves(g, (long long)tiles_x * tiles_y, 4);
    const int chunks = (g.n[2] + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles_x, tiles_y, chunks);
    k_fused_step3d<<<grid, NTHR, SMEM_BYTES, st>>>(map, a);
    return cudaGetLastError();
}

}  // namespace lks
