// Fused D3Q15 LKS step for the FP32 path on non-periodic grids: one kernel per time step.
//
// Algorithm 1's stencil part (Eqs. rho, u with the viscosity term of f^eq, the Brinkman update
// of Eq. u_ex_2 and the boundary rules of Eqs. bc_rho, bc_u) in one pass over the state:
//   * a block owns a 32 x 16 tile of output columns and marches along z over a chunk of planes;
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

#include "lks_device.cuh"

namespace lks {

namespace {

constexpr int TX = 32, TY = 16;             // output tile
constexpr int HX = TX + 4, HY = TY + 4;     // raw tile with a two-cell halo
constexpr int FX = TX + 2, FY = TY + 2;     // f^eq region with a one-cell halo
constexpr int NSLOT = 5;                    // raw-plane ring depth
constexpr int NTHR = TX * TY;               // 512
constexpr int NHALO = FX * FY - TX * TY;    // 100 extra f^eq nodes on the tile rim
constexpr int NCROSS = 12;                  // directions leaving the column
constexpr unsigned PLANE_BYTES = HX * HY * 16;

// shared-memory layout (bytes)
constexpr size_t OFF_RAW = 0;
constexpr size_t OFF_F = OFF_RAW + (size_t)NSLOT * PLANE_BYTES;
constexpr size_t OFF_BAR = OFF_F + (size_t)NCROSS * FX * FY * 4;
constexpr size_t SMEM_BYTES = OFF_BAR + NSLOT * 8;

// cross-direction slots in sF: 0 +x, 1 -x, 2 +y, 3 -y, 4..7 corners with cz=+1 (sx,sy) =
// (+,+),(-,+),(+,-),(-,-), 8..11 corners with cz=-1 in the same (sx,sy) order.
__device__ __forceinline__ int corner_slot(int sx, int sy, int sz) {
    return (sz > 0 ? 4 : 8) + (sx > 0 ? 0 : 1) + (sy > 0 ? 0 : 2);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_plane(uint32_t dst, const CUtensorMap* map, int x, int y,
                                               int z, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(PLANE_BYTES)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Bounded wait on an mbarrier phase: about a second of spinning, then give up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
}

struct FusedArgs {
    Geom g;
    float4* out;
    const float4* kus;
    const float4* src;    // same buffer the tensor map describes (for rare direct loads)
    int* err;
    int zchunk;
    float A, w0, w1, w2;
};

// Evaluate f^eq at one node of the f^eq region.  Stores the 12 cross-column values into sF and
// returns the rest, +z and -z values.
__device__ __forceinline__ void feq_node(const FusedArgs& a, const float4* __restrict__ rm,
                                         const float4* __restrict__ r0,
                                         const float4* __restrict__ rp, float* __restrict__ sF,
                                         int fx, int fy, int gx, int gy, int gz, float& f_rest,
                                         float& f_pz, float& f_mz) {
    const Geom& g = a.g;
    const int h = (fy + 1) * HX + (fx + 1);
    const float4 c = r0[h];
    // D_ab = 2 d u_a / d x_b : central differences, one-sided on boundary nodes
    float Dx[3], Dy[3], Dz[3];
    {
        const float4 e = r0[h + 1], w = r0[h - 1];
        if (gx == 0) {
            const float4 e2 = r0[h + 2];
            Dx[0] = -3.f * c.y + 4.f * e.y - e2.y;
            Dx[1] = -3.f * c.z + 4.f * e.z - e2.z;
            Dx[2] = -3.f * c.w + 4.f * e.w - e2.w;
        } else if (gx == g.n[0] - 1) {
            const float4 w2 = r0[h - 2];
            Dx[0] = 3.f * c.y - 4.f * w.y + w2.y;
            Dx[1] = 3.f * c.z - 4.f * w.z + w2.z;
            Dx[2] = 3.f * c.w - 4.f * w.w + w2.w;
        } else {
            Dx[0] = e.y - w.y;
            Dx[1] = e.z - w.z;
            Dx[2] = e.w - w.w;
        }
    }
    {
        const float4 nn = r0[h + HX], ss = r0[h - HX];
        if (gy == 0) {
            const float4 n2 = r0[h + 2 * HX];
            Dy[0] = -3.f * c.y + 4.f * nn.y - n2.y;
            Dy[1] = -3.f * c.z + 4.f * nn.z - n2.z;
            Dy[2] = -3.f * c.w + 4.f * nn.w - n2.w;
        } else if (gy == g.n[1] - 1) {
            const float4 s2 = r0[h - 2 * HX];
            Dy[0] = 3.f * c.y - 4.f * ss.y + s2.y;
            Dy[1] = 3.f * c.z - 4.f * ss.z + s2.z;
            Dy[2] = 3.f * c.w - 4.f * ss.w + s2.w;
        } else {
            Dy[0] = nn.y - ss.y;
            Dy[1] = nn.z - ss.z;
            Dy[2] = nn.w - ss.w;
        }
    }
    {
        const float4 up = rp[h], dn = rm[h];
        if (gz == 0 || gz == g.n[2] - 1) {
            // the plane two away is outside the ring: read it from global memory
            const bool lo = (gz == 0);
            const int z2 = lo ? 2 : g.n[2] - 3;
            float4 f2 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gx >= 0 && gx < g.n[0] && gy >= 0 && gy < g.n[1])
                f2 = a.src[((long long)z2 * g.n[1] + gy) * g.n[0] + gx];
            const float s = lo ? 1.f : -1.f;
            const float4 n1 = lo ? up : dn;
            Dz[0] = s * (-3.f * c.y + 4.f * n1.y - f2.y);
            Dz[1] = s * (-3.f * c.z + 4.f * n1.z - f2.z);
            Dz[2] = s * (-3.f * c.w + 4.f * n1.w - f2.w);
        } else {
            Dz[0] = up.y - dn.y;
            Dz[1] = up.z - dn.z;
            Dz[2] = up.w - dn.w;
        }
    }
    const float A = a.A, hA = 0.5f * a.A;
    const float ux = c.y, uy = c.z, uz = c.w;
    const float ASxx = A * Dx[0], ASyy = A * Dy[1], ASzz = A * Dz[2];
    const float ASxy = hA * (Dy[0] + Dx[1]);
    const float ASxz = hA * (Dz[0] + Dx[2]);
    const float ASyz = hA * (Dz[1] + Dy[2]);
    const float P = c.x - 1.5f * (ux * ux + uy * uy + uz * uz);
    const int fi = fy * FX + fx;
    constexpr int FS = FX * FY;
    // rest and axes: w (P + 4.5 u_a^2 + A S_aa) +- 3 w u_a
    f_rest = a.w0 * P;
    const float w1 = a.w1, w13 = 3.f * a.w1;
    {
        const float bx = w1 * (P + 4.5f * ux * ux + ASxx);
        sF[0 * FS + fi] = bx + w13 * ux;
        sF[1 * FS + fi] = bx - w13 * ux;
        const float by = w1 * (P + 4.5f * uy * uy + ASyy);
        sF[2 * FS + fi] = by + w13 * uy;
        sF[3 * FS + fi] = by - w13 * uy;
        const float bz = w1 * (P + 4.5f * uz * uz + ASzz);
        f_pz = bz + w13 * uz;
        f_mz = bz - w13 * uz;
    }
    // corners (sx, sy, +1) and their opposites (-sx, -sy, -1)
    const float w2 = a.w2, w23 = 3.f * a.w2, w245 = 4.5f * a.w2, w2A2 = 2.f * a.w2;
    const float T0 = w2 * (P + ASxx + ASyy + ASzz);
    const float s1 = ux + uy, d1 = ux - uy;
    const float q1 = ASxz + ASyz, q2 = ASyz - ASxz;
    {   // (+,+,+) / (-,-,-)
        const float cu = s1 + uz, off = ASxy + q1;
        const float sym = T0 + w245 * cu * cu + w2A2 * off;
        sF[4 * FS + fi] = sym + w23 * cu;
        sF[11 * FS + fi] = sym - w23 * cu;
    }
    {   // (-,+,+) / (+,-,-)
        const float cu = uz - d1, off = q2 - ASxy;
        const float sym = T0 + w245 * cu * cu + w2A2 * off;
        sF[5 * FS + fi] = sym + w23 * cu;
        sF[10 * FS + fi] = sym - w23 * cu;
    }
    {   // (+,-,+) / (-,+,-)
        const float cu = uz + d1, off = -ASxy - q2;
        const float sym = T0 + w245 * cu * cu + w2A2 * off;
        sF[6 * FS + fi] = sym + w23 * cu;
        sF[9 * FS + fi] = sym - w23 * cu;
    }
    {   // (-,-,+) / (+,+,-)
        const float cu = uz - s1, off = ASxy - q1;
        const float sym = T0 + w245 * cu * cu + w2A2 * off;
        sF[7 * FS + fi] = sym + w23 * cu;
        sF[8 * FS + fi] = sym - w23 * cu;
    }
}

__global__ void __launch_bounds__(NTHR, 2)
    k_fused_step3d(const __grid_constant__ CUtensorMap tmap, const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    float4* raw = reinterpret_cast<float4*>(smem + OFF_RAW);
    float* sF = reinterpret_cast<float*>(smem + OFF_F);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    const Geom& g = a.g;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int q0 = blockIdx.z * a.zchunk;
    const int q1 = min(g.n[2], q0 + a.zchunk);
    const int nplanes = q1 - q0 + 4;   // raw planes q0-2 .. q1+1
    // rim node handled by this thread (tid < NHALO)
    int hfx = -1, hfy = -1;
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
        for (int k = 0; k < 4 && k < nplanes; ++k)
            tma_load_plane(smem_addr(raw + (size_t)k * HX * HY), &tmap, x0 - 2, y0 - 2,
                           q0 - 2 + k, smem_addr(&bars[k]));
    }
    __syncthreads();

    const int gx = x0 + tx, gy = y0 + ty;
    const bool col_in = gx < g.n[0] && gy < g.n[1];
    const bool col_inner = gx >= 1 && gx <= g.n[0] - 2 && gy >= 1 && gy <= g.n[1] - 2;
    float acc0[4] = {0.f, 0.f, 0.f, 0.f};  // plane p (c_z = 0 and -1 groups still to come)
    float acc1[4] = {0.f, 0.f, 0.f, 0.f};  // plane p + 1
    constexpr int FS = FX * FY;
    const int fo = (ty + 1) * FX + (tx + 1);
    bool ok = true;

    for (int p = q0 - 1; p <= q1; ++p) {
        const int k_new = p - q0 + 3;  // plane p + 1 must have landed
        bool good = true;
        if (p == q0 - 1) {
            for (int k = 0; k <= 2 && good; ++k) good = mbar_wait(smem_addr(&bars[k % NSLOT]), (k / NSLOT) & 1);
        } else {
            good = mbar_wait(smem_addr(&bars[k_new % NSLOT]), (k_new / NSLOT) & 1);
        }
        if (__syncthreads_or(!good)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            const int k = p - q0 + 5;
            if (k < nplanes) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_plane(smem_addr(raw + (size_t)(k % NSLOT) * HX * HY), &tmap, x0 - 2,
                               y0 - 2, q0 - 2 + k, smem_addr(&bars[k % NSLOT]));
            }
        }
        const int km = p - q0 + 1;
        const float4* rm = raw + (size_t)(km % NSLOT) * HX * HY;
        const float4* r0 = raw + (size_t)((km + 1) % NSLOT) * HX * HY;
        const float4* rp = raw + (size_t)((km + 2) % NSLOT) * HX * HY;
        float f_rest, f_pz, f_mz;
        feq_node(a, rm, r0, rp, sF, tx + 1, ty + 1, gx, gy, p, f_rest, f_pz, f_mz);
        if (tid < NHALO) {
            float d0, d1, d2;
            feq_node(a, rm, r0, rp, sF, hfx, hfy, x0 - 1 + hfx, y0 - 1 + hfy, p, d0, d1, d2);
        }
        __syncthreads();
        // gather the three z-groups of plane p's f^eq into planes p-1, p, p+1
        const float fpx = sF[0 * FS + fo - 1], fmx = sF[1 * FS + fo + 1];
        const float fpy = sF[2 * FS + fo - FX], fmy = sF[3 * FS + fo + FX];
        // corners (sx, sy, sz) come from (x - sx, y - sy)
        const float cpp_p = sF[4 * FS + fo - 1 - FX], cmp_p = sF[5 * FS + fo + 1 - FX];
        const float cpm_p = sF[6 * FS + fo - 1 + FX], cmm_p = sF[7 * FS + fo + 1 + FX];
        const float cpp_m = sF[8 * FS + fo - 1 - FX], cmp_m = sF[9 * FS + fo + 1 - FX];
        const float cpm_m = sF[10 * FS + fo - 1 + FX], cmm_m = sF[11 * FS + fo + 1 + FX];
        // c_z = -1 group completes plane p-1
        {
            const float sxp = cpp_m + cpm_m, sxm = cmp_m + cmm_m;
            const float syp = cpp_m + cmp_m, sym = cpm_m + cmm_m;
            const float all = sxp + sxm + f_mz;
            const float r = acc0[0] + all;
            const float ux = acc0[1] + (sxp - sxm);
            const float uy = acc0[2] + (syp - sym);
            const float uz = acc0[3] - all;
            const int qz = p - 1;
            if (qz >= q0 && col_inner && qz >= 1 && qz <= g.n[2] - 2) {
                float4 o;
                o.x = r;
                long long bi;
                const float bfx = (float)g.body[0], bfy = (float)g.body[1], bfz = (float)g.body[2];
                if (in_box(g, gx, gy, qz, bi)) {
                    const float4 ks = a.kus[bi];
                    const float inv = 1.f / (1.f + ks.x);
                    o.y = (ux + bfx + ks.x * ks.y) * inv;
                    o.z = (uy + bfy + ks.x * ks.z) * inv;
                    o.w = (uz + bfz + ks.x * ks.w) * inv;
                } else {
                    o.y = ux + bfx;
                    o.z = uy + bfy;
                    o.w = uz + bfz;
                }
                const long long m = ((long long)qz * g.n[1] + gy) * g.n[0] + gx;
                a.out[m] = o;
                if (gx == 1 || gy == 1 || qz == 1 || gx == g.n[0] - 2 || gy == g.n[1] - 2 ||
                    qz == g.n[2] - 2) {
                    V4<float> v;
                    v.r = o.x;
                    v.x = o.y;
                    v.y = o.z;
                    v.z = o.w;
                    write_bc_from(g, gx, gy, qz, v, reinterpret_cast<V4<float>*>(a.out));
                }
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
    }
    (void)col_in;
    if (!ok) {
        // a copy did not land in time: record it, then give the copies still in flight a
        // bounded chance to finish before the block's shared memory goes away
        if (tid == 0) {
            atomicOr(a.err, 8);
            for (int s = 0; s < NSLOT; ++s) {
                uint32_t st;
                asm volatile(
                    "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;"
                    " selp.u32 %0, 1, 0, p; }"
                    : "=r"(st)
                    : "r"(smem_addr(&bars[s]))
                    : "memory");
                const long long t0 = clock64();
                while (clock64() - t0 < (1LL << 28)) {
                }
            }
        }
        __syncthreads();
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

// One fused forward step src -> dst.  Returns a CUDA error code (cudaSuccess on success).
cudaError_t launch_fused_step3d(const Geom& g, const V4<float>* src, const V4<float>* kus,
                                V4<float>* dst, int* err, cudaStream_t st) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    cuuint64_t dims[4] = {4, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    cuuint64_t strides[3] = {16, (cuuint64_t)g.n[0] * 16, (cuuint64_t)g.n[0] * g.n[1] * 16};
    cuuint32_t box[4] = {4, HX, HY, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)src, dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_step3d,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    FusedArgs a;
    a.g = g;
    a.out = reinterpret_cast<float4*>(dst);
    a.kus = reinterpret_cast<const float4*>(kus);
    a.src = reinterpret_cast<const float4*>(src);
    a.err = err;
    a.A = (float)g.A;
    a.w0 = (float)(2.0 / 9.0);
    a.w1 = (float)(1.0 / 9.0);
    a.w2 = (float)(1.0 / 72.0);
    const int tiles_x = (g.n[0] + TX - 1) / TX, tiles_y = (g.n[1] + TY - 1) / TY;
    // z chunks: about three resident waves of two blocks per SM
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)tiles_x * tiles_y;
    int chunks = (int)std::max(1LL, (6LL * nsm + tiles - 1) / tiles);
    chunks = std::min(chunks, std::max(1, g.n[2] / 16));
    a.zchunk = (g.n[2] + chunks - 1) / chunks;
    chunks = (g.n[2] + a.zchunk - 1) / a.zchunk;
    dim3 grid(tiles_x, tiles_y, chunks);
    k_fused_step3d<<<grid, NTHR, SMEM_BYTES, st>>>(map, a);
    return cudaGetLastError();
}

}  // namespace lks
