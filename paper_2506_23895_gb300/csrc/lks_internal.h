// Internal declarations shared by the host engine and the kernel translation units.
// Not part of the public ABI (include/lks.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace lks {

// One node of state (rho - rho0, ux, uy, uz) or adjoint (lam_rho, lam_u).  16 B (float) or
// 32 B (double), so one vector load/store moves a node.
template <class T>
struct alignas(4 * sizeof(T)) V4 {
    T r, x, y, z;
};

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTLET = 3 };

// Everything a kernel needs to know about the analysis grid, boundaries, objective and the
// transfer footprint box.  Passed by value.
struct Geom {
    int dim;
    int n[3];
    int periodic[3];
    long long nodes;
    int bc[6];
    double bcv[6][4];   // ux, uy, uz, rho per face
    double rho0, A;
    double body[3];
    // footprint box (union over all steps of the transfer support), may be empty
    int blo[3], bn[3];
    long long boxN;
    // objective region
    int okind;
    int obox[6];
    double odir[3];
    double ocyl_r, ocyl_c[2];
    double ocount;
    const int* otarget;   // node indices of the target region, ascending (device)
    const void* ks;       // static Brinkman coefficient per node (T, device) or nullptr
};

// Design grid and per-step rigid motion.
struct Design {
    int L[3];
    double xiG[3];
    float xiGf[3];      // the same in single precision
    long long nd;       // design nodes
    long long ncol;     // design columns lx*ly
};

struct Motion {
    double c, s, om;    // cos(theta), sin(theta), omega
    double xG[3], uG[3];
    // single-precision forms for FP32 kernels: cos and sin as float pairs (hi + lo), x_G split
    // into an integer and a float-pair fraction, and plain floats
    float ch, cl, sh, sl;
    int xgi[2];
    float xgh[2], xgl[2];
    float cf, sf, omf, xgf[2], ugf[3];
    // rotation matrix R(theta) (row-major) about the unit axis ax (3D general-axis transfer)
    double R[9], ax[3];
};

// Per-step scratch produced by the design-position kernel and consumed by the transfer,
// the fill and the sensitivity gather.
struct TransferScratch {
    int* col_base;       // [ncol][2] floor of x_ref, y_ref per design column
    void* col_frac;      // [ncol][2] T: fractional part in [0,1)
    float4* col_sc;      // [ncol] sin, cos of (pi f / 2) for f = x and y fractions (2D table path)
    int* zt_idx;         // [bn_z][4] design z index per analysis z of the box (-1: none)
    void* zt_w;          // [bn_z][4] T: kernel weight
    int* tap_cnt;        // [box columns]
    int* tap_idx;        // [box columns][kMaxTaps] design column index
    void* tap_w;         // [box columns][kMaxTaps] T
    void* col_m;         // [box columns][3] T: m0, m1x, m1y
    int* dz_base;        // [lz] floor of the moved z of each design plane
    void* dz_frac;       // [lz] T: its fractional part
    int* err;            // device error word (bit 0: tap overflow)
};

constexpr int kMaxTaps = 32;

// Scratch of the general-axis transfer: per design node the integer base of x_ref (int4) and
// its fraction (V4<T>); per footprint-box cell the design nodes whose base is that cell.
constexpr int kCellMax = 8;   // a unit cube holds at most 8 points at mutual distance >= 1
struct AxisScratch {
    int4* base;
    void* frac;
    int* cnt;    // [box cells]
    int* idx;    // [box cells][kCellMax], ascending design index
};

// Per-device once-only host state (kernel attributes are per device): bit d of `mask` records
// that the current device d has been set up.  Devices past 31 are set up on every call.  The
// mask is atomic, so host threads driving contexts at the same time may race to set a device up
// (the set-up is idempotent) but never lose a bit.
inline bool device_done(const std::atomic<unsigned>& mask) {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev < 32 && (mask.load(std::memory_order_acquire) >> dev & 1u);
}
inline void device_mark(std::atomic<unsigned>& mask) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 32) mask.fetch_or(1u << dev, std::memory_order_release);
}

// ---- kernel launchers (templated on T = float / double, explicitly instantiated) ----
template <class T>
void launch_init_state(const Geom& g, V4<T>* s, cudaStream_t st);
template <class T>
void launch_fill_uniform(const Geom& g, V4<T>* s, const double u[3], cudaStream_t st);
template <class T>
void launch_apply_bc(const Geom& g, V4<T>* s, cudaStream_t st);
template <class T>
void launch_feq(const Geom& g, const V4<T>* s, T* F, cudaStream_t st);
template <class T>
void launch_gather(const Geom& g, const T* F, const V4<T>* kus, V4<T>* out, cudaStream_t st);
template <class T>
void launch_objective(const Geom& g, const V4<T>* s, double* jstep, cudaStream_t st);
template <class T>
void launch_adj_bcT(const Geom& g, V4<T>* lam, double h, cudaStream_t st);
// u3 (optional): 3 U~ of the last moments, for the printed-ALKS variant (else nullptr).
template <class T>
void launch_adj_mu(const Geom& g, const V4<T>* lam, const V4<T>* kus, const V4<T>* sn,
                   V4<T>* mu, T* e, double h, cudaStream_t st, const V4<T>* u3 = nullptr);
template <class T>
void launch_adj_moments(const Geom& g, const V4<T>* mu, const V4<T>* sp, V4<T>* lam_out,
                        T* phi, cudaStream_t st, V4<T>* u3 = nullptr);
template <class T>
void launch_adj_divT(const Geom& g, const T* phi, V4<T>* lam_out, cudaStream_t st);
template <class T>
void launch_check_state(const Geom& g, const V4<T>* s, int* flag, cudaStream_t st);

// Fused FP32 D3Q15 step and adjoint step (non-periodic grids, TMA-fed z-march).
struct FaceOffsets {
    long long off[6];
};
bool fused3d_eligible(const Geom& g);
int fused_zchunk_waves(const Geom& g, long long tiles, int per_sm);
constexpr int kStep3dVariants = 3;
cudaError_t launch_fused_step3d(const Geom& g, const V4<float>* src, const V4<float>* kus,
                                V4<float>* dst, int* err, cudaStream_t st, int variant);
// Offsets of the six face arrays (3 floats per face node) and their total length.
void face_offsets(const Geom& g, FaceOffsets& fo, long long& total);
// variant 0: two block barriers per plane; 1: one barrier per plane (conversion one plane ahead)
constexpr int kAdj3dVariants = 2;
cudaError_t launch_fused_adj3d(const Geom& g, const V4<float>* lam_in, V4<float>* lam_out,
                               const V4<float>* kus, const V4<float>* sn, const V4<float>* sp,
                               float* e, float* face, double h, int* err, cudaStream_t st,
                               int variant);

template <class T>
void launch_design_prep(const Design& d, const double* gamma, double kappa_max, double q,
                        T* kref, T* kref_t, T* kprime, int* bad, cudaStream_t st);
template <class T>
void launch_design_pos(const Design& d, const Geom& g, const Motion& m, TransferScratch ts,
                       cudaStream_t st);
template <class T>
void launch_transfer(const Design& d, const Geom& g, const Motion& m, TransferScratch ts,
                     const T* kref_t, T* k2, V4<T>* kus, cudaStream_t st);
template <class T>
void launch_sens(const Design& d, const Geom& g, TransferScratch ts, const T* e,
                 const T* kprime, double* gacc, cudaStream_t st);
// Design chain (FP64): gb = H(F gamma), hp = H'(F gamma), wsum = filter normaliser; the
// transposed chain out = F^T (hp * g) (hp = nullptr: F^T g); a fixed-order sum.
void launch_filter(const Design& d, double R, double beta, double eta, const double* gamma,
                   double* gb, double* hp, double* wsum, cudaStream_t st);
void launch_filter_T(const Design& d, double R, const double* g, const double* hp,
                     const double* wsum, double* out, cudaStream_t st);
void launch_design_sum(long long nd, const double* a, double* out, cudaStream_t st);
void launch_fill_f64(double* a, long long n, double v, cudaStream_t st);
// General-axis transfer (kappa, u_S on the box) and its sensitivity gather.
template <class T>
void launch_transfer_axis(const Design& d, const Geom& g, const Motion& m, AxisScratch as,
                          const T* kref, V4<T>* kus, cudaStream_t st);
template <class T>
void launch_sens_axis(const Design& d, const Geom& g, AxisScratch as, const T* e,
                      const T* kprime, double* gacc, cudaStream_t st);
template <class T>
void launch_box_to_grid(const Geom& g, const V4<T>* kus, double* kappa, double* us,
                        cudaStream_t st);
template <class T>
void launch_state_to_f64(const Geom& g, const V4<T>* s, double* out, cudaStream_t st,
                         bool add_rho0 = true);
template <class T>
void launch_state_from_f64(const Geom& g, const double* in, V4<T>* s, cudaStream_t st);

}  // namespace lks
