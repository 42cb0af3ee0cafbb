// Instance tables: the D2Q9 FP32 kernels that take a table of contexts and cover all of them in
// one persistent launch per phase (one context is a table of one).  Each kernel walks a list of
// work units (tiles, blocks of box nodes, design columns, ...) concatenated over the
// instances; a prefix array per unit kind maps a unit to its instance.
#pragma once

#include "lks_internal.h"

namespace lks {

// Buffers of a context addressed by index, so that a captured launch sequence names buffers
// the same way for every instance: the two working states, the initial state, the two adjoint
// buffers, then the snapshot/tape pool.
enum { BUF_S0 = 0, BUF_S1 = 1, BUF_INIT = 2, BUF_LAM0 = 3, BUF_LAM1 = 4, BUF_POOL = 5 };

struct Inst {
    Geom g;
    Design d;
    int2* pos_b[2];           // design positions of the steps of each parity: integer base of
    float4* pos_sc[2];        // x_ref, y_ref and sin, cos of (pi f / 2) of their fractions
    const Motion* motion;     // rows 0..max_steps with cos/sin already evaluated (device)
    void* const* bufs;        // BUF_* (device)
    const float* kref;        // kappa_ref per design node
    const float* kprime;      // d kappa_ref / d gamma
    V4<float>* kus;           // kappa, u_S on the footprint box
    V4<float>* kus_tape;      // kappa, u_S of each taped step (slots of boxN records) or null
    float* e;                 // dJ/dkappa density on the box
    double* gacc;             // dJ/dgamma accumulator
    double* jstep;            // objective per step
    int win_begin, win_end;
    float Af, bf[2];          // A and the body force in single precision
    double hwin;              // 1 / (window length): the window weight h_n inside the window
    float src_r, src_x, src_y;   // h_n d j / d (rho, ux, uy) at a target node, inside the window
    float4 bcf[4];            // per face: prescribed (ux, uy, 0, rho - rho0) in single precision
    int bckeep[4];            // per face: 1 keeps the source's rho (wall, inlet), 0 prescribes
                              // it and copies the normal velocity (outlet)
};

// Configurations of the fused kernels, chosen per run by the autotuner.  Step: five tile
// shapes of 256 threads (0..4) and four row-marching strips (5..8: strips of 62, 126, 126 and
// 254 columns marching over chunks of 64, 64, 128 and 64 rows).  Adjoint: the five tile shapes
// (0..4).  tile_tx / tile_ty give the extent of one work unit.
constexpr int kTileCfgs = 9;
constexpr int kAdjCfgs = 5;
__host__ __device__ constexpr int tile_tx(int k) {
    return k == 0 ? 32 : (k == 1 ? 16 : (k == 2 ? 32 : (k <= 4 ? 64 :
           (k == 5 ? 62 : (k == 8 ? 254 : 126)))));
}
__host__ __device__ constexpr int tile_ty(int k) {
    return k == 0 ? 8 : (k == 1 ? 16 : (k == 2 ? 16 : (k == 3 ? 8 : (k == 4 ? 16 :
           (k == 7 ? 128 : 64)))));
}

// Work-unit kinds: design columns in blocks of kUnitThreads, footprint-box tiles, one unit per
// instance (objective), tiles of each shape.
constexpr int kUnitThreads = 256;
constexpr int kBoxTile = 16;   // box tiles of the 2D transfer: kBoxTile^2 = kUnitThreads nodes
enum { U_DCOL = 0, U_BOX, U_INST, U_TILE0, U_COUNT = U_TILE0 + kTileCfgs };

struct Plan {
    const Inst* tab;          // device
    const int* pre;           // device, [U_COUNT][count + 1]
    int count;
    int total[U_COUNT];
    int grid[U_COUNT + kAdjCfgs];    // persistent grid per kernel (set on the host)
    const int* nbase;         // device: step index base added to each launch's offset
};

// Tile origin along an axis of n nodes for tiles of T: -o with o in {0, 2} chosen so that the
// nodes 0..2 and n-3..n-1 of a non-periodic axis each fall in one tile (the one-sided
// gradient rows of boundary nodes reach two nodes inward, and the adjoint's transposed
// gradient then needs them inside the tile).  T >= 8.
__host__ __device__ inline int tile_origin(int n, int T, int periodic) {
    if (periodic) return 0;
    const int r1 = (n - 1) % T, r2 = (n - 2) % T;
    return (r1 == 0 || r2 == 0) ? 2 : 0;
}
__host__ __device__ inline int tile_count(int n, int T, int periodic) {
    return (n + tile_origin(n, T, periodic) + T - 1) / T;
}

// Host: persistent grid sizes for every kernel of a plan (occupancy x SMs, capped by work).
void plan_grids(Plan& p);

// Launchers (stream st; noff = step offset from *nbase; buffer arguments are BUF_* indices;
// kslot: the kappa, u_S records a launch writes (transfer) or reads (step, adjoint): -1 for the
// box buffer kus, else slot kslot of kus_tape; next: the transfer also forms the design positions
// of the following step).
cudaError_t launch_t_design_pos(const Plan& p, int noff, cudaStream_t st);
cudaError_t launch_t_transfer2d(const Plan& p, int noff, int kslot, bool next, cudaStream_t st);
cudaError_t launch_t_step2d(const Plan& p, int cfg, int src, int dst, int kslot, cudaStream_t st);
cudaError_t launch_t_objective(const Plan& p, int noff, int src, cudaStream_t st);
cudaError_t launch_t_adj2d(const Plan& p, int cfg, int noff, int lam_in, int lam_out, int sn,
                           int sp, int kslot, cudaStream_t st);
cudaError_t launch_t_sens(const Plan& p, int noff, cudaStream_t st);
cudaError_t launch_set_int(int* dst, int v, cudaStream_t st);

}  // namespace lks
