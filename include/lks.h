/*
 * lks.h -- C ABI of the GB300 library for the lattice kinetic scheme (LKS) with a rigidly moving
 * design grid and its discrete adjoint (arXiv 2506.23895).
 *
 * The calls follow the paper's statement of the problem:
 *   lks_set_design(gamma)      the pseudo-density gamma : D -> [0,1] on the design grid (Sec. 2.1,
 *                              Eq. 1), mapped to the Brinkman coefficient kappa_ref (Sec. 2.3);
 *   lks_set_motion(schedule)   the prescribed rigid motion theta(t), omega(t), x_G(t), u_G(t) of
 *                              the design grid (Sec. 2.3, Eqs. rigid_body_position/velocity);
 *   lks_forward(n) -> J        Algorithm 1 (Sec. 2.3) for n steps with the time-averaged
 *                              objective J1 or J2 (Sec. 2.5);
 *   lks_adjoint() -> dJ/dgamma the reverse-time adjoint sweep (Algorithm 2, Sec. 2.4) taken as the
 *                              exact discrete adjoint of the forward steps, with the design
 *                              sensitivity gathered back onto the design grid (Sec. 2.4).
 *
 * Conventions for every call:
 *   - Every function returns an lks_status; nothing throws across the ABI.  After an error,
 *     lks_last_error() returns a one-line message.
 *   - Input arrays are copied; the caller keeps ownership.  The library never frees caller
 *     memory.  Device memory is either the caller's workspace (lks_create) or allocated by the
 *     library and released by lks_destroy.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global memory on the
 *     context's device.  All work is issued on cfg.stream (NULL = legacy default stream); calls
 *     that return host values synchronise that stream.
 *   - Arrays are row-major with x fastest: analysis fields [nz][ny][nx], design fields
 *     [lz][ly][lx] (nz = lz = 1 in 2D).
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef LKS_H
#define LKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lks_ctx lks_ctx;

typedef enum {
    LKS_OK = 0,
    LKS_ERR_ARG = 1,      /* invalid argument or configuration (message says which) */
    LKS_ERR_ORDER = 2,    /* call out of order, e.g. adjoint before forward */
    LKS_ERR_NOMEM = 3,    /* workspace too small or device allocation failed */
    LKS_ERR_CUDA = 4,     /* a CUDA runtime call failed */
    LKS_ERR_DIVERGED = 5, /* non-finite or |u| > 0.5 state after a forward run */
    LKS_ERR_TIMEOUT = 6   /* reserved for bounded device waits */
} lks_status;

/* Face boundary types; faces are ordered x-, x+, y-, y+, z-, z+ (Eqs. bc_rho, bc_u).
 * PERIODIC must be set on both faces of an axis.  WALL and INLET prescribe u (bc_val[f][0..2])
 * and copy rho from the interior; OUTLET prescribes rho (bc_val[f][3]) and the tangential u and
 * copies the normal u.  A boundary node copies from the interior node one step inward along
 * every boundary normal it lies on; on edges and corners WALL > INLET > OUTLET, ties to the
 * lower face index. */
enum { LKS_BC_PERIODIC = 0, LKS_BC_WALL = 1, LKS_BC_INLET = 2, LKS_BC_OUTLET = 3 };

/* Objectives of Sec. 2.5: J1 = -mean pressure (p = rho/3) over the target region and J2 =
 * -mean n.u over it, both averaged over the steps win_begin..win_end. */
enum { LKS_OBJ_PRESSURE = 0, LKS_OBJ_VELOCITY = 1 };

/* Arithmetic of the state and adjoint stencils.  FP32 keeps rho - rho0 and u in float with
 * FP64 objective and sensitivity accumulation; FP64 is the plain double-precision path. */
enum { LKS_FP32 = 0, LKS_FP64 = 1 };

typedef struct {
    int dim;                 /* 2 (D2Q9) or 3 (D3Q15) */
    int nx, ny, nz;          /* analysis grid; nz = 1 in 2D; every active axis >= 3 nodes */
    int lx, ly, lz;          /* design grid (unit spacing); lx = 0: no moving body */
    int precision;           /* LKS_FP32 or LKS_FP64 */
    int max_steps;           /* largest n_steps passed to lks_forward (sizes the checkpoints) */
    double A;                /* viscosity parameter of f^eq, nu = 1/6 - 2A/9 (Sec. 2.2) */
    double kappa_max, q;     /* Brinkman interpolation kappa_ref(gamma) (Sec. 2.3) */
    double rho0;             /* reference density; the FP32 path stores rho - rho0 */
    int bc[6];               /* LKS_BC_* per face */
    double bc_val[6][4];     /* per face: ux, uy, uz, rho */
    double u_init[3];        /* initial uniform velocity (rho = rho0), then boundary values */
    double body_force[3];    /* constant body force added to u (u = u* + F); 0 normally */
    double xi_G[3];          /* rotation centre in design-grid coordinates */
    int obj_kind;            /* LKS_OBJ_* */
    int obj_box[6];          /* target region: inclusive x0,x1,y0,y1,z0,z1 */
    double obj_dir[3];       /* n for J2 */
    double obj_cyl_r;        /* > 0: region also limited to (x-cx)^2 + (y-cy)^2 <= r^2 */
    double obj_cyl_c[2];
    int win_begin, win_end;  /* objective window (inclusive step indices, 1-based) */
    size_t ckpt_bytes;       /* device bytes for adjoint snapshots; 0 = full history if it
                                fits in 8 GB, else the minimum of a two-level scheme */
    void* stream;            /* cudaStream_t the work is ordered on; NULL = legacy default
                                stream.  A 3D forward or adjoint run starts after the work
                                already on it and is complete on it when the call returns: the
                                run executes on two internal streams of the context (its steps
                                at the highest priority, the next step's transfer and the
                                sensitivity gathers at the lowest), forked from and joined back
                                to this stream by events. */
    int flags;               /* LKS_FLAG_* bits; 0 normally */
    double rot_axis[3];      /* 3D rotation axis of the design grid, a unit vector; all zero or
                                (0, 0, 1) is the z axis (the paper's 3D rotor, Sec. 3.3).  Any
                                other axis uses a cell-list transfer (R(theta) by Rodrigues'
                                formula).  Ignored in 2D. */
} lks_config;

/* Run every step on the plain per-node kernels even where the fused FP32 3D step applies. */
#define LKS_FLAG_PLAIN_KERNELS 1
/* Adjoint source update as printed in Sec. 2.4 instead of the exact discrete adjoint: the
 * (1 + kappa)^-1 of the Brinkman source (Eq. au_ex) divides only the gathered first moment and
 * the objective source.  For comparing the printed scheme's gradient with the exact one; uses
 * the plain kernels. */
#define LKS_FLAG_PAPER_ALKS 2

/* Prescribed rigid motion, rows n = 0..n_rows-1 for time t_n = n (Delta t = 1).
 * Each row: theta, omega, xG[3], uG[3] (8 doubles, host memory, copied).  In 3D the rotation
 * is about the z axis (the paper's 3D rotor, Sec. 3.3); x_ref = R(theta)(xi - xi_G) + x_G and
 * u_ref = R'(theta)(xi - xi_G) omega + u_G (Eqs. rigid_body_position / rigid_body_velocity). */
typedef struct {
    int n_rows;
    const double* rows;
} lks_motion;

/* Bytes of device workspace a context for cfg needs (0 on an invalid cfg). */
size_t lks_workspace_bytes(const lks_config* cfg);

/* Create a context.  workspace: device pointer of ws_bytes >= lks_workspace_bytes(cfg),
 * 256-byte aligned, owned by the caller and kept alive until lks_destroy; or NULL to let the
 * library allocate it.  Errors: LKS_ERR_ARG (bad cfg; *out = NULL), LKS_ERR_NOMEM. */
lks_status lks_create(const lks_config* cfg, void* workspace, size_t ws_bytes, lks_ctx** out);

/* Set gamma on the design grid (lx*ly*lz doubles; host if on_device = 0, else device).
 * Values must lie in [0,1] (LKS_ERR_ARG otherwise).  Invalidates any forward run. */
lks_status lks_set_design(lks_ctx* ctx, const double* gamma, int on_device);

/* Design chain around the solver: the density filter and Heaviside projection the paper uses
 * to binarise designs (Secs. 1 and 3.1: filter radius R = 2.4 cells, steepness beta from 1 in
 * continuation).  With R > 0 the solver sees gb = H(F gamma), F the linear-weight density
 * filter gt_i = sum_j w_ij gamma_j / sum_j w_ij, w_ij = max(0, R - |xi_i - xi_j|) over the
 * design grid, H(t) = [tanh(beta eta) + tanh(beta (t - eta))] / [tanh(beta eta) +
 * tanh(beta (1 - eta))]; lks_adjoint then returns dJ/dgamma = F^T (H'(F gamma) dJ/dgb).
 * R = 0 (the default) switches the chain off.  Re-applies to the current design and
 * invalidates any forward run.  LKS_ERR_ARG unless R >= 0 and, for R > 0, beta > 0 and
 * 0 < eta < 1. */
lks_status lks_set_filter(lks_ctx* ctx, double R, double beta, double eta);

/* Volume constraint of Sec. 2.1 (Eq. constraint) on the field the solver sees (gb with the
 * filter chain, else gamma), unit cell volumes: G = sum / (vmax * design nodes) - 1, written to
 * *G_out (host).  dGdgamma (design nodes doubles, host or device if on_device; may be NULL)
 * receives dG/dgamma through the chain.  LKS_ERR_ORDER without a design, LKS_ERR_ARG if
 * vmax <= 0.  Synchronises. */
lks_status lks_volume(lks_ctx* ctx, double vmax, double* G_out, double* dGdgamma, int on_device);

/* Static solids: a Brinkman coefficient kappa_s >= 0 per analysis node (host, nodes doubles,
 * copied; NULL removes it) for solid walls at rest inside the fluid, such as the inner wall of
 * the paper's 2D pump (Sec. 3.2) or the fixed outer cylinder of its rotating-cylinder check
 * (appendix).  The Brinkman update becomes u = (u* + kappa u_S) / (1 + kappa + kappa_s) and the
 * adjoint follows exactly.  The FP32 D3Q15 context then runs the plain kernels (the fused D2Q9
 * kernels support it).  Invalidates any forward run; LKS_ERR_ARG on a negative or non-finite
 * value. */
lks_status lks_set_static(lks_ctx* ctx, const double* kappa_s);

/* Warm starts for periodic flows (Secs. 3.2 and 3.3 reuse the terminal fields of the previous
 * optimisation step).  lks_warm_start: the initial state becomes the final state of the last
 * forward run (LKS_ERR_ORDER without one).  lks_set_adjoint_start(warm = 1): every later adjoint
 * starts from lambda^0 of the previous adjoint run instead of zero, which makes it the exact
 * adjoint of J + <lambda_prev, s^N>; warm = 0 (the default) returns to the exact adjoint of J.
 * lks_get_adjoint_state: lambda^0 of the last adjoint run as (rho, ux, uy, uz) planes of nodes
 * doubles (host); it is dJ/ds^0, the gradient with respect to the initial state. */
lks_status lks_warm_start(lks_ctx* ctx);
lks_status lks_set_adjoint_start(lks_ctx* ctx, int warm);
lks_status lks_get_adjoint_state(const lks_ctx* ctx, double* lambda_out);

/* Set the motion schedule; needs n_rows >= max_steps + 1.  The transfer footprint (every
 * analysis node within two cells of a moved design node) must stay inside the grid and off
 * boundary nodes for every step, else LKS_ERR_ARG.  Invalidates any forward run. */
lks_status lks_set_motion(lks_ctx* ctx, const lks_motion* motion);

/* Replace the initial state (rho, ux, uy, uz planes of nodes doubles each, host).  NULL
 * restores the default (rho0, u_init, then boundary values). */
lks_status lks_set_initial_state(lks_ctx* ctx, const double* state);

/* Algorithm 1 for n_steps (1 <= n_steps <= max_steps) from the initial state; writes J
 * (host double) and keeps what the adjoint needs.  LKS_ERR_ORDER without design/motion. */
lks_status lks_forward(lks_ctx* ctx, int n_steps, double* J_out);

/* Exact discrete adjoint of the last forward run; writes dJ/dgamma (lx*ly*lz doubles, host or
 * device).  LKS_ERR_ORDER if no valid forward run precedes it. */
lks_status lks_adjoint(lks_ctx* ctx, double* dJdgamma, int on_device);

/* Copy the current forward state to the host as (rho, ux, uy, uz) planes in double. */
lks_status lks_get_state(const lks_ctx* ctx, double* state_out);

/* Evaluate the transfer alone at step n of the motion schedule: kappa (nodes doubles) and
 * u_S (3 planes) on the whole analysis grid, host memory. */
lks_status lks_transfer(lks_ctx* ctx, int step, double* kappa_out, double* us_out);

/* Which kernels run the steps of this context: 1 the fused FP32 D3Q15 step and adjoint, 2 the
 * fused FP32 D2Q9 kernels (the instance-table kernels of the batches), 0 the plain per-node
 * kernels. */
int lks_uses_fused(const lks_ctx* ctx);

/* Variant of the fused FP32 D3Q15 forward step (lks_uses_fused == 1): 0 a shared-memory
 * z-march with two block barriers per plane, 1 (the default) a register z-march with one.  Both
 * evaluate the same arithmetic (Sec. 2.2 f^eq, Eqs. rho and u, the Brinkman update) and agree to
 * rounding, not bitwise.  request: 0..1 fixes a variant, -1 times every variant once on the
 * first fused step and keeps the fastest (results then depend on that choice at the rounding
 * level), -2 changes nothing.  *chosen (may be NULL) receives the variant in use, -1 before the
 * first fused step.  LKS_ERR_ARG for any other request. */
lks_status lks_step_variant(lks_ctx* ctx, int request, int* chosen);

/* Variant of the fused FP32 3D adjoint step (Sec. 2.4's adjoint equations, Eqs. arho, au, as;
 * used when lks_uses_fused returns 1): 0 converts lambda to mu one plane ahead of the moments
 * with two block barriers per plane, 1 converts two planes ahead with one barrier per plane.
 * Both evaluate the same arithmetic in the same order (results bitwise equal); 1 is the default.
 * request 0..1 fixes the variant, -2 changes nothing; *chosen (may be NULL) receives the variant
 * in use.
 * LKS_ERR_ARG for any other request.  Host only. */
lks_status lks_adjoint_variant(lks_ctx* ctx, int request, int* chosen);

/* Counters of the last forward+adjoint: [0] forward steps, [1] recomputed steps,
 * [2] snapshot slots, [3] tape length (steps per segment), [4] kernel launches. */
lks_status lks_get_stats(const lks_ctx* ctx, long long* stats5);

/* Time the stencil kernels with CUDA events recorded on the context's stream: the forward
 * step (everything after the transfer) and the adjoint step (everything but the transfer and
 * the sensitivity gather), every `stride` steps (0 switches timing off).  Adds two event
 * records per sampled step. */
lks_status lks_set_timing(lks_ctx* ctx, int stride);

/* Read and reset the timing: [0] forward-step ms summed, [1] forward samples, [2] adjoint-step
 * ms summed, [3] adjoint samples.  Synchronises the stream. */
lks_status lks_read_timing(lks_ctx* ctx, double* out4);

/* The checkpoint schedule the adjoint would follow, as (kind, a, b) triples, for inspection:
 * kind 0 restore a, 1 advance a->b (segment indices), 2 store a, 3 free a, 4 tape a,
 * 5 adjoint a.  Returns the number of triples written (<= cap) or -1 on bad arguments.
 * Host only; needs no device. */
int lks_checkpoint_schedule(int n_segments, int free_slots, int* triples, int cap);

/* One forward LKS step without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they need a step --
 * code running while a stream is captured into a CUDA graph, frameworks that own all device
 * memory through their own pool, loops that must not block on the driver's allocator.
 *
 * It runs the plain per-node step (f^eq of every node, gather from x - c_i, Brinkman update,
 * boundary rules) from state_in to state_out, both device arrays of one node record per node
 * in cfg->precision ((rho - rho0, ux, uy, uz) as float4 or double4, x fastest).  kappa_us is
 * a device array of (kappa, u_S x, u_S y, u_S z) per node over the whole grid in the same
 * precision, or NULL when no body is present.  Work goes to cfg->stream; nothing is
 * synchronised.  The f^eq planes live in a file-scope device array of 32 MiB that stays on
 * every device that loads the library until the process exits: grids needing more
 * (nodes x Q x element size > 32 MiB, e.g. more than about 559k nodes for D3Q15 in FP32) are
 * rejected with LKS_ERR_ARG and a message in err (err_len bytes, may be NULL), and so are
 * state_in, state_out or kappa_us not aligned to one node record (16 bytes in FP32, 32 in
 * FP64).  A call on a stream that is not being captured looks up that array's device address on
 * the current device; a call under stream capture reuses the address the last such call found,
 * so the first call on each device must come before any capture (else LKS_ERR_ORDER), and
 * after a device reset the next uncaptured call finds the array's new address.  A CUDA error
 * already pending on the calling thread is reported (LKS_ERR_CUDA) before anything is
 * launched.  All calls share the array, so calls that overlap on the GPU race and must be
 * serialised by the caller; each call rewrites all the scratch it reads.  cudaMalloc, cudaFree
 * and allocating library routines are never called. */
lks_status lks_step_noalloc(const lks_config* cfg, const void* state_in, void* state_out,
                            const void* kappa_us, char* err, size_t err_len);

const char* lks_last_error(const lks_ctx* ctx);
void lks_destroy(lks_ctx* ctx);

/* The device's measured fused multiply-add rate in precision (LKS_FP32 or LKS_FP64), in
 * floating-point operations per second (2 per FMA), for the arithmetic roofline of the paths
 * that are bound by it (the plain FP64 path).  The paper has no counterpart.  A kernel of
 * independent FMA chains over whole waves of every SM, timed with CUDA events on `stream`
 * (a cudaStream_t, may be NULL) over five launches after a warm-up; synchronises.  Allocates
 * nothing.  LKS_ERR_ARG on a bad precision or NULL output, LKS_ERR_CUDA on a failed launch. */
lks_status lks_fma_rate(int precision, void* stream, double* flops_per_s);

/* Host-side fault injection for failure-detection tests (the paper has no counterpart): the
 * nth device allocation the library makes from now on (1 = the next one) reports failure
 * without calling the allocator, as if the device were out of memory; 0 switches injection
 * off.  Allocations are those of lks_create without a caller workspace, lks_batch_create and
 * the temporary buffers of lks_get_state, lks_get_adjoint_state, lks_set_initial_state and
 * lks_transfer; each returns LKS_ERR_NOMEM when its allocation fails and frees what it had
 * taken.  Returns the previous setting.  Process-wide; host only, needs no device. */
int lks_inject_alloc_failure(int nth);

/* ---- batches: many problems in lock step (designs, finite-difference perturbations, grids of
 * different sizes).  The paper solves one problem at a time; a batch runs the same Algorithm 1
 * and adjoint sweep for every member context, with each phase of a step one persistent kernel
 * launch over all members, runs of steps captured into CUDA graphs and replayed, and the tile
 * shape of the fused step and adjoint kernels chosen by timing every candidate on the batch.
 * Each member keeps its own design, motion, objective, state and gradient: results are bitwise
 * those of the member run alone with lks_forward / lks_adjoint. */
typedef struct lks_batch lks_batch;

/* Group n contexts (not copied; they must outlive the batch).  Every member must be a D2Q9
 * FP32 context without LKS_FLAG_PLAIN_KERNELS / LKS_FLAG_PAPER_ALKS, with equal max_steps,
 * equal snapshot slots (ckpt_bytes = slots x state bytes of the member) and the same stream,
 * each context at most once; else LKS_ERR_ARG (*out = NULL).  The batch allocates a small
 * device table and its own CUDA stream, ordered after / before the members' stream by events
 * at every call.  LKS_ERR_NOMEM if that fails. */
lks_status lks_batch_create(lks_ctx* const* ctxs, int n, lks_batch** out);

/* use_graphs: 1 (default) capture and replay runs of steps, 0 launch directly.  tile_fwd:
 * configuration of the fused step kernel (0..4 tiles, 5..8 row-marching strips; see
 * lks_batch_tile_shapes); tile_adj: configuration of the fused adjoint kernel (0..4 tiles);
 * -1 (default) autotunes at the next forward.  LKS_ERR_ARG on an index out of range. */
lks_status lks_batch_set_options(lks_batch* b, int use_graphs, int tile_fwd, int tile_adj);

/* lks_forward for every member: J_out (host, n doubles, may be NULL) receives each member's
 * J.  Needs design and motion on every member (LKS_ERR_ORDER).  On an error the message of the
 * first failing member is in lks_batch_last_error.  Synchronises. */
lks_status lks_batch_forward(lks_batch* b, int n_steps, double* J_out);

/* lks_adjoint for every member: dJdgamma[i] (n pointers; an entry may be NULL) receives member
 * i's lx*ly doubles, host memory or device memory if on_device.  LKS_ERR_ORDER without a valid
 * forward on every member. */
lks_status lks_batch_adjoint(lks_batch* b, double* const* dJdgamma, int on_device);

/* The work-unit extent (tx, ty) of every step configuration (the adjoint uses the first
 * five); returns their number (writes <= cap pairs) or -1 on bad arguments.  Host only. */
int lks_batch_tile_shapes(int* txty, int cap);

/* chosen2: configuration indices in use for [step, adjoint] (-1 before the first forward);
 * ms (may be NULL): 2 x (number of step configurations) autotune timings in ms per launch,
 * step then adjoint, -1 where not timed. */
lks_status lks_batch_tuning(const lks_batch* b, int* chosen2, float* ms);

/* [0] kernels launched by the last forward or adjoint call (graph nodes included), [1] graphs
 * held, [2] kernel nodes in them. */
lks_status lks_batch_stats(const lks_batch* b, long long* stats3);

const char* lks_batch_last_error(const lks_batch* b);
void lks_batch_destroy(lks_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LKS_H */
