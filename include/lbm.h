/*
 * lbm.h - C ABI of the GB300 two-component Shan-Chen D3Q19 lattice Boltzmann
 * library (Otomo et al., "Multi-component lattice Boltzmann models for
 * accurate simulation of flows with wide viscosity variation",
 * arXiv:1711.03254).
 *
 * One update (lbm_step) is, per cell and per component alpha in {1, 2}:
 *   S1 pull streaming f_i(x) = f*_i(x - c_i), halfway bounce-back
 *      f_i(x) = f*_{-i}(x) when x - c_i is SOLID            (Eq. 1, Eq. 9, Sec. 2 walls)
 *   S2 rho_alpha = sum_i f_i, j = sum_alpha sum_i c_i f_i     (Eq. 4)
 *   S3 psi_beta = rho_beta in fluid, rho^s_beta in SOLID      (Eq. 7, Eq. 11)
 *   S4 F^alpha = G rho_alpha sum_i ws_i c_i psi_beta(x + c_i) (beta != alpha), with
 *      psi_beta of a SOLID neighbour set by the wall model, + rho_alpha g
 *                                                             (Eq. 7, Eq. 11)
 *   S5 u_F = (j + F/2) / rho, nu_mix = p nu_1 + (1-p) nu_2 with p = rho_1/rho in
 *      [0, 1], tau = nu_mix / T0 + 1/2                        (Eq. 5, 6, 8)
 *   S6 feq (Eq. 3), Pi^neq, f' = Phi : Pi (2nd-order Hermite, Eq. 10), forcing
 *   S7 f* = feq + (1 - 1/tau) f' + F_i                        (Eq. 9)
 * with D3Q19 weights w_i (1/3, 1/18, 1/36), T0 = 1/3, force-stencil weights
 * ws_i = 2 w_i, and F_i = w_i c_i.F/(2 T0) + (1 - 1/(2 tau)) w_i/(2 T0^2)
 * (c_i c_i - T0 I):(u_F F + F u_F).
 *
 * Conventions
 *  - Lattice units, Delta t = 1.  Grids are periodic in x, y and z; walls come
 *    from SOLID cells of the geometry.
 *  - Host arrays are C order [batch][nz][ny][nx] (x fastest); velocities have a
 *    trailing axis of 3: [batch][nz][ny][nx][3].
 *  - Cell types: 0 FLUID, 1 SOLID, 2 INLET (holds feq(rho_in, u_in)),
 *    3 OUTLET (takes the streamed distributions of its -x neighbour).
 *  - Ownership: the caller owns every host buffer it passes; the library owns
 *    all device memory, allocated through the allocator hook (default
 *    cudaMalloc) and released by lbm_destroy.
 *  - Errors: every call returns an lbm_status; nothing is thrown across the
 *    ABI.  lbm_last_error gives the message of the context's last failure.
 *    After LBM_ERR_DIVERGED the context stays valid for lbm_get_*,
 *    lbm_set_state and lbm_destroy.
 *  - Work is queued on the context's stream (lbm_set_stream; default: the
 *    legacy default stream).  Calls that return host data synchronise that
 *    stream; lbm_step does not.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument (sizes, tau <= 1/2, bad cell type, ...) */
    LBM_ERR_CUDA = 2,     /* a CUDA runtime call failed (message in lbm_last_error) */
    LBM_ERR_OOM = 3,      /* device allocation failed */
    LBM_ERR_DIVERGED = 4, /* non-finite value, or |u_F| above the sound speed 1/sqrt(3), found by lbm_reduce */
    LBM_ERR_TIMEOUT = 5,  /* lbm_run_to_steady used up its update budget before the tolerance, or a
                             grid-wide barrier of the persistent update gave up waiting */
    LBM_ERR_STATE = 6     /* call out of order (e.g. step before set_fields) */
} lbm_status;

/* Storage of the distributions.  Arithmetic is FP64 in LBM_FP64 and FP32 in
 * the other modes.  LBM_FP32 and the 16-bit modes store each value as its
 * deviation f_i - w_i R from a rest equilibrium, rounded to nearest even,
 * where R is the density (rounded to FP16, kept per cell and component) that
 * the cell the value streams into had at its last update.  FP16 holds that
 * deviation times 2^12 (an exact power of two), to keep small deviations out of
 * FP16's subnormal range. */
typedef enum {
    LBM_FP64 = 0,
    LBM_FP32 = 1,
    LBM_FP32_F16S = 2,
    LBM_FP32_BF16S = 3
} lbm_precision;

/* Kernel strategy for lbm_step. */
typedef enum {
    LBM_KERNEL_AUTO = 0,     /* compact when the grid fits its coordinate limits, else two-pass;
                                for n >= 8 updates of at most 65,536 non-solid cells in all
                                (32,768 inside lbm_run_to_steady's graphs; no wall slip) the
                                persistent update */
    LBM_KERNEL_TWO_PASS = 1, /* density pre-pass, then stream+collide, over the non-solid cells */
    LBM_KERNEL_FUSED = 2,    /* single read of f: z-marching tiles with a recomputed density halo */
    LBM_KERNEL_CLUSTER = 3,  /* persistent: one thread-block cluster per instance, n updates per launch */
    LBM_KERNEL_COMPACT = 4,  /* two-pass on a compact layout that stores only the non-solid cells
                                (in cell order; neighbours found from per-row occupancy words);
                                needs nx <= 2048, ny <= 2048, nz <= 1024 */
    LBM_KERNEL_FUSED_COMPACT = 5, /* single read of f on the compact layout: thread-block clusters
                                march bands of rows along z, densities kept in shared memory;
                                FP32 arithmetic only; where a plane's rows do not fit in shared
                                memory the compact two-pass update runs instead (see
                                lbm_resolved_kernel) */
    LBM_KERNEL_PERSISTENT = 6  /* the compact two-pass update, n updates in one cooperative launch
                                with grid-wide barriers between the passes (for small instances
                                and batches of them); no wall slip; a barrier
                                that waits about two seconds gives up, and the next
                                lbm_reduce, lbm_get_fields or lbm_run_to_steady returns
                                LBM_ERR_TIMEOUT */
} lbm_kernel;

typedef struct {
    int nx, ny, nz;          /* cells per axis, each >= 1 */
    int batch;               /* independent instances, >= 1 */
    lbm_precision precision;
    int eq_order;            /* 0: Eq. 3 as printed (no quadratic terms); 1: with them */
    int wall_model;          /* psi of a SOLID neighbour (Eq. 11): 0 rho^s_beta with the wall forces
                                balanced between components, 1 plain rho^s_beta, 2 the cell's own
                                rho_beta + rho^s_beta (neutral wall at rho^s = 0; recommended),
                                3 the cell's own rho_beta, with the wall potential's force
                                G rho_alpha sum_solid ws_i c_i rho^s_beta added balanced between
                                the components (neutral wall, and no net wall force on the
                                mixture: the permeability of Sec. 3.5) */
    int reg_order;           /* regularisation of the non-equilibrium part (Eq. 10): 2 (or 0, the
                                default of a zeroed struct) second-order Hermite projection of
                                Pi^neq; 3 adds the third-order Hermite terms, built from Pi^neq
                                and u_F recursively (a3_abg = u_a Pi_bg + u_b Pi_ag + u_g Pi_ab)
                                and projected onto the six third-order polynomials D3Q19
                                carries.  reg_order 3 runs in the TWO_PASS and COMPACT
                                strategies (and AUTO) only */
} lbm_config;

typedef struct {
    double tau[2];   /* relaxation time of each pure component, > 1/2; nu_k = (tau_k - 1/2)/3 */
    double G;        /* inter-component coupling of Eq. 7 (negative: repulsive) */
    double rho_s;    /* single wettability parameter: rho^s_1 = max(-rho_s, 0), rho^s_2 = max(rho_s, 0) */
    double g[3];     /* body acceleration applied to both components */
    double rho_in[2];/* INLET densities */
    double u_in[3];  /* INLET velocity */
    double slip;     /* surface scattering at SOLID walls (Sec. 2): the fraction of the particles a
                        wall reflects specularly about its voxel face, in [0, 1]; the rest bounce
                        back.  0 (a zeroed struct) is the no-slip wall.  Non-zero slip runs in the
                        TWO_PASS and COMPACT strategies (and AUTO) only */
} lbm_instance_params;

/* Create a context for cfg->batch instances with per-instance parameters
 * per_instance[batch] (host array, copied).  The parameters are those the
 * paper states its problems with: the relaxation times of the pure components
 * (Eq. 5, nu_k = T0 (tau_k - 1/2)), the coupling G of Eq. 7, the single
 * wettability parameter rho^s of the wall potential (Eq. 11 and the mapping to
 * rho^s_1, rho^s_2 kept beside it), and the body force of Sec. 3.2.
 * Allocates the device buffers.
 * Errors: LBM_ERR_ARG (null pointers, a dimension < 1, batch < 1 or
 * batch > 32767, more than 226 million cells per instance, tau <= 1/2, a
 * non-finite parameter, precision, eq_order, wall_model or reg_order out of
 * range),
 * LBM_ERR_OOM (an allocation through the hook returned NULL), LBM_ERR_CUDA.
 * On failure *out is NULL and nothing stays allocated. */
lbm_status lbm_create(const lbm_config *cfg, const lbm_instance_params *per_instance, lbm_ctx **out);

/* Upload the cell types, host uint8 [batch][nz][ny][nx] with values 0..3
 * (page-locked host memory makes the copy a DMA).  The types are checked, and
 * the cell lists and compact row tables built, on the device; the call returns
 * when they are done.  On LBM_ERR_ARG nothing of the context changes.
 * Errors: LBM_ERR_ARG (null, value > 3, an instance without any FLUID cell),
 * LBM_ERR_OOM (scratch allocation), LBM_ERR_CUDA. */
lbm_status lbm_set_geometry(lbm_ctx *ctx, const uint8_t *cell_type);

/* Initialise every non-solid cell to f = feq(rho_alpha, u) (Eq. 3, no force
 * correction); INLET cells take feq(rho_in, u_in).  Host FP64 arrays
 * rho1, rho2 [batch][nz][ny][nx] and u [batch][nz][ny][nx][3].  Resets the
 * residual snapshot.  Errors: LBM_ERR_ARG (null), LBM_ERR_STATE (no geometry). */
lbm_status lbm_set_fields(lbm_ctx *ctx, const double *rho1, const double *rho2, const double *u);

/* Advance every instance by n >= 0 updates (asynchronous on the context's
 * stream).  One update is the streaming-collision step of Eq. 1 / Eq. 9 with
 * the steps S1-S7 above: pull streaming and halfway bounce-back (Sec. 2,
 * volumetric wall in its voxel-aligned case), moments (Eq. 4), the
 * pseudo-potential and Shan-Chen force with the wall term (Eq. 7, Eq. 11),
 * u_F and the density-weighted tau_mix (Eq. 5, 6, 8), and the regularised
 * collision with forcing (Eq. 3, Eq. 9, Eq. 10).  The densities and velocity
 * u_F of the last update are kept for lbm_get_fields / lbm_reduce.
 * Errors: LBM_ERR_ARG (n < 0), LBM_ERR_STATE (no fields), LBM_ERR_CUDA
 * (launch failure). */
lbm_status lbm_step(lbm_ctx *ctx, int n);

/* Split update for a decomposition of one domain into z-slabs (one process
 * and context per slab; no counterpart in the paper, which runs one domain).
 * Each context holds its slab plus one ghost plane on either side (periodic in
 * z inside the context).  Per update the caller
 *   1. puts into its lower ghost plane the LBM_PLANE_F_UP values of the lower
 *      neighbour's last slab plane, and into its upper ghost plane the
 *      LBM_PLANE_F_DOWN values of the upper neighbour's first slab plane
 *      (the post-collision values that stream across the faces, Eq. 1);
 *   2. runs lbm_step_part(ctx, 0): the density pass, psi of every cell (Eq. 7);
 *   3. puts the neighbours' psi of those planes into its ghost planes
 *      (LBM_PLANE_PSI: the interaction force of Eq. 7 reaches one cell);
 *   4. runs lbm_step_part(ctx, 1): the collision pass, completing the update.
 * The slab cells then match the single-domain update bit for bit; the ghost
 * cells hold meaningless values (also in lbm_get_fields and lbm_reduce).
 * Needs the compact layout's limits (the split update is the compact
 * two-pass one, whatever lbm_set_kernel chose); part 1 must follow part 0, and
 * lbm_step is refused in between (LBM_ERR_STATE).
 * Errors: LBM_ERR_ARG (part not 0 or 1, grid beyond the compact limits),
 * LBM_ERR_STATE (no fields, parts out of order), LBM_ERR_CUDA. */
lbm_status lbm_step_part(lbm_ctx *ctx, int part);

typedef enum {
    LBM_PLANE_F_UP = 0,   /* f* of the 5 directions with c_z = +1: [5][cells of the plane] pairs */
    LBM_PLANE_F_DOWN = 1, /* f* of the 5 directions with c_z = -1 */
    LBM_PLANE_PSI = 2     /* psi pairs of the plane's cells: [cells] */
} lbm_plane_part;

/* Bytes of one plane's part (instance 0): cells of plane z x (5 f pairs, or
 * one psi pair); an f pair is both components in the storage format (2 x 8,
 * 4 or 2 bytes, as stored: deviations from the reference densities in the
 * shifted modes), a psi pair 2 x 8 (FP64) or 2 x 4 bytes.  Cells are the
 * plane's non-solid cells in cell order.  Errors: LBM_ERR_ARG (batch != 1, part
 * or plane out of range), LBM_ERR_STATE (no geometry within the compact
 * limits). */
lbm_status lbm_plane_bytes(lbm_ctx *ctx, int what, int z, size_t *bytes);

/* Copy one plane's part between the context's current state and buf (host or
 * device memory, lbm_plane_bytes long; to_buf != 0 reads the context, 0
 * writes it).  Synchronises the stream.  Errors as lbm_plane_bytes, plus
 * LBM_ERR_ARG (null buf), LBM_ERR_CUDA. */
lbm_status lbm_plane_copy(lbm_ctx *ctx, int what, int z, void *buf, int to_buf);

/* Copy the macroscopic fields of the last update (or of lbm_set_fields) to
 * host FP64 arrays rho1, rho2 [batch][nz][ny][nx], u [batch][nz][ny][nx][3]
 * (u is u_F of Eq. 8; zero in SOLID cells).  Any pointer may be NULL to skip
 * that field.  Synchronises the stream. */
lbm_status lbm_get_fields(lbm_ctx *ctx, double *rho1, double *rho2, double *u);

/* FP64 reductions per instance over non-solid cells (no counterpart in the
 * paper, which states no convergence test: M1 and M2 are the per-component
 * masses that Eq. 1 conserves, P the momentum that the forcing of Eq. 9 changes
 * by the total force, and the residual the steady-state test of the
 * warm-start comparison), written to the host
 * array out[batch][7] = {M1, M2, Px, Py, Pz, residual, max|u_F|} with
 * P = sum rho u_F and residual = |u - u_prev|_2 / (k |u|_2 + 1e-30), where
 * u_prev and k are the velocity at and the updates since the previous
 * lbm_reduce (0 when k = 0).  The sums use a fixed-order tree, so repeated
 * runs give identical bits.  Returns LBM_ERR_DIVERGED (after filling out) when a
 * value is not finite or max|u_F| > 1/sqrt(3).  Synchronises the stream. */
lbm_status lbm_reduce(lbm_ctx *ctx, double *out);

/* Post-collision distributions of the current state as FP64 (the shifted
 * storage modes are expanded back to f = stored + w_i R), host array
 * f[batch][2][19][nz][ny][nx] with the direction order 0 rest, then pairs
 * +x,-x, +y,-y, +z,-z, (1,1,0),(-1,-1,0), (1,-1,0),(-1,1,0), (1,0,1),(-1,0,-1),
 * (1,0,-1),(-1,0,1), (0,1,1),(0,-1,-1), (0,1,-1),(0,-1,1).  SOLID cells carry
 * no distributions: they are exported as 0 and ignored on import.
 * lbm_set_distributions uploads such an array (rounded to the storage format)
 * as the new state; the fields of the last update are kept.
 * Errors: LBM_ERR_ARG (null), LBM_ERR_STATE (no fields yet). */
lbm_status lbm_get_distributions(lbm_ctx *ctx, double *f);
lbm_status lbm_set_distributions(lbm_ctx *ctx, const double *f);

/* Checkpoint: with buf == NULL, *bytes receives the size needed; otherwise
 * the distributions, cell types, fields and counters are written to buf
 * (host, *bytes large enough).  lbm_set_state restores a buffer written by a
 * context of the same configuration; the continuation is bitwise identical.
 * Errors: LBM_ERR_ARG (size or configuration mismatch). */
lbm_status lbm_get_state(lbm_ctx *ctx, void *buf, size_t *bytes);
lbm_status lbm_set_state(lbm_ctx *ctx, const void *buf, size_t bytes);

/* Replace the per-instance parameters (host array [batch], copied; checked as
 * in lbm_create) for the updates that follow; the state is kept.  The paper
 * changes the driving force in stages this way to find the critical pressure
 * of slug displacement (Sec. 3.6).  Synchronises the stream.
 * Errors: LBM_ERR_ARG (null, tau <= 1/2, non-finite value), LBM_ERR_STATE
 * (between the parts of a split update), LBM_ERR_CUDA. */
lbm_status lbm_set_params(lbm_ctx *ctx, const lbm_instance_params *per_instance);

/* Failure test of the persistent update (LBM_KERNEL_PERSISTENT): its
 * grid-wide barriers wait at most wait_cycles SM clock cycles (default 4e9,
 * about two seconds) and, with missing > 0, wait for that many arrivals more
 * than the launch has, so that every barrier gives up after the bound; the
 * launch then ends early and the next lbm_reduce, lbm_get_fields or
 * lbm_run_to_steady returns LBM_ERR_TIMEOUT.  missing = 0 restores normal
 * barriers.  Errors: LBM_ERR_ARG (null, wait_cycles < 1000). */
lbm_status lbm_set_barrier_test(lbm_ctx *ctx, long long wait_cycles, unsigned missing);

/* Use the given cudaStream_t (cast to void*) for all later work; NULL selects
 * the legacy default stream.  The caller keeps ownership of the stream. */
lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Choose the kernel strategy (default LBM_KERNEL_AUTO).  LBM_ERR_ARG if the
 * strategy cannot run this configuration (e.g. CLUSTER on a large grid,
 * COMPACT beyond its coordinate limits, FUSED, CLUSTER or FUSED_COMPACT with
 * reg_order 3).  The compact strategy keeps the
 * distributions in its own layout; the library converts the state between the
 * layouts when a step, an export or an import needs the other one (one
 * gather of f, on the context's stream). */
lbm_status lbm_set_kernel(lbm_ctx *ctx, lbm_kernel kernel);

/* The strategy lbm_step(ctx, n) would run now (AUTO resolved; it depends on
 * the geometry, so call it after lbm_set_geometry).  Returns -1 for a NULL
 * context. */
int lbm_resolved_kernel(const lbm_ctx *ctx, int n);

/* Tiling of the fused kernel: tile 0 = 32x8, 1 = 32x4, 2 = 64x4, 3 = 32x16
 * cells per thread block, each marching zchunk planes; -1 selects the
 * built-in choice.  Errors: LBM_ERR_ARG (out of range). */
lbm_status lbm_set_tiling(lbm_ctx *ctx, int tile, int zchunk);

/* Autotuner: time every kernel strategy and fused tiling on the current state
 * (steps_per_trial updates each, CUDA events on the context's stream), keep the
 * fastest for later lbm_step calls, and restore the state, so the next update
 * is the one that would have followed without tuning.  With cache_path non-NULL
 * the choice is looked up in / appended to that file (one JSON object per line,
 * keyed by grid, batch, precision, equilibrium order and device name); a hit
 * skips the timing.  *chosen (may be NULL) receives the strategy, tile and
 * zchunk.  Errors: LBM_ERR_STATE (no fields), LBM_ERR_ARG (steps_per_trial < 1). */
lbm_status lbm_autotune(lbm_ctx *ctx, int steps_per_trial, const char *cache_path, int chosen[3]);

/* Advance until every instance's residual (as in lbm_reduce) is <= tol,
 * checking every check_every updates, for at most max_steps updates.  The
 * check_every updates and the reduction are captured once as a CUDA graph and
 * replayed.  *steps_done and residual[batch] (may be NULL) receive the update
 * count and the last residuals.  Returns LBM_ERR_DIVERGED if a reduction sees a
 * non-finite value or |u_F| above the lattice sound speed (as lbm_reduce), and
 * LBM_ERR_TIMEOUT if max_steps were used up first (both leave a valid state;
 * *steps_done and residual are filled either way).
 * Errors: LBM_ERR_ARG (check_every < 1, max_steps < 0). */
lbm_status lbm_run_to_steady(lbm_ctx *ctx, int check_every, double tol, int max_steps, int *steps_done,
                             double *residual);

/* Allocation-free FP64 field sums (no counterpart in the paper; a service for
 * callers that cannot allocate device memory when they need the check, e.g.
 * code inside a fixed-size memory pool, a real-time loop that must not call
 * cudaMalloc because it synchronises the device, or a host application that
 * owns all GPU memory).  Same sums as lbm_reduce, computed from caller-owned
 * device arrays: rho1, rho2 [batch][ncells] and u [batch][ncells][3] (FP64),
 * cell_type [batch][ncells] (uint8, SOLID cells skipped); writes the device
 * array out[batch][6] = {M1, M2, Px, Py, Pz, max|u|} (max|u| is NaN if a value
 * is not finite).  Work is queued on `stream` (a cudaStream_t, NULL = legacy
 * default) and not synchronised.  The per-block partial sums live in a fixed
 * 1 MiB device array inside the library (held by every GPU that loads it until
 * exit), so no call allocates; every call overwrites the part it uses, and two
 * calls that overlap on the GPU race on that array.  The first call on a
 * device looks up the array's device address; make that first call before any
 * stream capture.  Errors: LBM_ERR_ARG (null pointer, ncells < 1, batch < 1 or
 * batch > 64), LBM_ERR_CUDA (no device, lookup or launch failure). */
lbm_status lbm_field_sums_static(const double *rho1, const double *rho2, const double *u,
                                 const uint8_t *cell_type, long long ncells, int batch, double *out, void *stream);

/* Number of CUDA kernel launches the context has issued so far. */
long long lbm_launch_count(const lbm_ctx *ctx);

/* Per-kernel device time of lbm_step (no counterpart in the paper: it is how
 * the update kernels are measured against the memory roofline).  Parts: */
typedef enum {
    LBM_PART_PSI = 0,     /* two-pass: density and psi of every fluid cell */
    LBM_PART_COLLIDE = 1, /* two-pass: pull, forces, collision, store */
    LBM_PART_FUSED = 2,   /* single-read fused update */
    LBM_PART_CLUSTER = 3, /* persistent launch (several updates each): CLUSTER, PERSISTENT */
    LBM_PART_COUNT = 4
} lbm_part;

/* Start timing: until lbm_timing_end, every kernel launched by lbm_step on the
 * context's stream is bracketed by CUDA events (at most max_launches of them,
 * 1..65536; launches beyond that are not timed).  The events are created here.
 * Steps issued while the stream is being captured are not timed.
 * Errors: LBM_ERR_ARG (null ctx, max_launches out of range), LBM_ERR_STATE
 * (timing already on), LBM_ERR_CUDA (event creation). */
lbm_status lbm_timing_begin(lbm_ctx *ctx, int max_launches);

/* Stop timing: waits for the last recorded event, then writes, per lbm_part,
 * the summed device milliseconds to ms[LBM_PART_COUNT] and the number of timed
 * launches to launches[LBM_PART_COUNT] (both caller-owned host arrays), and
 * destroys the events.  Errors: LBM_ERR_ARG (null pointer), LBM_ERR_STATE
 * (timing not on), LBM_ERR_CUDA (event query). */
lbm_status lbm_timing_end(lbm_ctx *ctx, double *ms, long long *launches);

/* Process-wide device allocator hook used by contexts created afterwards:
 * alloc(bytes, stream) returns device memory or NULL; release(ptr, stream)
 * frees it.  Passing NULLs restores cudaMalloc / cudaFree. */
lbm_status lbm_set_allocator(void *(*alloc)(size_t bytes, void *stream),
                             void (*release)(void *ptr, void *stream));

/* Message of the context's last error ("" when none); ctx may be NULL for the
 * last lbm_create / lbm_set_allocator failure.  Valid until the next call. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Release the context and its device memory (synchronises its stream). */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
