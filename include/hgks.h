/*
 * hgks.h -- C-ABI of the GB300 (sm_103a) high-order gas-kinetic scheme (HGKS)
 * library, libhgks.so.
 *
 * The method is that of "Multiple-GPU accelerated high-order gas-kinetic
 * scheme for direct numerical simulation of compressible turbulence"
 * (arXiv 2207.01173), Sec. 2: the finite-volume semi-discretisation
 * dQ/dt = L(Q) (Eqs. "semi", "semi2") on a structured hexahedral grid, the
 * BGK gas-kinetic interface flux at the 2x2 Gauss points of every face
 * (Eq. "flux" and the compatibility / micro-slope conditions that follow it),
 * its linear-in-time fit (Eq. "expansion-1") and the two-stage fourth-order
 * time update (Eq. "two-stage"), with fifth-order WENO reconstruction applied
 * dimension by dimension.  The test problems are the Taylor-Green vortex
 * (Sec. 4.1) and the compressible channel flow (Sec. 4.2).
 *
 * Conventions
 *   - Every entry point returns an hgks_status; results go through
 *     out-pointers.  HGKS_OK is 0.
 *   - The library owns all device memory of a handle (allocated at
 *     hgks_create, freed at hgks_destroy).
 *   - Host buffers passed in are owned by the caller; the library copies
 *     them and never keeps a pointer.  Calls that read or write host
 *     buffers return only after the copy has completed.
 *   - Work is enqueued on the CUDA stream given at hgks_create (NULL = the
 *     legacy default stream).  hgks_step is asynchronous except for one
 *     status read at its end.
 *   - A handle is used by one host thread at a time.
 *   - Conservative state layout for host buffers: double[5][nz][ny][nx],
 *     components (rho, rho U, rho V, rho W, rho E), x fastest.
 *   - Units: gas constant R = 1, so p = rho T and lambda = rho / (2 p).
 *   - The product path never falls back to the CPU: if no usable CUDA
 *     device is present hgks_create fails with HGKS_ERR_CUDA.
 */
#ifndef HGKS_H
#define HGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hgks_s *hgks_t; /* opaque handle */

typedef enum {
    HGKS_OK = 0,
    HGKS_ERR_INVALID_ARG = 1, /* a NULL pointer, a size or parameter out of range */
    HGKS_ERR_OOM = 2,         /* device allocation failed */
    HGKS_ERR_CUDA = 3,        /* a CUDA runtime call failed (see hgks_last_error) */
    HGKS_ERR_NONFINITE = 4,   /* a step produced a non-finite value or rho <= 0 or p <= 0;
                                 the state is left at the last completed step */
    HGKS_ERR_TIMEOUT = 5,     /* reserved for bounded device-side waits */
    HGKS_ERR_STATE = 6        /* call not valid in the handle's current state */
} hgks_status;

/* HGKS_BC_EXTERNAL: the three ghost layers of that side belong to a
 * neighbouring sub-domain and are written by the caller (hgks_halo_set);
 * the library never fills them.  This is the sub-domain boundary of the
 * paper's domain decomposition (Sec. 3.2, Alg. 2), accepted in z only (the
 * slab direction). */
typedef enum { HGKS_BC_PERIODIC = 0, HGKS_BC_ISOTHERMAL_WALL = 1, HGKS_BC_EXTERNAL = 2 } hgks_bc;
typedef enum { HGKS_VISC_CONSTANT = 0, HGKS_VISC_POWER = 1 } hgks_visc_kind;
/* HGKS_FP64: all arithmetic in FP64.  HGKS_MIXED: FP64 for the state and
 * the stage update; reconstruction and flux arithmetic in FP32 on deviations
 * from the stencil centre; the reconstructed values, the equilibrium state
 * Q0 (mean of the two sides plus an FP32 compatibility correction), its
 * pressure and Euler flux as float-float pairs (two FP32 numbers, ~48 bits).
 * A MIXED handle allocates one more state-sized buffer (the state split into
 * hi / lo FP32 planes before each stage).
 * HGKS_MIXED_T64: HGKS_MIXED with the Maxwellian temperature T0 = p0/rho0 of
 * every Gauss point, its collision time tau = mu(T0)/p0 and the time-
 * integration coefficients (the exp(-delta/tau) terms of both windows) formed
 * in FP64 from the float-float Q0; the sums they weight stay FP32.  This is
 * the split that keeps the temperature / collision-time terms in FP64; it is
 * not accepted by hgks_batch_create. */
typedef enum { HGKS_FP64 = 0, HGKS_MIXED = 1, HGKS_MIXED_T64 = 2 } hgks_precision;

/* Structured grid (Sec. 2 "orthogonal structured mesh"; Sec. 4.2 mesh map).
 * nx, ny, nz >= 1 cells.  Uniform spacing lx/nx and lz/nz in x and z.
 * y_stretch_b = 0: uniform y; y_stretch_b = b > 0: y faces at
 *   y_j = y0 + ly/2 (1 + tanh(b (2j/ny - 1)) / tanh(b)), j = 0..ny,
 * which for y0 = -1, ly = 2 is the channel map of Sec. 4.2. */
typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    double x0, y0, z0;
    double y_stretch_b;
} hgks_grid;

/* Viscosity law (Sec. 4.2): mu = mu_ref (T / T_ref)^omega for POWER,
 * mu = mu_ref for CONSTANT.  The collision time is tau = mu / p (Sec. 2). */
typedef struct {
    hgks_visc_kind kind;
    double mu_ref, T_ref, omega;
} hgks_visc;

/* Boundary conditions per direction and side (Sec. 4: periodic in every
 * direction for the TGV; periodic x, z and no-slip isothermal walls in y for
 * the channel).  Walls need at least 3 cells in their direction, and so do
 * EXTERNAL sides (a neighbour's ghost layers come from this sub-domain's
 * three boundary layers alone). */
typedef struct {
    hgks_bc lo[3], hi[3];
    double T_wall;
} hgks_bcs;

/* Diagnostics (Sec. 4.1 definitions of E_k and eps_com). */
typedef struct {
    double t;          /* simulated time */
    int64_t step;      /* completed steps */
    double dt;         /* time step of the last completed step */
    double Ek;         /* (1 / (rho0 Omega)) sum 1/2 rho |u|^2 |Omega_i| */
    double enstrophy;  /* (1 / (rho0 Omega)) sum 1/2 rho |omega|^2 |Omega_i| */
    double eps_com;    /* (1 / (rho0 Omega)) sum mu (|omega|^2 + 4/3 (div u)^2) |Omega_i| */
    double mass, mom[3], energy; /* sums of Q |Omega_i| */
    double max_mach;   /* max |u| / c over cells */
    double wall_shear; /* mean x-momentum wall flux per unit wall area of the last step's
                          first stage (walls only, else 0) */
} hgks_stats_t;

/* Create a solver.
 *   grid, visc, bcs: see above (copied).  gamma > 1 (internal degrees of
 *   freedom K = (5 - 3 gamma)/(gamma - 1), Sec. 2).  Pr > 0 (Prandtl number,
 *   applied to the energy flux as F_E += (1/Pr - 1) q).
 *   body_force: constant acceleration (G_x, G_y, G_z) or NULL for none.  It
 *   enters L as the source (0, rho G, rho u.G) and dL/dt as its time
 *   derivative (0, G L_rho, G.L_mom); the interface flux's time slope comes
 *   from the force-free compatibility condition, so the forced terms are
 *   second order in time.
 *   precision: HGKS_FP64, HGKS_MIXED or HGKS_MIXED_T64 (see hgks_precision).
 *   cuda_stream: a cudaStream_t, or NULL.
 *   out: receives the handle.
 * Errors: INVALID_ARG, OOM, CUDA (no device / context failure). */
hgks_status hgks_create(const hgks_grid *grid, double gamma, double Pr, const hgks_visc *visc,
                        const hgks_bcs *bcs, const double body_force[3], hgks_precision precision,
                        void *cuda_stream, hgks_t *out);

/* Taylor-Green vortex of Sec. 4.1 on the grid's box as exact cell averages:
 * u = U0 sin x cos y cos z, v = -U0 cos x sin y cos z, w = 0, rho = rho0,
 * p = p0 + rho0 U0^2/16 (cos 2x + cos 2y)(cos 2z + 2), p0 = rho0 U0^2/(gamma Ma^2).
 * Resets t and step to 0.  Sets the stats reference density to rho0. */
hgks_status hgks_init_tgv(hgks_t h, double Ma, double U0, double rho0);

/* Perturbed Poiseuille channel of Sec. 4.2 (point values at cell centres):
 * rho = 1, T = T_w = 1/(gamma Ma_b^2) (U_b = 1), U = 1.5 (1 - yn^2) with yn the
 * wall-normal coordinate scaled to [-1, 1]; u = U (1 + a r0), v = a r1, w = a r2,
 * a = noise_amp, r_c uniform in [-1, 1) from splitmix64(seed ^ (3 idx + c)),
 * idx = (k ny + j) nx + i.  Sets the wall temperature to T_w. */
hgks_status hgks_init_channel(hgks_t h, double Ma_b, double noise_amp, uint64_t seed);

/* Smooth density wave for convergence studies: exact cell averages of
 * rho = 1 + amp sin(pi sum_d k_d x_d), U_d = k_d, p = 1, with k_d = 1 for every
 * direction that has more than one cell and 0 otherwise. */
hgks_status hgks_init_density_wave(hgks_t h, double amp);

/* Copy a host state double[5][nz][ny][nx] in / out (blocking). */
hgks_status hgks_set_state(hgks_t h, const double *host_q);
hgks_status hgks_get_state(hgks_t h, double *host_q);
/* Set the simulated time and step counter (e.g. when resuming). */
hgks_status hgks_set_time(hgks_t h, double t, int64_t step);

/* Advance nsteps S2O4 steps.  Each step fills the ghost cells, takes
 * dt = cfl * min over cells and directions of dx_d / (|u_d| + c) (Alg. 1 STEP 1)
 * and runs the two stages of Eq. "two-stage" with that dt.
 * Errors: INVALID_ARG (nsteps < 0, cfl <= 0), NONFINITE, CUDA. */
hgks_status hgks_step(hgks_t h, int nsteps, double cfl);
/* As hgks_step with a fixed time step dt > 0. */
hgks_status hgks_step_dt(hgks_t h, int nsteps, double dt);
/* The CFL time step of the current state (blocking). */
hgks_status hgks_compute_dt(hgks_t h, double cfl, double *dt);

/* L(Q) and dL/dt(Q) of the current state (Eq. "semi2" and its time
 * derivative, F^n and dF^n/dt from the fit over dt and dt/2), as host
 * arrays double[5][nz][ny][nx].  For testing the flux path in isolation. */
hgks_status hgks_rhs(hgks_t h, double dt, double *host_L, double *host_dL);

/* Device time of one step split by kernel kind (CUDA events recorded on the
 * handle's stream between the launches). */
typedef struct {
    double total_ms;                 /* first to last launch of the step */
    double ghost_ms, dt_ms;          /* ghost fill (2 per step), CFL reduction */
    double normal_ms, tan1_ms, flux_ms; /* the three sweep passes, summed over 2 stages x 3 sweeps */
    double update_ms, other_ms;      /* stage updates; wall stress and commit */
    int launches;                    /* kernels launched in the step */
    int flux_launches;               /* launches of the flux pass */
} hgks_step_times_t;
/* One step as hgks_step(h, 1, cfl) with the per-kind device times. */
hgks_status hgks_step_timed(hgks_t h, double cfl, hgks_step_times_t *out);

/* Measured FP64 fused-multiply-add throughput of the current device in
 * TFLOP/s (2 flops per FMA), from a short dependent-chain kernel. */
hgks_status hgks_fp64_probe(double *tflops);

/* Diagnostics of the current state (blocking). */
hgks_status hgks_stats(hgks_t h, hgks_stats_t *out);

/* Algorithmic floating-point work of the step, from the kernels' own
 * arithmetic run on the host with an operation-counting scalar type.
 * +, -, * count 1 (a fused multiply-add 2); division, sqrt, exp, erfc and pow
 * count 1 each and are also given on their own for the flux pass.  Index
 * arithmetic and comparisons count 0.  Host only; needs no device. */
typedef struct {
    double normal_per_face;       /* normal reconstruction, per position of its pass */
    double tan1_per_pos;          /* first tangential reconstruction, per position */
    double flux_per_face;         /* second tangential reconstruction + 4 Gauss-point fluxes, per face */
    double div_per_face_flux;     /* divisions inside flux_per_face */
    double special_per_face_flux; /* sqrt / exp / erfc / pow inside flux_per_face */
    double per_step;              /* all passes of one two-stage step on the grid */
} hgks_flop_model_t;
/* precision: HGKS_FP64 (the method's arithmetic; the mixed path runs the same
 * formulas, with some values carried as float-float pairs on top, and is
 * rejected here with INVALID_ARG).  Errors: INVALID_ARG (NULL, bad sizes,
 * precision other than FP64). */
hgks_status hgks_flop_model(const hgks_grid *grid, hgks_precision precision, hgks_flop_model_t *out);

/* ---- sub-domains: one step taken in phases -----------------------------
 * The paper splits the grid over GPUs and, before each stage of a step,
 * exchanges the ghost layers of neighbouring sub-domains and takes the
 * global minimum of the CFL limit (Sec. 3.2, Alg. 2 and the MPI+CUDA
 * communication figure).  A handle whose z sides are HGKS_BC_EXTERNAL is one
 * such sub-domain (a slab of whole z planes), and one step of the whole
 * domain runs as
 *     dt = min over sub-domains of hgks_compute_dt(h, cfl)     (global CFL)
 *     for stage s = 1, 2 (state 0 = the current state, 1 = the stage state):
 *         hgks_fill_ghosts(h, s - 1)       on every sub-domain
 *         hgks_halo_get(h, s - 1, 2, side, buf) on every sub-domain and side
 *         hgks_halo_set(h', s - 1, 2, other side, buf) on its neighbour h'
 *         hgks_stage(h, s, dt)             on every sub-domain
 * which gives, cell for cell, the same numbers as hgks_step on the whole
 * grid.  The diagnostics of a sub-domain (hgks_stats) are volume averages over
 * that sub-domain; set the halos of the current state first, since the
 * vorticity stencils reach into them.  Buffers are device memory owned by the caller; nothing is allocated
 * by these calls.  All work is enqueued on the handle's stream; to hand a
 * buffer from one handle to another on a different stream, order the two
 * streams (an event) or use one stream. */
enum { HGKS_STATE_CURRENT = 0, HGKS_STATE_STAGE = 1 };

/* Fill the ghost layers of a state (HGKS_STATE_CURRENT: the current state
 * Q^n; HGKS_STATE_STAGE: the stage state Q* of the step in progress) on every
 * side that is not EXTERNAL: periodic copies, wall mirrors, in the order x,
 * y, z as hgks_step does, so edge and corner ghosts are filled too.
 * Errors: INVALID_ARG (NULL handle, bad state index). */
hgks_status hgks_fill_ghosts(hgks_t h, int state);

/* Doubles in one halo buffer of direction dir (only dir = 2, z, is
 * supported): 5 components x 3 layers x (ny + 6) x (nx + 6), i.e. whole
 * padded planes with their x and y ghosts.  0 for an invalid argument. */
size_t hgks_halo_count(hgks_t h, int dir);

/* Copy the three boundary layers next to side (0: low, 1: high) of direction
 * dir (2) of a state, with the x and y ghost cells of each plane, into d_buf
 * (device pointer, hgks_halo_count(h, dir) doubles, layout
 * [5][3][ny + 6][nx + 6], layers ordered by increasing z).  Fill the x / y
 * ghosts (hgks_fill_ghosts) first: they travel with the planes, which makes
 * the stencil corners right.  Asynchronous on the handle's stream.
 * Errors: INVALID_ARG (NULL, dir != 2, side or state out of range). */
hgks_status hgks_halo_get(hgks_t h, int state, int dir, int side, double *d_buf);

/* Write d_buf (device pointer, layout as for hgks_halo_get) into the three
 * ghost layers on side (0: low, 1: high) of direction dir (2) of a state.
 * For a slab decomposition the low ghosts of a slab are the high boundary
 * layers of its lower neighbour, and the other way round.  Asynchronous on
 * the handle's stream.
 * Errors: INVALID_ARG (NULL, dir != 2, side or state out of range). */
hgks_status hgks_halo_set(hgks_t h, int state, int dir, int side, const double *d_buf);

/* One stage of the step with time step dt > 0 (Eq. "two-stage"), on a state
 * whose ghost layers are all set (hgks_fill_ghosts plus the halos):
 *   stage 1: the three sweeps on Q^n, then Q* = Q^n + dt/2 L + dt^2/8 dL and
 *            R = Q^n + dt L + dt^2/6 dL;
 *   stage 2: the three sweeps on Q*, then Q^{n+1} = R + dt^2/3 dL(Q*), and
 *            the step is committed (t += dt, step + 1).
 * Stage 2 reads the device status once (as hgks_step does) and reports a bad
 * state with NONFINITE, leaving the state at the last completed step.
 * Errors: INVALID_ARG (stage not 1 or 2, dt <= 0), STATE (stage 2 without a
 * stage 1 of the same step: a whole step, a state copy in or an initial field
 * in between also cancels the pending stage 1), NONFINITE, CUDA. */
hgks_status hgks_stage(hgks_t h, int stage, double dt);

/* Largest grid (cells) accepted by hgks_cfl_dt_noalloc. */
#define HGKS_NOALLOC_MAX_CELLS 33554432

/* The CFL time step of a caller-owned device state, with no device memory
 * allocated by this call or by the library (the paper has no counterpart;
 * this is a library service).
 *
 * For callers that cannot allocate device memory when they need a time step:
 * an application whose memory manager reserved the whole device at start-up,
 * a solver embedded in another program's time loop that must not change the
 * device footprint, or a loop that cannot afford the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.
 *
 *   grid:  cell counts, box lengths and y map as for hgks_create (host, read).
 *   gamma: ratio of specific heats (> 1).   cfl: CFL number (> 0).
 *   d_q:   device pointer, the conservative state double[5][nz][ny][nx]
 *          (no ghost cells), owned by the caller, read only.
 *   d_dt:  device pointer to one double, owned by the caller; receives
 *          cfl * min over cells and directions of dx_d / (|u_d| + c).
 *   cuda_stream: the stream the work is enqueued on (NULL = default stream);
 *          the call is asynchronous: d_dt holds the result once the stream
 *          reaches this work.
 * Scratch: a fixed 1 MiB array of device memory (one double per 256 cells)
 * that every GPU loading the library holds until the process exits.  Grids
 * with more than HGKS_NOALLOC_MAX_CELLS cells are rejected with
 * HGKS_ERR_INVALID_ARG.  Every call uses the same array (it keeps the last
 * call's partial minima; each call writes every slot it reads), so calls
 * whose work overlaps on the GPU race with each other: serialise them on one
 * stream.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  The address is kept per CUDA context:
 * after cudaDeviceReset, or under another current context, the next call
 * looks it up again (so that call, too, should come before a capture).
 * Invalid state: if any cell has a non-positive density or pressure, or a
 * non-finite value, *d_dt receives NaN (no cell is silently skipped).
 * Wall-stretched grids (y_stretch_b > 0): the cell heights are computed on
 * the device with the device tanh, while hgks_compute_dt takes them from a
 * host table, so on such grids the two agree to about 1e-13 relative (the
 * rounding of a difference of two tanh values), not bit for bit; on uniform
 * grids they agree to the last bit.
 * Errors: INVALID_ARG (NULL pointer, bad sizes, too many cells), CUDA (a
 * launch failed, or a CUDA error from earlier work was already pending: it is
 * reported with its own text and left pending). */
hgks_status hgks_cfl_dt_noalloc(const hgks_grid *grid, double gamma, double cfl, const double *d_q,
                                double *d_dt, void *cuda_stream);

/* ---- batches: many problems advanced together -------------------------
 * The paper advances one problem at a time; batching has no counterpart
 * there.  Every problem of a batch takes exactly the step of hgks_step (the
 * two-stage step of Eq. "two-stage" with the fluxes of Eq. "flux"), with the
 * same arithmetic, so a batch reproduces its problems stepped one by one bit
 * for bit.
 * A batch groups n solver handles (any grids, gas parameters and precisions,
 * all created on one CUDA stream) so that each pass of a step runs as one
 * persistent kernel over a tile work-list spanning all of them, and the whole
 * step is one captured CUDA graph replayed on the batch's own stream.
 * Ownership: the batch borrows the handles and their device buffers; destroy
 * the batch before any of its handles.  Between batch calls the handles stay
 * usable on their own (init, state copies, stats, hgks_step).
 * Each problem keeps its own time step, step counter and bad-state flag: a
 * problem whose stage produces a non-finite or non-positive state stops at
 * its last completed step for the rest of the call while the others advance,
 * and the call returns HGKS_ERR_NONFINITE naming it in
 * hgks_batch_last_error; its flag is cleared on return. */
typedef struct hgks_batch_s *hgks_batch_t;
typedef struct {
    int problems;          /* handles in the batch */
    int tile_sweep;        /* interface positions per tile of the FP64 flux pass */
    int tile_cells;        /* cells per tile of the cell passes (ghost fill, CFL, update, split) */
    int launches_per_step; /* kernel nodes of the per-step graph */
    long long tiles;       /* tiles over all passes */
    double last_ms;        /* device time of the graph steps of the last hgks_batch_step call */
    int last_steps;        /* steps of that call */
    int tile_normal;       /* positions per tile of the FP64 normal pass */
    int tile_tan1;         /* positions per tile of the FP64 first tangential pass */
    int tile_normal_mx;    /* positions per tile of the mixed normal pass */
} hgks_batch_info_t;
/* handles: n distinct handles on one stream (n >= 1).  *out receives the
 * batch.  Errors: INVALID_ARG (NULL, n < 1, a repeated handle, handles on
 * different streams, a handle with EXTERNAL sides or HGKS_MIXED_T64
 * precision), CUDA (allocation of the work-lists). */
hgks_status hgks_batch_create(hgks_t *handles, int n, hgks_batch_t *out);
/* nsteps (>= 0) steps of every problem, each with its own CFL time step
 * cfl * min over cells of dx_d / (|u_d| + c).  Work queued earlier on the
 * handles' stream completes first; the call returns after the steps have
 * completed.  The graph is captured on the first call and again whenever
 * cfl or the tile size changes.  Errors: INVALID_ARG, NONFINITE (see above),
 * CUDA. */
hgks_status hgks_batch_step(hgks_batch_t b, int nsteps, double cfl);
/* Autotuner: picks the tile size of each tunable pass by timing that pass
 * on the current states: the cell passes (candidates 2048, 8192, 32768
 * cells per tile) and, for each precision present, the normal, first
 * tangential (FP64) and flux (FP64) sweeps (candidates 256, 1024, 4096,
 * 16384 positions), one group after the other, each candidate timed once
 * after a warm-up run.  A timing run enqueues the ghost fill, the CFL
 * reduction, the state split and the sweeps of direction x: they write only
 * ghost cells (with the values they hold), the CFL minimum and scratch
 * buffers, so the problems stay where they were and nothing is allocated
 * but the tile lists.  best_ms (may be NULL) receives the summed time of the
 * tuned groups in one such run.  The chosen sizes are reported by
 * hgks_batch_info. */
hgks_status hgks_batch_tune(hgks_batch_t b, double cfl, double *best_ms);
/* steps[i] receives the step counter of problem i as read back at the end
 * of the last hgks_batch_step call (no device work); a problem that stopped
 * on a bad state shows fewer steps than the others.  steps: n entries, owned
 * by the caller.  Errors: INVALID_ARG (NULL), STATE (no step call yet). */
hgks_status hgks_batch_steps(hgks_batch_t b, long long *steps);
/* Fills *out.  Errors: INVALID_ARG (NULL). */
hgks_status hgks_batch_info(hgks_batch_t b, hgks_batch_info_t *out);
/* Message of the last error of this batch; owned by the batch. */
const char *hgks_batch_last_error(hgks_batch_t b);
/* Waits for the batch's work and frees it; the handles are untouched. */
void hgks_batch_destroy(hgks_batch_t b);

/* Device bytes a handle for this grid and precision allocates (admission). */
size_t hgks_footprint_bytes(const hgks_grid *grid, hgks_precision precision);

/* Message of the last error on this handle, or for h == NULL the last error
 * of a call without a handle made on the calling thread.  Valid until the
 * next call on the handle (or on the thread). */
const char *hgks_last_error(hgks_t h);

/* Wait for all work of the handle's stream. */
hgks_status hgks_synchronize(hgks_t h);

/* Release the handle and its device memory.  NULL is ignored. */
void hgks_destroy(hgks_t h);

#ifdef __cplusplus
}
#endif
#endif /* HGKS_H */
