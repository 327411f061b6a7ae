// hgks_api.cu -- host implementation of the C-ABI declared in include/hgks.h.
//
// One step (arXiv 2207.01173 Alg. 1 with the two stages of Eq. "two-stage"):
//   ghost fill Q^n -> CFL reduction -> dt
//   stage 1: three sweeps (normal / tangential / flux passes) -> F^n, dF^n
//            update: Q* = Q^n + dt/2 L + dt^2/8 dL,  R = Q^n + dt L + dt^2/6 dL
//   ghost fill Q* -> stage 2 sweeps -> Q^{n+1} = R + dt^2/3 dL(Q*)
//   commit (time, step counter, index of the good state buffer)
// All of it is enqueued on the handle's stream; the host reads the control
// block once per hgks_step call to report a bad state.
#include "../../include/hgks.h"
#include "hgks_handle.h"
#include "hgks_kernels.cuh"
#include "hgks_mesh.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace hgks;


static thread_local std::string g_err;

namespace hgks {
// message for hgks_last_error(NULL) from entry points that take no handle
void set_global_error(const char *msg) { g_err = msg; }
}  // namespace hgks

static hgks_status set_err(hgks_t h, hgks_status s, const std::string &msg)
{
    if (h) h->err = msg;
    else g_err = msg;
    return s;
}

static hgks_status cuda_check(hgks_t h, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HGKS_OK;
    return set_err(h, e == cudaErrorMemoryAllocation ? HGKS_ERR_OOM : HGKS_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(h, call)                                          \
    do {                                                     \
        hgks_status s_ = cuda_check((h), (call), #call);     \
        if (s_ != HGKS_OK) return s_;                        \
    } while (0)

// ---------------------------------------------------------------------------
// sizes
// ---------------------------------------------------------------------------
struct Sizes {
    size_t pad, cells, fq, t1, F[3], ytab, stats;
};

static Params shape_params(const hgks_grid &g)
{
    Params P;
    memset(&P, 0, sizeof P);
    P.n[0] = g.nx;
    P.n[1] = g.ny;
    P.n[2] = g.nz;
    for (int d = 0; d < 3; d++) P.np[d] = P.n[d] + 2 * NG;
    P.sy = P.np[0];
    P.sz = (long long)P.np[0] * P.np[1];
    P.cs = P.sz * P.np[2];
    P.ncell = (long long)g.nx * g.ny * g.nz;
    return P;
}

static Sizes sizes_of(const Params &P)
{
    Sizes s;
    s.pad = (size_t)P.cs * 5;
    s.cells = (size_t)P.ncell * 5;
    s.fq = 0;
    s.t1 = 0;
    for (int d = 0; d < 3; d++) {
        s.fq = std::max(s.fq, (size_t)box_count(box_fq(P, d)) * FQ_N);
        s.t1 = std::max(s.t1, (size_t)box_count(box_t1(P, d)) * T1_N);
        s.F[d] = (size_t)box_count(box_face(P, d)) * F_N;
    }
    s.ytab = (size_t)(P.n[1] + 1) * 2 + (size_t)P.n[1] * 5;
    s.stats = (size_t)stats_blocks(P) * 10 + 16;
    return s;
}

extern "C" size_t hgks_footprint_bytes(const hgks_grid *grid, hgks_precision precision)
{
    if (!grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return 0;
    Params P = shape_params(*grid);
    Sizes s = sizes_of(P);
    size_t doubles = 4 * s.pad + s.fq + s.t1 + s.F[0] + s.F[1] + s.F[2] + 2 * s.cells + s.ytab + s.stats;
    if (precision == HGKS_MIXED || precision == HGKS_MIXED_T64) doubles += s.pad;  // the split state
    return doubles * sizeof(double) + sizeof(Ctl);
}

// ---------------------------------------------------------------------------
// lifecycle
// ---------------------------------------------------------------------------
static void free_all(hgks_t h)
{
    double *bufs[] = { h->q[0], h->q[1], h->qs, h->r, h->fq, h->t1, h->qf, h->F[0], h->F[1], h->F[2],
                       h->io[0], h->io[1], h->ytab, h->stat_scratch, h->stat_out };
    for (double *b : bufs)
        if (b) cudaFree(b);
    if (h->ctl) cudaFree(h->ctl);
}

extern "C" void hgks_destroy(hgks_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->st);
    free_all(h);
    delete h;
}

extern "C" hgks_status hgks_create(const hgks_grid *grid, double gamma, double Pr, const hgks_visc *visc,
                                   const hgks_bcs *bcs, const double body_force[3], hgks_precision precision,
                                   void *cuda_stream, hgks_t *out)
{
    if (!grid || !visc || !bcs || !out) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->lx > 0) || !(grid->ly > 0) || !(grid->lz > 0))
        return set_err(nullptr, HGKS_ERR_INVALID_ARG, "grid sizes must be positive");
    if (!(gamma > 1.0) || !(Pr > 0.0)) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "need gamma > 1 and Pr > 0");
    if (precision != HGKS_FP64 && precision != HGKS_MIXED && precision != HGKS_MIXED_T64)
        return set_err(nullptr, HGKS_ERR_INVALID_ARG, "precision must be HGKS_FP64, HGKS_MIXED or HGKS_MIXED_T64");
    const bool mixed = precision != HGKS_FP64;
    if (visc->kind == HGKS_VISC_POWER && !(visc->T_ref > 0.0))
        return set_err(nullptr, HGKS_ERR_INVALID_ARG, "power-law viscosity needs T_ref > 0");
    if (!(visc->mu_ref >= 0.0)) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "mu_ref must be >= 0");
    const int n[3] = { grid->nx, grid->ny, grid->nz };
    for (int d = 0; d < 3; d++) {
        bool wall = bcs->lo[d] == HGKS_BC_ISOTHERMAL_WALL || bcs->hi[d] == HGKS_BC_ISOTHERMAL_WALL;
        bool ext = bcs->lo[d] == HGKS_BC_EXTERNAL || bcs->hi[d] == HGKS_BC_EXTERNAL;
        for (int side = 0; side < 2; side++) {
            const hgks_bc b = side ? bcs->hi[d] : bcs->lo[d];
            if (b != HGKS_BC_PERIODIC && b != HGKS_BC_ISOTHERMAL_WALL && b != HGKS_BC_EXTERNAL)
                return set_err(nullptr, HGKS_ERR_INVALID_ARG, "unknown boundary condition");
        }
        if (ext && d != 2)
            return set_err(nullptr, HGKS_ERR_INVALID_ARG, "EXTERNAL sides are accepted in z only (z slabs)");
        if (wall && n[d] < NG) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "walls need >= 3 cells");
        if (ext && n[d] < NG)
            return set_err(nullptr, HGKS_ERR_INVALID_ARG, "EXTERNAL sides need >= 3 cells in their direction");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return set_err(nullptr, HGKS_ERR_CUDA, "no CUDA device available");
    }

    hgks_t h = new hgks_s();
    h->grid = *grid;
    h->bcs = *bcs;
    h->prec = precision;
    h->st = (cudaStream_t)cuda_stream;
    Params P = shape_params(*grid);
    for (int d = 0; d < 3; d++) {
        P.bc_lo[d] = bcs->lo[d];
        P.bc_hi[d] = bcs->hi[d];
    }
    P.h[0] = grid->lx / grid->nx;
    P.h[1] = grid->ly / grid->ny;
    P.h[2] = grid->lz / grid->nz;
    P.stretched = grid->y_stretch_b > 0.0;
    P.gamma = gamma;
    P.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    P.Pr = Pr;
    P.visc_kind = visc->kind;
    P.mu_ref = visc->mu_ref;
    P.T_ref = visc->T_ref > 0.0 ? visc->T_ref : 1.0;
    P.omega = visc->omega;
    P.T_wall = bcs->T_wall;
    for (int d = 0; d < 3; d++) P.G[d] = body_force ? body_force[d] : 0.0;
    P.has_force = (P.G[0] != 0.0 || P.G[1] != 0.0 || P.G[2] != 0.0);
    P.f_gm1 = (float)(gamma - 1.0);
    P.f_gm1_lo = (float)((gamma - 1.0) - (double)P.f_gm1);
    P.f_K = (float)P.K;
    P.f_prc = (float)(1.0 / Pr - 1.0);
    P.f_mu_ref = (float)P.mu_ref;
    P.f_inv_Tref = (float)(1.0 / P.T_ref);
    P.f_omega = (float)P.omega;
    for (int d = 0; d < 3; d++) P.f_ih[d] = (float)(1.0 / P.h[d]);

    Sizes s = sizes_of(P);
    auto alloc = [&](double **p, size_t n) -> hgks_status {
        return cuda_check(h, cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(double)), "cudaMalloc");
    };
    hgks_status st = HGKS_OK;
    if (!st) st = alloc(&h->q[0], s.pad);
    if (!st) st = alloc(&h->q[1], s.pad);
    if (!st) st = alloc(&h->qs, s.pad);
    if (!st) st = alloc(&h->r, s.pad);
    if (!st) st = alloc(&h->fq, s.fq);
    if (!st) st = alloc(&h->t1, s.t1);
    if (!st && mixed) st = alloc(&h->qf, s.pad);
    if (!st) st = cuda_check(h, fp64_setup(), "flux kernel set-up");
    if (!st && mixed) st = cuda_check(h, mixed_setup(), "mixed-precision kernel set-up");
    for (int d = 0; d < 3 && !st; d++) st = alloc(&h->F[d], s.F[d]);
    if (!st) st = alloc(&h->io[0], s.cells);
    if (!st) st = alloc(&h->io[1], s.cells);
    if (!st) st = alloc(&h->ytab, s.ytab);
    if (!st) st = alloc(&h->stat_scratch, s.stats);
    if (!st) st = alloc(&h->stat_out, 16);
    if (!st) st = cuda_check(h, cudaMalloc((void **)&h->ctl, sizeof(Ctl)), "cudaMalloc");
    if (st) {
        g_err = h->err;
        free_all(h);
        delete h;
        return st;
    }
    std::vector<double> yt = mesh_y_tables(*grid);
    const int ny = grid->ny;
    P.my_face = h->ytab;
    P.my_gp = h->ytab + ny + 1;
    P.my_cen = h->ytab + 3 * ny + 1;
    P.hy_cell = h->ytab + 4 * ny + 1;
    h->P = P;
    Ctl c0;
    memset(&c0, 0, sizeof c0);
    cudaError_t e = cudaMemcpy(h->ytab, yt.data(), yt.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->ctl, &c0, sizeof c0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->q[0], 0, s.pad * sizeof(double));
    if (e != cudaSuccess) {
        cuda_check(h, e, "initial copies");
        g_err = h->err;
        free_all(h);
        delete h;
        return HGKS_ERR_CUDA;
    }
    *out = h;
    return HGKS_OK;
}

extern "C" const char *hgks_last_error(hgks_t h) { return h ? h->err.c_str() : g_err.c_str(); }

extern "C" hgks_status hgks_synchronize(hgks_t h)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    CK(h, cudaStreamSynchronize(h->st));
    return HGKS_OK;
}

static hgks_status read_ctl(hgks_t h, Ctl &c)
{
    CK(h, cudaMemcpyAsync(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return HGKS_OK;
}
static hgks_status write_ctl(hgks_t h, const Ctl &c)
{
    CK(h, cudaMemcpyAsync(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return HGKS_OK;
}

static hgks_status reset_clock(hgks_t h)
{
    h->stage1_done = false;  // a new state: no stage of a step in progress
    Ctl c;
    hgks_status s = read_ctl(h, c);
    if (s) return s;
    c.t = 0.0;
    c.step = 0;
    c.flag = 0;
    c.good = h->cur;
    c.wall_shear = 0.0;
    c.last_dt = 0.0;
    return write_ctl(h, c);
}

// ---------------------------------------------------------------------------
// initial fields and state transfer
// ---------------------------------------------------------------------------
extern "C" hgks_status hgks_init_tgv(hgks_t h, double Ma, double U0, double rho0)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if (!(Ma > 0.0) || !(rho0 > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need Ma > 0 and rho0 > 0");
    const double *yface = h->ytab + 5 * h->grid.ny + 1;
    launch_init_tgv(h->P, h->q[h->cur], yface, h->grid.x0, h->grid.z0, Ma, U0, rho0, h->st);
    CK(h, cudaGetLastError());
    h->rho_ref = rho0;
    return reset_clock(h);
}

extern "C" hgks_status hgks_init_channel(hgks_t h, double Ma_b, double noise_amp, uint64_t seed)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if (!(Ma_b > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need Ma_b > 0");
    const double *ycen = h->ytab + 6 * h->grid.ny + 2;
    launch_init_channel(h->P, h->q[h->cur], ycen, h->grid.y0 + 0.5 * h->grid.ly, 0.5 * h->grid.ly, Ma_b, noise_amp,
                        (unsigned long long)seed, h->st);
    CK(h, cudaGetLastError());
    h->P.T_wall = 1.0 / (h->P.gamma * Ma_b * Ma_b);
    h->bcs.T_wall = h->P.T_wall;
    h->rho_ref = 1.0;
    return reset_clock(h);
}

extern "C" hgks_status hgks_init_density_wave(hgks_t h, double amp)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    launch_init_wave(h->P, h->q[h->cur], h->grid.x0, h->grid.y0, h->grid.z0, h->grid.ly / h->grid.ny, amp, h->st);
    CK(h, cudaGetLastError());
    h->rho_ref = 1.0;
    return reset_clock(h);
}

extern "C" hgks_status hgks_set_state(hgks_t h, const double *host_q)
{
    if (!h || !host_q) return set_err(h, HGKS_ERR_INVALID_ARG, "null argument");
    h->stage1_done = false;
    CK(h, cudaMemcpyAsync(h->io[0], host_q, (size_t)h->P.ncell * 5 * sizeof(double), cudaMemcpyHostToDevice, h->st));
    launch_scatter(h->P, h->io[0], h->q[h->cur], h->st);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->st));
    return HGKS_OK;
}

extern "C" hgks_status hgks_get_state(hgks_t h, double *host_q)
{
    if (!h || !host_q) return set_err(h, HGKS_ERR_INVALID_ARG, "null argument");
    launch_gather(h->P, h->q[h->cur], h->io[0], h->st);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(host_q, h->io[0], (size_t)h->P.ncell * 5 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return HGKS_OK;
}

extern "C" hgks_status hgks_set_time(hgks_t h, double t, int64_t step)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    Ctl c;
    hgks_status s = read_ctl(h, c);
    if (s) return s;
    c.t = t;
    c.step = step;
    return write_ctl(h, c);
}

// ---------------------------------------------------------------------------
// the step
// ---------------------------------------------------------------------------
// optional per-kind timing of the launches of one step
struct StepTimer {
    static constexpr int MAXEV = 64;
    cudaEvent_t ev[MAXEV];
    int kind[MAXEV];
    int n = 0;
    bool on = false;
    cudaStream_t st = nullptr;
    int launches = 0, flux_launches = 0;
};
enum { TK_GHOST, TK_DT, TK_NORMAL, TK_TAN1, TK_FLUX, TK_UPDATE, TK_OTHER, TK_N };

// record the end of a launch of `kind` (and count the launch)
static void mark(StepTimer *T, int kind, int nlaunch = 1)
{
    if (!T) return;
    T->launches += nlaunch;
    if (kind == TK_FLUX) T->flux_launches += nlaunch;
    if (T->on && T->n < StepTimer::MAXEV) {
        cudaEventRecord(T->ev[T->n], T->st);
        T->kind[T->n] = kind;
        T->n++;
    }
}

static void enqueue_sweeps(hgks_t h, const double *q, bool record_wall, StepTimer *T)
{
    const Params &P = h->P;
    const bool mixed = h->prec != HGKS_FP64, t64 = h->prec == HGKS_MIXED_T64;
    if (mixed) {
        launch_split_mixed(P, q, h->qf, h->ctl, h->st);
        mark(T, TK_OTHER);
    }
    for (int d = 0; d < 3; d++) {
        int nl = 1;
        if (mixed) nl = launch_sweep_mixed(P, d, h->qf, h->fq, h->t1, h->F[d], h->ctl, h->st, 0, t64);
        else launch_normal(P, d, q, h->fq, h->ctl, h->st);
        mark(T, TK_NORMAL, nl);
        nl = 1;
        if (mixed) nl = launch_sweep_mixed(P, d, h->qf, h->fq, h->t1, h->F[d], h->ctl, h->st, 1, t64);
        else launch_tan1(P, d, h->fq, h->t1, h->ctl, h->st);
        mark(T, TK_TAN1, nl);
        if (mixed) launch_sweep_mixed(P, d, h->qf, h->fq, h->t1, h->F[d], h->ctl, h->st, 2, t64);
        else launch_flux(P, d, h->t1, h->F[d], h->ctl, h->st);
        mark(T, TK_FLUX);
        if (d == 1 && record_wall && (P.bc_lo[1] == HGKS_BC_ISOTHERMAL_WALL || P.bc_hi[1] == HGKS_BC_ISOTHERMAL_WALL)) {
            launch_wall(P, h->F[1], h->ctl, h->grid.lx * h->grid.lz, h->st);
            mark(T, TK_OTHER);
        }
    }
}

static void enqueue_step(hgks_t h, double cfl, double fixed_dt, StepTimer *T = nullptr)
{
    const Params &P = h->P;
    double *q = h->q[h->cur], *qn = h->q[1 - h->cur];
    const double *Fc[3] = { h->F[0], h->F[1], h->F[2] };
    if (T && T->on) {
        cudaEventRecord(T->ev[0], T->st);
        T->kind[0] = -1;
        T->n = 1;
    }
    launch_ghost(P, q, h->st);
    mark(T, TK_GHOST, 3);
    if (fixed_dt > 0.0) {
        launch_dt_final(h->ctl, 0.0, fixed_dt, h->st);
        mark(T, TK_DT);
    } else {
        launch_dt_reset(h->ctl, h->st);
        launch_cfl(P, q, h->ctl, h->st);
        launch_dt_final(h->ctl, cfl, 0.0, h->st);
        mark(T, TK_DT, 3);
    }
    enqueue_sweeps(h, q, true, T);
    launch_update(P, 1, q, Fc, h->qs, h->r, h->ctl, h->st);
    mark(T, TK_UPDATE);
    launch_ghost(P, h->qs, h->st);
    mark(T, TK_GHOST, 3);
    enqueue_sweeps(h, h->qs, false, T);
    launch_update(P, 2, h->qs, Fc, qn, h->r, h->ctl, h->st);
    mark(T, TK_UPDATE);
    launch_commit(h->ctl, 1 - h->cur, h->st);
    mark(T, TK_OTHER);
    h->cur = 1 - h->cur;
}

static hgks_status run_steps(hgks_t h, int nsteps, double cfl, double fixed_dt)
{
    h->stage1_done = false;  // whole steps overwrite the stage state
    for (int s = 0; s < nsteps; s++) enqueue_step(h, cfl, fixed_dt);
    CK(h, cudaGetLastError());
    Ctl c;
    hgks_status st = read_ctl(h, c);
    if (st) return st;
    if (c.flag) {
        h->cur = c.good;
        c.flag = 0;
        st = write_ctl(h, c);
        if (st) return st;
        return set_err(h, HGKS_ERR_NONFINITE, "a stage produced a non-finite or non-positive state; "
                                              "state left at the last completed step");
    }
    return HGKS_OK;
}

extern "C" hgks_status hgks_step(hgks_t h, int nsteps, double cfl)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if (nsteps < 0 || !(cfl > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need nsteps >= 0 and cfl > 0");
    return run_steps(h, nsteps, cfl, 0.0);
}

extern "C" hgks_status hgks_step_dt(hgks_t h, int nsteps, double dt)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if (nsteps < 0 || !(dt > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need nsteps >= 0 and dt > 0");
    return run_steps(h, nsteps, 0.0, dt);
}

// ---------------------------------------------------------------------------
// sub-domains: the step in phases (fill, halo exchange by the caller, stage)
// ---------------------------------------------------------------------------
static double *state_of(hgks_t h, int state) { return state == HGKS_STATE_CURRENT ? h->q[h->cur] : h->qs; }

extern "C" hgks_status hgks_fill_ghosts(hgks_t h, int state)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if (state != HGKS_STATE_CURRENT && state != HGKS_STATE_STAGE)
        return set_err(h, HGKS_ERR_INVALID_ARG, "state must be HGKS_STATE_CURRENT or HGKS_STATE_STAGE");
    launch_ghost(h->P, state_of(h, state), h->st);
    CK(h, cudaGetLastError());
    return HGKS_OK;
}

extern "C" size_t hgks_halo_count(hgks_t h, int dir)
{
    if (!h || dir != 2) return 0;
    return (size_t)5 * NG * (size_t)h->P.sz;
}

static hgks_status halo_args(hgks_t h, int state, int dir, int side, const void *buf)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if (!buf) return set_err(h, HGKS_ERR_INVALID_ARG, "null halo buffer");
    if (state != HGKS_STATE_CURRENT && state != HGKS_STATE_STAGE)
        return set_err(h, HGKS_ERR_INVALID_ARG, "state must be HGKS_STATE_CURRENT or HGKS_STATE_STAGE");
    if (dir != 2) return set_err(h, HGKS_ERR_INVALID_ARG, "halo exchange is supported in z (dir 2) only");
    if (side != 0 && side != 1) return set_err(h, HGKS_ERR_INVALID_ARG, "side must be 0 (low) or 1 (high)");
    return HGKS_OK;
}

extern "C" hgks_status hgks_halo_get(hgks_t h, int state, int dir, int side, double *d_buf)
{
    hgks_status s = halo_args(h, state, dir, side, d_buf);
    if (s) return s;
    launch_halo_z(h->P, state_of(h, state), side == 0 ? 0 : h->P.n[2] - NG, d_buf, true, h->st);
    CK(h, cudaGetLastError());
    return HGKS_OK;
}

extern "C" hgks_status hgks_halo_set(hgks_t h, int state, int dir, int side, const double *d_buf)
{
    hgks_status s = halo_args(h, state, dir, side, d_buf);
    if (s) return s;
    launch_halo_z(h->P, state_of(h, state), side == 0 ? -NG : h->P.n[2], const_cast<double *>(d_buf), false, h->st);
    CK(h, cudaGetLastError());
    return HGKS_OK;
}

extern "C" hgks_status hgks_stage(hgks_t h, int stage, double dt)
{
    if (!h) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null handle");
    if ((stage != 1 && stage != 2) || !(dt > 0.0))
        return set_err(h, HGKS_ERR_INVALID_ARG, "need stage 1 or 2 and dt > 0");
    const Params &P = h->P;
    const double *Fc[3] = { h->F[0], h->F[1], h->F[2] };
    if (stage == 1) {
        double *q = h->q[h->cur];
        launch_dt_final(h->ctl, 0.0, dt, h->st);
        enqueue_sweeps(h, q, true, nullptr);
        launch_update(P, 1, q, Fc, h->qs, h->r, h->ctl, h->st);
        CK(h, cudaGetLastError());
        h->stage1_done = true;
        return HGKS_OK;
    }
    if (!h->stage1_done) return set_err(h, HGKS_ERR_STATE, "hgks_stage(2) needs stage 1 of the same step first");
    h->stage1_done = false;
    launch_dt_final(h->ctl, 0.0, dt, h->st);
    enqueue_sweeps(h, h->qs, false, nullptr);
    launch_update(P, 2, h->qs, Fc, h->q[1 - h->cur], h->r, h->ctl, h->st);
    launch_commit(h->ctl, 1 - h->cur, h->st);
    h->cur = 1 - h->cur;
    CK(h, cudaGetLastError());
    Ctl c;
    hgks_status st = read_ctl(h, c);
    if (st) return st;
    if (c.flag) {
        h->cur = c.good;
        c.flag = 0;
        st = write_ctl(h, c);
        if (st) return st;
        return set_err(h, HGKS_ERR_NONFINITE, "a stage produced a non-finite or non-positive state; "
                                              "state left at the last completed step");
    }
    return HGKS_OK;
}

extern "C" hgks_status hgks_compute_dt(hgks_t h, double cfl, double *dt)
{
    if (!h || !dt) return set_err(h, HGKS_ERR_INVALID_ARG, "null argument");
    if (!(cfl > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need cfl > 0");
    launch_ghost(h->P, h->q[h->cur], h->st);
    launch_dt_reset(h->ctl, h->st);
    launch_cfl(h->P, h->q[h->cur], h->ctl, h->st);
    launch_dt_final(h->ctl, cfl, 0.0, h->st);
    CK(h, cudaGetLastError());
    Ctl c;
    hgks_status s = read_ctl(h, c);
    if (s) return s;
    *dt = c.dt;
    return HGKS_OK;
}

extern "C" hgks_status hgks_rhs(hgks_t h, double dt, double *host_L, double *host_dL)
{
    if (!h || !host_L || !host_dL) return set_err(h, HGKS_ERR_INVALID_ARG, "null argument");
    if (!(dt > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need dt > 0");
    double *q = h->q[h->cur];
    const double *Fc[3] = { h->F[0], h->F[1], h->F[2] };
    launch_ghost(h->P, q, h->st);
    launch_set_dt(h->ctl, dt, h->st);
    enqueue_sweeps(h, q, false, nullptr);
    launch_rhs_out(h->P, q, Fc, h->io[0], h->io[1], h->ctl, h->st);
    CK(h, cudaGetLastError());
    size_t bytes = (size_t)h->P.ncell * 5 * sizeof(double);
    CK(h, cudaMemcpyAsync(host_L, h->io[0], bytes, cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaMemcpyAsync(host_dL, h->io[1], bytes, cudaMemcpyDeviceToHost, h->st));
    CK(h, cudaStreamSynchronize(h->st));
    return HGKS_OK;
}

extern "C" hgks_status hgks_stats(hgks_t h, hgks_stats_t *out)
{
    if (!h || !out) return set_err(h, HGKS_ERR_INVALID_ARG, "null argument");
    launch_ghost(h->P, h->q[h->cur], h->st);
    launch_stats(h->P, h->q[h->cur], h->stat_scratch, h->stat_out, h->rho_ref, h->st);
    CK(h, cudaGetLastError());
    double v[10];
    CK(h, cudaMemcpyAsync(v, h->stat_out, sizeof v, cudaMemcpyDeviceToHost, h->st));
    Ctl c;
    hgks_status s = read_ctl(h, c);
    if (s) return s;
    out->t = c.t;
    out->step = c.step;
    out->dt = c.last_dt;
    out->Ek = v[0];
    out->enstrophy = v[1];
    out->eps_com = v[2];
    out->mass = v[3];
    out->mom[0] = v[4];
    out->mom[1] = v[5];
    out->mom[2] = v[6];
    out->energy = v[7];
    out->max_mach = v[8];
    out->wall_shear = c.wall_shear;
    return HGKS_OK;
}

extern "C" hgks_status hgks_step_timed(hgks_t h, double cfl, hgks_step_times_t *out)
{
    if (!h || !out) return set_err(h, HGKS_ERR_INVALID_ARG, "null argument");
    if (!(cfl > 0.0)) return set_err(h, HGKS_ERR_INVALID_ARG, "need cfl > 0");
    StepTimer T;
    T.on = true;
    T.st = h->st;
    for (int i = 0; i < StepTimer::MAXEV; i++) CK(h, cudaEventCreate(&T.ev[i]));
    enqueue_step(h, cfl, 0.0, &T);
    hgks_status st = HGKS_OK;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(T.ev[T.n - 1]);
    double ms[TK_N] = { 0 };
    double total = 0.0;
    if (e == cudaSuccess) {
        for (int i = 1; i < T.n && e == cudaSuccess; i++) {
            float f = 0.0f;
            e = cudaEventElapsedTime(&f, T.ev[i - 1], T.ev[i]);
            ms[T.kind[i]] += f;
            total += f;
        }
    }
    for (int i = 0; i < StepTimer::MAXEV; i++) cudaEventDestroy(T.ev[i]);
    if (e != cudaSuccess) return cuda_check(h, e, "step timing");
    Ctl c;
    st = read_ctl(h, c);
    if (st) return st;
    if (c.flag) {
        h->cur = c.good;
        c.flag = 0;
        st = write_ctl(h, c);
        if (st) return st;
        return set_err(h, HGKS_ERR_NONFINITE, "a stage produced a non-finite or non-positive state");
    }
    out->total_ms = total;
    out->ghost_ms = ms[TK_GHOST];
    out->dt_ms = ms[TK_DT];
    out->normal_ms = ms[TK_NORMAL];
    out->tan1_ms = ms[TK_TAN1];
    out->flux_ms = ms[TK_FLUX];
    out->update_ms = ms[TK_UPDATE];
    out->other_ms = ms[TK_OTHER];
    out->launches = T.launches;
    out->flux_launches = T.flux_launches;
    return HGKS_OK;
}

extern "C" hgks_status hgks_fp64_probe(double *tflops)
{
    if (!tflops) return set_err(nullptr, HGKS_ERR_INVALID_ARG, "null argument");
    double v = 0.0;
    cudaError_t e = fp64_probe(&v);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "fp64 probe");
    *tflops = v;
    return HGKS_OK;
}
