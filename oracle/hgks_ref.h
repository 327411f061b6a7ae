/*
 * hgks_ref.h -- the ORACLE: a plain, serial (optionally OpenMP over faces),
 * FP64 CPU implementation of the high-order gas-kinetic scheme (HGKS) of
 * "Multiple-GPU accelerated high-order gas-kinetic scheme for direct
 * numerical simulation of compressible turbulence" (arXiv 2207.01173).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * (the CUDA library) shares no code, header, table or constant generator
 * with it.
 *
 * The API mirrors the product's C-ABI with an hgks_ref_ prefix so that tests
 * can diff the two, plus unit-level entry points used by the pins.
 *
 * All velocities in the "rotated frame" entry points are ordered
 * (normal, tangential-1, tangential-2).
 */
#ifndef HGKS_REF_H
#define HGKS_REF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hgks_ref_s *hgks_ref_t;

enum { HGKS_REF_OK = 0, HGKS_REF_ERR_INVALID_ARG = 1, HGKS_REF_ERR_OOM = 2,
       HGKS_REF_ERR_NONFINITE = 4, HGKS_REF_ERR_STATE = 6 };
/* EXTERNAL: the ghost layers of that side are left to the caller (filled by
   the halo hook below); used to emulate a slab decomposition with CPU ranks */
enum { HGKS_REF_BC_PERIODIC = 0, HGKS_REF_BC_ISOTHERMAL_WALL = 1, HGKS_REF_BC_EXTERNAL = 2 };
enum { HGKS_REF_VISC_CONSTANT = 0, HGKS_REF_VISC_POWER = 1 };

typedef struct { int nx, ny, nz; double lx, ly, lz; double x0, y0, z0;
                 double y_stretch_b; } hgks_ref_grid;
typedef struct { int kind; double mu_ref, T_ref, omega; } hgks_ref_visc;
typedef struct { int lo[3], hi[3]; double T_wall; } hgks_ref_bcs;
typedef struct { double t; int64_t step; double dt, Ek, enstrophy, eps_com,
                 mass, mom[3], energy, max_mach, wall_shear; } hgks_ref_stats_t;

/* ---- solver (same shape as the product ABI) ---- */
int  hgks_ref_create(const hgks_ref_grid *grid, double gamma, double Pr,
                     const hgks_ref_visc *visc, const hgks_ref_bcs *bcs,
                     const double body_force[3], hgks_ref_t *out);
int  hgks_ref_init_tgv(hgks_ref_t h, double Ma, double U0, double rho0);
int  hgks_ref_init_channel(hgks_ref_t h, double Ma_b, double noise_amp, uint64_t seed);
int  hgks_ref_init_density_wave(hgks_ref_t h, double amp);
int  hgks_ref_set_state(hgks_ref_t h, const double *host_q);   /* [5][nz][ny][nx] */
int  hgks_ref_get_state(hgks_ref_t h, double *host_q);
int  hgks_ref_set_time(hgks_ref_t h, double t, int64_t step);
int  hgks_ref_step(hgks_ref_t h, int nsteps, double cfl);
int  hgks_ref_step_dt(hgks_ref_t h, int nsteps, double dt);
int  hgks_ref_compute_dt(hgks_ref_t h, double cfl, double *dt);
int  hgks_ref_rhs(hgks_ref_t h, double dt, double *L, double *dL); /* L(Q), dL/dt(Q) of current state */
/* L, dL/dt at sampled interior cells (index (k ny + j) nx + i); outputs [ncells][5] */
int  hgks_ref_rhs_cells(hgks_ref_t h, double dt, int ncells, const int64_t *cells, double *L, double *dL);
/* F^n and dF^n/dt (times the face area, global component order) of the
   interface of direction d between cells f-1 and f along d, at tangential
   cell indices (a, b) (Eq. "flux" summed over the 2x2 Gauss points) */
int  hgks_ref_face_flux(hgks_ref_t h, double dt, int d, int f, int a, int b, double F[5], double dF[5]);
int  hgks_ref_stats(hgks_ref_t h, hgks_ref_stats_t *out);
/* Hooks for slab ranks.  halo(user, q) runs after every ghost fill of a
   padded state q ([5][nz+6][ny+6][nx+6]; the physical boundary ghosts are
   already set, EXTERNAL ones are the hook's to write).  dtmin(user, m)
   turns this rank's CFL minimum m into the global one.  NULL: no hook. */
typedef void (*hgks_ref_halo_fn)(void *user, double *q);
typedef double (*hgks_ref_min_fn)(void *user, double local_min);
int  hgks_ref_set_hooks(hgks_ref_t h, hgks_ref_halo_fn halo, hgks_ref_min_fn dtmin, void *user);
const char *hgks_ref_last_error(hgks_ref_t h);
void hgks_ref_destroy(hgks_ref_t h);

/* ---- unit-level entry points used by the pins ---- */
/* normalised moments <u^n> (n = 0..nmax-1) of a 1-D Maxwellian with mean U,
   lambda lam, over range 0 = full, 1 = u>0, 2 = u<0 */
void hgks_ref_moments_1d(double U, double lam, int range, int nmax, double *out);
/* <xi^(2d)>, d = 0..2, for K internal degrees of freedom */
void hgks_ref_moments_xi(double lam, double K, double out[3]);
/* conservative (rho, rho U, rho V, rho W, rho E) -> (rho, U, V, W, lambda) */
void hgks_ref_prim(const double Q[5], double K, double W[5]);
/* solve <a psi> = dQ for the micro-slope a of a Maxwellian with primitives W */
void hgks_ref_micro_slope(const double W[5], double K, const double dQ[5], double a[5]);
/* sum_j (moment matrix of W)_ij a_j * rho : the left-hand side of the slope equation */
void hgks_ref_slope_moments(const double W[5], double K, const double a[5], double out[5]);
/* Q0 from the compatibility condition of g_l (u>0) and g_r (u<0) */
void hgks_ref_compat(const double Ql[5], const double Qr[5], double K, double Q0[5]);
/* time-integration coefficients over [0, delta]: q_eq, q_abar, q_Abar, q_f, q_fa */
void hgks_ref_time_coeffs(double tau, double delta, double q[5]);
/* F^n and dF^n/dt from the two time integrals I(dt), I(dt/2) */
void hgks_ref_time_fit(const double Ifull[5], const double Ihalf[5], double dt,
                       double Fn[5], double dFn[5]);
/* GKS flux through a unit-area interface point, rotated frame.  d?[3][5]
   are the physical derivatives (normal, t1, t2) of the conservative
   variables.  Writes the time integrals I(dt), I(dt/2) and F^n, dF^n/dt. */
void hgks_ref_point_flux(const double Ql[5], const double Qr[5],
                         const double dQl[15], const double dQr[15], const double dQ0[15],
                         double gamma, double Pr, const hgks_ref_visc *visc,
                         double dt, double Ifull[5], double Ihalf[5],
                         double Fn[5], double dFn[5]);
/* WENO-Z point value at offset sigma (cell widths from the centre cell) from
   five cell averages X[-2..2] */
double hgks_ref_weno_z(const double X[5], double sigma, double eps);
void   hgks_ref_weno_linear_weights(double sigma, double d[3]);
void   hgks_ref_weno_candidates(const double X[5], double sigma, double p[3], double beta[3]);
/* coefficients of the quartic through five cell averages: value and
   derivative at sigma */
void   hgks_ref_quartic_coeffs(double sigma, double Lc[5], double Dc[5]);
/* published splitmix64 of x, and the uniform [-1,1) number made from it */
uint64_t hgks_ref_splitmix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif
