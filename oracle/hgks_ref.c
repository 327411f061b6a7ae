/*
 * hgks_ref.c -- ORACLE for the high-order gas-kinetic scheme (HGKS),
 * arXiv 2207.01173 Sec. 2.  TEST INFRASTRUCTURE ONLY (see hgks_ref.h).
 *
 * Plain FP64, written for a reader checking it against the paper:
 *   - every velocity-space integral is evaluated by a small sparse-polynomial
 *     moment engine: the integrand psi * u * (polynomial) is expanded into
 *     monomials u^a v^b w^c xi^(2d) and each monomial is replaced by the
 *     product of the 1-D Maxwellian moments (full range, or u>0 / u<0);
 *   - micro-slopes are found by assembling the 5x5 moment matrix <psi psi^T>
 *     and solving it with Gaussian elimination;
 *   - WENO candidate polynomials, smoothness indicators, linear weights and
 *     the quartic value/derivative weights are obtained by fitting
 *     polynomials to cell averages (small linear solves), never from
 *     hand-expanded closed forms.
 * Loops over interfaces may run under OpenMP; every interface writes only its
 * own output, so results do not depend on the thread count.
 *
 * Readings of passages the paper leaves open are marked R-xxx; they are the
 * same readings the CUDA path follows (stated independently there).
 *
 * Pins: tests/test_oracle_*.py check every part against numerical quadrature,
 * closed forms, limits, symmetries, convergence orders and the time steps of
 * the paper's Table 3, and tests/test_oracle_mutants.py plants plausible
 * slips one at a time, each of which must fail a pin.  Parity unpinned:
 * agreement with the paper's own implementation, whose code and output the
 * paper does not print beyond Table 3; and one detail that no physical pin
 * resolves, the positivity tests of density and internal energy in the
 * bad-state check (guards that a non-finite value pre-empts).
 */
#include "hgks_ref.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 3              /* ghost layers: WENO5 needs 3 (Sec. 2, "fifth-order WENO") */
#define WENO_EPS 1e-6     /* R-W: WENO-Z epsilon */
static const double PI = 3.14159265358979323846;

/* ======================================================================
 * small dense linear algebra
 * ==================================================================== */
/* solve A x = b for n <= 8 by Gaussian elimination with partial pivoting */
static void gauss_solve(int n, const double *A_in, const double *b_in, double *x)
{
    double A[64], b[8];
    memcpy(A, A_in, sizeof(double) * n * n);
    memcpy(b, b_in, sizeof(double) * n);
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (p != c) {
            for (int k = 0; k < n; k++) { double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
}

/* ======================================================================
 * polynomial reconstruction from cell averages (unit cells, centre cell at 0)
 * ==================================================================== */
/* average of x^n over the unit cell centred at integer c */
static double cell_avg_pow(int c, int n)
{
    return (pow(c + 0.5, n + 1) - pow(c - 0.5, n + 1)) / (n + 1);
}

/* weights w_j (j over `m` cells) with P(sigma) = sum_j w_j X_j (deriv = 0) or
   P'(sigma) = sum_j w_j X_j (deriv = 1), where P is the degree m-1 polynomial
   whose cell averages equal X.  P(s) = sum_n c_n s^n with A c = X,
   A[r][n] = avg_r(x^n); hence w = A^{-T} s_vec. */
static void fit_weights(int m, const int *cells, double sigma, int deriv, double *w)
{
    double AT[64], s[8];
    for (int r = 0; r < m; r++)
        for (int n = 0; n < m; n++) AT[n * m + r] = cell_avg_pow(cells[r], n);
    for (int n = 0; n < m; n++) {
        if (deriv == 0) s[n] = pow(sigma, n);
        else s[n] = (n == 0) ? 0.0 : n * pow(sigma, n - 1);
    }
    gauss_solve(m, AT, s, w);
}

/* candidate quadratic coefficient maps: c_n(k) = sum_j cand_c[k][n][j] X_j */
static double cand_c[3][3][3];
static const int cand_cells[3][3] = { { -2, -1, 0 }, { -1, 0, 1 }, { 0, 1, 2 } };

typedef struct {
    double sigma;
    double cand[3][5];   /* p_k(sigma) = sum_j cand[k][j] X[j], j = 0..4 <-> cells -2..2 */
    double lin[3];       /* linear weights: sum_k lin_k p_k(sigma) = quartic(sigma) */
    double qv[5], qd[5]; /* quartic value and derivative weights at sigma */
} weno_point;

enum { WP_RIGHT = 0, WP_LEFT = 1, WP_GM = 2, WP_GP = 3, WP_COUNT = 4 };
static weno_point wp[WP_COUNT];
static int tables_ready = 0;

static void build_weno_point(weno_point *P, double sigma)
{
    static const int five[5] = { -2, -1, 0, 1, 2 };
    P->sigma = sigma;
    fit_weights(5, five, sigma, 0, P->qv);
    fit_weights(5, five, sigma, 1, P->qd);
    for (int k = 0; k < 3; k++) {
        double w[3];
        fit_weights(3, cand_cells[k], sigma, 0, w);
        for (int j = 0; j < 5; j++) P->cand[k][j] = 0.0;
        for (int r = 0; r < 3; r++) P->cand[k][cand_cells[k][r] + 2] = w[r];
    }
    /* linear weights: least-squares solution of sum_k d_k cand[k][j] = qv[j]
       (consistent for every sigma in the centre cell) */
    double N[9], rhs[3];
    for (int a = 0; a < 3; a++) {
        rhs[a] = 0.0;
        for (int j = 0; j < 5; j++) rhs[a] += P->cand[a][j] * P->qv[j];
        for (int b = 0; b < 3; b++) {
            double s = 0.0;
            for (int j = 0; j < 5; j++) s += P->cand[a][j] * P->cand[b][j];
            N[a * 3 + b] = s;
        }
    }
    gauss_solve(3, N, rhs, P->lin);
}

static void build_tables(void)
{
    if (tables_ready) return;
    for (int k = 0; k < 3; k++) {
        /* A c = X with A[r][n] = avg_r(x^n); store A^{-1} column by column */
        double A[9];
        for (int r = 0; r < 3; r++)
            for (int n = 0; n < 3; n++) A[r * 3 + n] = cell_avg_pow(cand_cells[k][r], n);
        for (int j = 0; j < 3; j++) {
            double e[3] = { 0, 0, 0 }, c[3];
            e[j] = 1.0;
            gauss_solve(3, A, e, c);
            for (int n = 0; n < 3; n++) cand_c[k][n][j] = c[n];
        }
    }
    const double g = sqrt(3.0) / 6.0; /* 2-point Gauss-Legendre abscissae on [-1/2, 1/2] */
    build_weno_point(&wp[WP_RIGHT], 0.5);
    build_weno_point(&wp[WP_LEFT], -0.5);
    build_weno_point(&wp[WP_GM], -g);
    build_weno_point(&wp[WP_GP], g);
    tables_ready = 1;
}

/* integral over [-1/2, 1/2] of a polynomial with coefficients c[0..n-1] */
static double poly_int_cell(const double *c, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; k++)
        if (k % 2 == 0) s += c[k] * 2.0 * pow(0.5, k + 1) / (k + 1);
    return s;
}

/* Jiang-Shu smoothness indicator: sum over l = 1, 2 of the integral over the
   centre cell of (d^l p / dx^l)^2 (unit cell width) */
static double smoothness(const double c[3])
{
    double d1[2] = { c[1], 2.0 * c[2] };           /* p'  */
    double sq1[3] = { d1[0] * d1[0], 2.0 * d1[0] * d1[1], d1[1] * d1[1] };
    double d2 = 2.0 * c[2];                        /* p'' */
    double sq2[1] = { d2 * d2 };
    return poly_int_cell(sq1, 3) + poly_int_cell(sq2, 1);
}

static void weno_parts(const double X[5], const weno_point *P, double p[3], double beta[3])
{
    for (int k = 0; k < 3; k++) {
        double c[3];
        for (int n = 0; n < 3; n++) {
            double s = 0.0;
            for (int r = 0; r < 3; r++) s += cand_c[k][n][r] * X[cand_cells[k][r] + 2];
            c[n] = s;
        }
        beta[k] = smoothness(c);
        double v = 0.0;
        for (int j = 0; j < 5; j++) v += P->cand[k][j] * X[j];
        p[k] = v;
    }
}

/* WENO-Z (Borges et al. 2008, p = 1) value at the point of P, R-W */
static double weno_z_eps(const double X[5], const weno_point *P, double eps)
{
    double p[3], beta[3], alpha[3];
    weno_parts(X, P, p, beta);
    double tau5 = fabs(beta[0] - beta[2]);
    double sa = 0.0;
    for (int k = 0; k < 3; k++) {
        alpha[k] = P->lin[k] * (1.0 + tau5 / (beta[k] + eps));
        sa += alpha[k];
    }
    double v = 0.0;
    for (int k = 0; k < 3; k++) v += (alpha[k] / sa) * p[k];
    return v;
}

static double weno_z_at(const double X[5], const weno_point *P) { return weno_z_eps(X, P, WENO_EPS); }

static double dot5(const double *w, const double *X)
{
    double s = 0.0;
    for (int j = 0; j < 5; j++) s += w[j] * X[j];
    return s;
}

/* ======================================================================
 * Maxwellian moments (Sec. 2: psi, internal degrees of freedom K)
 * ==================================================================== */
typedef struct {
    double rho, lam;
    double mu[3][8];       /* full-range <u_d^n>, d = normal, t1, t2 */
    double mpos[8], mneg[8];
    double mxi[3];         /* <xi^0>, <xi^2>, <xi^4> */
} maxw;

enum { R_FULL = 0, R_POS = 1, R_NEG = 2 };

static void moments_1d(double U, double lam, int range, int nmax, double *m)
{
    if (range == R_FULL) {
        m[0] = 1.0;
        m[1] = U;
    } else {
        double s = sqrt(lam);
        double e = exp(-lam * U * U) / (2.0 * sqrt(PI * lam));
        if (range == R_POS) { m[0] = 0.5 * erfc(-s * U); m[1] = U * m[0] + e; }
        else                { m[0] = 0.5 * erfc(s * U);  m[1] = U * m[0] - e; }
    }
    /* integration by parts: <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lam) <u^n> */
    for (int n = 0; n + 2 < nmax; n++) m[n + 2] = U * m[n + 1] + (n + 1) / (2.0 * lam) * m[n];
}

static void moments_xi(double lam, double K, double m[3])
{
    m[0] = 1.0;
    m[1] = K / (2.0 * lam);
    m[2] = K * (K + 2.0) / (4.0 * lam * lam);
}

static void maxw_build(maxw *g, const double W[5], double K)
{
    g->rho = W[0];
    g->lam = W[4];
    moments_1d(W[1], W[4], R_FULL, 8, g->mu[0]);
    moments_1d(W[2], W[4], R_FULL, 8, g->mu[1]);
    moments_1d(W[3], W[4], R_FULL, 8, g->mu[2]);
    moments_1d(W[1], W[4], R_POS, 8, g->mpos);
    moments_1d(W[1], W[4], R_NEG, 8, g->mneg);
    moments_xi(W[4], K, g->mxi);
}

/* ---- sparse polynomials in (u, v, w, xi^2) ---- */
#define PMAX 32
typedef struct { double c; int e[4]; } mono;
typedef struct { int n; mono m[PMAX]; } poly;

static void p_clear(poly *p) { p->n = 0; }
static void p_add(poly *p, double c, int eu, int ev, int ew, int ex)
{
    if (p->n >= PMAX) { fprintf(stderr, "hgks_ref: polynomial overflow\n"); abort(); }
    mono *m = &p->m[p->n++];
    m->c = c; m->e[0] = eu; m->e[1] = ev; m->e[2] = ew; m->e[3] = ex;
}
/* psi_i * u^extra_u (psi = (1, u, v, w, (u^2+v^2+w^2+xi^2)/2)) */
static void p_psi(poly *p, int i, int extra_u)
{
    p_clear(p);
    switch (i) {
    case 0: p_add(p, 1.0, extra_u, 0, 0, 0); break;
    case 1: p_add(p, 1.0, 1 + extra_u, 0, 0, 0); break;
    case 2: p_add(p, 1.0, extra_u, 1, 0, 0); break;
    case 3: p_add(p, 1.0, extra_u, 0, 1, 0); break;
    default:
        p_add(p, 0.5, 2 + extra_u, 0, 0, 0);
        p_add(p, 0.5, extra_u, 2, 0, 0);
        p_add(p, 0.5, extra_u, 0, 2, 0);
        p_add(p, 0.5, extra_u, 0, 0, 1);
    }
}
/* append s * a(u) * u_d^1 (d = -1: no velocity factor), a(u) = a0 + a1 u + a2 v + a3 w + a4 psi_4 */
static void p_add_slope(poly *p, const double a[5], int d, double s)
{
    int e[4] = { 0, 0, 0, 0 };
    if (d >= 0) e[d] = 1;
    p_add(p, s * a[0], e[0], e[1], e[2], e[3]);
    p_add(p, s * a[1], e[0] + 1, e[1], e[2], e[3]);
    p_add(p, s * a[2], e[0], e[1] + 1, e[2], e[3]);
    p_add(p, s * a[3], e[0], e[1], e[2] + 1, e[3]);
    p_add(p, s * 0.5 * a[4], e[0] + 2, e[1], e[2], e[3]);
    p_add(p, s * 0.5 * a[4], e[0], e[1] + 2, e[2], e[3]);
    p_add(p, s * 0.5 * a[4], e[0], e[1], e[2] + 2, e[3]);
    p_add(p, s * 0.5 * a[4], e[0], e[1], e[2], e[3] + 1);
}
/* heat-flux weight (u - U0) * (|u - U0|^2 + xi^2) / 2 expanded in monomials */
static void p_heat(poly *p, double U0, double V0, double W0)
{
    p_clear(p);
    /* (u-U0)^3 / 2 */
    p_add(p, 0.5, 3, 0, 0, 0);
    p_add(p, -1.5 * U0, 2, 0, 0, 0);
    p_add(p, 1.5 * U0 * U0, 1, 0, 0, 0);
    p_add(p, -0.5 * U0 * U0 * U0, 0, 0, 0, 0);
    /* (u-U0)(v-V0)^2 / 2 and (u-U0)(w-W0)^2 / 2 */
    for (int t = 1; t <= 2; t++) {
        double C = (t == 1) ? V0 : W0;
        int e2[3] = { 2, 1, 0 };
        double cc[3] = { 0.5, -C, 0.5 * C * C };
        for (int q = 0; q < 3; q++) {
            int ev = (t == 1) ? e2[q] : 0, ew = (t == 2) ? e2[q] : 0;
            p_add(p, cc[q], 1, ev, ew, 0);
            p_add(p, -U0 * cc[q], 0, ev, ew, 0);
        }
    }
    /* (u-U0) xi^2 / 2 */
    p_add(p, 0.5, 1, 0, 0, 1);
    p_add(p, -0.5 * U0, 0, 0, 0, 1);
}

static double mono_moment(const maxw *g, int range, const int e[4])
{
    const double *mu = (range == R_FULL) ? g->mu[0] : (range == R_POS ? g->mpos : g->mneg);
    return mu[e[0]] * g->mu[1][e[1]] * g->mu[2][e[2]] * g->mxi[e[3]];
}

/* integral of A(u) * B(u) * g over the velocity range */
static double moment2(const poly *A, const poly *B, const maxw *g, int range)
{
    double s = 0.0;
    for (int i = 0; i < A->n; i++)
        for (int j = 0; j < B->n; j++) {
            int e[4];
            for (int q = 0; q < 4; q++) e[q] = A->m[i].e[q] + B->m[j].e[q];
            if (e[0] > 7 || e[1] > 7 || e[2] > 7 || e[3] > 2) {
                fprintf(stderr, "hgks_ref: moment degree overflow\n");
                abort();
            }
            s += A->m[i].c * B->m[j].c * mono_moment(g, range, e);
        }
    return g->rho * s;
}

static const poly *one_poly(void)
{
    static poly one = { 1, { { 1.0, { 0, 0, 0, 0 } } } };
    return &one;
}

/* ======================================================================
 * conservative <-> primitive, micro-slopes, compatibility (Sec. 2)
 * ==================================================================== */
void hgks_ref_prim(const double Q[5], double K, double W[5])
{
    double rho = Q[0];
    double U = Q[1] / rho, V = Q[2] / rho, Wv = Q[3] / rho;
    double eint = Q[4] - 0.5 * rho * (U * U + V * V + Wv * Wv);
    W[0] = rho; W[1] = U; W[2] = V; W[3] = Wv;
    W[4] = (K + 3.0) * rho / (4.0 * eint); /* rho E = rho|U|^2/2 + (K+3) rho / (4 lambda) */
}

/* moment matrix M_ij = <psi_i psi_j> / rho (full range) */
static void moment_matrix(const maxw *g, double M[25])
{
    poly pi, pj;
    for (int i = 0; i < 5; i++) {
        p_psi(&pi, i, 0);
        for (int j = 0; j < 5; j++) {
            p_psi(&pj, j, 0);
            M[i * 5 + j] = moment2(&pi, &pj, g, R_FULL) / g->rho;
        }
    }
}

/* <a psi> = dQ  (moments taken with g, so  M a = dQ / rho) */
static void slope_solve(const maxw *g, const double dQ[5], double a[5])
{
    double M[25], b[5];
    moment_matrix(g, M);
    for (int i = 0; i < 5; i++) b[i] = dQ[i] / g->rho;
    gauss_solve(5, M, b, a);
}

/* <a_n u + a_t1 v + a_t2 w + A> = 0  ->  M A = -<psi (a.u)> / rho */
static void time_slope_solve(const maxw *g, const double a[3][5], double A[5])
{
    double M[25], b[5];
    poly pau, pp;
    p_clear(&pau);
    for (int d = 0; d < 3; d++) p_add_slope(&pau, a[d], d, 1.0);
    moment_matrix(g, M);
    for (int i = 0; i < 5; i++) {
        p_psi(&pp, i, 0);
        b[i] = -moment2(&pp, &pau, g, R_FULL) / g->rho;
    }
    gauss_solve(5, M, b, A);
}

static void compat_g(const maxw *gl, const maxw *gr, double Q0[5])
{
    poly pp;
    for (int i = 0; i < 5; i++) {
        p_psi(&pp, i, 0);
        Q0[i] = moment2(&pp, one_poly(), gl, R_POS) + moment2(&pp, one_poly(), gr, R_NEG);
    }
}

/* ======================================================================
 * GKS interface flux at one point (Sec. 2, Eq. "flux"; time fit Eq. "expansion-1")
 * ==================================================================== */
static double viscosity(const hgks_ref_visc *v, double T)
{
    if (v->kind == HGKS_REF_VISC_POWER) return v->mu_ref * pow(T / v->T_ref, v->omega);
    return v->mu_ref;
}

void hgks_ref_time_coeffs(double tau, double d, double q[5])
{
    double e = (tau > 0.0) ? exp(-d / tau) : 0.0;
    q[0] = d - tau * (1.0 - e);                                 /* int (1 - e^{-t/tau})           */
    q[1] = 2.0 * tau * tau * (1.0 - e) - tau * d - tau * d * e; /* int ((t+tau)e^{-t/tau} - tau)  */
    q[2] = 0.5 * d * d - tau * d + tau * tau * (1.0 - e);       /* int (t - tau + tau e^{-t/tau}) */
    q[3] = tau * (1.0 - e);                                     /* int e^{-t/tau}                 */
    q[4] = 2.0 * tau * tau * (1.0 - e) - tau * d * e;           /* int (tau + t) e^{-t/tau}       */
}

void hgks_ref_time_fit(const double If[5], const double Ih[5], double dt, double Fn[5], double dFn[5])
{
    /* F dt + F' dt^2/2 = If ; F dt/2 + F' dt^2/8 = Ih */
    for (int i = 0; i < 5; i++) {
        Fn[i] = (4.0 * Ih[i] - If[i]) / dt;
        dFn[i] = 4.0 * (If[i] - 2.0 * Ih[i]) / (dt * dt);
    }
}

typedef struct { double gamma, Pr, K; hgks_ref_visc visc; } gas_params;

/* integrals over [0, dt] and [0, dt/2] of the flux of psi (components 0..4)
   through a unit-area interface point, rotated frame, including the Prandtl
   correction (R-PR) */
static void point_flux(const gas_params *gp, const double Ql[5], const double Qr[5],
                       const double dQl[3][5], const double dQr[3][5], const double dQ0[3][5],
                       double dt, double Ifull[5], double Ihalf[5])
{
    const double K = gp->K;
    double Wl[5], Wr[5], W0[5], Q0[5];
    maxw gl, gr, g0;
    hgks_ref_prim(Ql, K, Wl);
    hgks_ref_prim(Qr, K, Wr);
    maxw_build(&gl, Wl, K);
    maxw_build(&gr, Wr, K);
    /* equilibrium g0 from the compatibility condition: Q0 = int_{u>0} psi g_l + int_{u<0} psi g_r */
    compat_g(&gl, &gr, Q0);
    hgks_ref_prim(Q0, K, W0);
    maxw_build(&g0, W0, K);
    /* collision time tau = mu / p with p from Q0 (smooth flows) */
    double T0 = 1.0 / (2.0 * W0[4]);
    double p0 = W0[0] * T0;
    double tau = viscosity(&gp->visc, T0) / p0;

    /* spatial micro-slopes: <a^k_d> = dQ_k / dx_d  */
    double al[3][5], ar[3][5], a0[3][5], Al[5], Ar[5], A0[5];
    for (int d = 0; d < 3; d++) {
        slope_solve(&gl, dQl[d], al[d]);
        slope_solve(&gr, dQr[d], ar[d]);
        slope_solve(&g0, dQ0[d], a0[d]);
    }
    /* time slopes from <a.u + A> = 0 */
    time_slope_solve(&gl, al, Al);
    time_slope_solve(&gr, ar, Ar);
    time_slope_solve(&g0, a0, A0);

    poly au_l, au_r, au_0, pA_l, pA_r, pA_0;
    p_clear(&au_l); p_clear(&au_r); p_clear(&au_0);
    for (int d = 0; d < 3; d++) {
        p_add_slope(&au_l, al[d], d, 1.0);
        p_add_slope(&au_r, ar[d], d, 1.0);
        p_add_slope(&au_0, a0[d], d, 1.0);
    }
    p_clear(&pA_l); p_add_slope(&pA_l, Al, -1, 1.0);
    p_clear(&pA_r); p_add_slope(&pA_r, Ar, -1, 1.0);
    p_clear(&pA_0); p_add_slope(&pA_0, A0, -1, 1.0);

    /* basis integrals B[term][component], component 5 = heat flux about U0 */
    double B[6][6];
    poly wgt;
    for (int i = 0; i < 6; i++) {
        if (i < 5) p_psi(&wgt, i, 1); /* u psi_i */
        else p_heat(&wgt, W0[1], W0[2], W0[3]);
        B[0][i] = moment2(&wgt, one_poly(), &g0, R_FULL);
        B[1][i] = moment2(&wgt, &au_0, &g0, R_FULL);
        B[2][i] = moment2(&wgt, &pA_0, &g0, R_FULL);
        B[3][i] = moment2(&wgt, one_poly(), &gl, R_POS) + moment2(&wgt, one_poly(), &gr, R_NEG);
        B[4][i] = moment2(&wgt, &au_l, &gl, R_POS) + moment2(&wgt, &au_r, &gr, R_NEG);
        B[5][i] = moment2(&wgt, &pA_l, &gl, R_POS) + moment2(&wgt, &pA_r, &gr, R_NEG);
    }

    for (int pass = 0; pass < 2; pass++) {
        double delta = (pass == 0) ? dt : 0.5 * dt;
        double q[5];
        hgks_ref_time_coeffs(tau, delta, q);
        double I[6];
        for (int i = 0; i < 6; i++)
            I[i] = q[0] * B[0][i] + q[1] * B[1][i] + q[2] * B[2][i] + q[3] * B[3][i]
                 - q[4] * B[4][i] - tau * q[3] * B[5][i];
        /* R-PR: energy flux corrected by (1/Pr - 1) times the heat flux */
        I[4] += (1.0 / gp->Pr - 1.0) * I[5];
        double *out = (pass == 0) ? Ifull : Ihalf;
        for (int i = 0; i < 5; i++) out[i] = I[i];
    }
}

/* ======================================================================
 * solver state
 * ==================================================================== */
struct hgks_ref_s {
    hgks_ref_grid g;
    gas_params gas;
    hgks_ref_bcs bcs;
    double G[3];
    double rho_ref;
    int np[3];           /* padded sizes */
    size_t ncell_pad, ncell;
    double *q, *qs, *qn; /* padded [5][nzp][nyp][nxp] */
    double *L1, *dL1, *L2, *dL2;  /* interior [5][nz][ny][nx] */
    double *F[3], *dF[3];         /* face fluxes [5][faces] per direction */
    double *yface;       /* ny+1 face coordinates of the (possibly stretched) y mesh */
    double t, dt_last, wall_shear;
    int64_t step;
    hgks_ref_halo_fn halo_hook;
    hgks_ref_min_fn min_hook;
    void *hook_user;
    char err[256];
};

static int n_of(const hgks_ref_t h, int d) { return d == 0 ? h->g.nx : (d == 1 ? h->g.ny : h->g.nz); }

static size_t pidx(const hgks_ref_t h, int i, int j, int k)
{
    return ((size_t)(k + NG) * h->np[1] + (size_t)(j + NG)) * h->np[0] + (size_t)(i + NG);
}
static size_t iidx(const hgks_ref_t h, int i, int j, int k)
{
    return ((size_t)k * h->g.ny + j) * h->g.nx + i;
}

/* ---- mesh (Sec. 4.2 coordinate transformation; R-MESH) ---- */
static int stretched(const hgks_ref_t h) { return h->g.y_stretch_b > 0.0; }

static double y_of_s(const hgks_ref_t h, double s) /* s = 2 j / ny in [0, 2] */
{
    if (!stretched(h)) return h->g.y0 + 0.5 * s * h->g.ly;
    double b = h->g.y_stretch_b;
    return h->g.y0 + 0.5 * h->g.ly * (1.0 + tanh(b * (s - 1.0)) / tanh(b));
}
/* dy / dj (one cell of index space) at fractional index position jj (cells start at integer) */
static double dy_dj(const hgks_ref_t h, double jj)
{
    double ds = 2.0 / h->g.ny;
    if (!stretched(h)) return h->g.ly / h->g.ny;
    double b = h->g.y_stretch_b, s = jj * ds;
    double th = tanh(b * (s - 1.0));
    return 0.5 * h->g.ly * b * (1.0 - th * th) / tanh(b) * ds;
}
static double dx_(const hgks_ref_t h) { return h->g.lx / h->g.nx; }
static double dz_(const hgks_ref_t h) { return h->g.lz / h->g.nz; }
static double dy_cell(const hgks_ref_t h, int j)
{
    if (!stretched(h)) return h->g.ly / h->g.ny;
    return h->yface[j + 1] - h->yface[j];
}

/* metric (physical length per index step) of direction d at fractional index position */
static double metric(const hgks_ref_t h, int d, double pos)
{
    if (d == 0) return dx_(h);
    if (d == 2) return dz_(h);
    return dy_dj(h, pos);
}

/* ---- boundary / ghost fill (Alg. 2 boundary step; R-BC) ---- */
static void wall_ghost(const hgks_ref_t h, const double *src, double *dst)
{
    const double K = h->gas.K;
    double W[5];
    hgks_ref_prim(src, K, W);
    double p = W[0] / (2.0 * W[4]);
    double T = p / W[0];
    double Tw = h->bcs.T_wall;
    double Tg = 2.0 * Tw - T;
    if (Tg < 0.5 * Tw) Tg = 0.5 * Tw;
    double rho = p / Tg;
    double U = -W[1], V = -W[2], Wv = -W[3];
    dst[0] = rho;
    dst[1] = rho * U;
    dst[2] = rho * V;
    dst[3] = rho * Wv;
    dst[4] = p / (h->gas.gamma - 1.0) + 0.5 * rho * (U * U + V * V + Wv * Wv);
}

static void ghost_fill(const hgks_ref_t h, double *q)
{
    const size_t S = h->ncell_pad;
    for (int d = 0; d < 3; d++) {
        int n = n_of(h, d);
        /* ranges of the other two indices: interior for directions not yet
           filled, padded for directions already filled */
        int lo[3], hi[3];
        for (int e = 0; e < 3; e++) {
            if (e < d) { lo[e] = -NG; hi[e] = n_of(h, e) + NG; }
            else { lo[e] = 0; hi[e] = n_of(h, e); }
        }
        lo[d] = 0; hi[d] = 1; /* placeholder, ghost loop below */
        for (int c2 = lo[(d + 2) % 3]; c2 < hi[(d + 2) % 3]; c2++)
            for (int c1 = lo[(d + 1) % 3]; c1 < hi[(d + 1) % 3]; c1++)
                for (int side = 0; side < 2; side++)
                    for (int m = 0; m < NG; m++) {
                        int g = side == 0 ? -1 - m : n + m;
                        int bc = side == 0 ? h->bcs.lo[d] : h->bcs.hi[d];
                        if (bc == HGKS_REF_BC_EXTERNAL) continue;
                        int s;
                        if (bc == HGKS_REF_BC_PERIODIC) s = ((g % n) + n) % n;
                        else s = side == 0 ? m : n - 1 - m;
                        int ig[3], is[3];
                        ig[d] = g; is[d] = s;
                        ig[(d + 1) % 3] = is[(d + 1) % 3] = c1;
                        ig[(d + 2) % 3] = is[(d + 2) % 3] = c2;
                        size_t pg = pidx(h, ig[0], ig[1], ig[2]);
                        size_t ps = pidx(h, is[0], is[1], is[2]);
                        if (bc == HGKS_REF_BC_PERIODIC) {
                            for (int c = 0; c < 5; c++) q[c * S + pg] = q[c * S + ps];
                        } else {
                            double src[5], dst[5];
                            for (int c = 0; c < 5; c++) src[c] = q[c * S + ps];
                            wall_ghost(h, src, dst);
                            for (int c = 0; c < 5; c++) q[c * S + pg] = dst[c];
                        }
                    }
    }
    if (h->halo_hook) h->halo_hook(h->hook_user, q);
}

/* ---- time step (Alg. 1 STEP 1; R-DT: convective, per direction) ---- */
static double dt_limit(const hgks_ref_t h, const double *q)
{
    const size_t S = h->ncell_pad;
    double best = INFINITY;
    for (int k = 0; k < h->g.nz; k++)
        for (int j = 0; j < h->g.ny; j++)
            for (int i = 0; i < h->g.nx; i++) {
                size_t p = pidx(h, i, j, k);
                double Q[5], W[5];
                for (int c = 0; c < 5; c++) Q[c] = q[c * S + p];
                hgks_ref_prim(Q, h->gas.K, W);
                double pr = W[0] / (2.0 * W[4]);
                double cs = sqrt(h->gas.gamma * pr / W[0]);
                double hd[3] = { dx_(h), dy_cell(h, j), dz_(h) };
                for (int d = 0; d < 3; d++) {
                    double v = hd[d] / (fabs(W[1 + d]) + cs);
                    if (v < best) best = v;
                }
            }
    return best;
}

/* ---- face fluxes of one direction ---- */
/* rotated component order: rho, normal mom, t1 mom, t2 mom, energy */
static const int perm[3][5] = { { 0, 1, 2, 3, 4 }, { 0, 2, 1, 3, 4 }, { 0, 3, 1, 2, 4 } };
/* tangential directions of each sweep, in reconstruction order */
static const int tdir[3][2] = { { 1, 2 }, { 0, 2 }, { 0, 1 } };

enum { FQ_QL = 0, FQ_QR, FQ_DQL, FQ_DQR, FQ_Q0, FQ_DQ0, FQ_N };

/* cell index triple for (normal position, t1 position, t2 position) */
static void cell_ijk(int d, int cn, int a, int b, int ijk[3])
{
    ijk[d] = cn;
    ijk[tdir[d][0]] = a;
    ijk[tdir[d][1]] = b;
}

/* normal reconstruction for face f (between cells f-1 and f) on the line (a, b):
   Ql, Qr, their normal slopes, Q0 by compatibility and its normal slope, in
   index units (R-W, R-SL, R-EQ) */
static void normal_recon(const hgks_ref_t h, const double *q, int d, int f, int a, int b,
                         double out[FQ_N][5])
{
    const size_t S = h->ncell_pad;
    double X[5][6]; /* X[c][m] for cells f-3..f+2 */
    for (int m = 0; m < 6; m++) {
        int ijk[3];
        cell_ijk(d, f - 3 + m, a, b, ijk);
        size_t p = pidx(h, ijk[0], ijk[1], ijk[2]);
        for (int c = 0; c < 5; c++) X[c][m] = q[perm[d][c] * S + p];
    }
    for (int c = 0; c < 5; c++) {
        /* cell f-1 <-> X index 2; cell f <-> X index 3 */
        const double *sl = &X[c][0], *sr = &X[c][1];
        double lm_r = weno_z_at(sl, &wp[WP_RIGHT]); /* cell f-1, right edge */
        double lm_l = weno_z_at(sl, &wp[WP_LEFT]);  /* cell f-1, left edge  */
        double r_l = weno_z_at(sr, &wp[WP_LEFT]);   /* cell f, left edge    */
        double r_r = weno_z_at(sr, &wp[WP_RIGHT]);  /* cell f, right edge   */
        out[FQ_QL][c] = lm_r;
        out[FQ_QR][c] = r_l;
        /* parabola through (left edge, cell average, right edge) of a cell */
        out[FQ_DQL][c] = 2.0 * lm_l + 4.0 * lm_r - 6.0 * X[c][2];  /* at its right end */
        out[FQ_DQR][c] = -4.0 * r_l - 2.0 * r_r + 6.0 * X[c][3];   /* at its left end  */
        /* cubic through the four averages f-2..f+1, derivative at the face */
        out[FQ_DQ0][c] = (15.0 * (X[c][3] - X[c][2]) - (X[c][4] - X[c][1])) / 12.0;
    }
    double Wl[5], Wr[5];
    maxw gl, gr;
    hgks_ref_prim(out[FQ_QL], h->gas.K, Wl);
    hgks_ref_prim(out[FQ_QR], h->gas.K, Wr);
    maxw_build(&gl, Wl, h->gas.K);
    maxw_build(&gr, Wr, h->gas.K);
    compat_g(&gl, &gr, out[FQ_Q0]);
}

/* flux of one face (f, a, b) of sweep d from the normal-reconstruction records
   of its 5x5 tangential neighbourhood: rec[jj][kk] is the record at tangential
   offsets (jj - 2, kk - 2).  Returns F^n and dF^n/dt times the face area, in
   the global component order. */
static void face_flux_one(const hgks_ref_t h, int d, int f, int a, int b, double dt, const double *rec[5][5],
                          double Fout[5], double dFout[5])
{
    const weno_point *gpt[2] = { &wp[WP_GM], &wp[WP_GP] };
    static const int wq[5] = { FQ_QL, FQ_QR, FQ_DQL, FQ_DQR, FQ_DQ0 }; /* WENO-Z tangentially */
    static const int lq[3] = { FQ_QL, FQ_QR, FQ_Q0 };                  /* linear value/derivative */
    double Fsum[5] = { 0, 0, 0, 0, 0 }, dFsum[5] = { 0, 0, 0, 0, 0 };
    int ijk[3];
    cell_ijk(d, f, a, b, ijk);
    double area;
    if (d == 0) area = dy_cell(h, ijk[1]) * dz_(h);
    else if (d == 1) area = dx_(h) * dz_(h);
    else area = dx_(h) * dy_cell(h, ijk[1]);
    double hn = metric(h, d, (double)f);
    for (int m = 0; m < 2; m++) {
        double T1V[5][5][5], T1L[5][3][5], T1D[5][3][5]; /* [t2 row][quantity][comp] */
        for (int kk = 0; kk < 5; kk++) {
            for (int c = 0; c < 5; c++) {
                double X[5];
                for (int qi = 0; qi < 5; qi++) {
                    for (int jj = 0; jj < 5; jj++) X[jj] = rec[jj][kk][wq[qi] * 5 + c];
                    T1V[kk][qi][c] = weno_z_at(X, gpt[m]);
                }
                for (int qi = 0; qi < 3; qi++) {
                    for (int jj = 0; jj < 5; jj++) X[jj] = rec[jj][kk][lq[qi] * 5 + c];
                    T1L[kk][qi][c] = dot5(gpt[m]->qv, X);
                    T1D[kk][qi][c] = dot5(gpt[m]->qd, X);
                }
            }
        }
        double h1 = metric(h, tdir[d][0], a + 0.5 + gpt[m]->sigma);
        for (int n = 0; n < 2; n++) {
            double h2 = metric(h, tdir[d][1], b + 0.5 + gpt[n]->sigma);
            double V[5][5], Dt1[3][5], Dt2[3][5];
            for (int c = 0; c < 5; c++) {
                double X[5];
                for (int qi = 0; qi < 5; qi++) {
                    for (int kk = 0; kk < 5; kk++) X[kk] = T1V[kk][qi][c];
                    V[qi][c] = weno_z_at(X, gpt[n]);
                }
                for (int qi = 0; qi < 3; qi++) {
                    for (int kk = 0; kk < 5; kk++) X[kk] = T1D[kk][qi][c];
                    Dt1[qi][c] = dot5(gpt[n]->qv, X);
                    for (int kk = 0; kk < 5; kk++) X[kk] = T1L[kk][qi][c];
                    Dt2[qi][c] = dot5(gpt[n]->qd, X);
                }
            }
            double dQl[3][5], dQr[3][5], dQ0[3][5];
            for (int c = 0; c < 5; c++) {
                dQl[0][c] = V[2][c] / hn;
                dQr[0][c] = V[3][c] / hn;
                dQ0[0][c] = V[4][c] / hn;
                dQl[1][c] = Dt1[0][c] / h1;
                dQr[1][c] = Dt1[1][c] / h1;
                dQ0[1][c] = Dt1[2][c] / h1;
                dQl[2][c] = Dt2[0][c] / h2;
                dQr[2][c] = Dt2[1][c] / h2;
                dQ0[2][c] = Dt2[2][c] / h2;
            }
            double If[5], Ih[5], Fn[5], dFn[5];
            point_flux(&h->gas, V[0], V[1], dQl, dQr, dQ0, dt, If, Ih);
            hgks_ref_time_fit(If, Ih, dt, Fn, dFn);
            for (int c = 0; c < 5; c++) {
                Fsum[c] += 0.25 * Fn[c];
                dFsum[c] += 0.25 * dFn[c];
            }
        }
    }
    for (int c = 0; c < 5; c++) {
        Fout[perm[d][c]] = Fsum[c] * area;
        dFout[perm[d][c]] = dFsum[c] * area;
    }
}

static void face_fluxes(const hgks_ref_t h, const double *q, int d, double dt, double *Fo, double *dFo)
{
    const int nd = n_of(h, d), n1 = n_of(h, tdir[d][0]), n2 = n_of(h, tdir[d][1]);
    const int e1 = n1 + 4, e2 = n2 + 4; /* tangential extents including 2 ghost rows each side */
    const size_t nface = (size_t)(nd + 1) * n1 * n2;
    double *FQ = (double *)malloc(sizeof(double) * FQ_N * 5 * (size_t)(nd + 1) * e1 * e2);
    if (!FQ) { fprintf(stderr, "hgks_ref: out of memory\n"); abort(); }

    /* 1. normal reconstruction on every face, including two tangential ghost rows */
    const long nfq = (long)(nd + 1) * e1 * e2;
#pragma omp parallel for schedule(dynamic, 64)
    for (long idx = 0; idx < nfq; idx++) {
        int f = (int)(idx % (nd + 1));
        int a = (int)((idx / (nd + 1)) % e1) - 2;
        int b = (int)(idx / ((long)(nd + 1) * e1)) - 2;
        normal_recon(h, q, d, f, a, b, (double(*)[5]) & FQ[(size_t)idx * FQ_N * 5]);
    }

    /* 2. tangential reconstruction to the 2x2 Gauss points and the GKS flux */
#pragma omp parallel for schedule(dynamic, 16)
    for (long fidx = 0; fidx < (long)nface; fidx++) {
        int f = (int)(fidx % (nd + 1));
        int a = (int)((fidx / (nd + 1)) % n1);
        int b = (int)(fidx / ((long)(nd + 1) * n1));
        const double *rec[5][5];
        for (int jj = 0; jj < 5; jj++)
            for (int kk = 0; kk < 5; kk++) {
                size_t fi = ((size_t)(b + kk) * e1 + (size_t)(a + jj)) * (nd + 1) + f; /* offsets -2..2, shifted */
                rec[jj][kk] = &FQ[fi * FQ_N * 5];
            }
        double Fl[5], dFl[5];
        face_flux_one(h, d, f, a, b, dt, rec, Fl, dFl);
        for (int c = 0; c < 5; c++) {
            Fo[(size_t)c * nface + fidx] = Fl[c];
            dFo[(size_t)c * nface + fidx] = dFl[c];
        }
    }
    free(FQ);
}

/* the same face flux with the 25 neighbouring normal reconstructions done on
   the spot (for sampled interfaces of large grids) */
static void face_flux_local(const hgks_ref_t h, const double *q, int d, int f, int a, int b, double dt,
                            double Fl[5], double dFl[5])
{
    double recs[5][5][FQ_N * 5];
    const double *rec[5][5];
    for (int jj = 0; jj < 5; jj++)
        for (int kk = 0; kk < 5; kk++) {
            normal_recon(h, q, d, f, a - 2 + jj, b - 2 + kk, (double(*)[5])recs[jj][kk]);
            rec[jj][kk] = recs[jj][kk];
        }
    face_flux_one(h, d, f, a, b, dt, rec, Fl, dFl);
}

/* R-F: a constant body force G is the source S = (0, rho G, rho U.G) in L and
   its time derivative dS/dt = (0, G L_rho, G.L_rhoU) in dL/dt, where L_rhoU
   already holds the momentum source */
static void add_body_force(const hgks_ref_t h, const double *q, size_t p, double Lc[5], double dLc[5])
{
    const size_t S = h->ncell_pad;
    if (h->G[0] == 0.0 && h->G[1] == 0.0 && h->G[2] == 0.0) return;
    double rho = q[0 * S + p];
    for (int e = 0; e < 3; e++) Lc[1 + e] += rho * h->G[e];
    Lc[4] += q[1 * S + p] * h->G[0] + q[2 * S + p] * h->G[1] + q[3 * S + p] * h->G[2];
    for (int e = 0; e < 3; e++) dLc[1 + e] += h->G[e] * Lc[0];
    dLc[4] += h->G[0] * Lc[1] + h->G[1] * Lc[2] + h->G[2] * Lc[3];
}

/* L(Q) and dL/dt(Q) (Eq. "semi2" and its time derivative) of a ghost-filled state */
static void eval_rhs(const hgks_ref_t h, const double *q, double dt, double *L, double *dL, int record_wall)
{
    const int nx = h->g.nx, ny = h->g.ny, nz = h->g.nz;
    const size_t N = h->ncell;
    for (int d = 0; d < 3; d++) face_fluxes(h, q, d, dt, h->F[d], h->dF[d]);
    size_t nf[3] = { (size_t)(nx + 1) * ny * nz, (size_t)(ny + 1) * nx * nz, (size_t)(nz + 1) * nx * ny };
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                size_t ci = iidx(h, i, j, k);
                double vol = dx_(h) * dy_cell(h, j) * dz_(h);
                /* face indices: direction d, face f, tangential (a, b) -> f + (nd+1)(a + n1 b) */
                size_t fx = ((size_t)k * ny + j) * (nx + 1) + i;
                size_t fy = ((size_t)k * nx + i) * (ny + 1) + j;
                size_t fz = ((size_t)j * nx + i) * (nz + 1) + k;
                double Lc[5], dLc[5];
                for (int c = 0; c < 5; c++) {
                    double sx = h->F[0][c * nf[0] + fx + 1] - h->F[0][c * nf[0] + fx];
                    double sy = h->F[1][c * nf[1] + fy + 1] - h->F[1][c * nf[1] + fy];
                    double sz = h->F[2][c * nf[2] + fz + 1] - h->F[2][c * nf[2] + fz];
                    Lc[c] = -((sx + sy) + sz) / vol;
                    double tx = h->dF[0][c * nf[0] + fx + 1] - h->dF[0][c * nf[0] + fx];
                    double ty = h->dF[1][c * nf[1] + fy + 1] - h->dF[1][c * nf[1] + fy];
                    double tz = h->dF[2][c * nf[2] + fz + 1] - h->dF[2][c * nf[2] + fz];
                    dLc[c] = -((tx + ty) + tz) / vol;
                }
                add_body_force(h, q, pidx(h, i, j, k), Lc, dLc);
                for (int c = 0; c < 5; c++) {
                    L[c * N + ci] = Lc[c];
                    dL[c * N + ci] = dLc[c];
                }
            }
    if (record_wall) {
        /* mean wall shear from the x-momentum flux through the y walls */
        double s = 0.0;
        int walls = 0;
        if (h->bcs.lo[1] == HGKS_REF_BC_ISOTHERMAL_WALL) {
            double acc = 0.0;
            for (int k = 0; k < nz; k++)
                for (int i = 0; i < nx; i++) acc += h->F[1][1 * nf[1] + ((size_t)k * nx + i) * (ny + 1) + 0];
            s += -acc; walls++;
        }
        if (h->bcs.hi[1] == HGKS_REF_BC_ISOTHERMAL_WALL) {
            double acc = 0.0;
            for (int k = 0; k < nz; k++)
                for (int i = 0; i < nx; i++) acc += h->F[1][1 * nf[1] + ((size_t)k * nx + i) * (ny + 1) + ny];
            s += acc; walls++;
        }
        h->wall_shear = walls ? s / (walls * h->g.lx * h->g.lz) : 0.0;
    }
}

/* ======================================================================
 * public API
 * ==================================================================== */
static int fail(hgks_ref_t h, int code, const char *msg)
{
    if (h) snprintf(h->err, sizeof h->err, "%s", msg);
    return code;
}

int hgks_ref_create(const hgks_ref_grid *grid, double gamma, double Pr, const hgks_ref_visc *visc,
                    const hgks_ref_bcs *bcs, const double body_force[3], hgks_ref_t *out)
{
    if (!grid || !visc || !bcs || !out) return HGKS_REF_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(gamma > 1.0) || !(Pr > 0.0))
        return HGKS_REF_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++) {
        int n = d == 0 ? grid->nx : (d == 1 ? grid->ny : grid->nz);
        if ((bcs->lo[d] == HGKS_REF_BC_ISOTHERMAL_WALL || bcs->hi[d] == HGKS_REF_BC_ISOTHERMAL_WALL) && n < NG)
            return HGKS_REF_ERR_INVALID_ARG;
    }
    build_tables();
    hgks_ref_t h = (hgks_ref_t)calloc(1, sizeof *h);
    if (!h) return HGKS_REF_ERR_OOM;
    h->g = *grid;
    h->gas.gamma = gamma;
    h->gas.Pr = Pr;
    h->gas.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    h->gas.visc = *visc;
    h->bcs = *bcs;
    for (int d = 0; d < 3; d++) h->G[d] = body_force ? body_force[d] : 0.0;
    h->rho_ref = 1.0;
    h->np[0] = grid->nx + 2 * NG;
    h->np[1] = grid->ny + 2 * NG;
    h->np[2] = grid->nz + 2 * NG;
    h->ncell_pad = (size_t)h->np[0] * h->np[1] * h->np[2];
    h->ncell = (size_t)grid->nx * grid->ny * grid->nz;
    h->q = (double *)calloc(5 * h->ncell_pad, sizeof(double));
    h->yface = (double *)calloc((size_t)grid->ny + 1, sizeof(double));
    if (!h->q || !h->yface) { hgks_ref_destroy(h); return HGKS_REF_ERR_OOM; }
    for (int j = 0; j <= grid->ny; j++) h->yface[j] = y_of_s(h, 2.0 * j / grid->ny);
    *out = h;
    return HGKS_REF_OK;
}

static int ensure_work(hgks_ref_t h)
{
    if (h->qs) return HGKS_REF_OK;
    size_t N = h->ncell;
    h->qs = (double *)calloc(5 * h->ncell_pad, sizeof(double));
    h->qn = (double *)calloc(5 * h->ncell_pad, sizeof(double));
    h->L1 = (double *)calloc(5 * N, sizeof(double));
    h->dL1 = (double *)calloc(5 * N, sizeof(double));
    h->L2 = (double *)calloc(5 * N, sizeof(double));
    h->dL2 = (double *)calloc(5 * N, sizeof(double));
    size_t nf[3] = { (size_t)(h->g.nx + 1) * h->g.ny * h->g.nz, (size_t)(h->g.ny + 1) * h->g.nx * h->g.nz,
                     (size_t)(h->g.nz + 1) * h->g.nx * h->g.ny };
    for (int d = 0; d < 3; d++) {
        h->F[d] = (double *)calloc(5 * nf[d], sizeof(double));
        h->dF[d] = (double *)calloc(5 * nf[d], sizeof(double));
        if (!h->F[d] || !h->dF[d]) return HGKS_REF_ERR_OOM;
    }
    if (!h->qs || !h->qn || !h->L1 || !h->dL1 || !h->L2 || !h->dL2) return HGKS_REF_ERR_OOM;
    return HGKS_REF_OK;
}

void hgks_ref_destroy(hgks_ref_t h)
{
    if (!h) return;
    free(h->q); free(h->qs); free(h->qn);
    free(h->L1); free(h->dL1); free(h->L2); free(h->dL2);
    for (int d = 0; d < 3; d++) { free(h->F[d]); free(h->dF[d]); }
    free(h->yface);
    free(h);
}

const char *hgks_ref_last_error(hgks_ref_t h) { return h ? h->err : "null handle"; }

static void set_cons(const hgks_ref_t h, int i, int j, int k, double rho, double u, double v, double w, double p)
{
    size_t S = h->ncell_pad, pp = pidx(h, i, j, k);
    h->q[0 * S + pp] = rho;
    h->q[1 * S + pp] = rho * u;
    h->q[2 * S + pp] = rho * v;
    h->q[3 * S + pp] = rho * w;
    h->q[4 * S + pp] = p / (h->gas.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
}

/* Taylor-Green vortex (Sec. 4.1) as exact cell averages (R-INIT) */
int hgks_ref_init_tgv(hgks_ref_t h, double Ma, double U0, double rho0)
{
    if (!h || !(Ma > 0.0) || !(rho0 > 0.0)) return fail(h, HGKS_REF_ERR_INVALID_ARG, "bad TGV parameters");
    const double gm1 = h->gas.gamma - 1.0;
    const double p0 = rho0 * U0 * U0 / (h->gas.gamma * Ma * Ma);
    const size_t S = h->ncell_pad;
    double *avs[3][5]; /* per direction: avg sin, cos, cos2, sin^2, cos^2 */
    int n[3] = { h->g.nx, h->g.ny, h->g.nz };
    for (int d = 0; d < 3; d++) {
        for (int t = 0; t < 5; t++) avs[d][t] = (double *)malloc(sizeof(double) * n[d]);
        for (int i = 0; i < n[d]; i++) {
            double xl, xr;
            if (d == 0) { xl = h->g.x0 + i * dx_(h); xr = xl + dx_(h); }
            else if (d == 1 && stretched(h)) { xl = h->yface[i]; xr = h->yface[i + 1]; }
            else if (d == 1) { xl = h->g.y0 + i * (h->g.ly / h->g.ny); xr = xl + h->g.ly / h->g.ny; }
            else { xl = h->g.z0 + i * dz_(h); xr = xl + dz_(h); }
            double w = xr - xl;
            avs[d][0][i] = (cos(xl) - cos(xr)) / w;
            avs[d][1][i] = (sin(xr) - sin(xl)) / w;
            avs[d][2][i] = (sin(2.0 * xr) - sin(2.0 * xl)) / (2.0 * w);
            avs[d][3][i] = 0.5 - 0.5 * avs[d][2][i];
            avs[d][4][i] = 0.5 + 0.5 * avs[d][2][i];
        }
    }
    for (int k = 0; k < n[2]; k++)
        for (int j = 0; j < n[1]; j++)
            for (int i = 0; i < n[0]; i++) {
                size_t pp = pidx(h, i, j, k);
                double Sx = avs[0][0][i], Cx = avs[0][1][i], C2x = avs[0][2][i], ssx = avs[0][3][i], ccx = avs[0][4][i];
                double Sy = avs[1][0][j], Cy = avs[1][1][j], C2y = avs[1][2][j], ssy = avs[1][3][j], ccy = avs[1][4][j];
                double Cz = avs[2][1][k], C2z = avs[2][2][k], ccz = avs[2][4][k];
                double pbar = p0 + rho0 * U0 * U0 / 16.0 * (C2x + C2y) * (C2z + 2.0);
                h->q[0 * S + pp] = rho0;
                h->q[1 * S + pp] = rho0 * U0 * Sx * Cy * Cz;
                h->q[2 * S + pp] = -rho0 * U0 * Cx * Sy * Cz;
                h->q[3 * S + pp] = 0.0;
                h->q[4 * S + pp] = pbar / gm1 + 0.5 * rho0 * U0 * U0 * (ssx * ccy * ccz + ccx * ssy * ccz);
            }
    for (int d = 0; d < 3; d++)
        for (int t = 0; t < 5; t++) free(avs[d][t]);
    h->rho_ref = rho0;
    h->t = 0.0; h->step = 0; h->dt_last = 0.0; h->wall_shear = 0.0;
    return HGKS_REF_OK;
}

uint64_t hgks_ref_splitmix64(uint64_t x)
{
    /* SplitMix64 (Steele, Lea, Flood 2014): golden-gamma increment, two
       xor-shift-multiply rounds and a final xor-shift */
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double uniform_pm1(uint64_t x)
{
    return (double)(hgks_ref_splitmix64(x) >> 11) * (1.0 / 4503599627370496.0) - 1.0; /* [-1, 1) */
}

/* perturbed Poiseuille channel (Sec. 4.2; R-NOISE), point values at cell centres */
int hgks_ref_init_channel(hgks_ref_t h, double Ma_b, double noise_amp, uint64_t seed)
{
    if (!h || !(Ma_b > 0.0)) return fail(h, HGKS_REF_ERR_INVALID_ARG, "bad channel parameters");
    const double Ub = 1.0, rho = 1.0;
    const double Tw = Ub * Ub / (h->gas.gamma * Ma_b * Ma_b);
    const double p = rho * Tw;
    const double ymid = h->g.y0 + 0.5 * h->g.ly, hh = 0.5 * h->g.ly;
    h->bcs.T_wall = Tw;
    for (int k = 0; k < h->g.nz; k++)
        for (int j = 0; j < h->g.ny; j++)
            for (int i = 0; i < h->g.nx; i++) {
                double yc = y_of_s(h, 2.0 * (j + 0.5) / h->g.ny);
                double yn = (yc - ymid) / hh;
                double U = 1.5 * Ub * (1.0 - yn * yn);
                uint64_t idx = ((uint64_t)k * h->g.ny + j) * h->g.nx + i;
                double r0 = uniform_pm1(seed ^ (3 * idx + 0));
                double r1 = uniform_pm1(seed ^ (3 * idx + 1));
                double r2 = uniform_pm1(seed ^ (3 * idx + 2));
                set_cons(h, i, j, k, rho, U + noise_amp * U * r0, noise_amp * Ub * r1, noise_amp * Ub * r2, p);
            }
    h->rho_ref = rho;
    h->t = 0.0; h->step = 0; h->dt_last = 0.0; h->wall_shear = 0.0;
    return HGKS_REF_OK;
}

/* smooth density wave advected by a uniform velocity: exact cell averages of
   rho = 1 + amp sin(pi sum_d k_d x_d), U_d = k_d, p = 1, with k_d = 1 for
   every direction with more than one cell and 0 otherwise */
int hgks_ref_init_density_wave(hgks_ref_t h, double amp)
{
    if (!h) return HGKS_REF_ERR_INVALID_ARG;
    double kd[3] = { h->g.nx > 1, h->g.ny > 1, h->g.nz > 1 };
    double hs[3] = { dx_(h), h->g.ly / h->g.ny, dz_(h) };
    double fac = 1.0;
    for (int d = 0; d < 3; d++)
        if (kd[d] > 0) fac *= sin(PI * hs[d] / 2.0) / (PI * hs[d] / 2.0);
    for (int k = 0; k < h->g.nz; k++)
        for (int j = 0; j < h->g.ny; j++)
            for (int i = 0; i < h->g.nx; i++) {
                double xc = h->g.x0 + (i + 0.5) * hs[0], yc = h->g.y0 + (j + 0.5) * hs[1], zc = h->g.z0 + (k + 0.5) * hs[2];
                double ph = PI * (kd[0] * xc + kd[1] * yc + kd[2] * zc);
                double rho = 1.0 + amp * sin(ph) * fac;
                size_t S = h->ncell_pad, pp = pidx(h, i, j, k);
                h->q[0 * S + pp] = rho;
                for (int d = 0; d < 3; d++) h->q[(1 + d) * S + pp] = rho * kd[d];
                h->q[4 * S + pp] = 1.0 / (h->gas.gamma - 1.0) + 0.5 * rho * (kd[0] + kd[1] + kd[2]);
            }
    h->rho_ref = 1.0;
    h->t = 0.0; h->step = 0; h->dt_last = 0.0; h->wall_shear = 0.0;
    return HGKS_REF_OK;
}

int hgks_ref_set_state(hgks_ref_t h, const double *hq)
{
    if (!h || !hq) return HGKS_REF_ERR_INVALID_ARG;
    for (int c = 0; c < 5; c++)
        for (int k = 0; k < h->g.nz; k++)
            for (int j = 0; j < h->g.ny; j++)
                for (int i = 0; i < h->g.nx; i++)
                    h->q[c * h->ncell_pad + pidx(h, i, j, k)] = hq[c * h->ncell + iidx(h, i, j, k)];
    return HGKS_REF_OK;
}

int hgks_ref_get_state(hgks_ref_t h, double *hq)
{
    if (!h || !hq) return HGKS_REF_ERR_INVALID_ARG;
    for (int c = 0; c < 5; c++)
        for (int k = 0; k < h->g.nz; k++)
            for (int j = 0; j < h->g.ny; j++)
                for (int i = 0; i < h->g.nx; i++)
                    hq[c * h->ncell + iidx(h, i, j, k)] = h->q[c * h->ncell_pad + pidx(h, i, j, k)];
    return HGKS_REF_OK;
}

int hgks_ref_set_time(hgks_ref_t h, double t, int64_t step)
{
    if (!h) return HGKS_REF_ERR_INVALID_ARG;
    h->t = t;
    h->step = step;
    return HGKS_REF_OK;
}

int hgks_ref_compute_dt(hgks_ref_t h, double cfl, double *dt)
{
    if (!h || !dt || !(cfl > 0.0)) return HGKS_REF_ERR_INVALID_ARG;
    double m = dt_limit(h, h->q);
    if (h->min_hook) m = h->min_hook(h->hook_user, m);
    *dt = cfl * m;
    return HGKS_REF_OK;
}

int hgks_ref_set_hooks(hgks_ref_t h, hgks_ref_halo_fn halo, hgks_ref_min_fn dtmin, void *user)
{
    if (!h) return HGKS_REF_ERR_INVALID_ARG;
    h->halo_hook = halo;
    h->min_hook = dtmin;
    h->hook_user = user;
    return HGKS_REF_OK;
}

int hgks_ref_rhs(hgks_ref_t h, double dt, double *L, double *dL)
{
    if (!h || !L || !dL || !(dt > 0.0)) return HGKS_REF_ERR_INVALID_ARG;
    int st = ensure_work(h);
    if (st) return fail(h, st, "out of memory");
    ghost_fill(h, h->q);
    eval_rhs(h, h->q, dt, L, dL, 0);
    return HGKS_REF_OK;
}

/* L and dL/dt at a list of interior cells only (cell index (k ny + j) nx + i) */
int hgks_ref_rhs_cells(hgks_ref_t h, double dt, int ncells, const int64_t *cells, double *L, double *dL)
{
    if (!h || !cells || !L || !dL || ncells < 0 || !(dt > 0.0)) return HGKS_REF_ERR_INVALID_ARG;
    ghost_fill(h, h->q);
    const int nx = h->g.nx, ny = h->g.ny;
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < ncells; s++) {
        int64_t ci = cells[s];
        int i = (int)(ci % nx), j = (int)((ci / nx) % ny), k = (int)(ci / ((int64_t)nx * ny));
        int ijk[3] = { i, j, k };
        double sd[3][5], tdd[3][5];
        for (int d = 0; d < 3; d++) {
            int f = ijk[d], a = ijk[tdir[d][0]], b = ijk[tdir[d][1]];
            double Fm[5], dFm[5], Fp[5], dFp[5];
            face_flux_local(h, h->q, d, f, a, b, dt, Fm, dFm);
            face_flux_local(h, h->q, d, f + 1, a, b, dt, Fp, dFp);
            for (int c = 0; c < 5; c++) { sd[d][c] = Fp[c] - Fm[c]; tdd[d][c] = dFp[c] - dFm[c]; }
        }
        double vol = dx_(h) * dy_cell(h, j) * dz_(h);
        double Lc[5], dLc[5];
        for (int c = 0; c < 5; c++) {
            Lc[c] = -((sd[0][c] + sd[1][c]) + sd[2][c]) / vol;
            dLc[c] = -((tdd[0][c] + tdd[1][c]) + tdd[2][c]) / vol;
        }
        add_body_force(h, h->q, pidx(h, i, j, k), Lc, dLc);
        for (int c = 0; c < 5; c++) { L[(size_t)s * 5 + c] = Lc[c]; dL[(size_t)s * 5 + c] = dLc[c]; }
    }
    return HGKS_REF_OK;
}

int hgks_ref_face_flux(hgks_ref_t h, double dt, int d, int f, int a, int b, double F[5], double dF[5])
{
    if (!h || !F || !dF || d < 0 || d > 2 || !(dt > 0.0)) return HGKS_REF_ERR_INVALID_ARG;
    if (f < 0 || f > n_of(h, d) || a < 0 || a >= n_of(h, tdir[d][0]) || b < 0 || b >= n_of(h, tdir[d][1]))
        return HGKS_REF_ERR_INVALID_ARG;
    ghost_fill(h, h->q);
    face_flux_local(h, h->q, d, f, a, b, dt, F, dF);
    return HGKS_REF_OK;
}

static int state_ok(const hgks_ref_t h, const double *q)
{
    for (int k = 0; k < h->g.nz; k++)
        for (int j = 0; j < h->g.ny; j++)
            for (int i = 0; i < h->g.nx; i++) {
                double Q[5];
                size_t p = pidx(h, i, j, k);
                for (int c = 0; c < 5; c++) {
                    Q[c] = q[c * h->ncell_pad + p];
                    if (!isfinite(Q[c])) return 0;
                }
                double e = Q[4] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]) / Q[0];
                if (!(Q[0] > 0.0) || !(e > 0.0)) return 0;
            }
    return 1;
}

/* one S2O4 step (Eq. "two-stage") with the same dt and delta in both stages (R-S2) */
static int one_step(hgks_ref_t h, double dt)
{
    const size_t N = h->ncell, S = h->ncell_pad;
    /* stage 1 on Q^n (already ghost-filled) */
    eval_rhs(h, h->q, dt, h->L1, h->dL1, 1);
    memcpy(h->qs, h->q, sizeof(double) * 5 * S);
    for (int c = 0; c < 5; c++)
        for (int k = 0; k < h->g.nz; k++)
            for (int j = 0; j < h->g.ny; j++)
                for (int i = 0; i < h->g.nx; i++) {
                    size_t p = pidx(h, i, j, k), ci = iidx(h, i, j, k);
                    h->qs[c * S + p] = h->q[c * S + p] + 0.5 * dt * h->L1[c * N + ci]
                                     + 0.125 * dt * dt * h->dL1[c * N + ci];
                }
    ghost_fill(h, h->qs);
    /* stage 2 on Q* */
    eval_rhs(h, h->qs, dt, h->L2, h->dL2, 0);
    memcpy(h->qn, h->q, sizeof(double) * 5 * S);
    for (int c = 0; c < 5; c++)
        for (int k = 0; k < h->g.nz; k++)
            for (int j = 0; j < h->g.ny; j++)
                for (int i = 0; i < h->g.nx; i++) {
                    size_t p = pidx(h, i, j, k), ci = iidx(h, i, j, k);
                    h->qn[c * S + p] = h->q[c * S + p] + dt * h->L1[c * N + ci]
                                     + dt * dt / 6.0 * (h->dL1[c * N + ci] + 2.0 * h->dL2[c * N + ci]);
                }
    if (!state_ok(h, h->qn)) return fail(h, HGKS_REF_ERR_NONFINITE, "non-finite or non-positive state");
    double *t = h->q; h->q = h->qn; h->qn = t;
    h->t += dt;
    h->step += 1;
    h->dt_last = dt;
    return HGKS_REF_OK;
}

int hgks_ref_step(hgks_ref_t h, int nsteps, double cfl)
{
    if (!h || nsteps < 0 || !(cfl > 0.0)) return fail(h, HGKS_REF_ERR_INVALID_ARG, "bad step arguments");
    int st = ensure_work(h);
    if (st) return fail(h, st, "out of memory");
    for (int s = 0; s < nsteps; s++) {
        ghost_fill(h, h->q);
        double m = dt_limit(h, h->q);
        if (h->min_hook) m = h->min_hook(h->hook_user, m);
        double dt = cfl * m;
        st = one_step(h, dt);
        if (st) return st;
    }
    return HGKS_REF_OK;
}

int hgks_ref_step_dt(hgks_ref_t h, int nsteps, double dt)
{
    if (!h || nsteps < 0 || !(dt > 0.0)) return fail(h, HGKS_REF_ERR_INVALID_ARG, "bad step arguments");
    int st = ensure_work(h);
    if (st) return fail(h, st, "out of memory");
    for (int s = 0; s < nsteps; s++) {
        ghost_fill(h, h->q);
        st = one_step(h, dt);
        if (st) return st;
    }
    return HGKS_REF_OK;
}

/* diagnostics (Sec. 4.1 E_k, eps_com; R-STAT) */
int hgks_ref_stats(hgks_ref_t h, hgks_ref_stats_t *o)
{
    if (!h || !o) return HGKS_REF_ERR_INVALID_ARG;
    ghost_fill(h, h->q);
    const size_t S = h->ncell_pad;
    const double K = h->gas.K;
    double vol_tot = 0, ek = 0, ens = 0, eps = 0, mass = 0, mom[3] = { 0, 0, 0 }, en = 0, mmax = 0;
    for (int k = 0; k < h->g.nz; k++)
        for (int j = 0; j < h->g.ny; j++)
            for (int i = 0; i < h->g.nx; i++) {
                size_t p = pidx(h, i, j, k);
                double vol = dx_(h) * dy_cell(h, j) * dz_(h);
                double Q[5], W[5];
                for (int c = 0; c < 5; c++) Q[c] = h->q[c * S + p];
                hgks_ref_prim(Q, K, W);
                double pr = W[0] / (2.0 * W[4]), T = pr / W[0];
                double u2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
                double cs = sqrt(h->gas.gamma * pr / W[0]);
                if (sqrt(u2) / cs > mmax) mmax = sqrt(u2) / cs;
                /* velocity gradient by fourth-order central differences of cell-centre u */
                double gr[3][3]; /* gr[a][b] = d u_a / d x_b */
                for (int b = 0; b < 3; b++) {
                    int o1[3] = { 0, 0, 0 };
                    o1[b] = 1;
                    double hb = (b == 0) ? dx_(h) : (b == 1 ? dy_dj(h, j + 0.5) : dz_(h));
                    double uu[4][3];
                    const int offs[4] = { -2, -1, 1, 2 };
                    for (int s = 0; s < 4; s++) {
                        size_t ps = pidx(h, i + offs[s] * o1[0], j + offs[s] * o1[1], k + offs[s] * o1[2]);
                        for (int a = 0; a < 3; a++) uu[s][a] = h->q[(1 + a) * S + ps] / h->q[ps];
                    }
                    for (int a = 0; a < 3; a++)
                        gr[a][b] = (uu[0][a] - 8.0 * uu[1][a] + 8.0 * uu[2][a] - uu[3][a]) / (12.0 * hb);
                }
                double wx = gr[2][1] - gr[1][2], wy = gr[0][2] - gr[2][0], wz = gr[1][0] - gr[0][1];
                double w2 = wx * wx + wy * wy + wz * wz;
                double div = gr[0][0] + gr[1][1] + gr[2][2];
                double mu = viscosity(&h->gas.visc, T);
                vol_tot += vol;
                ek += 0.5 * W[0] * u2 * vol;
                ens += 0.5 * W[0] * w2 * vol;
                eps += mu * (w2 + 4.0 / 3.0 * div * div) * vol;
                mass += Q[0] * vol;
                for (int a = 0; a < 3; a++) mom[a] += Q[1 + a] * vol;
                en += Q[4] * vol;
            }
    o->t = h->t;
    o->step = h->step;
    o->dt = h->dt_last;
    o->Ek = ek / (h->rho_ref * vol_tot);
    o->enstrophy = ens / (h->rho_ref * vol_tot);
    o->eps_com = eps / (h->rho_ref * vol_tot);
    o->mass = mass;
    for (int a = 0; a < 3; a++) o->mom[a] = mom[a];
    o->energy = en;
    o->max_mach = mmax;
    o->wall_shear = h->wall_shear;
    return HGKS_REF_OK;
}

/* ======================================================================
 * unit-level exports for the pins
 * ==================================================================== */
void hgks_ref_moments_1d(double U, double lam, int range, int nmax, double *out)
{
    double m[16];
    if (nmax > 16) nmax = 16;
    moments_1d(U, lam, range, nmax < 2 ? 2 : nmax, m);
    for (int n = 0; n < nmax; n++) out[n] = m[n];
}

void hgks_ref_moments_xi(double lam, double K, double out[3]) { moments_xi(lam, K, out); }

void hgks_ref_micro_slope(const double W[5], double K, const double dQ[5], double a[5])
{
    maxw g;
    maxw_build(&g, W, K);
    slope_solve(&g, dQ, a);
}

void hgks_ref_slope_moments(const double W[5], double K, const double a[5], double out[5])
{
    maxw g;
    double M[25];
    maxw_build(&g, W, K);
    moment_matrix(&g, M);
    for (int i = 0; i < 5; i++) {
        double s = 0.0;
        for (int j = 0; j < 5; j++) s += M[i * 5 + j] * a[j];
        out[i] = s * W[0];
    }
}

void hgks_ref_compat(const double Ql[5], const double Qr[5], double K, double Q0[5])
{
    double Wl[5], Wr[5];
    maxw gl, gr;
    hgks_ref_prim(Ql, K, Wl);
    hgks_ref_prim(Qr, K, Wr);
    maxw_build(&gl, Wl, K);
    maxw_build(&gr, Wr, K);
    compat_g(&gl, &gr, Q0);
}

void hgks_ref_point_flux(const double Ql[5], const double Qr[5], const double dQl[15], const double dQr[15],
                         const double dQ0[15], double gamma, double Pr, const hgks_ref_visc *visc, double dt,
                         double Ifull[5], double Ihalf[5], double Fn[5], double dFn[5])
{
    gas_params gp;
    gp.gamma = gamma;
    gp.Pr = Pr;
    gp.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    gp.visc = *visc;
    double l[3][5], r[3][5], z[3][5];
    for (int d = 0; d < 3; d++)
        for (int c = 0; c < 5; c++) { l[d][c] = dQl[d * 5 + c]; r[d][c] = dQr[d * 5 + c]; z[d][c] = dQ0[d * 5 + c]; }
    point_flux(&gp, Ql, Qr, l, r, z, dt, Ifull, Ihalf);
    hgks_ref_time_fit(Ifull, Ihalf, dt, Fn, dFn);
}

static const weno_point *point_for(double sigma, weno_point *tmp)
{
    build_tables();
    for (int i = 0; i < WP_COUNT; i++)
        if (wp[i].sigma == sigma) return &wp[i];
    build_weno_point(tmp, sigma);
    return tmp;
}

double hgks_ref_weno_z(const double X[5], double sigma, double eps)
{
    weno_point tmp;
    return weno_z_eps(X, point_for(sigma, &tmp), eps);
}

void hgks_ref_weno_linear_weights(double sigma, double d[3])
{
    weno_point tmp;
    const weno_point *P = point_for(sigma, &tmp);
    for (int k = 0; k < 3; k++) d[k] = P->lin[k];
}

void hgks_ref_weno_candidates(const double X[5], double sigma, double p[3], double beta[3])
{
    weno_point tmp;
    const weno_point *P = point_for(sigma, &tmp);
    weno_parts(X, P, p, beta);
}

void hgks_ref_quartic_coeffs(double sigma, double Lc[5], double Dc[5])
{
    weno_point tmp;
    const weno_point *P = point_for(sigma, &tmp);
    for (int j = 0; j < 5; j++) { Lc[j] = P->qv[j]; Dc[j] = P->qd[j]; }
}
