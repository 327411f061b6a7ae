// Host instantiation of the arithmetic of the CUDA flux path, applied case
// by case over arrays for tests/test_kernel_host.py: the FP64 templates of
// paper_2207_01173_gb300/csrc/hgks_device.cuh (the Gauss-point GKS flux,
// WENO-Z at the cell edges and Gauss points, the quartic value and slope
// weights), the mixed-precision Gauss-point flux of hgks_passes_mx.cuh, and
// the whole FP64 flux of one interface through the three pass bodies of
// hgks_bodies.cuh with the library's mesh tables and face geometry.
// Host libm stands in for CUDA's erfc/exp/sqrt/pow here.
#include "../paper_2207_01173_gb300/csrc/hgks_bodies.cuh"
#include "../paper_2207_01173_gb300/csrc/hgks_device.cuh"
#include "../paper_2207_01173_gb300/csrc/hgks_mesh.h"
#include "../paper_2207_01173_gb300/csrc/hgks_passes.cuh"
#include "../paper_2207_01173_gb300/csrc/hgks_passes_mx.cuh"

extern "C" {

// per case: Ql, Qr [5]; dl, dr, d0 [3][5] (normal, t1, t2); outputs Fn, dFn [5]
void kh_point_flux(int n, const double *Ql, const double *Qr, const double *dl, const double *dr, const double *d0,
                   double gamma, double Pr, int visc_kind, double mu_ref, double T_ref, double omega, double dt,
                   double *Fn, double *dFn)
{
    hgks::Params P{};
    P.gamma = gamma;
    P.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    P.Pr = Pr;
    P.visc_kind = visc_kind;
    P.mu_ref = mu_ref;
    P.T_ref = T_ref;
    P.omega = omega;
    for (int i = 0; i < n; i++)
        hgks::gks_point_flux<double>(Ql + 5 * i, Qr + 5 * i, (const double(*)[5])(dl + 15 * i),
                                     (const double(*)[5])(dr + 15 * i), (const double(*)[5])(d0 + 15 * i), P, dt,
                                     Fn + 5 * i, dFn + 5 * i);
}

// the time change of a side's primitives (rho, U, V, W, T) along its time
// slope, as the flux forms it from the spatial changes of the three
// directions (primitive-form Euler equations); per case Q [5], dq [3][5]
void kh_side_time_rate(int n, const double *Q, const double *dq, double gamma, double *out)
{
    const double gm1 = gamma - 1.0, K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    for (int i = 0; i < n; i++) {
        hgks::HalfSide<double> h;
        hgks::half_side_setup(Q + 5 * i, gm1, K, true, h);
        hgks::HalfDelta<double> d;
        hgks::HalfRate<double> r;
        const double *g = dq + 15 * i;
        hgks::half_delta(h, g, gm1, K, d);
        hgks::half_rate_add<0>(h, d, gm1, r);
        hgks::half_delta(h, g + 5, gm1, K, d);
        hgks::half_rate_add<1>(h, d, gm1, r);
        hgks::half_delta(h, g + 10, gm1, K, d);
        hgks::half_rate_add<2>(h, d, gm1, r);
        hgks::half_delta_time(h, r, K, d);
        double *o = out + 5 * i;
        o[0] = d.rho;
        for (int k = 0; k < 4; k++) o[1 + k] = d.dP[k];
    }
}

// per case: five averages X; outputs (left edge, right edge, value at -sqrt3/6,
// value at +sqrt3/6) by WENO-Z and (value -, value +, slope -, slope +) of the
// quartic, slopes in index units
void kh_reconstruct(int n, const double *X, double *weno, double *quartic)
{
    for (int i = 0; i < n; i++) {
        hgks::WenoPrep<double> W;
        hgks::weno_prep(X + 5 * i, W);
        double *w = weno + 4 * i, *q = quartic + 4 * i;
        hgks::weno_edge_pair(W, w[0], w[1]);
        hgks::weno_gauss_pair(W, w[2], w[3]);
        hgks::quartic_value_pair(X + 5 * i, q[0], q[1]);
        hgks::quartic_deriv_pair(X + 5 * i, q[2], q[3]);
    }
}

// the mixed-precision Gauss-point flux: per case Ql, Qr as float-float
// pairs (hi, lo) [5], slopes dl, dr, d0 [3][5] in FP32 (physical units);
// outputs F^n (float-float, returned as hi + lo in FP64) and dF^n/dt (FP32)
// (t64 != 0: the HGKS_MIXED_T64 variant, FP64 temperature, collision time
// and time coefficients)
void kh_point_flux_mixed(int n, const float *Ql_hi, const float *Ql_lo, const float *Qr_hi, const float *Qr_lo,
                         const float *dl, const float *dr, const float *d0, double gamma, double Pr, int visc_kind,
                         double mu_ref, double T_ref, double omega, double dt, double *Fn, double *dFn, int t64)
{
    hgks::Params P{};
    P.gamma = gamma;
    P.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    P.Pr = Pr;
    P.visc_kind = visc_kind;
    P.mu_ref = mu_ref;
    P.T_ref = T_ref;
    P.omega = omega;
    P.f_gm1 = (float)(gamma - 1.0);
    P.f_gm1_lo = (float)((gamma - 1.0) - (double)P.f_gm1);
    P.f_K = (float)P.K;
    P.f_prc = (float)(1.0 / Pr - 1.0);
    P.f_mu_ref = (float)mu_ref;
    P.f_inv_Tref = (float)(1.0 / T_ref);
    P.f_omega = (float)omega;
    const hgks::MxGas G = hgks::mx_gas(P);
    float col[hgks::GP_SLOTS];
    for (int i = 0; i < n; i++) {
        for (int c = 0; c < 5; c++) {
            col[GP_VAL(0, c, 0)] = Ql_hi[5 * i + c];
            col[GP_VAL(0, c, 1)] = Ql_lo[5 * i + c];
            col[GP_VAL(0, 5 + c, 0)] = Qr_hi[5 * i + c];
            col[GP_VAL(0, 5 + c, 1)] = Qr_lo[5 * i + c];
        }
        const float *sl[3] = { dl + 15 * i, dr + 15 * i, d0 + 15 * i };
        for (int which = 0; which < 3; which++)
            for (int c = 0; c < 5; c++) {
                col[GP_SN(0, which * 5 + c)] = sl[which][c];
                col[GP_S1(0, which * 5 + c)] = sl[which][5 + c];
                col[GP_S2(0, which * 5 + c)] = sl[which][10 + c];
            }
        hgks::ff F[5];
        float dF[5];
        if (t64) hgks::gks_point_flux_mixed<true>(col, 1, 0, 1.0f, 1.0f, 1.0f, G, (float)dt, F, dF, dt);
        else hgks::gks_point_flux_mixed<false>(col, 1, 0, 1.0f, 1.0f, 1.0f, G, (float)dt, F, dF, dt);
        for (int c = 0; c < 5; c++) {
            Fn[5 * i + c] = hgks::ff_to_double(F[c]);
            dFn[5 * i + c] = dF[c];
        }
    }
}

// equilibrium state Q0 of the mixed path from float-float Ql, Qr (per case
// 5 hi + 5 lo each); output as hi + lo in FP64
void kh_compat_mixed(int n, const float *Ql_hi, const float *Ql_lo, const float *Qr_hi, const float *Qr_lo,
                     double gamma, double *Q0)
{
    const float gm1 = (float)(gamma - 1.0), K = (float)((5.0 - 3.0 * gamma) / (gamma - 1.0));
    for (int i = 0; i < n; i++) {
        hgks::ff l[5], r[5], q[5];
        for (int c = 0; c < 5; c++) {
            l[c] = hgks::ff{ Ql_hi[5 * i + c], Ql_lo[5 * i + c] };
            r[c] = hgks::ff{ Qr_hi[5 * i + c], Qr_lo[5 * i + c] };
        }
        hgks::compat_mixed(l, r, gm1, K, q);
        for (int c = 0; c < 5; c++) Q0[5 * i + c] = hgks::ff_to_double(q[c]);
    }
}

// F^n and dF^n/dt (times the face area, global component order) of face f of
// sweep d at tangential cell indices (a, b), by the FP64 pass bodies: the
// normal pass on the 5 x 5 tangential neighbourhood, the first tangential
// pass on its 5 rows, then the flux pass.  q: a ghost-filled padded state
// [5][nz+6][ny+6][nx+6].
void kh_face_flux(const double *q, const hgks_grid *grid, double gamma, double Pr, int visc_kind, double mu_ref,
                  double T_ref, double omega, int d, int f, int a, int b, double dt, double *F, double *dF)
{
    using namespace hgks;
    const std::vector<double> yt = mesh_y_tables(*grid);
    const int n[3] = { grid->nx, grid->ny, grid->nz };
    Params P{};
    for (int e = 0; e < 3; e++) {
        P.n[e] = n[e];
        P.np[e] = n[e] + 2 * NG;
    }
    P.h[0] = grid->lx / grid->nx;
    P.h[1] = grid->ly / grid->ny;
    P.h[2] = grid->lz / grid->nz;
    P.stretched = grid->y_stretch_b > 0.0;
    P.my_face = yt.data();
    P.my_gp = yt.data() + n[1] + 1;
    P.my_cen = yt.data() + 3 * n[1] + 1;
    P.hy_cell = yt.data() + 4 * n[1] + 1;
    P.gamma = gamma;
    P.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    P.Pr = Pr;
    P.visc_kind = visc_kind;
    P.mu_ref = mu_ref;
    P.T_ref = T_ref;
    P.omega = omega;
    const long long cs = (long long)P.np[0] * P.np[1] * P.np[2];
    auto at = [&](int c, int i, int j, int k) {
        return q[c * cs + ((long long)(k + NG) * P.np[1] + (j + NG)) * P.np[0] + (i + NG)];
    };
    const int e1 = tdir(d, 0), e2 = tdir(d, 1);
    double rec[5][5][30], t1[5][110];  // rec[t2 offset][t1 offset][slot], t1[t2 offset][slot]
    for (int jb = 0; jb < 5; jb++)
        for (int ja = 0; ja < 5; ja++) {
            auto load = [&](int c, int m) {
                int ijk[3];
                ijk[d] = f - 3 + m;
                ijk[e1] = a - 2 + ja;
                ijk[e2] = b - 2 + jb;
                return at(perm_of(d, c), ijk[0], ijk[1], ijk[2]);
            };
            auto store = [&](int slot, double v) { rec[jb][ja][slot] = v; };
            normal_body<double>(load, store, P.K);
        }
    for (int jb = 0; jb < 5; jb++) {
        auto load = [&](int slot, int j) { return rec[jb][j][slot]; };
        auto store = [&](int slot, double v) { t1[jb][slot] = v; };
        tan1_body<double>(load, store);
    }
    const FaceGeom G = face_geom(P, d, f, a, b);
    auto load = [&](int slot, int j) { return t1[j][slot]; };
    double col[110], Fs[5], dFs[5];
    flux_body<double>(load, G, P, dt, col, Fs, dFs);
    for (int c = 0; c < 5; c++) {
        F[perm_of(d, c)] = Fs[c];
        dF[perm_of(d, c)] = dFs[c];
    }
}

}  // extern "C"
