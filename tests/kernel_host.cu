// Host instantiation of the arithmetic of the CUDA flux path, applied case
// by case over arrays for tests/test_kernel_host.py: the FP64 templates of
// paper_2207_01173_gb300/csrc/hgks_device.cuh (the Gauss-point GKS flux,
// WENO-Z at the cell edges and Gauss points, the quartic value and slope
// weights) and the mixed-precision Gauss-point flux of hgks_passes_mx.cuh.
// Host libm stands in for CUDA's erfc/exp/sqrt/pow here.
#include "../paper_2207_01173_gb300/csrc/hgks_device.cuh"
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
void kh_point_flux_mixed(int n, const float *Ql_hi, const float *Ql_lo, const float *Qr_hi, const float *Qr_lo,
                         const float *dl, const float *dr, const float *d0, double gamma, double Pr, int visc_kind,
                         double mu_ref, double T_ref, double omega, double dt, double *Fn, double *dFn)
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
        hgks::gks_point_flux_mixed(col, 1, 0, 1.0f, 1.0f, 1.0f, G, (float)dt, F, dF);
        for (int c = 0; c < 5; c++) {
            Fn[5 * i + c] = hgks::ff_to_double(F[c]);
            dFn[5 * i + c] = dF[c];
        }
    }
}

}  // extern "C"
