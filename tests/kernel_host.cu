// Host instantiation of the FP64 arithmetic templates of the CUDA flux path
// (paper_2207_01173_gb300/csrc/hgks_device.cuh): the Gauss-point GKS flux,
// WENO-Z at the cell edges and Gauss points, and the quartic value and slope
// weights, applied case by case over arrays for tests/test_kernel_host.py.
// Host libm stands in for CUDA's erfc/exp/sqrt/pow here.
#include "../paper_2207_01173_gb300/csrc/hgks_device.cuh"

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

}  // extern "C"
