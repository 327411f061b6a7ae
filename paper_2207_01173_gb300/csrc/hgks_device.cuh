// hgks_device.cuh -- device-side building blocks of the HGKS step (FP64).
//
// Method: arXiv 2207.01173, Sec. 2.  Closed forms used here:
//   * WENO-Z candidate quadratics written as c0 + c1 s + c2 s^2 about the centre
//     cell (s in cell widths), Jiang-Shu smoothness beta = c1^2 + 13/3 c2^2,
//     Borges et al. (2008) weights alpha_k = d_k (1 + tau5 / (beta_k + eps)),
//     evaluated with one division per point: alpha_k is proportional to
//     d_k (b_k + tau5) prod_{j != k} b_j with b = beta + eps.
//   * Gauss abscissae s = +-sqrt(3)/6 satisfy s^2 = 1/12, so every candidate
//     value there is X_0 +- s c1 and the quartic value/derivative weights have
//     the closed forms below (derived symbolically from cell averages).
//   * Maxwellian moments <u^n> by <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lambda) <u^n>,
//     half-range starts 1/2 erfc(-+sqrt(lambda) U) and e^{-lambda U^2}/(2 sqrt(pi lambda)).
//   * the micro-slope terms of the flux (a g = dg/dQ . dQ for a Maxwellian)
//     as directional derivatives of moment functions: Euler-flux Jacobians for
//     the full-range equilibrium terms, differentiated half-range moments for
//     the l/r terms, so no 5x5 slope system is ever solved; the time slope of
//     each l/r side enters through its primitives' time changes, taken from
//     the Euler equations in primitive form.
// The arithmetic routines are templates on the scalar type T (double on the
// device; a host operation-counting type instantiates the same code to count
// the scheme's floating-point work).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HGKS_HD __host__ __device__ __forceinline__

// Reciprocal of the WENO weight normaliser.  In FP32 (the mixed path) the
// approximate reciprocal (at most 2 ulp) is enough: it scales a deviation
// from the stencil centre, so it moves the reconstruction by ~1e-7 of a
// deviation, never the centre value, and consistency (weights summing to one)
// is exact because numerator and denominator share it.  FP64 divides.
template <typename T>
__host__ __device__ __forceinline__ T weno_recip(T x)
{
    return T(1.0) / x;
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ float weno_recip<float>(float x)
{
    return __fdividef(1.0f, x);
}
#endif

// a * b + c rounded once.  Written out where a sum has two products, because
// there the compiler may fuse either one, and its choice can differ between
// kernels that inline the same code (so the batch kernels would not repeat
// the single-problem kernels bit for bit).  The counting type of the flop
// model takes the generic form (one multiply, one add).
template <typename T>
__host__ __device__ __forceinline__ T fmad(T a, T b, T c)
{
    return a * b + c;
}
__host__ __device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }

namespace hgks {

constexpr int NG = 3;            // ghost layers (fifth-order WENO needs three)
constexpr double WENO_EPS = 1e-6;

// ---------------------------------------------------------------------------
// solver parameters passed by value to every kernel
// ---------------------------------------------------------------------------
struct Params {
    int n[3];               // interior cells per direction
    int np[3];              // padded extents n + 2 NG
    long long sy, sz, cs;   // strides of the padded array (x stride 1), component stride
    long long ncell;        // interior cells
    double h[3];            // uniform spacings (h[1] unused when stretched)
    int stretched;
    const double *my_face;  // [ny+1]  dy/dj at y faces (index units)
    const double *my_gp;    // [ny][2] dy/dj at the two Gauss abscissae of each cell
    const double *my_cen;   // [ny]    dy/dj at cell centres
    const double *hy_cell;  // [ny]    physical cell heights
    double gamma, K, Pr;
    int visc_kind;
    double mu_ref, T_ref, omega;
    double G[3];            // body force (acceleration)
    int has_force;
    int bc_lo[3], bc_hi[3];
    double T_wall;
    // FP32 copies for the mixed-precision passes: gamma - 1 as a float-float
    // pair, K, 1/Pr - 1, the viscosity law, and 1/h of the uniform directions
    float f_gm1, f_gm1_lo, f_K, f_prc, f_mu_ref, f_inv_Tref, f_omega;
    float f_ih[3];
};

// device control block of one handle
struct Ctl {
    unsigned long long dtmin_bits;  // min over cells of dx/(|u|+c), as ordered bits
    double dt;                      // time step of the step in flight
    double t;                       // time of the last good state
    long long step;                 // steps completed
    int flag;                       // set when a stage produced a bad state
    int good;                       // state buffer that holds the last good state
    double wall_shear;              // wall stress from the last step's first stage
    double last_dt;
};

__device__ __forceinline__ long long pidx(const Params &P, int i, int j, int k)
{
    return ((long long)(k + NG) * P.np[1] + (j + NG)) * (long long)P.np[0] + (i + NG);
}

// ---------------------------------------------------------------------------
// reconstruction
// ---------------------------------------------------------------------------
// Gauss abscissa sqrt(3)/6 and WENO-Z linear weights there (stencils ordered
// left, centre, right): ((210 - sqrt3)/1080, 11/18, (210 + sqrt3)/1080).
#define HGKS_SQ3 1.7320508075688772935
#define HGKS_GAUSS (HGKS_SQ3 / 6.0)
#define HGKS_DGL ((210.0 - HGKS_SQ3) / 1080.0)
#define HGKS_DGC (11.0 / 18.0)
#define HGKS_DGR ((210.0 + HGKS_SQ3) / 1080.0)

template <typename T>
struct WenoPrep {
    T c1[3], c2[3], cw[3];  // candidate slopes/curvatures, unnormalised nonlinear factors
    T x0;
};

template <typename T>
HGKS_HD void weno_prep(const T X[5], WenoPrep<T> &W)
{
    // candidate slopes and curvatures from the first differences of the averages
    const T d1 = X[1] - X[0], d2 = X[2] - X[1], d3 = X[3] - X[2], d4 = X[4] - X[3];
    W.x0 = X[2];
    const T h = T(0.5), t3 = T(1.5);
    W.c2[0] = h * (d2 - d1);
    W.c1[0] = t3 * d2 - h * d1;
    W.c2[1] = h * (d3 - d2);
    W.c1[1] = h * (d3 + d2);
    W.c2[2] = h * (d4 - d3);
    W.c1[2] = t3 * d3 - h * d4;
    T b[3];
#pragma unroll
    for (int k = 0; k < 3; k++) b[k] = W.c1[k] * W.c1[k] + T(13.0 / 3.0) * W.c2[k] * W.c2[k] + T(WENO_EPS);
    T tau5 = fabs(b[0] - b[2]);
    W.cw[0] = (b[0] + tau5) * (b[1] * b[2]);
    W.cw[1] = (b[1] + tau5) * (b[0] * b[2]);
    W.cw[2] = (b[2] + tau5) * (b[0] * b[1]);
}

// both Gauss abscissae from one reciprocal: the two denominators D- and D+
// (mirrored linear weights) are inverted together as 1/(D- D+)
template <typename T>
HGKS_HD void weno_gauss_pair(const WenoPrep<T> &W, T &vm, T &vp)
{
    const T dgl = T(HGKS_DGL), dgr = T(HGKS_DGR);
    const T e0 = dgl * W.cw[0], e2 = dgr * W.cw[2], f0 = dgr * W.cw[0], f2 = dgl * W.cw[2];
    const T a1 = T(HGKS_DGC) * W.cw[1];
    const T dp = e0 + a1 + e2, dm = f0 + a1 + f2;  // plus: (DGL, DGC, DGR), minus: mirrored
    const T np = e0 * W.c1[0] + a1 * W.c1[1] + e2 * W.c1[2];
    const T nm = f0 * W.c1[0] + a1 * W.c1[1] + f2 * W.c1[2];
    const T r = weno_recip<T>(dp * dm);
    vp = W.x0 + T(HGKS_GAUSS) * (np * dm * r);
    vm = W.x0 - T(HGKS_GAUSS) * (nm * dp * r);
}

// both cell edges (-1/2: vl, +1/2: vr) from one reciprocal
template <typename T>
HGKS_HD void weno_edge_pair(const WenoPrep<T> &W, T &vl, T &vr)
{
    const T c01 = T(0.1), c03 = T(0.3), c06 = T(0.6), c16 = T(1.0 / 6.0), h = T(0.5);
    const T a1 = c06 * W.cw[1];
    const T r0 = c01 * W.cw[0], r2 = c03 * W.cw[2];  // right edge weights
    const T l0 = c03 * W.cw[0], l2 = c01 * W.cw[2];  // left edge weights
    const T p0 = W.x0 + W.c2[0] * c16, p1 = W.x0 + W.c2[1] * c16, p2 = W.x0 + W.c2[2] * c16;
    const T nr = r0 * (p0 + h * W.c1[0]) + a1 * (p1 + h * W.c1[1]) + r2 * (p2 + h * W.c1[2]);
    const T nl = l0 * (p0 - h * W.c1[0]) + a1 * (p1 - h * W.c1[1]) + l2 * (p2 - h * W.c1[2]);
    const T dr = r0 + a1 + r2, dl = l0 + a1 + l2;
    const T r = weno_recip<T>(dr * dl);
    vr = nr * dl * r;
    vl = nl * dr * r;
}

// quartic through five cell averages: point value and derivative (index units)
// at -sqrt(3)/6 (plus = 0) or +sqrt(3)/6 (plus = 1).
// value = E.X +- sqrt3 O.X,  E = (-1/4320, 1/1080, 719/720, 1/1080, -1/4320),
//                           O = (7/432, -25/216, 0, 25/216, -7/432)
// deriv = C.X -+ sqrt3 S.X,  C = (1/12, -2/3, 0, 2/3, -1/12),
//                           S = (1/54, -13/54, 24/54, -13/54, 1/54)
template <typename T>
HGKS_HD void quartic_value_pair(const T X[5], T &vm, T &vp)
{
    const T e = T(-1.0 / 4320.0) * (X[0] + X[4]) + T(1.0 / 1080.0) * (X[1] + X[3]) + T(719.0 / 720.0) * X[2];
    const T o = T(HGKS_SQ3) * (T(7.0 / 432.0) * (X[0] - X[4]) + T(25.0 / 216.0) * (X[3] - X[1]));
    vm = e - o;
    vp = e + o;
}
template <typename T>
HGKS_HD void quartic_deriv_pair(const T X[5], T &dm, T &dp)
{
    const T c = T(1.0 / 12.0) * (X[0] - X[4]) + T(2.0 / 3.0) * (X[3] - X[1]);
    const T s = T(HGKS_SQ3) * (T(1.0 / 54.0) * (X[0] + X[4]) - T(13.0 / 54.0) * (X[1] + X[3]) + T(24.0 / 54.0) * X[2]);
    dm = c + s;
    dp = c - s;
}

// ---------------------------------------------------------------------------
// Maxwellian moments and the gas-kinetic flux
// ---------------------------------------------------------------------------
template <typename T>
struct Prim {
    T rho, U, V, W, lam;
};

template <typename T, typename S>
HGKS_HD Prim<T> prim_of(const T Q[5], S K)
{
    Prim<T> g;
    T ir = T(1.0) / Q[0];
    g.rho = Q[0];
    g.U = Q[1] * ir;
    g.V = Q[2] * ir;
    g.W = Q[3] * ir;
    T eint = Q[4] - T(0.5) * Q[0] * (g.U * g.U + g.V * g.V + g.W * g.W);
    g.lam = T(K + 3.0) * Q[0] / (T(4.0) * eint);
    return g;
}

// full-range normalised moments <x^n>, n < N, of a Gaussian with mean U
template <int N, typename T>
HGKS_HD void mom_full(T U, T i2l, T *m)
{
    m[0] = T(1.0);
    m[1] = U;
#pragma unroll
    for (int n = 0; n + 2 < N; n++) m[n + 2] = U * m[n + 1] + T(n + 1) * i2l * m[n];
}

// half-range moments over u > 0 (pos) or u < 0
template <int N, typename T>
HGKS_HD void mom_half(T U, T lam, T i2l, bool pos, T *m)
{
    const T inv_2sqrtpi = T(0.28209479177387814347); // 1 / (2 sqrt(pi))
    T sl = sqrt(lam);
    T e = exp(-lam * U * U) * inv_2sqrtpi / sl;
    if (pos) {
        m[0] = T(0.5) * erfc(-sl * U);
        m[1] = U * m[0] + e;
    } else {
        m[0] = T(0.5) * erfc(sl * U);
        m[1] = U * m[0] - e;
    }
#pragma unroll
    for (int n = 0; n + 2 < N; n++) m[n + 2] = U * m[n + 1] + T(n + 1) * i2l * m[n];
}

// moments of one state: u (range specific), v, w (full), xi
template <typename T>
struct Mom {
    const T *u;
    const T *v;
    const T *w;
    T xi1, xi2;  // <xi^2>, <xi^4>
};

// <psi_i u^A v^B w^C>
template <int A, int B, int C, typename T>
HGKS_HD void psi_mom(const Mom<T> &m, T o[5])
{
    T uvw = m.u[A] * m.v[B] * m.w[C];
    o[0] = uvw;
    o[1] = m.u[A + 1] * m.v[B] * m.w[C];
    o[2] = m.u[A] * m.v[B + 1] * m.w[C];
    o[3] = m.u[A] * m.v[B] * m.w[C + 1];
    o[4] = T(0.5) * (m.u[A + 2] * m.v[B] * m.w[C] + m.u[A] * m.v[B + 2] * m.w[C] + m.u[A] * m.v[B] * m.w[C + 2]
                     + uvw * m.xi1);
}

template <typename T>
HGKS_HD T viscosity(const Params &P, T Tm)
{
    return P.visc_kind == 1 ? T(P.mu_ref) * pow(Tm * T(1.0 / P.T_ref), T(P.omega)) : T(P.mu_ref);
}

// ---------------------------------------------------------------------------
// flux-economic form of the point flux
// ---------------------------------------------------------------------------
// A Maxwellian g(Q) and the micro-slope a of a change dQ of its conserved
// variables satisfy a g = (dg/dQ) dQ.  Full-range moments of a g are therefore
// directional derivatives of moment functions of the Maxwellian:
//   sum_d <psi u_d a_d> rho = sum_d DF_d(Q)[d_d Q]    (F_d the Euler flux)
//   sum_d <psi u u_d a_d> rho = sum_d DH_d(Q)[d_d Q]  (H_d = rho <psi u u_d>)
//   <psi u A> rho = DF_n(Q)[d_t Q],  <psi A> rho = d_t Q,
// with d_t Q = -sum_d DF_d(Q)[d_d Q] from <a.u + A> = 0.  These closed forms
// replace the generic moment sums for the equilibrium terms; the half-range
// (u > 0, u < 0) terms keep the moment sums.

// primitive and derived quantities of one Maxwellian (R = 1)
template <typename T>
struct Gas {
    T rho, ir, U[3], uu, p, Tm, E;  // Tm = p / rho, E = rho E
};

template <typename T, typename S>
HGKS_HD Gas<T> gas_of(const T Q[5], S gm1)
{
    Gas<T> g;
    g.rho = Q[0];
    g.ir = T(1.0) / Q[0];
    g.U[0] = Q[1] * g.ir;
    g.U[1] = Q[2] * g.ir;
    g.U[2] = Q[3] * g.ir;
    g.uu = g.U[0] * g.U[0] + g.U[1] * g.U[1] + g.U[2] * g.U[2];
    g.E = Q[4];
    g.p = T(gm1) * (Q[4] - T(0.5) * Q[0] * g.uu);
    g.Tm = g.p * g.ir;
    return g;
}

// directional derivative of the Euler flux F_D (D = 0 normal, 1, 2) along dQ
template <int D, typename T, typename S>
HGKS_HD void euler_dflux(const Gas<T> &g, const T dQ[5], S gm1, T o[5])
{
    const T dp = T(gm1) * (dQ[4] - (g.U[0] * dQ[1] + g.U[1] * dQ[2] + g.U[2] * dQ[3]) + T(0.5) * g.uu * dQ[0]);
    const T dUd = (dQ[1 + D] - g.U[D] * dQ[0]) * g.ir;
    o[0] = dQ[1 + D];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T v = g.U[k] * dQ[1 + D] + g.U[D] * (dQ[1 + k] - g.U[k] * dQ[0]);
        o[1 + k] = k == D ? v + dp : v;
    }
    o[4] = dUd * (g.E + g.p) + g.U[D] * (dQ[4] + dp);
}

// directional derivative of H_D = rho <psi u u_D> (u the normal velocity):
// H_D = (rho U Ud + p d0D,
//        rho U Ud U_k + p (d0D U_k + d0k Ud + dDk U),
//        U Ud (rho E + 2p) + d0D p (|U|^2 + (K+5) T) / 2)
template <int D, typename T, typename S>
HGKS_HD void second_dmoment(const Gas<T> &g, const T dQ[5], S gm1, S Kp5, T o[5])
{
    const T drho = dQ[0];
    T dU[3];
#pragma unroll
    for (int k = 0; k < 3; k++) dU[k] = (dQ[1 + k] - g.U[k] * drho) * g.ir;
    const T dp = T(gm1) * (dQ[4] - (g.U[0] * dQ[1] + g.U[1] * dQ[2] + g.U[2] * dQ[3]) + T(0.5) * g.uu * drho);
    const T Un = g.U[0], Ud = g.U[D], dUn = dU[0], dUd = dU[D];
    const T dUnUd = dUn * Ud + Un * dUd;  // d(Un Ud)
    const T UnUd = Un * Ud;
    o[0] = drho * UnUd + g.rho * dUnUd;
    if (D == 0) o[0] += dp;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        T v = (drho * UnUd + g.rho * dUnUd) * g.U[k] + g.rho * UnUd * dU[k];
        if (D == 0) v += dp * g.U[k] + g.p * dU[k];
        if (k == 0) v += dp * Ud + g.p * dUd;
        if (k == D) v += dp * Un + g.p * dUn;
        o[1 + k] = v;
    }
    o[4] = dUnUd * (g.E + T(2.0) * g.p) + UnUd * (dQ[4] + T(2.0) * dp);
    if (D == 0) {
        const T UdU = g.U[0] * dU[0] + g.U[1] * dU[1] + g.U[2] * dU[2];
        const T kp5 = T(Kp5);
        o[4] += T(0.5) * (dp * (g.uu + kp5 * g.Tm) + g.p * (T(2.0) * UdU + kp5 * (dp - g.Tm * drho) * g.ir));
    }
}

template <typename T>
HGKS_HD T heat_of_g(const T B[5], const T W[5], const Gas<T> &g0)
{
    const T U0 = g0.U[0], V0 = g0.U[1], W0 = g0.U[2], uu = g0.uu;
    return B[4] - U0 * B[1] - V0 * B[2] - W0 * B[3] + T(0.5) * uu * B[0]
         - U0 * W[4] + U0 * U0 * W[1] + U0 * V0 * W[2] + U0 * W0 * W[3] - T(0.5) * U0 * uu * W[0];
}

// ---------------------------------------------------------------------------
// half-range moments by differentiation
// ---------------------------------------------------------------------------
// For a half-range Maxwellian (u > 0: sigma = +1, u < 0: sigma = -1) the
// micro-slope terms are directional derivatives of half-range moment
// functions Phi_m(Q) = rho <m psi>_sigma of monomials m (the range boundary
// u = 0 does not move), so neither a nor A has to be solved for:
//   <m psi a_d> rho = DPhi_m(Q)[d_d Q],   <m psi A> rho = DPhi_m(Q)[d_t Q].
// In primitives P = (rho, U, V, W, T) (T = 1/(2 lambda) = p/rho):
//   M_n (half, normal velocity), with phi0 = exp(-U^2/(2T)) / sqrt(2 pi T):
//     M_0 = erfc(-sigma U / sqrt(2T)) / 2,  M_1 = U M_0 + sigma T phi0,
//     M_{n+2} = U M_{n+1} + (n+1) T M_n,
//     dM_n/dU = n M_{n-1} + sigma phi0 [n = 0],
//     dM_n/dT = n(n-1)/2 M_{n-2} + sigma phi0 / 2 [n = 1] - sigma U phi0 / (2T) [n = 0];
//   full-range tangential moments: dM_n/dV = n M_{n-1}, dM_n/dT = n(n-1)/2 M_{n-2};
//   <xi^2> = K T.

template <typename T>
struct HalfSide {
    T rho, ir, U[3], uu, Tm, E, p;
    T u[5], v[4], w[4], xi1;              // moments (u: half range)
    T uU[5], uT[5], vV[4], vT[4], wW[4], wT[4];  // their partial derivatives
};

template <typename T, typename S>
HGKS_HD void half_side_setup(const T Q[5], S gm1, S K, bool pos, HalfSide<T> &h)
{
    h.rho = Q[0];
    h.ir = T(1.0) / Q[0];
    h.U[0] = Q[1] * h.ir;
    h.U[1] = Q[2] * h.ir;
    h.U[2] = Q[3] * h.ir;
    h.uu = h.U[0] * h.U[0] + h.U[1] * h.U[1] + h.U[2] * h.U[2];
    h.E = Q[4];
    h.p = T(gm1) * (Q[4] - T(0.5) * Q[0] * h.uu);
    h.Tm = h.p * h.ir;
    const T sg = T(pos ? 1.0 : -1.0);
    const T inv_sqrt2pi = T(0.39894228040143267794);  // 1/sqrt(2 pi)
    const T iTm = T(1.0) / h.Tm;
    const T isq = sqrt(iTm);                            // 1/sqrt(T)
    const T U = h.U[0];
    const T phi0 = exp(T(-0.5) * U * U * iTm) * (inv_sqrt2pi * isq);
    h.u[0] = T(0.5) * erfc(T(pos ? -0.70710678118654752440 : 0.70710678118654752440) * U * isq);
    h.u[1] = U * h.u[0] + sg * h.Tm * phi0;
#pragma unroll
    for (int n = 0; n < 3; n++) h.u[n + 2] = U * h.u[n + 1] + T(n + 1) * h.Tm * h.u[n];
    h.uU[0] = sg * phi0;
    h.uT[0] = T(pos ? -0.5 : 0.5) * U * iTm * phi0;
    h.uU[1] = h.u[0];
    h.uT[1] = T(pos ? 0.5 : -0.5) * phi0;
#pragma unroll
    for (int n = 2; n < 5; n++) {
        h.uU[n] = T(n) * h.u[n - 1];
        h.uT[n] = T(0.5 * n * (n - 1)) * h.u[n - 2];
    }
    mom_full<4>(h.U[1], h.Tm, h.v);
    mom_full<4>(h.U[2], h.Tm, h.w);
    h.vV[0] = T(0.0);
    h.wW[0] = T(0.0);
    h.vT[0] = T(0.0);
    h.wT[0] = T(0.0);
    h.vT[1] = T(0.0);
    h.wT[1] = T(0.0);
#pragma unroll
    for (int n = 1; n < 4; n++) {
        h.vV[n] = T(n) * h.v[n - 1];
        h.wW[n] = T(n) * h.w[n - 1];
    }
#pragma unroll
    for (int n = 2; n < 4; n++) {
        h.vT[n] = T(0.5 * n * (n - 1)) * h.v[n - 2];
        h.wT[n] = T(0.5 * n * (n - 1)) * h.w[n - 2];
    }
    h.xi1 = T(K) * h.Tm;
}

// value of Phi_m = rho <u^E v^J w^L psi>_sigma
template <int E, int J, int L, typename T>
HGKS_HD void half_phi(const HalfSide<T> &h, T o[5])
{
    const T bc = h.v[J] * h.w[L];
    const T abc = h.u[E] * bc;
    o[0] = h.rho * abc;
    o[1] = h.rho * (h.u[E + 1] * bc);
    o[2] = h.rho * (h.u[E] * h.v[J + 1] * h.w[L]);
    o[3] = h.rho * (h.u[E] * h.v[J] * h.w[L + 1]);
    o[4] = (T(0.5) * h.rho) * (h.u[E + 2] * bc + h.u[E] * (h.v[J + 2] * h.w[L] + h.v[J] * h.w[L + 2]) + h.xi1 * abc);
}

// changes of the primitives and of the 1-D moments along a change dQ of the
// conserved variables
template <typename T>
struct HalfDelta {
    T rho, du[5], dv[4], dw[4], dxi1;
    T dP[4];  // changes of U, V, W and T (rho: above)
    T dp;     // change of the pressure (set by half_delta only)
};

// the moment changes from the primitive changes (drho, dU, dV, dW, dT)
template <typename T, typename S>
HGKS_HD void half_delta_prim(const HalfSide<T> &h, T drho, T dU, T dV, T dW, T dT, S K, HalfDelta<T> &d)
{
    d.rho = drho;
    d.dP[0] = dU;
    d.dP[1] = dV;
    d.dP[2] = dW;
    d.dP[3] = dT;
#pragma unroll
    for (int n = 0; n < 5; n++) d.du[n] = fmad(h.uU[n], dU, h.uT[n] * dT);
    // <v^0> = 1 and <v^1> = V exactly: their changes are 0 and dV (index 0 is
    // never read, see half_dphi)
    d.dv[0] = T(0.0);
    d.dw[0] = T(0.0);
    d.dv[1] = dV;
    d.dw[1] = dW;
#pragma unroll
    for (int n = 2; n < 4; n++) {
        d.dv[n] = fmad(h.vV[n], dV, h.vT[n] * dT);
        d.dw[n] = fmad(h.wW[n], dW, h.wT[n] * dT);
    }
    d.dxi1 = T(K) * dT;
}

template <typename T, typename S>
HGKS_HD void half_delta(const HalfSide<T> &h, const T dQ[5], S gm1, S K, HalfDelta<T> &d)
{
    const T dU = fmad(-h.U[0], dQ[0], dQ[1]) * h.ir;
    const T dV = fmad(-h.U[1], dQ[0], dQ[2]) * h.ir;
    const T dW = fmad(-h.U[2], dQ[0], dQ[3]) * h.ir;
    const T Ud = fmad(h.U[2], dQ[3], fmad(h.U[1], dQ[2], h.U[0] * dQ[1]));
    const T dp = T(gm1) * fmad(T(0.5) * h.uu, dQ[0], dQ[4] - Ud);
    const T dT = fmad(-h.Tm, dQ[0], dp) * h.ir;
    half_delta_prim(h, dQ[0], dU, dV, dW, dT, K, d);
    d.dp = dp;
}

// Minus the time change of a side's primitives, summed over the three
// directions from their primitive changes.  The Euler equations in primitive
// form (R = 1, p = rho T) give
//   d_t rho = -(U.grad rho + rho div U),   d_t U_k = -(U.grad U_k + d_k p / rho),
//   d_t T = -(U.grad T + (gamma - 1) T div U),
// the linear map d_t Q = -sum_d DF_d(Q)[d_d Q] (the Euler-flux Jacobians)
// written in primitives.  Direction D adds its terms; D = 0 starts the sums.
template <typename T>
struct HalfRate {
    T rho, U[3], Tm;
};

template <int D, typename T, typename S>
HGKS_HD void half_rate_add(const HalfSide<T> &h, const HalfDelta<T> &d, S gm1, HalfRate<T> &r)
{
    const T Ud = h.U[D], div = d.dP[D];  // U_D and d_D U_D
    const T gT = T(gm1) * h.Tm;
    if constexpr (D == 0) {
        r.rho = fmad(Ud, d.rho, h.rho * div);
#pragma unroll
        for (int k = 0; k < 3; k++) r.U[k] = k == D ? fmad(Ud, d.dP[k], h.ir * d.dp) : Ud * d.dP[k];
        r.Tm = fmad(Ud, d.dP[3], gT * div);
    } else {
        r.rho = fmad(Ud, d.rho, fmad(h.rho, div, r.rho));
#pragma unroll
        for (int k = 0; k < 3; k++) r.U[k] = fmad(Ud, d.dP[k], k == D ? fmad(h.ir, d.dp, r.U[k]) : r.U[k]);
        r.Tm = fmad(Ud, d.dP[3], fmad(gT, div, r.Tm));
    }
}

// the side's moment changes along its time slope
template <typename T, typename S>
HGKS_HD void half_delta_time(const HalfSide<T> &h, const HalfRate<T> &r, S K, HalfDelta<T> &d)
{
    half_delta_prim(h, -r.rho, -r.U[0], -r.U[1], -r.U[2], -r.Tm, K, d);
}

// tangential factor X = <v^j><w^l> of a monomial and its change dX; the exact
// <v^0> = <w^0> = 1 (change 0) is taken out at compile time, so X = 1 (j = l = 0)
// never reaches here
template <int j, int l, typename T>
HGKS_HD void vw_factor(const HalfSide<T> &h, const HalfDelta<T> &d, T &X, T &dX)
{
    static_assert(j > 0 || l > 0, "X = 1 is handled by the caller");
    if constexpr (j == 0) {
        X = h.w[l];
        dX = d.dw[l];
    } else if constexpr (l == 0) {
        X = h.v[j];
        dX = d.dv[j];
    } else {
        X = h.v[j] * h.w[l];
        dX = fmad(d.dv[j], h.w[l], h.v[j] * d.dw[l]);
    }
}

// D(rho a X) = (drho a + rho da) X + (rho a) dX = al X + be dX for a = <u^k>_sigma
template <int j, int l, typename T>
HGKS_HD T dphi_term(const HalfSide<T> &h, const HalfDelta<T> &d, T al, T be)
{
    if constexpr (j == 0 && l == 0) {
        return al;
    } else {
        T X, dX;
        vw_factor<j, l>(h, d, X, dX);
        return fmad(al, X, be * dX);
    }
}

// directional derivative of Phi_m along the change d (product rule)
template <int E, int J, int L, typename T>
HGKS_HD void half_dphi(const HalfSide<T> &h, const HalfDelta<T> &d, T o[5])
{
    // a = <u^(E+k)>_sigma, k = 0, 1, 2: al_k = D(rho a) and be_k = rho a
    T al[3], be[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        al[k] = fmad(d.rho, h.u[E + k], h.rho * d.du[E + k]);
        be[k] = h.rho * h.u[E + k];
    }
    o[0] = dphi_term<J, L>(h, d, al[0], be[0]);
    o[1] = dphi_term<J, L>(h, d, al[1], be[1]);
    o[2] = dphi_term<J + 1, L>(h, d, al[0], be[0]);
    o[3] = dphi_term<J, L + 1>(h, d, al[0], be[0]);
    const T p4 = dphi_term<J, L>(h, d, al[2], be[2]);
    const T p5 = dphi_term<J + 2, L>(h, d, al[0], be[0]);
    const T p6 = dphi_term<J, L + 2>(h, d, al[0], be[0]);
    // xi^2 term: D(rho <xi^2> a X) = <xi^2> D(rho a X) + (rho a X) d<xi^2>
    T v0;
    if constexpr (J == 0 && L == 0) {
        v0 = be[0];
    } else {
        T X, dX;
        vw_factor<J, L>(h, d, X, dX);
        v0 = be[0] * X;
    }
    o[4] = T(0.5) * fmad(v0, d.dxi1, fmad(h.xi1, o[0], p4 + p5 + p6));
}

// all half-range terms of one side: Q0 part and B4 (values), W5, B5 (slopes),
// W6, B6 (time slope), summed over the three derivative directions
template <typename T, typename S>
HGKS_HD void half_terms(const T Q[5], const T dq[3][5], S gm1, S K, bool pos, T q0[5], T b4[5],
                        T w5[5], T b5[5], T w6[5], T b6[5])
{
    HalfSide<T> h;
    half_side_setup(Q, gm1, K, pos, h);
    half_phi<0, 0, 0>(h, q0);
    half_phi<1, 0, 0>(h, b4);
    HalfDelta<T> dd;
    HalfRate<T> rt;
    T s[5];
    half_delta(h, dq[0], gm1, K, dd);  // normal direction: m = u (W5), u^2 (B5)
    half_dphi<1, 0, 0>(h, dd, w5);
    half_dphi<2, 0, 0>(h, dd, b5);
    half_rate_add<0>(h, dd, gm1, rt);
    half_delta(h, dq[1], gm1, K, dd);  // first tangential: m = v, u v
    half_dphi<0, 1, 0>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) w5[c] += s[c];
    half_dphi<1, 1, 0>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) b5[c] += s[c];
    half_rate_add<1>(h, dd, gm1, rt);
    half_delta(h, dq[2], gm1, K, dd);  // second tangential: m = w, u w
    half_dphi<0, 0, 1>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) w5[c] += s[c];
    half_dphi<1, 0, 1>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) b5[c] += s[c];
    half_rate_add<2>(h, dd, gm1, rt);
    // time slope of the side's Maxwellian
    half_delta_time(h, rt, K, dd);
    half_dphi<0, 0, 0>(h, dd, w6);
    half_dphi<1, 0, 0>(h, dd, b6);
}

// GKS flux through a unit-area point of an interface (rotated frame: velocity
// components normal, t1, t2).  dl/dr/d0[d][c] are physical derivatives of the
// conservative variables along (normal, t1, t2).  Writes F^n and dF^n/dt
// obtained from the time integrals over [0, dt] and [0, dt/2] (Eq. "expansion-1").
template <typename T>
__host__ __device__ __noinline__ void gks_point_flux(const T Ql[5], const T Qr[5], const T dl[3][5],
                                                          const T dr[3][5], const T d0[3][5], const Params &P, T dt,
                                                          T Fn[5], T dFn[5])
{
    const double gm1 = P.gamma - 1.0, K = P.K;
    // half-range terms of the two sides (values and directional derivatives)
    T ql[5], b4l[5], w5l[5], b5l[5], w6l[5], b6l[5], qr[5], b4r[5], w5r[5], b5r[5], w6r[5], b6r[5];
    half_terms(Ql, dl, gm1, K, true, ql, b4l, w5l, b5l, w6l, b6l);
    half_terms(Qr, dr, gm1, K, false, qr, b4r, w5r, b5r, w6r, b6r);
    // equilibrium state from the compatibility condition
    T Q0[5];
#pragma unroll
    for (int i = 0; i < 5; i++) Q0[i] = ql[i] + qr[i];
    const Gas<T> g0 = gas_of(Q0, gm1);
    const T tau = viscosity(P, g0.Tm) / g0.p;

    // equilibrium terms: B1 = F_n(Q0), B2 = sum_d DH_d(Q0)[d_d Q0], B3 = DF_n(Q0)[d_t Q0],
    // W2 = -d_t Q0 = R0, W3 = d_t Q0
    T B1[5], B2[5], B3[5], R0[5];
    {
        T s[5];
        B1[0] = Q0[1];
        B1[1] = Q0[1] * g0.U[0] + g0.p;
        B1[2] = Q0[1] * g0.U[1];
        B1[3] = Q0[1] * g0.U[2];
        B1[4] = g0.U[0] * (g0.E + g0.p);
        euler_dflux<0>(g0, d0[0], gm1, R0);
        euler_dflux<1>(g0, d0[1], gm1, s);
#pragma unroll
        for (int c = 0; c < 5; c++) R0[c] += s[c];
        euler_dflux<2>(g0, d0[2], gm1, s);
#pragma unroll
        for (int c = 0; c < 5; c++) R0[c] += s[c];
        T dtQ0[5];
#pragma unroll
        for (int c = 0; c < 5; c++) dtQ0[c] = -R0[c];
        euler_dflux<0>(g0, dtQ0, gm1, B3);
        second_dmoment<0>(g0, d0[0], gm1, K + 5.0, B2);
        second_dmoment<1>(g0, d0[1], gm1, K + 5.0, s);
#pragma unroll
        for (int c = 0; c < 5; c++) B2[c] += s[c];
        second_dmoment<2>(g0, d0[2], gm1, K + 5.0, s);
#pragma unroll
        for (int c = 0; c < 5; c++) B2[c] += s[c];
    }
    T B4[5], B5[5], B6[5], W5[5], W6[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        B4[i] = b4l[i] + b4r[i];
        W5[i] = w5l[i] + w5r[i];
        B5[i] = b5l[i] + b5r[i];
        W6[i] = w6l[i] + w6r[i];
        B6[i] = b6l[i] + b6r[i];
    }
    T W3[5];
#pragma unroll
    for (int i = 0; i < 5; i++) W3[i] = -R0[i];
    const T h2 = heat_of_g(B2, R0, g0), h3 = heat_of_g(B3, W3, g0), h4 = heat_of_g(B4, Q0, g0),
            h5 = heat_of_g(B5, W5, g0), h6 = heat_of_g(B6, W6, g0);

    const T prc = T(1.0 / P.Pr - 1.0);
    // e^{-dt/(2 tau)} once; e^{-dt/tau} is its square
    const T eh = tau > T(0.0) ? T(exp(T(-0.5) * dt / tau)) : T(0.0);
    T I[2][5];
#pragma unroll
    for (int pass = 0; pass < 2; pass++) {
        const T dd = pass == 0 ? dt : T(0.5) * dt;
        const T e = pass == 0 ? eh * eh : eh;
        const T om = T(1.0) - e;
        const T q0 = dd - tau * om;
        const T q1 = tau * (T(2.0) * tau * om - dd - dd * e);
        const T q2 = T(0.5) * dd * dd - tau * dd + tau * tau * om;
        const T q3 = tau * om;
        const T q4 = tau * (T(2.0) * tau * om - dd * e);
        const T q5 = tau * q3;
#pragma unroll
        for (int i = 0; i < 5; i++)
            I[pass][i] = q0 * B1[i] + q1 * B2[i] + q2 * B3[i] + q3 * B4[i] - q4 * B5[i] - q5 * B6[i];
        I[pass][4] += prc * (q1 * h2 + q2 * h3 + q3 * h4 - q4 * h5 - q5 * h6);
    }
    const T idt = T(1.0) / dt;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        Fn[i] = (T(4.0) * I[1][i] - I[0][i]) * idt;
        dFn[i] = T(4.0) * (I[0][i] - T(2.0) * I[1][i]) * idt * idt;
    }
}

}  // namespace hgks
