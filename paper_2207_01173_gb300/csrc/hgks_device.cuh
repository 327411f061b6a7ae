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
//   * micro-slopes from the moment equations solved in central variables
//     c = u - U (closed-form inverse of the 5x5 moment matrix).
// The arithmetic routines are templates on the scalar type T (double on the
// device; a host operation-counting type instantiates the same code to count
// the scheme's floating-point work).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define HGKS_HD __host__ __device__ __forceinline__

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
    W.x0 = X[2];
    W.c2[0] = 0.5 * (X[0] - 2.0 * X[1] + X[2]);
    W.c1[0] = 0.5 * (X[0] - 4.0 * X[1] + 3.0 * X[2]);
    W.c2[1] = 0.5 * (X[1] - 2.0 * X[2] + X[3]);
    W.c1[1] = 0.5 * (X[3] - X[1]);
    W.c2[2] = 0.5 * (X[2] - 2.0 * X[3] + X[4]);
    W.c1[2] = 0.5 * (-3.0 * X[2] + 4.0 * X[3] - X[4]);
    T b[3];
#pragma unroll
    for (int k = 0; k < 3; k++) b[k] = W.c1[k] * W.c1[k] + (13.0 / 3.0) * W.c2[k] * W.c2[k] + WENO_EPS;
    T tau5 = fabs(b[0] - b[2]);
    W.cw[0] = (b[0] + tau5) * b[1] * b[2];
    W.cw[1] = (b[1] + tau5) * b[0] * b[2];
    W.cw[2] = (b[2] + tau5) * b[0] * b[1];
}

// value at the right (+1/2) or left (-1/2) cell edge; linear weights (1,6,3)/10 mirrored
template <typename T>
HGKS_HD T weno_edge(const WenoPrep<T> &W, int right)
{
    double d0 = right ? 0.1 : 0.3, d2 = right ? 0.3 : 0.1, s = right ? 0.5 : -0.5;
    T a0 = d0 * W.cw[0], a1 = 0.6 * W.cw[1], a2 = d2 * W.cw[2];
    T p0 = W.x0 + s * W.c1[0] + W.c2[0] * (1.0 / 6.0);
    T p1 = W.x0 + s * W.c1[1] + W.c2[1] * (1.0 / 6.0);
    T p2 = W.x0 + s * W.c1[2] + W.c2[2] * (1.0 / 6.0);
    return (a0 * p0 + a1 * p1 + a2 * p2) / (a0 + a1 + a2);
}

// value at the Gauss abscissa -sqrt(3)/6 (plus = 0) or +sqrt(3)/6 (plus = 1)
template <typename T>
HGKS_HD T weno_gauss(const WenoPrep<T> &W, int plus)
{
    double d0 = plus ? HGKS_DGL : HGKS_DGR, d2 = plus ? HGKS_DGR : HGKS_DGL;
    double s = plus ? HGKS_GAUSS : -HGKS_GAUSS;
    T a0 = d0 * W.cw[0], a1 = HGKS_DGC * W.cw[1], a2 = d2 * W.cw[2];
    T num = a0 * W.c1[0] + a1 * W.c1[1] + a2 * W.c1[2];
    return W.x0 + s * num / (a0 + a1 + a2);
}

// quartic through five cell averages: point value and derivative (index units)
// at -sqrt(3)/6 (plus = 0) or +sqrt(3)/6 (plus = 1).
// value = E.X +- sqrt3 O.X,  E = (-1/4320, 1/1080, 719/720, 1/1080, -1/4320),
//                           O = (7/432, -25/216, 0, 25/216, -7/432)
// deriv = C.X -+ sqrt3 S.X,  C = (1/12, -2/3, 0, 2/3, -1/12),
//                           S = (1/54, -13/54, 24/54, -13/54, 1/54)
template <typename T>
HGKS_HD T quartic_value(const T X[5], int plus)
{
    T e = (-1.0 / 4320.0) * (X[0] + X[4]) + (1.0 / 1080.0) * (X[1] + X[3]) + (719.0 / 720.0) * X[2];
    T o = (7.0 / 432.0) * (X[0] - X[4]) + (25.0 / 216.0) * (X[3] - X[1]);
    return plus ? e + HGKS_SQ3 * o : e - HGKS_SQ3 * o;
}
template <typename T>
HGKS_HD T quartic_deriv(const T X[5], int plus)
{
    T c = (1.0 / 12.0) * (X[0] - X[4]) + (2.0 / 3.0) * (X[3] - X[1]);
    T s = (1.0 / 54.0) * (X[0] + X[4]) - (13.0 / 54.0) * (X[1] + X[3]) + (24.0 / 54.0) * X[2];
    return plus ? c - HGKS_SQ3 * s : c + HGKS_SQ3 * s;
}

// ---------------------------------------------------------------------------
// Maxwellian moments and the gas-kinetic flux
// ---------------------------------------------------------------------------
template <typename T>
struct Prim {
    T rho, U, V, W, lam;
};

template <typename T>
HGKS_HD Prim<T> prim_of(const T Q[5], double K)
{
    Prim<T> g;
    T ir = 1.0 / Q[0];
    g.rho = Q[0];
    g.U = Q[1] * ir;
    g.V = Q[2] * ir;
    g.W = Q[3] * ir;
    T eint = Q[4] - 0.5 * Q[0] * (g.U * g.U + g.V * g.V + g.W * g.W);
    g.lam = (K + 3.0) * Q[0] / (4.0 * eint);
    return g;
}

// full-range normalised moments <x^n>, n < N, of a Gaussian with mean U
template <int N, typename T>
HGKS_HD void mom_full(T U, T i2l, T *m)
{
    m[0] = 1.0;
    m[1] = U;
#pragma unroll
    for (int n = 0; n + 2 < N; n++) m[n + 2] = U * m[n + 1] + (double)(n + 1) * i2l * m[n];
}

// half-range moments over u > 0 (pos) or u < 0
template <int N, typename T>
HGKS_HD void mom_half(T U, T lam, T i2l, bool pos, T *m)
{
    const double inv_2sqrtpi = 0.28209479177387814347; // 1 / (2 sqrt(pi))
    T sl = sqrt(lam);
    T e = exp(-lam * U * U) * inv_2sqrtpi / sl;
    if (pos) {
        m[0] = 0.5 * erfc(-sl * U);
        m[1] = U * m[0] + e;
    } else {
        m[0] = 0.5 * erfc(sl * U);
        m[1] = U * m[0] - e;
    }
#pragma unroll
    for (int n = 0; n + 2 < N; n++) m[n + 2] = U * m[n + 1] + (double)(n + 1) * i2l * m[n];
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
    o[4] = 0.5 * (m.u[A + 2] * m.v[B] * m.w[C] + m.u[A] * m.v[B + 2] * m.w[C] + m.u[A] * m.v[B] * m.w[C + 2]
                  + uvw * m.xi1);
}

// <a(u) psi_i u^A v^B w^C>, a(u) = a0 + a1 u + a2 v + a3 w + a4 (u^2 + v^2 + w^2 + xi^2)/2
template <int A, int B, int C, typename T>
HGKS_HD void mom_a(const Mom<T> &m, const T a[5], T o[5])
{
    T t[5];
    psi_mom<A, B, C>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) o[i] = a[0] * t[i];
    psi_mom<A + 1, B, C>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) o[i] += a[1] * t[i];
    psi_mom<A, B + 1, C>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) o[i] += a[2] * t[i];
    psi_mom<A, B, C + 1>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) o[i] += a[3] * t[i];
    // psi_5 part: (u^2 + v^2 + w^2)/2 and xi^2/2
    T s[5];
    psi_mom<A + 2, B, C>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) s[i] = t[i];
    psi_mom<A, B + 2, C>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) s[i] += t[i];
    psi_mom<A, B, C + 2>(m, t);
#pragma unroll
    for (int i = 0; i < 5; i++) s[i] += t[i];
    // xi^2 psi_i u^A v^B w^C: psi_0..3 carry no xi; psi_4 carries xi^2/2
    psi_mom<A, B, C>(m, t);
    T uvw = m.u[A] * m.v[B] * m.w[C];
#pragma unroll
    for (int i = 0; i < 4; i++) s[i] += m.xi1 * t[i];
    s[4] += 0.5 * (m.xi1 * (m.u[A + 2] * m.v[B] * m.w[C] + m.u[A] * m.v[B + 2] * m.w[C]
                            + m.u[A] * m.v[B] * m.w[C + 2]) + m.xi2 * uvw);
#pragma unroll
    for (int i = 0; i < 5; i++) o[i] += 0.5 * a[4] * s[i];
}

// <a psi> = rho b for a Maxwellian (U, V, W, lambda):
// a5 = 8 lam^2/(K+3) (b5 - U.b_mom + b1 (|U|^2 - E)),  E = |U|^2/2 + (K+3)/(4 lam)
// a2..4 = 2 lam (b_mom - U b1) - a5 U,  a1 = b1 - U.a_mom - a5 E
template <typename T>
HGKS_HD void micro_slope(const T b[5], const Prim<T> &g, double K, T a[5])
{
    T uu = g.U * g.U + g.V * g.V + g.W * g.W;
    T E = 0.5 * uu + (K + 3.0) / (4.0 * g.lam);
    T tl = 2.0 * g.lam;
    a[4] = 2.0 * tl * tl / (K + 3.0) * (b[4] - g.U * b[1] - g.V * b[2] - g.W * b[3] + b[0] * (uu - E));
    a[1] = tl * (b[1] - g.U * b[0]) - a[4] * g.U;
    a[2] = tl * (b[2] - g.V * b[0]) - a[4] * g.V;
    a[3] = tl * (b[3] - g.W * b[0]) - a[4] * g.W;
    a[0] = b[0] - g.U * a[1] - g.V * a[2] - g.W * a[3] - a[4] * E;
}

template <typename T>
HGKS_HD T viscosity(const Params &P, T Tm)
{
    return P.visc_kind == 1 ? P.mu_ref * pow(Tm / P.T_ref, P.omega) : T(P.mu_ref);
}

// heat flux about U0 of a term with flux moments B (of u psi) and moments W (of psi):
// q = int (u - U0) (|c|^2 + xi^2)/2 f, c = velocity relative to (U0, V0, W0)
template <typename T>
HGKS_HD T heat_of(const T B[5], const T W[5], const Prim<T> &g0)
{
    T U0 = g0.U, V0 = g0.V, W0 = g0.W, uu = U0 * U0 + V0 * V0 + W0 * W0;
    return B[4] - U0 * B[1] - V0 * B[2] - W0 * B[3] + 0.5 * uu * B[0]
         - U0 * W[4] + U0 * U0 * W[1] + U0 * V0 * W[2] + U0 * W0 * W[3] - 0.5 * U0 * uu * W[0];
}

// GKS flux through a unit-area point of an interface (rotated frame: velocity
// components normal, t1, t2).  dl/dr/d0[d][c] are physical derivatives of the
// conservative variables along (normal, t1, t2).  Writes F^n and dF^n/dt
// obtained from the time integrals over [0, dt] and [0, dt/2] (Eq. "expansion-1").
template <typename T>
__host__ __device__ __noinline__ void gks_point_flux(const T Ql[5], const T Qr[5], const T dl[3][5], const T dr[3][5],
                                                     const T d0[3][5], const Params &P, T dt, T Fn[5], T dFn[5])
{
    const double K = P.K;
    Prim<T> gl = prim_of(Ql, K), gr = prim_of(Qr, K);
    T il = 0.5 / gl.lam, ir = 0.5 / gr.lam;
    T ulf[7], ulp[7], vl[6], wl[6], urf[7], urn[7], vr[6], wr[6];
    mom_full<7>(gl.U, il, ulf);
    mom_half<7>(gl.U, gl.lam, il, true, ulp);
    mom_full<6>(gl.V, il, vl);
    mom_full<6>(gl.W, il, wl);
    mom_full<7>(gr.U, ir, urf);
    mom_half<7>(gr.U, gr.lam, ir, false, urn);
    mom_full<6>(gr.V, ir, vr);
    mom_full<6>(gr.W, ir, wr);
    Mom<T> Ml_f{ulf, vl, wl, K * il, K * (K + 2.0) * il * il};
    Mom<T> Ml_p{ulp, vl, wl, Ml_f.xi1, Ml_f.xi2};
    Mom<T> Mr_f{urf, vr, wr, K * ir, K * (K + 2.0) * ir * ir};
    Mom<T> Mr_n{urn, vr, wr, Mr_f.xi1, Mr_f.xi2};

    // equilibrium state from the compatibility condition
    T Q0[5], t5[5];
    psi_mom<0, 0, 0>(Ml_p, Q0);
    psi_mom<0, 0, 0>(Mr_n, t5);
#pragma unroll
    for (int i = 0; i < 5; i++) Q0[i] = gl.rho * Q0[i] + gr.rho * t5[i];
    Prim<T> g0 = prim_of(Q0, K);
    T i0 = 0.5 / g0.lam;
    T u0[7], v0[6], w0[6];
    mom_full<7>(g0.U, i0, u0);
    mom_full<6>(g0.V, i0, v0);
    mom_full<6>(g0.W, i0, w0);
    Mom<T> M0{u0, v0, w0, K * i0, K * (K + 2.0) * i0 * i0};
    const T T0 = i0, p0 = g0.rho * i0;
    const T tau = viscosity(P, T0) / p0;

    // spatial micro-slopes a = M^{-1} dQ / rho
    T al[3][5], ar[3][5], ab[3][5];
    {
        const T rl = 1.0 / gl.rho, rr = 1.0 / gr.rho, r0 = 1.0 / g0.rho;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            T b[5];
#pragma unroll
            for (int c = 0; c < 5; c++) b[c] = dl[d][c] * rl;
            micro_slope(b, gl, K, al[d]);
#pragma unroll
            for (int c = 0; c < 5; c++) b[c] = dr[d][c] * rr;
            micro_slope(b, gr, K, ar[d]);
#pragma unroll
            for (int c = 0; c < 5; c++) b[c] = d0[d][c] * r0;
            micro_slope(b, g0, K, ab[d]);
        }
    }
    // time slopes from <a.u + A> = 0 (full-range moments)
    T Al[5], Ar[5], Ab[5], R0[5];
    {
        T s[5], t[5];
        mom_a<1, 0, 0>(Ml_f, al[0], s);
        mom_a<0, 1, 0>(Ml_f, al[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) s[i] += t[i];
        mom_a<0, 0, 1>(Ml_f, al[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) s[i] = -(s[i] + t[i]);
        micro_slope(s, gl, K, Al);
        mom_a<1, 0, 0>(Mr_f, ar[0], s);
        mom_a<0, 1, 0>(Mr_f, ar[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) s[i] += t[i];
        mom_a<0, 0, 1>(Mr_f, ar[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) s[i] = -(s[i] + t[i]);
        micro_slope(s, gr, K, Ar);
        mom_a<1, 0, 0>(M0, ab[0], R0);
        mom_a<0, 1, 0>(M0, ab[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) R0[i] += t[i];
        mom_a<0, 0, 1>(M0, ab[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) { R0[i] += t[i]; s[i] = -R0[i]; }
        micro_slope(s, g0, K, Ab);
    }

    // flux moments of the six terms (B) and conserved moments (W) for the heat flux
    T B[6][5], W5[5], W6[5];
    {
        T t[5];
        psi_mom<1, 0, 0>(M0, B[0]);
        mom_a<2, 0, 0>(M0, ab[0], B[1]);
        mom_a<1, 1, 0>(M0, ab[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) B[1][i] += t[i];
        mom_a<1, 0, 1>(M0, ab[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) B[1][i] += t[i];
        mom_a<1, 0, 0>(M0, Ab, B[2]);
#pragma unroll
        for (int i = 0; i < 5; i++) { B[0][i] *= g0.rho; B[1][i] *= g0.rho; B[2][i] *= g0.rho; }

        T x[5], y[5];
        psi_mom<1, 0, 0>(Ml_p, x);
        psi_mom<1, 0, 0>(Mr_n, y);
#pragma unroll
        for (int i = 0; i < 5; i++) B[3][i] = gl.rho * x[i] + gr.rho * y[i];

        mom_a<2, 0, 0>(Ml_p, al[0], x);
        mom_a<1, 1, 0>(Ml_p, al[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) x[i] += t[i];
        mom_a<1, 0, 1>(Ml_p, al[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) x[i] += t[i];
        mom_a<2, 0, 0>(Mr_n, ar[0], y);
        mom_a<1, 1, 0>(Mr_n, ar[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) y[i] += t[i];
        mom_a<1, 0, 1>(Mr_n, ar[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) { y[i] += t[i]; B[4][i] = gl.rho * x[i] + gr.rho * y[i]; }

        mom_a<1, 0, 0>(Ml_p, Al, x);
        mom_a<1, 0, 0>(Mr_n, Ar, y);
#pragma unroll
        for (int i = 0; i < 5; i++) B[5][i] = gl.rho * x[i] + gr.rho * y[i];

        mom_a<1, 0, 0>(Ml_p, al[0], x);
        mom_a<0, 1, 0>(Ml_p, al[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) x[i] += t[i];
        mom_a<0, 0, 1>(Ml_p, al[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) x[i] += t[i];
        mom_a<1, 0, 0>(Mr_n, ar[0], y);
        mom_a<0, 1, 0>(Mr_n, ar[1], t);
#pragma unroll
        for (int i = 0; i < 5; i++) y[i] += t[i];
        mom_a<0, 0, 1>(Mr_n, ar[2], t);
#pragma unroll
        for (int i = 0; i < 5; i++) { y[i] += t[i]; W5[i] = gl.rho * x[i] + gr.rho * y[i]; }

        mom_a<0, 0, 0>(Ml_p, Al, x);
        mom_a<0, 0, 0>(Mr_n, Ar, y);
#pragma unroll
        for (int i = 0; i < 5; i++) W6[i] = gl.rho * x[i] + gr.rho * y[i];
    }
    // heat-flux moments of terms 2..6 (term 1, the equilibrium, carries none)
    T W2[5], W3[5];
#pragma unroll
    for (int i = 0; i < 5; i++) { W2[i] = g0.rho * R0[i]; W3[i] = -W2[i]; }
    const T h2 = heat_of(B[1], W2, g0), h3 = heat_of(B[2], W3, g0), h4 = heat_of(B[3], Q0, g0),
                 h5 = heat_of(B[4], W5, g0), h6 = heat_of(B[5], W6, g0);

    const double prc = 1.0 / P.Pr - 1.0;
    T I[2][5];
#pragma unroll
    for (int pass = 0; pass < 2; pass++) {
        const T dd = pass == 0 ? dt : 0.5 * dt;
        T e = tau > 0.0 ? T(exp(-dd / tau)) : T(0.0);
        T q0 = dd - tau * (1.0 - e);
        T q1 = 2.0 * tau * tau * (1.0 - e) - tau * dd - tau * dd * e;
        T q2 = 0.5 * dd * dd - tau * dd + tau * tau * (1.0 - e);
        T q3 = tau * (1.0 - e);
        T q4 = 2.0 * tau * tau * (1.0 - e) - tau * dd * e;
        T q5 = tau * q3;
#pragma unroll
        for (int i = 0; i < 5; i++)
            I[pass][i] = q0 * B[0][i] + q1 * B[1][i] + q2 * B[2][i] + q3 * B[3][i] - q4 * B[4][i] - q5 * B[5][i];
        T hq = q1 * h2 + q2 * h3 + q3 * h4 - q4 * h5 - q5 * h6;
        I[pass][4] += prc * hq;
    }
    const T idt = 1.0 / dt;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        Fn[i] = (4.0 * I[1][i] - I[0][i]) * idt;
        dFn[i] = 4.0 * (I[0][i] - 2.0 * I[1][i]) * idt * idt;
    }
}

}  // namespace hgks
