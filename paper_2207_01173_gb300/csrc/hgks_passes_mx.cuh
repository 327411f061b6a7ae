// hgks_passes_mx.cuh -- the mixed-precision sweep passes (HGKS_MIXED): FP32 reconstruction
// and flux arithmetic, FP64 state, equilibrium state and equilibrium flux.
//
// Where FP64 stays, and why (low-Mach flows lose digits to cancellation):
//   * cell averages, stage sums and the S2O4 update (the k_update kernel) --
//     a step changes rho E by ~1e-6 of its value;
//   * every reconstructed VALUE is an FP64 centre value plus an FP32
//     deviation: WENO-Z and the quartics act on differences from the centre
//     of their stencil, which are small and keep full FP32 relative
//     precision (the nonlinear weights depend on differences only);
//   * the equilibrium state Q0 = (Ql + Qr)/2 + C at each Gauss point: the
//     compatibility correction C is small for smooth data and is evaluated in
//     FP32 as -(DPhi+(Ql) - DPhi-(Qr))[Qr - Ql]/2 (trapezoidal rule for the
//     difference of half-range moment functions whose sum is the identity;
//     error O(|Qr - Ql|^3)), or directly as Phi+(Ql) + Phi-(Qr) when the jump
//     is not small;
//   * the temperature and pressure of Q0 and its Euler flux B1 = F_n(Q0),
//     which carries the pressure whose face-to-face differences drive L.
// Everything else -- slopes, half-range moments, the collision time and the
// non-equilibrium / time-derivative terms, all scaled by tau or dt -- is
// FP32.  The flux becomes F^n = B1 + (4 S(dt/2) - S(dt))/dt and
// dF^n/dt = 4 (S(dt) - 2 S(dt/2))/dt^2 with S the FP32 sum of the small
// terms, because the B1 part of I(delta) is exactly delta B1.
#pragma once
#include "hgks_bodies.cuh"
#include "hgks_kernels.cuh"

namespace hgks {


__host__ __device__ inline int perm_mx(int d, int c)
{
    if (c == 0 || c == 4) return c;
    if (d == 0) return c;
    if (d == 1) return c == 1 ? 2 : (c == 2 ? 1 : 3);
    return c == 1 ? 3 : (c == 2 ? 1 : 2);
}

static __device__ __forceinline__ void bpos(const Box &b, long long t, int p[3])
{
    p[0] = (int)(t % b.E[0]) + b.O[0];
    t /= b.E[0];
    p[1] = (int)(t % b.E[1]) + b.O[1];
    p[2] = (int)(t / b.E[1]) + b.O[2];
}
static __device__ __forceinline__ long long blin(const Box &b, const int p[3])
{
    return ((long long)(p[2] - b.O[2]) * b.E[1] + (p[1] - b.O[1])) * b.E[0] + (p[0] - b.O[0]);
}
static __device__ __forceinline__ long long bstride(const Box &b, int e)
{
    return e == 0 ? 1 : (e == 1 ? (long long)b.E[0] : (long long)b.E[0] * b.E[1]);
}

// ---------------------------------------------------------------------------
// equilibrium state from left/right states (FP64 values)
// ---------------------------------------------------------------------------
// Q0 = Qm + C; hl, hr: half-range setups of Ql (u > 0) and Qr (u < 0) in FP32
static __device__ __forceinline__ void compat_mixed(const double Ql[5], const double Qr[5], const HalfSide<float> &hl,
                                             const HalfSide<float> &hr, double gm1, double K, double Q0[5])
{
    double Qm[5];
    float dq[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        Qm[c] = 0.5 * (Ql[c] + Qr[c]);
        dq[c] = (float)(Qr[c] - Ql[c]);
    }
    const float jump = fabsf(dq[0]) / (float)Qm[0] + fabsf(dq[4]) / (float)Qm[4];
    if (jump < 1e-3f) {
        HalfDelta<float> d;
        float a[5], b[5];
        half_delta(hl, dq, gm1, K, d);
        half_dphi<0, 0, 0>(hl, d, a);  // DPhi+(Ql)[dq]
        half_delta(hr, dq, gm1, K, d);
        half_dphi<0, 0, 0>(hr, d, b);  // DPhi-(Qr)[dq]
#pragma unroll
        for (int c = 0; c < 5; c++) Q0[c] = Qm[c] - 0.5 * (double)(a[c] - b[c]);
    } else {
        float a[5], b[5];
        half_phi<0, 0, 0>(hl, a);
        half_phi<0, 0, 0>(hr, b);
#pragma unroll
        for (int c = 0; c < 5; c++) Q0[c] = (double)a[c] + (double)b[c];
    }
}

// ---------------------------------------------------------------------------
// Gauss-point flux, mixed precision
// ---------------------------------------------------------------------------
static __device__ __noinline__ void gks_point_flux_mixed(const double Ql[5], const double Qr[5], const float dl[3][5],
                                                  const float dr[3][5], const float d0[3][5], const Params &P,
                                                  double dt, double Fn[5], double dFn[5])
{
    const double gm1 = P.gamma - 1.0, K = P.K;
    float qlf[5], qrf[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        qlf[c] = (float)Ql[c];
        qrf[c] = (float)Qr[c];
    }
    // half-range terms of the two sides (FP32)
    HalfSide<float> hl, hr;
    half_side_setup(qlf, gm1, K, true, hl);
    half_side_setup(qrf, gm1, K, false, hr);
    float b4l[5], w5l[5], b5l[5], w6l[5], b6l[5], b4r[5], w5r[5], b5r[5], w6r[5], b6r[5];
    {
        HalfDelta<float> dd;
        float s[5];
        half_phi<1, 0, 0>(hl, b4l);
        half_phi<1, 0, 0>(hr, b4r);
        half_delta(hl, dl[0], gm1, K, dd);
        half_dphi<1, 0, 0>(hl, dd, w5l);
        half_dphi<2, 0, 0>(hl, dd, b5l);
        half_delta(hl, dl[1], gm1, K, dd);
        half_dphi<0, 1, 0>(hl, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) w5l[c] += s[c];
        half_dphi<1, 1, 0>(hl, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) b5l[c] += s[c];
        half_delta(hl, dl[2], gm1, K, dd);
        half_dphi<0, 0, 1>(hl, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) w5l[c] += s[c];
        half_dphi<1, 0, 1>(hl, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) b5l[c] += s[c];
        half_delta(hr, dr[0], gm1, K, dd);
        half_dphi<1, 0, 0>(hr, dd, w5r);
        half_dphi<2, 0, 0>(hr, dd, b5r);
        half_delta(hr, dr[1], gm1, K, dd);
        half_dphi<0, 1, 0>(hr, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) w5r[c] += s[c];
        half_dphi<1, 1, 0>(hr, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) b5r[c] += s[c];
        half_delta(hr, dr[2], gm1, K, dd);
        half_dphi<0, 0, 1>(hr, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) w5r[c] += s[c];
        half_dphi<1, 0, 1>(hr, dd, s);
#pragma unroll
        for (int c = 0; c < 5; c++) b5r[c] += s[c];
        // time slopes of the two sides
        const Gas<float> gl = gas_of(qlf, gm1), gr = gas_of(qrf, gm1);
        float tq[5];
        euler_dtq(gl, dl, gm1, tq);
        half_delta(hl, tq, gm1, K, dd);
        half_dphi<0, 0, 0>(hl, dd, w6l);
        half_dphi<1, 0, 0>(hl, dd, b6l);
        euler_dtq(gr, dr, gm1, tq);
        half_delta(hr, tq, gm1, K, dd);
        half_dphi<0, 0, 0>(hr, dd, w6r);
        half_dphi<1, 0, 0>(hr, dd, b6r);
    }

    // equilibrium state and its Euler flux in FP64
    double Q0[5];
    compat_mixed(Ql, Qr, hl, hr, gm1, K, Q0);
    const double ir0 = 1.0 / Q0[0];
    const double U0 = Q0[1] * ir0, V0 = Q0[2] * ir0, W0 = Q0[3] * ir0;
    const double p0 = gm1 * (Q0[4] - 0.5 * Q0[0] * (U0 * U0 + V0 * V0 + W0 * W0));
    double B1[5];
    B1[0] = Q0[1];
    B1[1] = Q0[1] * U0 + p0;
    B1[2] = Q0[1] * V0;
    B1[3] = Q0[1] * W0;
    B1[4] = U0 * (Q0[4] + p0);

    // FP32: equilibrium slope terms, collision time, the small terms S(delta)
    float q0f[5];
#pragma unroll
    for (int c = 0; c < 5; c++) q0f[c] = (float)Q0[c];
    const Gas<float> g0 = gas_of(q0f, gm1);
    const float T0 = (float)(p0 * ir0);
    const float tau = viscosity(P, T0) / (float)p0;
    float B2[5], B3[5], R0[5], B4m1[5], W5[5], B5[5], W6[5], B6[5];
    {
        float s[5];
        euler_dflux<0>(g0, d0[0], gm1, R0);
        euler_dflux<1>(g0, d0[1], gm1, s);
#pragma unroll
        for (int c = 0; c < 5; c++) R0[c] += s[c];
        euler_dflux<2>(g0, d0[2], gm1, s);
#pragma unroll
        for (int c = 0; c < 5; c++) R0[c] += s[c];
        float dtQ0[5];
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
#pragma unroll
        for (int c = 0; c < 5; c++) {
            B4m1[c] = (b4l[c] + b4r[c]) - (float)B1[c];  // half-range flux minus the equilibrium flux
            W5[c] = w5l[c] + w5r[c];
            B5[c] = b5l[c] + b5r[c];
            W6[c] = w6l[c] + w6r[c];
            B6[c] = b6l[c] + b6r[c];
        }
    }
    // heat fluxes of the terms (the equilibrium carries none; the B4 - B1 term
    // carries that of the half-range part: h(B4, Q0) - h(B1, Q0) = h(B4, Q0))
    float W3[5], Q0f[5], b4s[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        W3[c] = -R0[c];
        Q0f[c] = q0f[c];
        b4s[c] = b4l[c] + b4r[c];
    }
    const float h2 = heat_of_g(B2, R0, g0), h3 = heat_of_g(B3, W3, g0), h4 = heat_of_g(b4s, Q0f, g0),
                h5 = heat_of_g(B5, W5, g0), h6 = heat_of_g(B6, W6, g0);
    const float prc = (float)(1.0 / P.Pr - 1.0);
    const float dtf = (float)dt;
    const float eh = tau > 0.0f ? expf(-0.5f * dtf / tau) : 0.0f;
    float S[2][5];
#pragma unroll
    for (int pass = 0; pass < 2; pass++) {
        const float dd = pass == 0 ? dtf : 0.5f * dtf;
        const float e = pass == 0 ? eh * eh : eh;
        const float om = 1.0f - e;
        const float q1 = tau * (2.0f * tau * om - dd - dd * e);
        const float q2 = 0.5f * dd * dd - tau * dd + tau * tau * om;
        const float q3 = tau * om;
        const float q4 = tau * (2.0f * tau * om - dd * e);
        const float q5 = tau * q3;
#pragma unroll
        for (int i = 0; i < 5; i++)
            S[pass][i] = q1 * B2[i] + q2 * B3[i] + q3 * B4m1[i] - q4 * B5[i] - q5 * B6[i];
        S[pass][4] += prc * (q1 * h2 + q2 * h3 + q3 * h4 - q4 * h5 - q5 * h6);
    }
    const float idt = 1.0f / dtf;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        Fn[i] = B1[i] + (double)((4.0f * S[1][i] - S[0][i]) * idt);
        dFn[i] = (double)(4.0f * (S[0][i] - 2.0f * S[1][i]) * idt * idt);
    }
}

// ---------------------------------------------------------------------------
// pass 1: normal reconstruction (values FP64 = centre + FP32 deviation)
// ---------------------------------------------------------------------------
// fqd[15][nq] doubles: Ql, Qr, Q0 values; fqf[15][nq] floats: dQl, dQr, dQ0 (index units)
static __device__ __forceinline__ void pos_normal_mx(const Params &P, int d, const Box &B,
                                                     const double *__restrict__ q, double *__restrict__ fqd,
                                                     float *__restrict__ fqf, long long t)
{
    const long long nq = box_count(B);
    int p[3];
    bpos(B, t, p);
    int c0[3] = { p[0], p[1], p[2] };
    c0[d] = p[d] - 3;
    const long long base = pidx(P, c0[0], c0[1], c0[2]);
    const long long sd = d == 0 ? 1 : (d == 1 ? P.sy : P.sz);
    double Ql[5], Qr[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        const double *src = q + (long long)perm_mx(d, c) * P.cs + base;
        double X[6];
#pragma unroll
        for (int m = 0; m < 6; m++) X[m] = src[m * sd];
        float xl[5], xr[5];
#pragma unroll
        for (int m = 0; m < 5; m++) {
            xl[m] = (float)(X[m] - X[2]);      // cell f-1 stencil, about its centre
            xr[m] = (float)(X[m + 1] - X[3]);  // cell f stencil
        }
        WenoPrep<float> wl, wr;
        weno_prep(xl, wl);
        weno_prep(xr, wr);
        float lm_l, lm_r, r_l, r_r;
        weno_edge_pair(wl, lm_l, lm_r);
        weno_edge_pair(wr, r_l, r_r);
        Ql[c] = X[2] + (double)lm_r;
        Qr[c] = X[3] + (double)r_l;
        fqd[(0 * 5 + c) * nq + t] = Ql[c];
        fqd[(1 * 5 + c) * nq + t] = Qr[c];
        fqf[(0 * 5 + c) * nq + t] = 2.0f * lm_l + 4.0f * lm_r;  // parabola slopes (centre cancels)
        fqf[(1 * 5 + c) * nq + t] = -4.0f * r_l - 2.0f * r_r;
        fqf[(2 * 5 + c) * nq + t] = (15.0f * (float)(X[3] - X[2]) - (float)(X[4] - X[1])) * (1.0f / 12.0f);
    }
    float qlf[5], qrf[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        qlf[c] = (float)Ql[c];
        qrf[c] = (float)Qr[c];
    }
    HalfSide<float> hl, hr;
    half_side_setup(qlf, P.gamma - 1.0, P.K, true, hl);
    half_side_setup(qrf, P.gamma - 1.0, P.K, false, hr);
    double Q0[5];
    compat_mixed(Ql, Qr, hl, hr, P.gamma - 1.0, P.K, Q0);
#pragma unroll
    for (int c = 0; c < 5; c++) fqd[(2 * 5 + c) * nq + t] = Q0[c];
}

// ---------------------------------------------------------------------------
// pass 2: first tangential direction
// ---------------------------------------------------------------------------
// t1d[2][25][nt] doubles per Gauss line m: WENO values of Ql, Qr (10), quartic
// values of Ql, Qr, Q0 (15); t1f[2][30][nt] floats: WENO of dQl, dQr, dQ0 (15),
// quartic derivatives of Ql, Qr, Q0 (15)
static __device__ __forceinline__ void pos_tan1_mx(const Params &P, int d, const Box &Bt, const Box &Bq,
                                                   const double *__restrict__ fqd, const float *__restrict__ fqf,
                                                   double *__restrict__ t1d, float *__restrict__ t1f, long long t)
{
    const long long nt = box_count(Bt), nq = box_count(Bq);
    int p[3];
    bpos(Bt, t, p);
    const long long base = blin(Bq, p), s1 = bstride(Bq, tdir(d, 0));
    // values: Ql, Qr (WENO + quartic), Q0 (quartic)
#pragma unroll 1
    for (int v = 0; v < 3; v++) {
#pragma unroll
        for (int c = 0; c < 5; c++) {
            const double *src = fqd + (v * 5 + c) * nq + base;
            double X[5];
#pragma unroll
            for (int j = 0; j < 5; j++) X[j] = src[(j - 2) * s1];
            float x[5];
#pragma unroll
            for (int j = 0; j < 5; j++) x[j] = (float)(X[j] - X[2]);
            if (v < 2) {
                WenoPrep<float> W;
                weno_prep(x, W);
                float vm, vp;
                weno_gauss_pair(W, vm, vp);
                t1d[(0 * 25 + v * 5 + c) * nt + t] = X[2] + (double)vm;
                t1d[(1 * 25 + v * 5 + c) * nt + t] = X[2] + (double)vp;
            }
            float qm, qp, dm, dp;
            quartic_value_pair(x, qm, qp);
            quartic_deriv_pair(x, dm, dp);
            t1d[(0 * 25 + 10 + v * 5 + c) * nt + t] = X[2] + (double)qm;
            t1d[(1 * 25 + 10 + v * 5 + c) * nt + t] = X[2] + (double)qp;
            t1f[(0 * 30 + 15 + v * 5 + c) * nt + t] = dm;
            t1f[(1 * 30 + 15 + v * 5 + c) * nt + t] = dp;
        }
    }
    // slopes: WENO-Z in FP32
#pragma unroll 1
    for (int w = 0; w < 3; w++) {
#pragma unroll
        for (int c = 0; c < 5; c++) {
            const float *src = fqf + (w * 5 + c) * nq + base;
            float x[5];
#pragma unroll
            for (int j = 0; j < 5; j++) x[j] = src[(j - 2) * s1];
            WenoPrep<float> W;
            weno_prep(x, W);
            float vm, vp;
            weno_gauss_pair(W, vm, vp);
            t1f[(0 * 30 + w * 5 + c) * nt + t] = vm;
            t1f[(1 * 30 + w * 5 + c) * nt + t] = vp;
        }
    }
}

// ---------------------------------------------------------------------------
// pass 3: second tangential direction and the four Gauss-point fluxes
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void pos_flux_mx(const Params &P, int d, const Box &Bf, const Box &Bt,
                                                   const double *__restrict__ t1d, const float *__restrict__ t1f,
                                                   double *__restrict__ F, double dt, long long t)
{
    const long long nf = box_count(Bf), nt = box_count(Bt);
    int p[3];
    bpos(Bf, t, p);
    const int e1 = tdir(d, 0), e2 = tdir(d, 1);
    const int f = p[d], a = p[e1], b = p[e2];
    const long long base = blin(Bt, p), s2 = bstride(Bt, e2);
    const float ihn = (float)(1.0 / (d == 1 ? P.my_face[f] : P.h[d]));
    double area;
    if (d == 0) area = P.hy_cell[a] * P.h[2];
    else if (d == 1) area = P.h[0] * P.h[2];
    else area = P.h[0] * P.hy_cell[b];

    double Fs[5] = { 0, 0, 0, 0, 0 }, dFs[5] = { 0, 0, 0, 0, 0 };
#pragma unroll 1
    for (int m = 0; m < 2; m++) {
        const float ih1 = (float)(1.0 / (e1 == 1 ? P.my_gp[2 * a + m] : P.h[e1]));
        double gq[2][10];
        float gs[2][15], gd1[2][15], gd2[2][15];
        // values Ql, Qr at the two Gauss points of this line
#pragma unroll 1
        for (int k = 0; k < 10; k++) {
            const double *src = t1d + (m * 25 + k) * nt + base;
            double X[5];
#pragma unroll
            for (int j = 0; j < 5; j++) X[j] = src[(j - 2) * s2];
            float x[5];
#pragma unroll
            for (int j = 0; j < 5; j++) x[j] = (float)(X[j] - X[2]);
            WenoPrep<float> W;
            weno_prep(x, W);
            float vm, vp;
            weno_gauss_pair(W, vm, vp);
            gq[0][k] = X[2] + (double)vm;
            gq[1][k] = X[2] + (double)vp;
        }
        // derivatives along the second tangential direction of the quartic values
#pragma unroll 1
        for (int k = 0; k < 15; k++) {
            const double *src = t1d + (m * 25 + 10 + k) * nt + base;
            double X[5];
#pragma unroll
            for (int j = 0; j < 5; j++) X[j] = src[(j - 2) * s2];
            float x[5];
#pragma unroll
            for (int j = 0; j < 5; j++) x[j] = (float)(X[j] - X[2]);
            quartic_deriv_pair(x, gd2[0][k], gd2[1][k]);
        }
        // normal slopes (WENO) and first-direction derivatives (quartic value)
#pragma unroll 1
        for (int k = 0; k < 15; k++) {
            const float *ss = t1f + (m * 30 + k) * nt + base;
            const float *sd = t1f + (m * 30 + 15 + k) * nt + base;
            float x[5], y[5];
#pragma unroll
            for (int j = 0; j < 5; j++) {
                x[j] = ss[(j - 2) * s2];
                y[j] = sd[(j - 2) * s2];
            }
            WenoPrep<float> W;
            weno_prep(x, W);
            weno_gauss_pair(W, gs[0][k], gs[1][k]);
            quartic_value_pair(y, gd1[0][k], gd1[1][k]);
        }
#pragma unroll 1
        for (int n = 0; n < 2; n++) {
            const float ih2 = (float)(1.0 / (e2 == 1 ? P.my_gp[2 * b + n] : P.h[e2]));
            float dl[3][5], dr[3][5], d0[3][5];
#pragma unroll
            for (int c = 0; c < 5; c++) {
                dl[0][c] = gs[n][c] * ihn;
                dr[0][c] = gs[n][5 + c] * ihn;
                d0[0][c] = gs[n][10 + c] * ihn;
                dl[1][c] = gd1[n][c] * ih1;
                dr[1][c] = gd1[n][5 + c] * ih1;
                d0[1][c] = gd1[n][10 + c] * ih1;
                dl[2][c] = gd2[n][c] * ih2;
                dr[2][c] = gd2[n][5 + c] * ih2;
                d0[2][c] = gd2[n][10 + c] * ih2;
            }
            double Fn[5], dFn[5];
            gks_point_flux_mixed(&gq[n][0], &gq[n][5], dl, dr, d0, P, dt, Fn, dFn);
#pragma unroll
            for (int c = 0; c < 5; c++) {
                Fs[c] += 0.25 * Fn[c];
                dFs[c] += 0.25 * dFn[c];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 5; c++) {
        F[(long long)perm_mx(d, c) * nf + t] = Fs[c] * area;
        F[(long long)(5 + perm_mx(d, c)) * nf + t] = dFs[c] * area;
    }
}

}  // namespace hgks
