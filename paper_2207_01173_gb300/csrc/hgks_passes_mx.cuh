// hgks_passes_mx.cuh -- the mixed-precision sweep passes (HGKS_MIXED): FP32
// reconstruction and flux arithmetic, FP64 state and update, float-float
// (two-FP32, ~48-bit) values wherever FP32 alone would lose digits.
//
// Where the extra precision stays, and why (low-Mach flows lose digits to
// cancellation: a step changes rho E by ~1e-6 of its value, and the flux
// differences of neighbouring faces cancel all but ~h/L of the flux):
//   * cell averages, stage sums and the S2O4 update (k_update) -- FP64;
//   * every reconstructed VALUE -- float-float.  Before each stage the state
//     is split once into hi + lo FP32 planes (k_split_mx), so the passes need
//     no FP64 instruction: WENO-Z and the quartics act on differences from
//     the centre of their stencil, formed as (hi_j - hi_c) + (lo_j - lo_c),
//     which keep full FP32 relative precision (the nonlinear weights depend
//     on differences only), and a value is the centre pair plus that FP32
//     deviation;
//   * the equilibrium state Q0 = (Ql + Qr)/2 + C at each Gauss point: the
//     compatibility correction C is small for smooth data and is evaluated in
//     FP32 as -(DPhi+(Ql) - DPhi-(Qr))[Qr - Ql]/2 (trapezoidal rule for the
//     difference of half-range moment functions whose sum is the identity;
//     error O(|Qr - Ql|^3)), or directly as Phi+(Ql) + Phi-(Qr) when the jump
//     is not small;
//   * the pressure of Q0 and its Euler flux B1 = F_n(Q0), whose face-to-face
//     differences drive L -- float-float.
// Everything else -- slopes, half-range moments, the collision time and the
// non-equilibrium / time-derivative terms, all scaled by tau or dt -- is
// FP32.  The flux becomes F^n = B1 + (4 S(dt/2) - S(dt))/dt and
// dF^n/dt = 4 (S(dt) - 2 S(dt/2))/dt^2 with S the FP32 sum of the small
// terms, because the B1 part of I(delta) is exactly delta B1.  Only the final
// face flux is converted to FP64 for the update.
#pragma once
#include "hgks_bodies.cuh"
#include "hgks_f32x2.cuh"
#include "hgks_ff.cuh"
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
// buffer views of the mixed passes (inside the FP64-sized handle buffers)
// ---------------------------------------------------------------------------
// state split: q2[5][cs] float2 (hi, lo)
// pass 1 (fq): v[15][nq] float2 (Ql, Qr, Q0 values), vs[15][nq] floats (dQl, dQr, dQ0 in index units)
// pass 2 (t1), per Gauss line m: th[2][25][nt], tl[2][25][nt] (WENO values of Ql, Qr (10), quartic
//   values of Ql, Qr, Q0 (15)), ts[2][30][nt] (WENO of the slopes (15), quartic derivatives (15))
// The state and the pass-1 values are read as one 8-byte (hi, lo) element
// each; the t1 values stay as hi and lo planes, which the flux pass stages
// faster (measured: 87 against 92-100 ms per 256^3 step with pairs).
struct FqMx {
    float2 *v;
    float *vs;
};
struct T1Mx {
    float *th, *tl, *ts;
};
__host__ __device__ inline FqMx fq_mx(double *fq, long long nq)
{
    float2 *v = (float2 *)fq;
    return FqMx{ v, (float *)(v + 15 * nq) };
}
__host__ __device__ inline T1Mx t1_mx(double *t1, long long nt)
{
    float *f = (float *)t1;
    return T1Mx{ f, f + 50 * nt, f + 100 * nt };
}

// the state as (hi, lo) float pairs
static __device__ __forceinline__ void pos_split_mx(const Params &P, const double *__restrict__ q,
                                                    float2 *__restrict__ q2, long long t)
{
#pragma unroll
    for (int c = 0; c < 5; c++) {
        const ff v = ff_of_double(q[c * P.cs + t]);
        q2[c * P.cs + t] = make_float2(v.hi, v.lo);
    }
}

// stencil deviations x_j = X_j - X_c of float-float values
static __host__ __device__ __forceinline__ float ff_dev(float hj, float lj, float hc, float lc)
{
    return (hj - hc) + (lj - lc);
}

// the gas constants of the FP32 flux, held in registers (the batched kernels
// read Params from global memory, so the point flux takes them by value)
struct MxGas {
    float gm1, gm1_lo, K, prc, mu_ref, inv_Tref, omega;
    int power_law;
    double mu_ref_d, inv_Tref_d, omega_d;  // the viscosity law in FP64 (HGKS_MIXED_T64)
};
static __host__ __device__ __forceinline__ MxGas mx_gas(const Params &P)
{
    return MxGas{ P.f_gm1,     P.f_gm1_lo,         P.f_K,          P.f_prc,   P.f_mu_ref, P.f_inv_Tref,
                  P.f_omega,   P.visc_kind == 1,   P.mu_ref,       1.0 / P.T_ref, P.omega };
}

// FP32 viscosity law
static __host__ __device__ __forceinline__ float viscosity_f(const MxGas &G, float Tm)
{
    return G.power_law ? G.mu_ref * powf(Tm * G.inv_Tref, G.omega) : G.mu_ref;
}

// ---------------------------------------------------------------------------
// one side's half-range terms (FP32)
// ---------------------------------------------------------------------------
// For the side of Ql (POS: u > 0) or Qr (u < 0): the half-range flux b4, the
// slope terms w5/b5 (the three spatial slopes dq), the time-slope terms w6/b6,
// and the side's part of the compatibility condition: DPhi(q)[jq] when the
// jump is small (trapezoidal form), else Phi(q) itself.  The two sides are
// done one after the other so that only one side's moment set is live.
template <bool POS>
static __host__ __device__ __forceinline__ void side_terms_mx(const float q[5], const float dq[3][5],
                                                              const float jq[5], bool small_jump, float gm1, float K,
                                                              float b4[5], float w5[5], float b5[5], float w6[5],
                                                              float b6[5], float cp[5])
{
    HalfSide<float> h;
    half_side_setup(q, gm1, K, POS, h);
    HalfDelta<float> dd;
    HalfRate<float> rt;
    float s[5];
    half_phi<1, 0, 0>(h, b4);
    half_delta(h, dq[0], gm1, K, dd);
    half_dphi<1, 0, 0>(h, dd, w5);
    half_dphi<2, 0, 0>(h, dd, b5);
    half_rate_add<0>(h, dd, gm1, rt);
    half_delta(h, dq[1], gm1, K, dd);
    half_dphi<0, 1, 0>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) w5[c] += s[c];
    half_dphi<1, 1, 0>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) b5[c] += s[c];
    half_rate_add<1>(h, dd, gm1, rt);
    half_delta(h, dq[2], gm1, K, dd);
    half_dphi<0, 0, 1>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) w5[c] += s[c];
    half_dphi<1, 0, 1>(h, dd, s);
#pragma unroll
    for (int c = 0; c < 5; c++) b5[c] += s[c];
    half_rate_add<2>(h, dd, gm1, rt);
    // time slope of the side
    half_delta_time(h, rt, K, dd);
    half_dphi<0, 0, 0>(h, dd, w6);
    half_dphi<1, 0, 0>(h, dd, b6);
    if (small_jump) {
        half_delta(h, jq, gm1, K, dd);
        half_dphi<0, 0, 0>(h, dd, cp);
    } else {
        half_phi<0, 0, 0>(h, cp);
    }
}

// Q0 = Qm + C from the two sides' compatibility parts: with a small jump
// C = -(DPhi+(Ql) - DPhi-(Qr))[Qr - Ql] / 2, else Q0 = Phi+(Ql) + Phi-(Qr)
static __host__ __device__ __forceinline__ bool compat_prepare(const ff Ql[5], const ff Qr[5], ff Qm[5], float dq[5])
{
#pragma unroll
    for (int c = 0; c < 5; c++) {
        Qm[c] = ff_scale(ff_add(Ql[c], Qr[c]), 0.5f);
        dq[c] = ff_dev(Qr[c].hi, Qr[c].lo, Ql[c].hi, Ql[c].lo);
    }
    return fabsf(dq[0]) / Qm[0].hi + fabsf(dq[4]) / Qm[4].hi < 1e-3f;
}
static __host__ __device__ __forceinline__ void compat_finish(bool small_jump, const ff Qm[5], const float cl[5],
                                                              const float cr[5], ff Q0[5])
{
#pragma unroll
    for (int c = 0; c < 5; c++)
        Q0[c] = small_jump ? ff_add_f(Qm[c], -0.5f * (cl[c] - cr[c])) : ff_two_sum(cl[c], cr[c]);
}

// the equilibrium state alone (pass 1): both sides' compatibility parts
static __host__ __device__ __forceinline__ void compat_mixed(const ff Ql[5], const ff Qr[5], float gm1, float K,
                                                             ff Q0[5])
{
    ff Qm[5];
    float dq[5], cl[5], cr[5];
    const bool small_jump = compat_prepare(Ql, Qr, Qm, dq);
    float q[5];
    {
#pragma unroll
        for (int c = 0; c < 5; c++) q[c] = ff_to_float(Ql[c]);
        HalfSide<float> h;
        half_side_setup(q, gm1, K, true, h);
        if (small_jump) {
            HalfDelta<float> dd;
            half_delta(h, dq, gm1, K, dd);
            half_dphi<0, 0, 0>(h, dd, cl);
        } else {
            half_phi<0, 0, 0>(h, cl);
        }
    }
    {
#pragma unroll
        for (int c = 0; c < 5; c++) q[c] = ff_to_float(Qr[c]);
        HalfSide<float> h;
        half_side_setup(q, gm1, K, false, h);
        if (small_jump) {
            HalfDelta<float> dd;
            half_delta(h, dq, gm1, K, dd);
            half_dphi<0, 0, 0>(h, dd, cr);
        } else {
            half_phi<0, 0, 0>(h, cr);
        }
    }
    compat_finish(small_jump, Qm, cl, cr, Q0);
}

// ---------------------------------------------------------------------------
// Gauss-point flux, mixed precision
// ---------------------------------------------------------------------------
// Inputs of one Gauss point, kept by the flux pass in shared memory as one
// column per thread (slot-major, so a warp's accesses fall in distinct banks):
//   values of Ql (0..4), Qr (5..9) as hi/lo pairs   GP_VAL(n, k, part)
//   WENO slopes along the normal                     GP_SN(n, k)   k = 0..14 (l, r, 0)
//   derivatives along the first tangential dir.      GP_S1(n, k)
//   derivatives along the second tangential dir.     GP_S2(n, k)
// for the two Gauss points n of one Gauss line; all slopes in index units.
#define GP_VAL(n, k, part) (((n) * 10 + (k)) * 2 + (part))
#define GP_SN(n, k) (40 + (n) * 15 + (k))
#define GP_S1(n, k) (70 + (n) * 15 + (k))
#define GP_S2(n, k) (100 + (n) * 15 + (k))
constexpr int GP_SLOTS = 130;
constexpr int FLUX_MX_BLOCK = 128;
constexpr int FLUX_MX_SMEM = GP_SLOTS * FLUX_MX_BLOCK * (int)sizeof(float);

// the slopes of one state (which = 0: Ql, 1: Qr, 2: Q0) in physical units
static __host__ __device__ __forceinline__ void gp_slopes(const float *col, int st, int n, int which, float ihn,
                                                          float ih1, float ih2, float dq[3][5])
{
#pragma unroll
    for (int c = 0; c < 5; c++) {
        dq[0][c] = col[GP_SN(n, which * 5 + c) * st] * ihn;
        dq[1][c] = col[GP_S1(n, which * 5 + c) * st] * ih1;
        dq[2][c] = col[GP_S2(n, which * 5 + c) * st] * ih2;
    }
}

// T64 = true (HGKS_MIXED_T64): the Maxwellian temperature T0 = p0 / rho0 of the
// Gauss point, its collision time tau = mu(T0) / p0 and the time-integration
// coefficients of both windows (dt, dt/2) are formed in FP64 from the
// float-float Q0 (dtd: the time step in FP64); the sums they weight stay FP32.
template <bool T64 = false>
static __host__ __device__ __forceinline__ void gks_point_flux_mixed(const float *col, int st, int n, float ihn,
                                                                  float ih1, float ih2, const MxGas G, float dtf,
                                                                  ff Fn[5], float dFn[5], double dtd = 0.0)
{
    const float gm1 = G.gm1, K = G.K;
    ff Ql[5], Qr[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        Ql[c] = ff{ col[GP_VAL(n, c, 0) * st], col[GP_VAL(n, c, 1) * st] };
        Qr[c] = ff{ col[GP_VAL(n, 5 + c, 0) * st], col[GP_VAL(n, 5 + c, 1) * st] };
    }
    ff Qm[5];
    float jq[5];
    const bool small_jump = compat_prepare(Ql, Qr, Qm, jq);
    // half-range terms of the two sides (FP32), one side at a time
    float b4l[5], w5l[5], b5l[5], w6l[5], b6l[5], b4r[5], w5r[5], b5r[5], w6r[5], b6r[5], cl[5], cr[5];
    {
        float q[5], dq[3][5];
#pragma unroll
        for (int c = 0; c < 5; c++) q[c] = ff_to_float(Ql[c]);
        gp_slopes(col, st, n, 0, ihn, ih1, ih2, dq);
        side_terms_mx<true>(q, dq, jq, small_jump, gm1, K, b4l, w5l, b5l, w6l, b6l, cl);
    }
    {
        float q[5], dq[3][5];
#pragma unroll
        for (int c = 0; c < 5; c++) q[c] = ff_to_float(Qr[c]);
        gp_slopes(col, st, n, 1, ihn, ih1, ih2, dq);
        side_terms_mx<false>(q, dq, jq, small_jump, gm1, K, b4r, w5r, b5r, w6r, b6r, cr);
    }

    // equilibrium state and its Euler flux in float-float
    ff Q0[5];
    compat_finish(small_jump, Qm, cl, cr, Q0);
    const ff gm1ff{ G.gm1, G.gm1_lo };
    const ff ir0 = ff_recip(Q0[0]);
    const ff U0 = ff_mul(Q0[1], ir0), V0 = ff_mul(Q0[2], ir0), W0 = ff_mul(Q0[3], ir0);
    const ff mU = ff_mul(Q0[1], U0);  // rho U^2
    const ff m2 = ff_add(ff_add(mU, ff_mul(Q0[2], V0)), ff_mul(Q0[3], W0));
    const ff p0 = ff_mul(gm1ff, ff_sub(Q0[4], ff_scale(m2, 0.5f)));
    ff B1[5];
    B1[0] = Q0[1];
    B1[1] = ff_add(mU, p0);
    B1[2] = ff_mul(Q0[1], V0);
    B1[3] = ff_mul(Q0[1], W0);
    B1[4] = ff_mul(U0, ff_add(Q0[4], p0));

    // FP32: equilibrium slope terms, collision time, the small terms S(delta)
    float q0f[5];
#pragma unroll
    for (int c = 0; c < 5; c++) q0f[c] = ff_to_float(Q0[c]);
    const Gas<float> g0 = gas_of(q0f, gm1);
    // time-integration coefficients q1..q5 of the windows dt (pass 0) and
    // dt/2 (pass 1): q1 = tau (2 tau (1 - e) - d - d e), q2 = d^2/2 - tau d +
    // tau^2 (1 - e), q3 = tau (1 - e), q4 = tau (2 tau (1 - e) - d e),
    // q5 = tau q3, with e = exp(-d / tau)
    float qc[2][5];
    if (T64) {
        const double p0d = ff_to_double(p0), T0d = p0d / ff_to_double(Q0[0]);
        const double mud = G.power_law ? G.mu_ref_d * pow(T0d * G.inv_Tref_d, G.omega_d) : G.mu_ref_d;
        const double taud = mud / p0d;
        const double ehd = taud > 0.0 ? exp(-0.5 * dtd / taud) : 0.0;
#pragma unroll
        for (int pass = 0; pass < 2; pass++) {
            const double dd = pass == 0 ? dtd : 0.5 * dtd;
            const double e = pass == 0 ? ehd * ehd : ehd;
            const double om = 1.0 - e;
            qc[pass][0] = (float)(taud * (2.0 * taud * om - dd - dd * e));
            qc[pass][1] = (float)(0.5 * dd * dd - taud * dd + taud * taud * om);
            qc[pass][2] = (float)(taud * om);
            qc[pass][3] = (float)(taud * (2.0 * taud * om - dd * e));
            qc[pass][4] = (float)(taud * taud * om);
        }
    } else {
        const float p0f = ff_to_float(p0);
        const float T0 = p0f * ff_to_float(ir0);
        const float tau = viscosity_f(G, T0) / p0f;
        const float eh = tau > 0.0f ? expf(-0.5f * dtf / tau) : 0.0f;
#pragma unroll
        for (int pass = 0; pass < 2; pass++) {
            const float dd = pass == 0 ? dtf : 0.5f * dtf;
            const float x = dd / tau;  // +inf for tau = 0
            if (x < 1.0f) {
                // a window shorter than the collision time: in q1 = tau^2 f1(x)
                // and q2 = tau^2 f2(x) the closed forms cancel to O(x^3) and
                // lose ~2 log10(1/x) digits in FP32, so they are summed as
                // their Taylor series, f1 = sum_k>=3 (-1)^(k+1) (2 - k) x^k / k!,
                // f2 = sum_k>=3 (-1)^(k+1) x^k / k! (k <= 13: below 1e-9 of the
                // first term at x = 1), and 1 - e as -expm1(-x)
                const float om = -expm1f(-x);
                const float f1 =
                    x * x * x *
                    (-1.0f / 6.0f +
                     x * (1.0f / 12.0f +
                          x * (-1.0f / 40.0f +
                               x * (1.0f / 180.0f +
                                    x * (-1.0f / 1008.0f +
                                         x * (1.0f / 6720.0f +
                                              x * (-1.0f / 51840.0f +
                                                   x * (1.0f / 453600.0f +
                                                        x * (-1.0f / 4435200.0f +
                                                             x * (1.0f / 47900160.0f +
                                                                  x * (-11.0f / 6227020800.0f)))))))))));
                const float f2 =
                    x * x * x *
                    (1.0f / 6.0f +
                     x * (-1.0f / 24.0f +
                          x * (1.0f / 120.0f +
                               x * (-1.0f / 720.0f +
                                    x * (1.0f / 5040.0f +
                                         x * (-1.0f / 40320.0f +
                                              x * (1.0f / 362880.0f +
                                                   x * (-1.0f / 3628800.0f +
                                                        x * (1.0f / 39916800.0f +
                                                             x * (-1.0f / 479001600.0f +
                                                                  x * (1.0f / 6227020800.0f)))))))))));
                const float t2 = tau * tau;
                qc[pass][0] = t2 * f1;
                qc[pass][1] = t2 * f2;
                qc[pass][2] = tau * om;
                qc[pass][3] = t2 * (2.0f * om - x * (1.0f - om));
                qc[pass][4] = tau * qc[pass][2];
            } else {
                const float e = pass == 0 ? eh * eh : eh;
                const float om = 1.0f - e;
                qc[pass][0] = tau * (2.0f * tau * om - dd - dd * e);
                qc[pass][1] = 0.5f * dd * dd - tau * dd + tau * tau * om;
                qc[pass][2] = tau * om;
                qc[pass][3] = tau * (2.0f * tau * om - dd * e);
                qc[pass][4] = tau * qc[pass][2];
            }
        }
    }
    float B2[5], B3[5], R0[5], B4m1[5], W5[5], B5[5], W6[5], B6[5];
    {
        float s[5], d0[3][5];
        gp_slopes(col, st, n, 2, ihn, ih1, ih2, d0);
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
        const float Kp5 = K + 5.0f;
        second_dmoment<0>(g0, d0[0], gm1, Kp5, B2);
        second_dmoment<1>(g0, d0[1], gm1, Kp5, s);
#pragma unroll
        for (int c = 0; c < 5; c++) B2[c] += s[c];
        second_dmoment<2>(g0, d0[2], gm1, Kp5, s);
#pragma unroll
        for (int c = 0; c < 5; c++) B2[c] += s[c];
#pragma unroll
        for (int c = 0; c < 5; c++) {
            // half-range flux minus the equilibrium flux
            B4m1[c] = ff_to_float(ff_sub(ff_two_sum(b4l[c], b4r[c]), B1[c]));
            W5[c] = w5l[c] + w5r[c];
            B5[c] = b5l[c] + b5r[c];
            W6[c] = w6l[c] + w6r[c];
            B6[c] = b6l[c] + b6r[c];
        }
    }
    // heat fluxes of the terms (the equilibrium carries none; the B4 - B1 term
    // carries that of the half-range part: h(B4, Q0) - h(B1, Q0) = h(B4, Q0))
    float W3[5], b4s[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        W3[c] = -R0[c];
        b4s[c] = b4l[c] + b4r[c];
    }
    const float h2 = heat_of_g(B2, R0, g0), h3 = heat_of_g(B3, W3, g0), h4 = heat_of_g(b4s, q0f, g0),
                h5 = heat_of_g(B5, W5, g0), h6 = heat_of_g(B6, W6, g0);
    const float prc = G.prc;
    float S[2][5];
#pragma unroll
    for (int pass = 0; pass < 2; pass++) {
        const float q1 = qc[pass][0], q2 = qc[pass][1], q3 = qc[pass][2], q4 = qc[pass][3], q5 = qc[pass][4];
#pragma unroll
        for (int i = 0; i < 5; i++)
            S[pass][i] = q1 * B2[i] + q2 * B3[i] + q3 * B4m1[i] - q4 * B5[i] - q5 * B6[i];
        S[pass][4] += prc * (q1 * h2 + q2 * h3 + q3 * h4 - q4 * h5 - q5 * h6);
    }
    const float idt = 1.0f / dtf;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        Fn[i] = ff_add_f(B1[i], (4.0f * S[1][i] - S[0][i]) * idt);
        dFn[i] = 4.0f * (S[0][i] - 2.0f * S[1][i]) * idt * idt;
    }
}

// ---------------------------------------------------------------------------
// pass 1: normal reconstruction from the split state
// ---------------------------------------------------------------------------
// the normal reconstruction at interface position p (its pass-1 record goes
// to ov / ovs at index t, planes S apart)
static __device__ __forceinline__ void normal_mx_at(const Params &P, int d, const int p[3],
                                                    const float2 *__restrict__ q2, float2 *__restrict__ ov,
                                                    float *__restrict__ ovs, long long S, long long t)
{
    const long long nq = S;
    FqMx o{ ov, ovs };
    int c0[3] = { p[0], p[1], p[2] };
    c0[d] = p[d] - 3;
    const long long base = pidx(P, c0[0], c0[1], c0[2]);
    const long long sd = d == 0 ? 1 : (d == 1 ? P.sy : P.sz);
    ff Ql[5], Qr[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        const long long off = (long long)perm_mx(d, c) * P.cs + base;
        float H[6], L[6];
#pragma unroll
        for (int m = 0; m < 6; m++) {
            const float2 e = q2[off + m * sd];
            H[m] = e.x;
            L[m] = e.y;
        }
        // the stencils of cell f-1 (lane x) and cell f (lane y), each as
        // deviations about its centre, reconstructed together on packed pairs
        f2 X[5];
        const f2 Hc = f2_pack(H[2], H[3]), Lc = f2_pack(L[2], L[3]);
#pragma unroll
        for (int m = 0; m < 5; m++) X[m] = f2_ff_dev(f2_pack(H[m], H[m + 1]), f2_pack(L[m], L[m + 1]), Hc, Lc);
        f2 vl, vr;
        f2_weno_edge(X, vl, vr);  // (cell f-1, cell f) at their left and right edges
        float lm_l, r_l, lm_r, r_r;
        f2_unpack(vl, lm_l, r_l);
        f2_unpack(vr, lm_r, r_r);
        // Ql: cell f-1's right edge; Qr: cell f's left edge
        f2 qh, ql;
        f2_ff_add_f(Hc, Lc, f2_pack(lm_r, r_l), qh, ql);
        f2_unpack(qh, Ql[c].hi, Qr[c].hi);
        f2_unpack(ql, Ql[c].lo, Qr[c].lo);
        o.v[(0 * 5 + c) * nq + t] = make_float2(Ql[c].hi, Ql[c].lo);
        o.v[(1 * 5 + c) * nq + t] = make_float2(Qr[c].hi, Qr[c].lo);
        // parabola slopes (centre cancels): 2 lm_l + 4 lm_r and -4 r_l - 2 r_r
        float sl, sr;
        f2_unpack(f2_fma(f2_pack(2.0f, -4.0f), vl, f2_mul(f2_pack(4.0f, -2.0f), vr)), sl, sr);
        o.vs[(0 * 5 + c) * nq + t] = sl;
        o.vs[(1 * 5 + c) * nq + t] = sr;
        float x1, x1r, x3, x3r, x4, x4r;
        f2_unpack(X[1], x1, x1r);
        f2_unpack(X[3], x3, x3r);
        f2_unpack(X[4], x4, x4r);
        o.vs[(2 * 5 + c) * nq + t] = (15.0f * x3 - (x4 - x1)) * (1.0f / 12.0f);
    }
    ff Q0[5];
    compat_mixed(Ql, Qr, P.f_gm1, P.f_K, Q0);
#pragma unroll
    for (int c = 0; c < 5; c++) {
        o.v[(2 * 5 + c) * nq + t] = make_float2(Q0[c].hi, Q0[c].lo);
    }
}

static __device__ __forceinline__ void pos_normal_mx(const Params &P, int d, const Box &B,
                                                     const float2 *__restrict__ q2, FqMx o, long long t)
{
    int p[3];
    bpos(B, t, p);
    normal_mx_at(P, d, p, q2, o.v, o.vs, box_count(B), t);
}

// ---------------------------------------------------------------------------
// pass 2: first tangential direction
// ---------------------------------------------------------------------------
// The row loops are fully unrolled: all rows' loads are in flight together
// (the pass is latency-bound), and with every index a compile-time constant
// the pass needs fewer registers than with a rolled loop (80 against 128).
// The first tangential reconstruction of one position from pass-1 records
// v2 / vs (planes Sq apart, the position's record at base, its neighbours
// along the first tangential direction s1 apart), written to th / tl / ts at
// index t (planes nt apart).
static __device__ __forceinline__ void tan1_mx_from(const float2 *__restrict__ v2, const float *__restrict__ vs,
                                                    long long Sq, long long base, long long s1,
                                                    float *__restrict__ th, float *__restrict__ tl,
                                                    float *__restrict__ ts, long long nt, long long t)
{
    // Rows are reduced two at a time on packed FP32 pairs (hgks_f32x2.cuh):
    // the Ql and Qr rows of one component together (WENO + quartic), the Q0
    // rows of components (0, 1) and (2, 3) (quartic), and the slope rows in
    // consecutive pairs (WENO); the Q0 row of component 4 and the last slope
    // row run alone.  Value index k (0..24) of a Gauss point: 0..9 WENO values
    // of Ql, Qr; 10..24 quartic values of Ql, Qr, Q0.
    auto put_value = [&](int k, f2 m, f2 p, int step) {  // hi parts of float-float values, both Gauss points
        float a0, a1, b0, b1;
        f2_unpack(m, a0, a1);
        f2_unpack(p, b0, b1);
        th[(0 * 25 + k) * nt + t] = a0;
        th[(1 * 25 + k) * nt + t] = b0;
        th[(0 * 25 + k + step) * nt + t] = a1;
        th[(1 * 25 + k + step) * nt + t] = b1;
    };
    auto put_lo = [&](int k, f2 m, f2 p, int step) {
        float a0, a1, b0, b1;
        f2_unpack(m, a0, a1);
        f2_unpack(p, b0, b1);
        tl[(0 * 25 + k) * nt + t] = a0;
        tl[(1 * 25 + k) * nt + t] = b0;
        tl[(0 * 25 + k + step) * nt + t] = a1;
        tl[(1 * 25 + k + step) * nt + t] = b1;
    };
    auto put_slope = [&](int k, f2 m, f2 p, int step) {  // FP32 slopes / derivatives, index k of 30
        float a0, a1, b0, b1;
        f2_unpack(m, a0, a1);
        f2_unpack(p, b0, b1);
        ts[(0 * 30 + k) * nt + t] = a0;
        ts[(1 * 30 + k) * nt + t] = b0;
        ts[(0 * 30 + k + step) * nt + t] = a1;
        ts[(1 * 30 + k + step) * nt + t] = b1;
    };
    // two value rows (planes r0, r1 of the pass-1 record) as packed (hi, lo)
    // deviations about their centres
    auto load_pair = [&](int r0, int r1, f2 H[5], f2 L[5], f2 x[5]) {
        const long long o0 = (long long)r0 * Sq + base, o1 = (long long)r1 * Sq + base;
#pragma unroll
        for (int j = 0; j < 5; j++) {
            const float2 a = v2[o0 + (j - 2) * s1], b = v2[o1 + (j - 2) * s1];
            H[j] = f2_pack(a.x, b.x);
            L[j] = f2_pack(a.y, b.y);
        }
#pragma unroll
        for (int j = 0; j < 5; j++) x[j] = f2_ff_dev(H[j], L[j], H[2], L[2]);
    };
    // values of Ql and Qr, component c: WENO and quartic values, quartic derivatives
#pragma unroll
    for (int c = 0; c < 5; c++) {
        f2 H[5], L[5], x[5], m, p, rh0, rl0, rh1, rl1;
        load_pair(c, 5 + c, H, L, x);
        f2_weno_gauss(x, m, p);
        f2_ff_add_f(H[2], L[2], m, rh0, rl0);
        f2_ff_add_f(H[2], L[2], p, rh1, rl1);
        put_value(c, rh0, rh1, 5);
        put_lo(c, rl0, rl1, 5);
        f2_quartic_value(x, m, p);
        f2_ff_add_f(H[2], L[2], m, rh0, rl0);
        f2_ff_add_f(H[2], L[2], p, rh1, rl1);
        put_value(10 + c, rh0, rh1, 5);
        put_lo(10 + c, rl0, rl1, 5);
        f2_quartic_deriv(x, m, p);
        put_slope(15 + c, m, p, 5);
    }
    // values of Q0, components (0, 1) and (2, 3): quartic values and derivatives
#pragma unroll
    for (int c = 0; c < 4; c += 2) {
        f2 H[5], L[5], x[5], m, p, rh0, rl0, rh1, rl1;
        load_pair(10 + c, 11 + c, H, L, x);
        f2_quartic_value(x, m, p);
        f2_ff_add_f(H[2], L[2], m, rh0, rl0);
        f2_ff_add_f(H[2], L[2], p, rh1, rl1);
        put_value(20 + c, rh0, rh1, 1);
        put_lo(20 + c, rl0, rl1, 1);
        f2_quartic_deriv(x, m, p);
        put_slope(25 + c, m, p, 1);
    }
    {  // Q0, component 4, alone
        const long long off = (long long)14 * Sq + base;
        float H[5], L[5], x[5];
#pragma unroll
        for (int j = 0; j < 5; j++) {
            const float2 e = v2[off + (j - 2) * s1];
            H[j] = e.x;
            L[j] = e.y;
        }
#pragma unroll
        for (int j = 0; j < 5; j++) x[j] = ff_dev(H[j], L[j], H[2], L[2]);
        const ff ctr{ H[2], L[2] };
        float qm, qp, dm, dp;
        quartic_value_pair(x, qm, qp);
        quartic_deriv_pair(x, dm, dp);
        const ff bm = ff_add_f(ctr, qm), bp = ff_add_f(ctr, qp);
        th[(0 * 25 + 24) * nt + t] = bm.hi;
        tl[(0 * 25 + 24) * nt + t] = bm.lo;
        th[(1 * 25 + 24) * nt + t] = bp.hi;
        tl[(1 * 25 + 24) * nt + t] = bp.lo;
        ts[(0 * 30 + 29) * nt + t] = dm;
        ts[(1 * 30 + 29) * nt + t] = dp;
    }
    // slopes (15 rows, w * 5 + c): WENO-Z of pairs of rows, the last alone
#pragma unroll
    for (int r = 0; r < 14; r += 2) {
        const float *s0 = vs + (long long)r * Sq + base, *s1p = vs + (long long)(r + 1) * Sq + base;
        f2 X[5], m, p;
#pragma unroll
        for (int j = 0; j < 5; j++) X[j] = f2_pack(s0[(j - 2) * s1], s1p[(j - 2) * s1]);
        f2_weno_gauss(X, m, p);
        put_slope(r, m, p, 1);
    }
    {
        const float *src = vs + (long long)14 * Sq + base;
        float x[5];
#pragma unroll
        for (int j = 0; j < 5; j++) x[j] = src[(j - 2) * s1];
        WenoPrep<float> W;
        weno_prep(x, W);
        float vm, vp;
        weno_gauss_pair(W, vm, vp);
        ts[(0 * 30 + 14) * nt + t] = vm;
        ts[(1 * 30 + 14) * nt + t] = vp;
    }
}

static __device__ __forceinline__ void tan1_mx_rows(int d, const Box &Bt, const Box &Bq,
                                                    const float2 *__restrict__ v2, const float *__restrict__ vs,
                                                    float *__restrict__ th,
                                                    float *__restrict__ tl, float *__restrict__ ts, long long t)
{
    int p[3];
    bpos(Bt, t, p);
    tan1_mx_from(v2, vs, box_count(Bq), blin(Bq, p), bstride(Bq, tdir(d, 0)), th, tl, ts, box_count(Bt), t);
}

// the input and output planes never overlap: passing them as restricted
// pointers lets the compiler move the loads of later rows ahead of the
// stores of earlier ones
static __device__ __forceinline__ void pos_tan1_mx(const Params &P, int d, const Box &Bt, const Box &Bq, FqMx in,
                                                   T1Mx o, long long t)
{
    (void)P;
    tan1_mx_rows(d, Bt, Bq, in.v, in.vs, o.th, o.tl, o.ts, t);
}

// ---------------------------------------------------------------------------
// pass 3: second tangential direction and the four Gauss-point fluxes
// ---------------------------------------------------------------------------
static __device__ __forceinline__ float inv_metric_f(const Params &P, int e, const double *tab, int idx)
{
    return e == 1 && P.stretched ? 1.0f / (float)tab[idx] : P.f_ih[e];
}

// ---------------------------------------------------------------------------
// pass 3 on block tiles: 32 face columns by 4 positions along the second
// tangential direction e2 (one warp per e2 position).  The columns are 32
// consecutive (x, other-axis) pairs of the plane normal to e2, flattened so
// that no lane idles at the end of an x row.  The four e2 positions of a tile
// share the eight t1 rows b0-2 .. b0+5 of every row type, so the block stages
// those in shared memory once (8 instead of 20 row loads per 4 faces) and
// prefetches the next row types with cp.async while it reduces the current
// ones; each lane stages its own column.  A stage holds two row types
// interleaved, [array][row][x][type], so that one 8-byte shared load gives a
// thread the pair of values it reduces together with the packed FP32
// instructions (hgks_f32x2.cuh).
// ---------------------------------------------------------------------------
constexpr int FT_X = 32, FT_B = 4, FT_ROWS = FT_B + 4;
constexpr int FT_TYPE = 2 * FT_ROWS * FT_X;     // floats of one row type: [array][row][x]
constexpr int FT_STAGE = 2 * 2 * FT_TYPE;       // [buffer][array][row][x][two row types]
constexpr int FLUX_MX_TILE_SMEM = FLUX_MX_SMEM + FT_STAGE * (int)sizeof(float);

struct FluxTiling {
    int e2, other, E0, no, nbt;
    long long ncol, ngt, count;  // columns (x, other) of the plane, column tiles, tiles
};
__host__ __device__ inline FluxTiling flux_tiling(const Params &P, int d)
{
    FluxTiling f;
    f.e2 = tdir(d, 1);
    f.other = d == 2 ? 2 : 1;  // the axis that is neither x nor e2
    f.E0 = P.n[0] + (d == 0 ? 1 : 0);
    f.no = P.n[f.other] + (f.other == d ? 1 : 0);
    f.nbt = (P.n[f.e2] + FT_B - 1) / FT_B;
    f.ncol = (long long)f.E0 * f.no;
    f.ngt = (f.ncol + FT_X - 1) / FT_X;
    f.count = f.ngt * f.nbt;
    return f;
}

static __device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
static __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// the two source arrays of row type it (0..79: line m = it / 40; 0..9 WENO
// values, 10..24 quartic values, 25..39 slopes and first-direction derivatives)
static __device__ __forceinline__ void ft_planes(const T1Mx &in, long long nt, int it, const float *&A,
                                                 const float *&B)
{
    const int m = it / 40, k = it % 40;
    if (k < 25) {
        A = in.th + (long long)(m * 25 + k) * nt;
        B = in.tl + (long long)(m * 25 + k) * nt;
    } else {
        A = in.ts + (long long)(m * 30 + (k - 25)) * nt;
        B = in.ts + (long long)(m * 30 + 15 + (k - 25)) * nt;
    }
}

// sm: GP_SLOTS floats per thread (Gauss-point inputs), then FT_STAGE floats
template <bool T64>
static __device__ __forceinline__ void flux_mx_tile(const Params &P, int d, const Box &Bf, const Box &Bt, T1Mx in,
                                                    double *__restrict__ F, double dt, long long T, float *sm)
{
    const FluxTiling ft = flux_tiling(P, d);
    const long long nf = box_count(Bf), nt = box_count(Bt);
    const long long gt = T % ft.ngt;
    const int b0 = (int)(T / ft.ngt) * FT_B;
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int e1 = tdir(d, 0), e2 = ft.e2;
    // this lane's column and this thread's face
    const long long g = gt * FT_X + lane;
    const bool col_ok = g < ft.ncol;
    int p[3];
    p[0] = col_ok ? (int)(g % ft.E0) : 0;
    p[ft.other] = col_ok ? (int)(g / ft.E0) : 0;
    p[e2] = b0 + wb;
    const bool valid = col_ok && p[e2] < Bf.E[e2];
    // this lane's first staged t1 row (e2 index b0 - 2) and the row stride
    int q0[3] = { p[0], p[1], p[2] };
    q0[e2] = b0 - 2;
    const long long base_l = blin(Bt, q0), s2 = bstride(Bt, e2);
    const int rlim = P.n[e2] + 3 - b0;  // rows r with e2 index b0 - 2 + r <= n + 1
    float *gp = sm, *stage = sm + GP_SLOTS * FLUX_MX_BLOCK;
    constexpr int st = FLUX_MX_BLOCK;  // every launch uses this block size: slot offsets become immediates
    float *col = gp + threadIdx.x;

    // cooperative staging: thread (lane, wb) copies rows wb, wb + 4 of both
    // arrays for its lane's column (segments wb + 4 i, i = 0..3); a stage
    // holds two row types u = 0, 1, interleaved
    auto issue = [&](int pair) {
        float *buf = stage + (pair & 1) * (2 * FT_TYPE);
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const float *A, *B;
            ft_planes(in, nt, 2 * pair + u, A, B);
#pragma unroll
            for (int i = 0; i < FT_TYPE / FLUX_MX_BLOCK; i++) {
                const int seg = wb + 4 * i, arr = seg / FT_ROWS, r = seg % FT_ROWS;
                if (col_ok && r <= rlim)
                    cp_async4(buf + (seg * FT_X + lane) * 2 + u, (arr ? B : A) + base_l + r * s2);
            }
        }
        cp_async_commit();
    };

    const float ihn = valid ? inv_metric_f(P, d, P.my_face, p[d]) : 0.0f;
    const float dtf = (float)dt;
    const MxGas G = mx_gas(P);
    ff Fs[5];
    float dFs[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        Fs[c] = ff{ 0.0f, 0.0f };
        dFs[c] = 0.0f;
    }
    // both row types of a stage at once (it0 even), two lanes per packed
    // instruction.  Kinds by k = it % 40: 0..9 float-float WENO values,
    // 10..24 quartic derivatives of float-float values, 25..39 WENO slopes
    // with quartic values; the pair (24, 25) mixes the last two kinds, so it
    // runs both and each lane keeps its own kind's results.
    auto reduce2 = [&](const float *buf, int it0) {
        const int k = it0 % 40;
        f2 X[5], Y[5];
#pragma unroll
        for (int j = 0; j < 5; j++) {
            X[j] = f2_load(buf + ((0 * FT_ROWS + wb + j) * FT_X + lane) * 2);
            Y[j] = f2_load(buf + ((1 * FT_ROWS + wb + j) * FT_X + lane) * 2);
        }
        float a0, a1, b0, b1;
        if (k < 10) {  // float-float values: deviations about the centre row
            f2 x[5];
#pragma unroll
            for (int j = 0; j < 5; j++) x[j] = f2_ff_dev(X[j], Y[j], X[2], Y[2]);
            f2 vm, vp, h, l;
            f2_weno_gauss(x, vm, vp);
            f2_ff_add_f(X[2], Y[2], vm, h, l);
            f2_unpack(h, a0, a1);
            f2_unpack(l, b0, b1);
            col[GP_VAL(0, k, 0) * st] = a0;
            col[GP_VAL(0, k + 1, 0) * st] = a1;
            col[GP_VAL(0, k, 1) * st] = b0;
            col[GP_VAL(0, k + 1, 1) * st] = b1;
            f2_ff_add_f(X[2], Y[2], vp, h, l);
            f2_unpack(h, a0, a1);
            f2_unpack(l, b0, b1);
            col[GP_VAL(1, k, 0) * st] = a0;
            col[GP_VAL(1, k + 1, 0) * st] = a1;
            col[GP_VAL(1, k, 1) * st] = b0;
            col[GP_VAL(1, k + 1, 1) * st] = b1;
            return;
        }
        if (k < 25) {  // derivatives along e2 of float-float values (quartic)
            f2 x[5], dm, dp;
#pragma unroll
            for (int j = 0; j < 5; j++) x[j] = f2_ff_dev(X[j], Y[j], X[2], Y[2]);
            f2_quartic_deriv(x, dm, dp);
            f2_unpack(dm, a0, a1);
            f2_unpack(dp, b0, b1);
            col[GP_S2(0, k - 10) * st] = a0;
            col[GP_S2(1, k - 10) * st] = b0;
            if (k + 1 < 25) {
                col[GP_S2(0, k - 9) * st] = a1;
                col[GP_S2(1, k - 9) * st] = b1;
            }
        }
        if (k + 1 >= 25) {  // normal slopes (WENO) and first-direction derivatives (quartic value)
            f2 s0, s1, q0v, q1v;
            f2_weno_gauss(X, s0, s1);
            f2_quartic_value(Y, q0v, q1v);
            f2_unpack(s0, a0, a1);
            f2_unpack(s1, b0, b1);
            float c0, c1, e0, e1;
            f2_unpack(q0v, c0, c1);
            f2_unpack(q1v, e0, e1);
            if (k >= 25) {
                col[GP_SN(0, k - 25) * st] = a0;
                col[GP_SN(1, k - 25) * st] = b0;
                col[GP_S1(0, k - 25) * st] = c0;
                col[GP_S1(1, k - 25) * st] = e0;
            }
            col[GP_SN(0, k - 24) * st] = a1;
            col[GP_SN(1, k - 24) * st] = b1;
            col[GP_S1(0, k - 24) * st] = c1;
            col[GP_S1(1, k - 24) * st] = e1;
        }
    };
    issue(0);
#pragma unroll 1
    for (int pair = 0; pair < 40; pair++) {
        if (pair + 1 < 40) {
            issue(pair + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *buf = stage + (pair & 1) * (2 * FT_TYPE);
        if (valid) {
            reduce2(buf, 2 * pair);
            if (pair % 20 == 19) {  // all inputs of line m: the two Gauss-point fluxes
                const int m = pair / 20;
                const float ih1 = inv_metric_f(P, e1, P.my_gp, 2 * p[e1] + m);
#pragma unroll 1
                for (int n = 0; n < 2; n++) {
                    const float ih2 = inv_metric_f(P, e2, P.my_gp, 2 * p[e2] + n);
                    ff Fn[5];
                    float dFn[5];
                    gks_point_flux_mixed<T64>(col, st, n, ihn, ih1, ih2, G, dtf, Fn, dFn, dt);
#pragma unroll
                    for (int c = 0; c < 5; c++) {
                        Fs[c] = ff_add(Fs[c], ff_scale(Fn[c], 0.25f));  // Gauss weights 1/4 (exact)
                        dFs[c] += 0.25f * dFn[c];
                    }
                }
            }
        }
        __syncthreads();  // this buffer is refilled two iterations later
    }
    if (!valid) return;
    double area;
    if (d == 0) area = P.hy_cell[p[1]] * P.h[2];
    else if (d == 1) area = P.h[0] * P.h[2];
    else area = P.h[0] * P.hy_cell[p[1]];
    const long long t = blin(Bf, p);
#pragma unroll
    for (int c = 0; c < 5; c++) {
        F[(long long)perm_mx(d, c) * nf + t] = ff_to_double(Fs[c]) * area;
        F[(long long)(5 + perm_mx(d, c)) * nf + t] = (double)dFs[c] * area;
    }
}

}  // namespace hgks
