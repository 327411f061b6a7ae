// hgks_f32x2.cuh -- pairs of FP32 values in one 64-bit register, operated on
// by the packed FP32 instructions of sm_100-class GPUs (add / sub / mul / fma
// with the .f32x2 type): one instruction issues the work of two.  Each lane
// is rounded to nearest exactly as the scalar instruction would round it, so
// error-free transformations (TwoSum) stay exact lane by lane.
//
// The mixed-precision passes use them for their reconstructions: the normal
// pass runs the left and right stencils of a component as one pair (WENO-Z
// to the cell edges), the first tangential pass reduces its rows two at a
// time, and the flux pass reduces the two row types of each staging step
// together (WENO-Z to the two Gauss abscissae, the quartic point values and
// derivatives, and the float-float additions that rebuild a value from its
// stencil centre).  The formulas are those of the scalar templates of
// hgks_device.cuh and hgks_ff.cuh, written out per lane pair.
#pragma once
#include <cuda_runtime.h>

#include "hgks_device.cuh"

namespace hgks {

struct f2 {
    unsigned long long v;
};

static __device__ __forceinline__ f2 f2_pack(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
static __device__ __forceinline__ void f2_unpack(f2 a, float &x, float &y)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
}
static __device__ __forceinline__ f2 f2_bcast(float a) { return f2_pack(a, a); }
static __device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
static __device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
static __device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
static __device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
static __device__ __forceinline__ f2 f2_abs(f2 a)
{
    f2 r;
    r.v = a.v & 0x7FFFFFFF7FFFFFFFull;  // clear both sign bits
    return r;
}
// one 8-byte load of an adjacent pair (lane x at the lower address)
static __device__ __forceinline__ f2 f2_load(const float *p)
{
    f2 r;
    r.v = *reinterpret_cast<const unsigned long long *>(p);
    return r;
}

// stencil deviation (X_j - X_c) + (Y_j - Y_c) of float-float values, per lane
static __device__ __forceinline__ f2 f2_ff_dev(f2 hj, f2 lj, f2 hc, f2 lc)
{
    return f2_add(f2_sub(hj, hc), f2_sub(lj, lc));
}

// float-float (hi, lo) + b per lane: TwoSum(hi, b) then FastTwoSum with lo
// added to the error (hgks_ff.cuh ff_add_f)
static __device__ __forceinline__ void f2_ff_add_f(f2 hi, f2 lo, f2 b, f2 &rh, f2 &rl)
{
    const f2 s = f2_add(hi, b);
    const f2 bb = f2_sub(s, hi);
    const f2 e = f2_add(f2_sub(hi, f2_sub(s, bb)), f2_sub(b, bb));
    const f2 t = f2_add(e, lo);
    rh = f2_add(s, t);
    rl = f2_sub(t, f2_sub(rh, s));
}

// WENO-Z of two stencils (hgks_device.cuh weno_prep + weno_gauss_pair): the
// values at the Gauss abscissae -sqrt(3)/6 (vm) and +sqrt(3)/6 (vp)
static __device__ __forceinline__ void f2_weno_gauss(const f2 X[5], f2 &vm, f2 &vp)
{
    const f2 h = f2_bcast(0.5f), t3 = f2_bcast(1.5f), mh = f2_bcast(-0.5f);
    const f2 d1 = f2_sub(X[1], X[0]), d2 = f2_sub(X[2], X[1]), d3 = f2_sub(X[3], X[2]), d4 = f2_sub(X[4], X[3]);
    const f2 c20 = f2_mul(h, f2_sub(d2, d1)), c10 = f2_fma(t3, d2, f2_mul(mh, d1));
    const f2 c21 = f2_mul(h, f2_sub(d3, d2)), c11 = f2_mul(h, f2_add(d3, d2));
    const f2 c22 = f2_mul(h, f2_sub(d4, d3)), c12 = f2_fma(t3, d3, f2_mul(mh, d4));
    const f2 k133 = f2_bcast((float)(13.0 / 3.0)), eps = f2_bcast((float)WENO_EPS);
    const f2 b0 = f2_fma(c10, c10, f2_fma(f2_mul(k133, c20), c20, eps));
    const f2 b1 = f2_fma(c11, c11, f2_fma(f2_mul(k133, c21), c21, eps));
    const f2 b2 = f2_fma(c12, c12, f2_fma(f2_mul(k133, c22), c22, eps));
    const f2 tau5 = f2_abs(f2_sub(b0, b2));
    const f2 cw0 = f2_mul(f2_add(b0, tau5), f2_mul(b1, b2));
    const f2 cw1 = f2_mul(f2_add(b1, tau5), f2_mul(b0, b2));
    const f2 cw2 = f2_mul(f2_add(b2, tau5), f2_mul(b0, b1));
    const f2 dgl = f2_bcast((float)HGKS_DGL), dgr = f2_bcast((float)HGKS_DGR), dgc = f2_bcast((float)HGKS_DGC);
    const f2 e0 = f2_mul(dgl, cw0), e2 = f2_mul(dgr, cw2), g0 = f2_mul(dgr, cw0), g2 = f2_mul(dgl, cw2);
    const f2 a1 = f2_mul(dgc, cw1);
    const f2 dp = f2_add(f2_add(e0, a1), e2), dm = f2_add(f2_add(g0, a1), g2);
    const f2 np = f2_fma(e0, c10, f2_fma(a1, c11, f2_mul(e2, c12)));
    const f2 nm = f2_fma(g0, c10, f2_fma(a1, c11, f2_mul(g2, c12)));
    float den_x, den_y;
    f2_unpack(f2_mul(dp, dm), den_x, den_y);
    const f2 r = f2_pack(weno_recip<float>(den_x), weno_recip<float>(den_y));
    const f2 ga = f2_bcast((float)HGKS_GAUSS), mga = f2_bcast((float)-HGKS_GAUSS);
    vp = f2_fma(ga, f2_mul(f2_mul(np, dm), r), X[2]);
    vm = f2_fma(mga, f2_mul(f2_mul(nm, dp), r), X[2]);
}

// WENO-Z of two stencils (hgks_device.cuh weno_prep + weno_edge_pair): the
// values at the two cell edges, -1/2 (vl) and +1/2 (vr)
static __device__ __forceinline__ void f2_weno_edge(const f2 X[5], f2 &vl, f2 &vr)
{
    const f2 h = f2_bcast(0.5f), t3 = f2_bcast(1.5f), mh = f2_bcast(-0.5f);
    const f2 d1 = f2_sub(X[1], X[0]), d2 = f2_sub(X[2], X[1]), d3 = f2_sub(X[3], X[2]), d4 = f2_sub(X[4], X[3]);
    const f2 c20 = f2_mul(h, f2_sub(d2, d1)), c10 = f2_fma(t3, d2, f2_mul(mh, d1));
    const f2 c21 = f2_mul(h, f2_sub(d3, d2)), c11 = f2_mul(h, f2_add(d3, d2));
    const f2 c22 = f2_mul(h, f2_sub(d4, d3)), c12 = f2_fma(t3, d3, f2_mul(mh, d4));
    const f2 k133 = f2_bcast((float)(13.0 / 3.0)), eps = f2_bcast((float)WENO_EPS);
    const f2 b0 = f2_fma(c10, c10, f2_fma(f2_mul(k133, c20), c20, eps));
    const f2 b1 = f2_fma(c11, c11, f2_fma(f2_mul(k133, c21), c21, eps));
    const f2 b2 = f2_fma(c12, c12, f2_fma(f2_mul(k133, c22), c22, eps));
    const f2 tau5 = f2_abs(f2_sub(b0, b2));
    const f2 cw0 = f2_mul(f2_add(b0, tau5), f2_mul(b1, b2));
    const f2 cw1 = f2_mul(f2_add(b1, tau5), f2_mul(b0, b2));
    const f2 cw2 = f2_mul(f2_add(b2, tau5), f2_mul(b0, b1));
    const f2 c01 = f2_bcast(0.1f), c03 = f2_bcast(0.3f), c06 = f2_bcast(0.6f), c16 = f2_bcast((float)(1.0 / 6.0));
    const f2 a1 = f2_mul(c06, cw1);
    const f2 r0 = f2_mul(c01, cw0), r2 = f2_mul(c03, cw2);  // right edge weights
    const f2 l0 = f2_mul(c03, cw0), l2 = f2_mul(c01, cw2);  // left edge weights
    const f2 p0 = f2_fma(c20, c16, X[2]), p1 = f2_fma(c21, c16, X[2]), p2 = f2_fma(c22, c16, X[2]);
    const f2 nr = f2_fma(r0, f2_fma(h, c10, p0), f2_fma(a1, f2_fma(h, c11, p1), f2_mul(r2, f2_fma(h, c12, p2))));
    const f2 nl = f2_fma(l0, f2_fma(mh, c10, p0), f2_fma(a1, f2_fma(mh, c11, p1), f2_mul(l2, f2_fma(mh, c12, p2))));
    const f2 dr = f2_add(f2_add(r0, a1), r2), dl = f2_add(f2_add(l0, a1), l2);
    float den_x, den_y;
    f2_unpack(f2_mul(dr, dl), den_x, den_y);
    const f2 r = f2_pack(weno_recip<float>(den_x), weno_recip<float>(den_y));
    vr = f2_mul(f2_mul(nr, dl), r);
    vl = f2_mul(f2_mul(nl, dr), r);
}

// quartic through five averages (hgks_device.cuh quartic_value_pair /
// quartic_deriv_pair): values and derivatives at -+sqrt(3)/6
static __device__ __forceinline__ void f2_quartic_value(const f2 X[5], f2 &vm, f2 &vp)
{
    const f2 e = f2_fma(f2_bcast((float)(-1.0 / 4320.0)), f2_add(X[0], X[4]),
                        f2_fma(f2_bcast((float)(1.0 / 1080.0)), f2_add(X[1], X[3]),
                               f2_mul(f2_bcast((float)(719.0 / 720.0)), X[2])));
    const f2 o = f2_mul(f2_bcast((float)HGKS_SQ3),
                        f2_fma(f2_bcast((float)(7.0 / 432.0)), f2_sub(X[0], X[4]),
                               f2_mul(f2_bcast((float)(25.0 / 216.0)), f2_sub(X[3], X[1]))));
    vm = f2_sub(e, o);
    vp = f2_add(e, o);
}
static __device__ __forceinline__ void f2_quartic_deriv(const f2 X[5], f2 &dm, f2 &dp)
{
    const f2 c = f2_fma(f2_bcast((float)(1.0 / 12.0)), f2_sub(X[0], X[4]),
                        f2_mul(f2_bcast((float)(2.0 / 3.0)), f2_sub(X[3], X[1])));
    const f2 s = f2_mul(f2_bcast((float)HGKS_SQ3),
                        f2_fma(f2_bcast((float)(1.0 / 54.0)), f2_add(X[0], X[4]),
                               f2_fma(f2_bcast((float)(-13.0 / 54.0)), f2_add(X[1], X[3]),
                                      f2_mul(f2_bcast((float)(24.0 / 54.0)), X[2]))));
    dm = f2_add(c, s);
    dp = f2_sub(c, s);
}

}  // namespace hgks
