// hgks_ff.cuh -- float-float ("double-float") arithmetic: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, which
// carries about 48 significant bits in FP32 operations only.
//
// The error-free transformations are the classical ones: Knuth's TwoSum (the
// rounding error of a + b, no ordering needed), Dekker's FastTwoSum (the same
// when |a| >= |b|), and the product error from one fused multiply-add
// (fma(a, b, -p) is exact for p = fl(a b)).  The compound operations below
// follow the usual double-word algorithms built from them; each keeps a
// relative error of a few units of 2^-46 or better away from underflow.
// Nothing here may be compiled with fast-math reassociation.  The functions
// are host-callable too, so the same source can be checked on the CPU.
#pragma once
#include <cuda_runtime.h>

#define HGKS_FF __host__ __device__ __forceinline__

namespace hgks {

struct ff {
    float hi, lo;
};

HGKS_FF ff ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return ff{ s, e };
}

HGKS_FF ff ff_fast_two_sum(float a, float b)  // needs |a| >= |b| (or a == 0)
{
    const float s = a + b;
    const float e = b - (s - a);
    return ff{ s, e };
}

HGKS_FF ff ff_from(float a) { return ff{ a, 0.0f }; }

// nearest float-float of an FP64 value (two roundings; exact up to 2^-48 relative)
HGKS_FF ff ff_of_double(double x)
{
#ifdef __CUDA_ARCH__
    const float h = __double2float_rn(x);
    return ff{ h, __double2float_rn(x - (double)h) };
#else
    const float h = (float)x;  // round to nearest, the host's default mode
    return ff{ h, (float)(x - (double)h) };
#endif
}
HGKS_FF double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
HGKS_FF float ff_to_float(ff a) { return a.hi + a.lo; }

// x + y, both float-float (accurate even under cancellation)
HGKS_FF ff ff_add(ff x, ff y)
{
    ff s = ff_two_sum(x.hi, y.hi);
    const ff t = ff_two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return ff_fast_two_sum(s.hi, s.lo);
}
HGKS_FF ff ff_neg(ff x) { return ff{ -x.hi, -x.lo }; }
HGKS_FF ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// x + b, b a float
HGKS_FF ff ff_add_f(ff x, float b)
{
    const ff s = ff_two_sum(x.hi, b);
    return ff_fast_two_sum(s.hi, s.lo + x.lo);
}

// x * y
HGKS_FF ff ff_mul(ff x, ff y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return ff_fast_two_sum(p, e);
}

// x * b, b a float
HGKS_FF ff ff_mul_f(ff x, float b)
{
    const float p = x.hi * b;
    const float e = fmaf(x.lo, b, fmaf(x.hi, b, -p));
    return ff_fast_two_sum(p, e);
}

// x * 2^k for an exact power-of-two factor s (no rounding)
HGKS_FF ff ff_scale(ff x, float s) { return ff{ x.hi * s, x.lo * s }; }

// 1 / x: FP32 reciprocal refined by one Newton step on the float-float residual
HGKS_FF ff ff_recip(ff x)
{
    const float r = 1.0f / x.hi;
    float e = fmaf(-x.hi, r, 1.0f);  // exact residual of the leading part
    e = fmaf(-x.lo, r, e);
    return ff_fast_two_sum(r, r * e);
}

}  // namespace hgks
