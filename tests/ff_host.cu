// Host instantiation of the float-float operations that the mixed-precision
// path builds on (paper_2207_01173_gb300/csrc/hgks_ff.cuh), applied
// element-wise over arrays, for the CPU checks in tests/test_ff.py.
#include "../paper_2207_01173_gb300/csrc/hgks_ff.cuh"

using hgks::ff;

extern "C" {

void ff_host_two_sum(int n, const float *a, const float *b, float *hi, float *lo, int fast)
{
    for (int i = 0; i < n; i++) {
        const ff r = fast ? hgks::ff_fast_two_sum(a[i], b[i]) : hgks::ff_two_sum(a[i], b[i]);
        hi[i] = r.hi;
        lo[i] = r.lo;
    }
}

void ff_host_of_double(int n, const double *x, float *hi, float *lo)
{
    for (int i = 0; i < n; i++) {
        const ff r = hgks::ff_of_double(x[i]);
        hi[i] = r.hi;
        lo[i] = r.lo;
    }
}

// op: 0 add, 1 sub, 2 mul (x, y float-float); 3 add_f, 4 mul_f (y = yh, a float); 5 recip (x only)
void ff_host_binary(int n, int op, const float *xh, const float *xl, const float *yh, const float *yl, float *hi,
                    float *lo)
{
    for (int i = 0; i < n; i++) {
        const ff x{ xh[i], xl[i] }, y{ yh[i], yl[i] };
        ff r;
        switch (op) {
        case 0: r = hgks::ff_add(x, y); break;
        case 1: r = hgks::ff_sub(x, y); break;
        case 2: r = hgks::ff_mul(x, y); break;
        case 3: r = hgks::ff_add_f(x, yh[i]); break;
        case 4: r = hgks::ff_mul_f(x, yh[i]); break;
        default: r = hgks::ff_recip(x); break;
        }
        hi[i] = r.hi;
        lo[i] = r.lo;
    }
}

}  // extern "C"
