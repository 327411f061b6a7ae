// hgks_mixed.cu -- kernels of the mixed-precision sweep (HGKS_MIXED); the
// per-position work and the precision split are in hgks_passes_mx.cuh.
#include "hgks_passes_mx.cuh"

namespace hgks {

__global__ void __launch_bounds__(128) k_normal_mx(Params P, int d, Box B, const double *__restrict__ q,
                                                   double *__restrict__ fqd, float *__restrict__ fqf,
                                                   const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(B) || ctl->flag) return;
    pos_normal_mx(P, d, B, q, fqd, fqf, t);
}

__global__ void __launch_bounds__(128) k_tan1_mx(Params P, int d, Box Bt, Box Bq, const double *__restrict__ fqd,
                                                 const float *__restrict__ fqf, double *__restrict__ t1d,
                                                 float *__restrict__ t1f, const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(Bt) || ctl->flag) return;
    pos_tan1_mx(P, d, Bt, Bq, fqd, fqf, t1d, t1f, t);
}

__global__ void __launch_bounds__(128) k_flux_mx(Params P, int d, Box Bf, Box Bt, const double *__restrict__ t1d,
                                                 const float *__restrict__ t1f, double *__restrict__ F,
                                                 const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(Bf) || ctl->flag) return;
    pos_flux_mx(P, d, Bf, Bt, t1d, t1f, F, ctl->dt, t);
}

static inline unsigned gridx(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// the FP64 fq / t1 buffers hold the mixed arrays: doubles first, then floats
void launch_sweep_mixed(const Params &P, int d, const double *q, double *fq, double *t1, double *F, const Ctl *ctl,
                        cudaStream_t st, int which)
{
    Box Bq = box_fq(P, d), Bt = box_t1(P, d), Bf = box_face(P, d);
    const long long nq = box_count(Bq), nt = box_count(Bt);
    double *fqd = fq;
    float *fqf = (float *)(fq + 15 * nq);
    double *t1d = t1;
    float *t1f = (float *)(t1 + 50 * nt);
    if (which == 0) k_normal_mx<<<gridx(nq, 128), 128, 0, st>>>(P, d, Bq, q, fqd, fqf, ctl);
    else if (which == 1) k_tan1_mx<<<gridx(nt, 128), 128, 0, st>>>(P, d, Bt, Bq, fqd, fqf, t1d, t1f, ctl);
    else k_flux_mx<<<gridx(box_count(Bf), 128), 128, 0, st>>>(P, d, Bf, Bt, t1d, t1f, F, ctl);
}

}  // namespace hgks
