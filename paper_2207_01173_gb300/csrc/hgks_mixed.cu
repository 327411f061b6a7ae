// hgks_mixed.cu -- kernels of the mixed-precision sweep (HGKS_MIXED); the
// per-position work and the precision split are in hgks_passes_mx.cuh.
#include "hgks_passes_mx.cuh"

namespace hgks {

__global__ void __launch_bounds__(256) k_split_mx(Params P, const double *__restrict__ q, float2 *__restrict__ q2,
                                                  const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.cs || ctl->flag) return;
    pos_split_mx(P, q, q2, t);
}

__global__ void __launch_bounds__(128) k_normal_mx(Params P, int d, Box B, const float2 *__restrict__ q2, FqMx o,
                                                   const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(B) || ctl->flag) return;
    pos_normal_mx(P, d, B, q2, o, t);
}

__global__ void __launch_bounds__(128, 4) k_tan1_mx(Params P, int d, Box Bt, Box Bq, FqMx in, T1Mx o,
                                                 const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(Bt) || ctl->flag) return;
    pos_tan1_mx(P, d, Bt, Bq, in, o, t);
}

// One block per tile of 32 x 4 faces (flux_mx_tile); dynamic shared memory
// holds the Gauss-point inputs (GP_SLOTS floats per thread, 66.5 kB) and the
// staged t1 rows (4 kB), which allows three blocks per SM and so 170
// registers per thread.
// T64: the HGKS_MIXED_T64 variant (temperature, collision time and time
// coefficients of each Gauss point in FP64).
template <bool T64>
__global__ void __launch_bounds__(FLUX_MX_BLOCK, 3) k_flux_mx(Params P, int d, Box Bf, Box Bt, T1Mx in,
                                                              double *__restrict__ F, const Ctl *__restrict__ ctl)
{
    extern __shared__ float gp_sm[];
    if (ctl->flag) return;
    flux_mx_tile<T64>(P, d, Bf, Bt, in, F, ctl->dt, blockIdx.x, gp_sm);
}

// opt in to the dynamic shared memory of the mixed flux kernels on the current
// device; called when a mixed handle is created, before any launch or capture
cudaError_t mixed_setup()
{
    cudaError_t e = cudaFuncSetAttribute((const void *)k_flux_mx<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FLUX_MX_TILE_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_flux_mx<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                FLUX_MX_TILE_SMEM);
}

static inline unsigned gridx(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// qf holds the split state: 5 planes of cs (hi, lo) float pairs
void launch_split_mixed(const Params &P, const double *q, double *qf, const Ctl *ctl, cudaStream_t st)
{
    k_split_mx<<<gridx(P.cs, 256), 256, 0, st>>>(P, q, (float2 *)qf, ctl);
}

// the FP64-sized fq / t1 buffers hold the float planes of the mixed passes
void launch_sweep_mixed(const Params &P, int d, const double *qf, double *fq, double *t1, double *F, const Ctl *ctl,
                        cudaStream_t st, int which, bool t64)
{
    Box Bq = box_fq(P, d), Bt = box_t1(P, d), Bf = box_face(P, d);
    const long long nq = box_count(Bq), nt = box_count(Bt);
    if (which == 0) k_normal_mx<<<gridx(nq, 128), 128, 0, st>>>(P, d, Bq, (const float2 *)qf, fq_mx(fq, nq), ctl);
    else if (which == 1) k_tan1_mx<<<gridx(nt, 128), 128, 0, st>>>(P, d, Bt, Bq, fq_mx(fq, nq), t1_mx(t1, nt), ctl);
    else if (t64)
        k_flux_mx<true><<<(unsigned)flux_tiling(P, d).count, FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM, st>>>(
            P, d, Bf, Bt, t1_mx(t1, nt), F, ctl);
    else
        k_flux_mx<false><<<(unsigned)flux_tiling(P, d).count, FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM, st>>>(
            P, d, Bf, Bt, t1_mx(t1, nt), F, ctl);
}

}  // namespace hgks
