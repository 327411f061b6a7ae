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

// Normal and first tangential passes fused, for the sweeps whose first
// tangential direction is x (y and z): one block per segment of NT_X
// consecutive positions of an x row of the first-tangential box.  The block
// reconstructs the NT_X + 4 pass-1 records the segment reads into shared
// memory (pos_normal_mx's arithmetic), then the first tangential values from
// there (tan1_mx_rows' arithmetic), so the pass-1 records never travel
// through HBM and the tangential stencils read shared memory instead of
// waiting on global loads.
constexpr int NT_X = 128, NT_Q = NT_X + 4;

__global__ void __launch_bounds__(NT_X, 4) k_nt1x_mx(Params P, int d, Box Bq, Box Bt, const float2 *__restrict__ q2,
                                                    T1Mx o, const Ctl *__restrict__ ctl)
{
    __shared__ float2 sv[15 * NT_Q];
    __shared__ float svs[15 * NT_Q];
    if (ctl->flag) return;
    const int nseg = (Bt.E[0] + NT_X - 1) / NT_X;
    const long long row = blockIdx.x / nseg;
    const int x0 = (int)(blockIdx.x % nseg) * NT_X;
    int p[3];
    p[1] = (int)(row % Bt.E[1]) + Bt.O[1];
    p[2] = (int)(row / Bt.E[1]) + Bt.O[2];
    // pass-1 records of x0 - 2 .. x0 + NT_X + 1 (those inside the box)
    for (int k = threadIdx.x; k < NT_Q; k += NT_X) {
        p[0] = x0 - 2 + k;
        if (p[0] < Bq.E[0] + Bq.O[0]) normal_mx_at(P, d, p, q2, sv, svs, NT_Q, k);
    }
    __syncthreads();
    const int x = x0 + (int)threadIdx.x;
    if (x < Bt.E[0]) {
        p[0] = x;
        tan1_mx_from(sv, svs, NT_Q, threadIdx.x + 2, 1, o.th, o.tl, o.ts, box_count(Bt), blin(Bt, p));
    }
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
// returns the number of kernels launched (the y and z sweeps run passes 0
// and 1 as one fused kernel, launched for which == 0)
int launch_sweep_mixed(const Params &P, int d, const double *qf, double *fq, double *t1, double *F, const Ctl *ctl,
                       cudaStream_t st, int which, bool t64)
{
    Box Bq = box_fq(P, d), Bt = box_t1(P, d), Bf = box_face(P, d);
    const long long nq = box_count(Bq), nt = box_count(Bt);
    const bool fused = tdir(d, 0) == 0;
    if (which == 0 && fused) {
        const long long rows = (long long)Bt.E[1] * Bt.E[2], nseg = (Bt.E[0] + NT_X - 1) / NT_X;
        k_nt1x_mx<<<(unsigned)(rows * nseg), NT_X, 0, st>>>(P, d, Bq, Bt, (const float2 *)qf, t1_mx(t1, nt), ctl);
    } else if (which == 1 && fused) {
        return 0;
    } else if (which == 0) k_normal_mx<<<gridx(nq, 128), 128, 0, st>>>(P, d, Bq, (const float2 *)qf, fq_mx(fq, nq), ctl);
    else if (which == 1) k_tan1_mx<<<gridx(nt, 128), 128, 0, st>>>(P, d, Bt, Bq, fq_mx(fq, nq), t1_mx(t1, nt), ctl);
    else if (t64)
        k_flux_mx<true><<<(unsigned)flux_tiling(P, d).count, FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM, st>>>(
            P, d, Bf, Bt, t1_mx(t1, nt), F, ctl);
    else
        k_flux_mx<false><<<(unsigned)flux_tiling(P, d).count, FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM, st>>>(
            P, d, Bf, Bt, t1_mx(t1, nt), F, ctl);
    return 1;
}

}  // namespace hgks
