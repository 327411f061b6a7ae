// hgks_flux.cu -- per-sweep reconstruction and gas-kinetic flux kernels (FP64).
//
// One sweep (direction d) of the interface fluxes of arXiv 2207.01173 Sec. 2
// runs as three passes over interface positions, each one thread per position
// with x-adjacent threads on x-adjacent memory:
//   k_normal: fifth-order WENO-Z of the cell averages normal to the face
//             (left/right states, parabola slopes, equilibrium by the
//             compatibility condition and its central slope) on every face of
//             the sweep, including two tangential ghost rows on each side;
//   k_tan1:   WENO-Z / quartic reconstruction along the first tangential
//             direction to the two Gauss lines of each face;
//   k_flux:   reconstruction along the second tangential direction to the
//             2x2 Gauss points, the BGK flux of Eq. "flux" there, the
//             linear-in-time fit of Eq. "expansion-1" and the Gauss sum
//             (weights 1/4) times the face area.
#include "hgks_passes.cuh"

namespace hgks {

__global__ void __launch_bounds__(128) k_normal(Params P, int d, Box B, const double *__restrict__ q,
                                                double *__restrict__ fq, const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(B) || ctl->flag) return;
    pos_normal(P, d, B, q, fq, t);
}

__global__ void __launch_bounds__(128) k_tan1(Params P, int d, Box Bt, Box Bq, const double *__restrict__ fq,
                                              double *__restrict__ t1, const Ctl *__restrict__ ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(Bt) || ctl->flag) return;
    pos_tan1(P, d, Bt, Bq, fq, t1, t);
}

// two blocks of 128 per SM: 255 registers and FLUX_SMEM (113.7 kB) of staged
// Gauss-point inputs each
__global__ void __launch_bounds__(FLUX_BLOCK, 2) k_flux(Params P, int d, Box Bf, Box Bt,
                                                        const double *__restrict__ t1, double *__restrict__ F,
                                                        const Ctl *__restrict__ ctl)
{
    extern __shared__ double flux_sm[];
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= box_count(Bf) || ctl->flag) return;
    pos_flux(P, d, Bf, Bt, t1, F, ctl->dt, t, flux_sm);
}

// opt in to the dynamic shared memory of the FP64 flux kernel on the current
// device; called when a handle is created, before any launch or capture
cudaError_t fp64_setup()
{
    return cudaFuncSetAttribute((const void *)k_flux, cudaFuncAttributeMaxDynamicSharedMemorySize, FLUX_SMEM);
}

static inline unsigned grid_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

void launch_normal(const Params &P, int d, const double *q, double *fq, const Ctl *ctl, cudaStream_t st)
{
    Box B = box_fq(P, d);
    k_normal<<<grid_for(box_count(B), 128), 128, 0, st>>>(P, d, B, q, fq, ctl);
}
void launch_tan1(const Params &P, int d, const double *fq, double *t1, const Ctl *ctl, cudaStream_t st)
{
    Box Bt = box_t1(P, d), Bq = box_fq(P, d);
    k_tan1<<<grid_for(box_count(Bt), 128), 128, 0, st>>>(P, d, Bt, Bq, fq, t1, ctl);
}
void launch_flux(const Params &P, int d, const double *t1, double *F, const Ctl *ctl, cudaStream_t st)
{
    Box Bf = box_face(P, d), Bt = box_t1(P, d);
    k_flux<<<grid_for(box_count(Bf), FLUX_BLOCK), FLUX_BLOCK, FLUX_SMEM, st>>>(P, d, Bf, Bt, t1, F, ctl);
}

}  // namespace hgks
