// hgks_kernels.cuh -- launch interface between the host API and the kernels.
#pragma once
#include "hgks_device.cuh"

namespace hgks {

// a box of interface (or cell) positions, x fastest; position = index + offset
struct Box {
    int E[3];
    int O[3];
};

__host__ __device__ inline long long box_count(const Box &b) { return (long long)b.E[0] * b.E[1] * b.E[2]; }

// tangential directions of each sweep in reconstruction order, and the
// velocity-component permutation into the sweep's (normal, t1, t2) frame
__host__ __device__ inline int tdir(int d, int t) { return d == 0 ? (t == 0 ? 1 : 2) : (d == 1 ? (t == 0 ? 0 : 2) : (t == 0 ? 0 : 1)); }

// number of doubles per position in the intermediate arrays
constexpr int FQ_N = 30;   // Ql, Qr, dQl, dQr, Q0, dQ0 (x5 components), normal reconstruction
constexpr int T1_N = 110;  // per Gauss line (2): 25 WENO values, 15 linear values, 15 linear derivatives
constexpr int F_N = 10;    // F^n and dF^n/dt (x5 components), global component order

// boxes of sweep d: the normal pass (all faces, two tangential ghost rows
// each side), the first tangential pass (ghost rows along t2 only), the faces
__host__ __device__ inline Box box_fq(const Params &P, int d)
{
    Box b;
    for (int e = 0; e < 3; e++) {
        b.E[e] = e == d ? P.n[e] + 1 : P.n[e] + 4;
        b.O[e] = e == d ? 0 : -2;
    }
    return b;
}
__host__ __device__ inline Box box_t1(const Params &P, int d)
{
    Box b;
    const int t2 = tdir(d, 1);
    for (int e = 0; e < 3; e++) {
        b.E[e] = e == d ? P.n[e] + 1 : (e == t2 ? P.n[e] + 4 : P.n[e]);
        b.O[e] = e == t2 ? -2 : 0;
    }
    return b;
}
__host__ __device__ inline Box box_face(const Params &P, int d)
{
    Box b;
    for (int e = 0; e < 3; e++) {
        b.E[e] = e == d ? P.n[e] + 1 : P.n[e];
        b.O[e] = 0;
    }
    return b;
}

// launches (all on `st`)
void launch_ghost(const Params &P, double *q, cudaStream_t st);
// three z planes starting at interior layer k0 to (to_buf) or from a buffer [5][3][ny+6][nx+6]
void launch_halo_z(const Params &P, double *q, int k0, double *buf, bool to_buf, cudaStream_t st);
void launch_dt_reset(Ctl *ctl, cudaStream_t st);
void launch_cfl(const Params &P, const double *q, Ctl *ctl, cudaStream_t st);
void launch_dt_final(Ctl *ctl, double cfl, double fixed_dt, cudaStream_t st);
void launch_normal(const Params &P, int d, const double *q, double *fq, const Ctl *ctl, cudaStream_t st);
void launch_tan1(const Params &P, int d, const double *fq, double *t1, const Ctl *ctl, cudaStream_t st);
void launch_flux(const Params &P, int d, const double *t1, double *F, const Ctl *ctl, cudaStream_t st);
void launch_wall(const Params &P, const double *Fy, Ctl *ctl, double lxlz, cudaStream_t st);
// mixed-precision sweep passes (which: 0 normal, 1 first tangential, 2 flux),
// using the same fq / t1 buffers as the FP64 passes
cudaError_t fp64_setup();
cudaError_t mixed_setup();
void launch_split_mixed(const Params &P, const double *q, double *qf, const Ctl *ctl, cudaStream_t st);
// t64: the HGKS_MIXED_T64 flux (FP64 temperature, collision time and time
// coefficients).  Returns the kernels launched (0 for the first tangential
// pass of the y and z sweeps, which the normal pass's fused kernel does).
int launch_sweep_mixed(const Params &P, int d, const double *qf, double *fq, double *t1, double *F, const Ctl *ctl,
                       cudaStream_t st, int which, bool t64 = false);
// stage 1: qs = q + dt/2 L + dt^2/8 dL, r = q + dt L + dt^2/6 dL;  stage 2: qn = r + dt^2/3 dL
void launch_update(const Params &P, int stage, const double *q, const double *const F[3], double *out_a,
                   double *out_b, Ctl *ctl, cudaStream_t st);
// L and dL/dt into interior arrays [5][N]
void launch_rhs_out(const Params &P, const double *q, const double *const F[3], double *L, double *dL, const Ctl *ctl,
                    cudaStream_t st);
void launch_commit(Ctl *ctl, int newbuf, cudaStream_t st);
void launch_set_dt(Ctl *ctl, double dt, cudaStream_t st);
void launch_scatter(const Params &P, const double *in, double *q, cudaStream_t st);
void launch_gather(const Params &P, const double *q, double *out, cudaStream_t st);
// diagnostics: partial sums per block into scratch, then one block folds them
int stats_blocks(const Params &P);
void launch_stats(const Params &P, const double *q, double *scratch, double *out12, double rho_ref, cudaStream_t st);
// FP64 FMA throughput of the device (TFLOP/s)
cudaError_t fp64_probe(double *tflops);
// initial fields
void launch_init_tgv(const Params &P, double *q, const double *yface, double x0, double z0, double Ma, double U0,
                     double rho0, cudaStream_t st);
void launch_init_channel(const Params &P, double *q, const double *ycen, double ymid, double hh, double Ma_b,
                         double amp, unsigned long long seed, cudaStream_t st);
void launch_init_wave(const Params &P, double *q, double x0, double y0, double z0, double hy, double amp,
                      cudaStream_t st);

}  // namespace hgks
