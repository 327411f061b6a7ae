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
#include "hgks_bodies.cuh"
#include "hgks_kernels.cuh"

namespace hgks {

__host__ __device__ inline int perm_of(int d, int c)
{
    // velocity components of the (normal, t1, t2) frame of sweep d
    if (c == 0 || c == 4) return c;
    if (d == 0) return c;
    if (d == 1) return c == 1 ? 2 : (c == 2 ? 1 : 3);
    return c == 1 ? 3 : (c == 2 ? 1 : 2);
}

__device__ __forceinline__ void box_pos(const Box &b, long long t, int p[3])
{
    p[0] = (int)(t % b.E[0]) + b.O[0];
    t /= b.E[0];
    p[1] = (int)(t % b.E[1]) + b.O[1];
    p[2] = (int)(t / b.E[1]) + b.O[2];
}
__device__ __forceinline__ long long box_lin(const Box &b, const int p[3])
{
    return ((long long)(p[2] - b.O[2]) * b.E[1] + (p[1] - b.O[1])) * b.E[0] + (p[0] - b.O[0]);
}
__device__ __forceinline__ long long box_stride(const Box &b, int e)
{
    return e == 0 ? 1 : (e == 1 ? (long long)b.E[0] : (long long)b.E[0] * b.E[1]);
}

Box box_fq(const Params &P, int d)
{
    Box b;
    for (int e = 0; e < 3; e++) {
        b.E[e] = e == d ? P.n[e] + 1 : P.n[e] + 4;
        b.O[e] = e == d ? 0 : -2;
    }
    return b;
}
Box box_t1(const Params &P, int d)
{
    Box b;
    int t2 = tdir(d, 1);
    for (int e = 0; e < 3; e++) {
        b.E[e] = e == d ? P.n[e] + 1 : (e == t2 ? P.n[e] + 4 : P.n[e]);
        b.O[e] = e == t2 ? -2 : 0;
    }
    return b;
}
Box box_face(const Params &P, int d)
{
    Box b;
    for (int e = 0; e < 3; e++) {
        b.E[e] = e == d ? P.n[e] + 1 : P.n[e];
        b.O[e] = 0;
    }
    return b;
}

// ---------------------------------------------------------------------------
// pass 1: normal reconstruction
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_normal(Params P, int d, Box B, const double *__restrict__ q,
                                                double *__restrict__ fq, const Ctl *__restrict__ ctl)
{
    const long long nq = box_count(B);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq || ctl->flag) return;
    int p[3];
    box_pos(B, t, p);
    int c0[3] = { p[0], p[1], p[2] };
    c0[d] = p[d] - 3;
    const long long base = pidx(P, c0[0], c0[1], c0[2]);
    const long long sd = d == 0 ? 1 : (d == 1 ? P.sy : P.sz);
    auto load = [&](int c, int m) { return q[(long long)perm_of(d, c) * P.cs + base + m * sd]; };
    auto store = [&](int slot, double v) { fq[slot * nq + t] = v; };
    normal_body<double>(load, store, P.K);
}

// ---------------------------------------------------------------------------
// pass 2: first tangential direction
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_tan1(Params P, int d, Box Bt, Box Bq, const double *__restrict__ fq,
                                              double *__restrict__ t1, const Ctl *__restrict__ ctl)
{
    const long long nt = box_count(Bt), nq = box_count(Bq);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt || ctl->flag) return;
    int p[3];
    box_pos(Bt, t, p);
    const long long base = box_lin(Bq, p), s1 = box_stride(Bq, tdir(d, 0));
    auto load = [&](int slot, int j) { return fq[slot * nq + base + (j - 2) * s1]; };
    auto store = [&](int slot, double v) { t1[slot * nt + t] = v; };
    tan1_body<double>(load, store);
}

// ---------------------------------------------------------------------------
// pass 3: second tangential direction, Gauss-point fluxes, Gauss sum
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_flux(Params P, int d, Box Bf, Box Bt, const double *__restrict__ t1,
                                              double *__restrict__ F, const Ctl *__restrict__ ctl)
{
    const long long nf = box_count(Bf), nt = box_count(Bt);
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf || ctl->flag) return;
    int p[3];
    box_pos(Bf, t, p);
    const int e1 = tdir(d, 0), e2 = tdir(d, 1);
    const int f = p[d], a = p[e1], b = p[e2];
    const long long base = box_lin(Bt, p), s2 = box_stride(Bt, e2);
    FaceGeom G;
    G.ihn = 1.0 / (d == 1 ? P.my_face[f] : P.h[d]);
    if (d == 0) G.area = P.hy_cell[a] * P.h[2];
    else if (d == 1) G.area = P.h[0] * P.h[2];
    else G.area = P.h[0] * P.hy_cell[b];
    for (int m = 0; m < 2; m++) {
        G.ih1[m] = 1.0 / (e1 == 1 ? P.my_gp[2 * a + m] : P.h[e1]);
        G.ih2[m] = 1.0 / (e2 == 1 ? P.my_gp[2 * b + m] : P.h[e2]);
    }
    auto load = [&](int slot, int j) { return t1[slot * nt + base + (j - 2) * s2]; };
    double Fs[5], dFs[5];
    flux_body<double>(load, G, P, ctl->dt, Fs, dFs);
#pragma unroll
    for (int c = 0; c < 5; c++) {
        F[(long long)perm_of(d, c) * nf + t] = Fs[c];
        F[(long long)(5 + perm_of(d, c)) * nf + t] = dFs[c];
    }
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
    k_flux<<<grid_for(box_count(Bf), 128), 128, 0, st>>>(P, d, Bf, Bt, t1, F, ctl);
}

}  // namespace hgks
