// hgks_misc.cu -- ghost fill, time step, stage update, diagnostics and initial
// fields of the HGKS step (FP64), arXiv 2207.01173 Sec. 2 and Sec. 4.
#include "hgks_passes.cuh"

namespace hgks {

static inline unsigned grid_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// ghost cells (three layers; periodic copy or isothermal no-slip mirror).
// Directions are filled in the order x, y, z, each over the already filled
// extent of the earlier directions, so edges and corners are filled too.
// ---------------------------------------------------------------------------
__global__ void k_ghost(Params P, double *q, int d)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ghost_count(P, d)) return;
    pos_ghost(P, q, d, t);
}

void launch_ghost(const Params &P, double *q, cudaStream_t st)
{
    for (int d = 0; d < 3; d++) k_ghost<<<grid_for(ghost_count(P, d), 256), 256, 0, st>>>(P, q, d);
}

// ---------------------------------------------------------------------------
// halo layers of a z slab: the three z planes next to a side, whole padded
// planes (their x / y ghosts included), to or from a caller's buffer
// [5][3][ny + 6][nx + 6].  get: interior layers k0 .. k0 + 2 -> buffer;
// set: buffer -> ghost layers.  The planes of one component are contiguous.
// ---------------------------------------------------------------------------
__global__ void k_halo_z(Params P, double *q, int k0, double *buf, int to_buf)
{
    const long long per_c = 3 * P.sz;  // doubles of one component
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 5 * per_c) return;
    const int c = (int)(t / per_c);
    const long long r = t - c * per_c;  // offset within the three planes
    const long long qi = (long long)c * P.cs + (long long)(k0 + NG) * P.sz + r;
    if (to_buf) buf[t] = q[qi];
    else q[qi] = buf[t];
}

// k0: first of the three z layers (interior index; -3 or nz for the ghosts)
void launch_halo_z(const Params &P, double *q, int k0, double *buf, bool to_buf, cudaStream_t st)
{
    const long long n = 5 * 3 * P.sz;
    k_halo_z<<<grid_for(n, 256), 256, 0, st>>>(P, q, k0, buf, to_buf ? 1 : 0);
}

// ---------------------------------------------------------------------------
// time step: dt = cfl * min over cells, directions of dx_d / (|u_d| + c)
// ---------------------------------------------------------------------------
__global__ void k_dt_reset(Ctl *ctl) { ctl->dtmin_bits = 0x7FF0000000000000ull; /* +inf */ }

__global__ void __launch_bounds__(256) k_cfl(Params P, const double *__restrict__ q, Ctl *ctl)
{
    __shared__ double red[8];
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = INFINITY;
    if (t < P.ncell && !ctl->flag) v = pos_cfl(P, q, t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
        // positive doubles order like their bit patterns
        if (threadIdx.x == 0 && v < INFINITY) atomicMin(&ctl->dtmin_bits, (unsigned long long)__double_as_longlong(v));
    }
}

__global__ void k_dt_final(Ctl *ctl, double cfl, double fixed_dt)
{
    if (ctl->flag) return;
    ctl->dt = fixed_dt > 0.0 ? fixed_dt : cfl * __longlong_as_double((long long)ctl->dtmin_bits);
}
__global__ void k_set_dt(Ctl *ctl, double dt) { ctl->dt = dt; }

void launch_dt_reset(Ctl *ctl, cudaStream_t st) { k_dt_reset<<<1, 1, 0, st>>>(ctl); }
void launch_cfl(const Params &P, const double *q, Ctl *ctl, cudaStream_t st)
{
    k_cfl<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, q, ctl);
}
void launch_dt_final(Ctl *ctl, double cfl, double fixed_dt, cudaStream_t st)
{
    k_dt_final<<<1, 1, 0, st>>>(ctl, cfl, fixed_dt);
}
void launch_set_dt(Ctl *ctl, double dt, cudaStream_t st) { k_set_dt<<<1, 1, 0, st>>>(ctl, dt); }

// ---------------------------------------------------------------------------
// flux divergence (Eq. "semi2"), body force and the S2O4 stages (Eq. "two-stage")
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_update(Params P, int stage, const double *__restrict__ q,
                                                const double *__restrict__ F0, const double *__restrict__ F1,
                                                const double *__restrict__ F2, double *__restrict__ oa,
                                                double *__restrict__ ob, Ctl *ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell || ctl->flag) return;
    if (!pos_update(P, stage, q, F0, F1, F2, oa, ob, ctl->dt, t)) atomicOr(&ctl->flag, 1);
}

void launch_update(const Params &P, int stage, const double *q, const double *const F[3], double *out_a,
                   double *out_b, Ctl *ctl, cudaStream_t st)
{
    k_update<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, stage, q, F[0], F[1], F[2], out_a, out_b, ctl);
}

__global__ void k_rhs_out(Params P, const double *q, const double *F0, const double *F1, const double *F2, double *L,
                          double *dL, const Ctl *ctl)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell || ctl->flag) return;
    int i = (int)(t % P.n[0]);
    long long r = t / P.n[0];
    int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
    const double *F[3] = { F0, F1, F2 };
    double a[5], b[5];
    cell_rhs(P, q, F, i, j, k, pidx(P, i, j, k), a, b);
#pragma unroll
    for (int c = 0; c < 5; c++) {
        L[c * P.ncell + t] = a[c];
        dL[c * P.ncell + t] = b[c];
    }
}

void launch_rhs_out(const Params &P, const double *q, const double *const F[3], double *L, double *dL, const Ctl *ctl,
                    cudaStream_t st)
{
    k_rhs_out<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, q, F[0], F[1], F[2], L, dL, ctl);
}

__global__ void k_commit(Ctl *ctl, int newbuf)
{
    if (ctl->flag) return;
    ctl->t += ctl->dt;
    ctl->step += 1;
    ctl->good = newbuf;
    ctl->last_dt = ctl->dt;
}
void launch_commit(Ctl *ctl, int newbuf, cudaStream_t st) { k_commit<<<1, 1, 0, st>>>(ctl, newbuf); }

// mean wall stress from the x-momentum flux through the y walls (first stage)
__global__ void k_wall(Params P, const double *Fy, Ctl *ctl, double lxlz)
{
    __shared__ double red[2][256];
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const long long n1 = (long long)nx * (ny + 1) * nz;
    double lo = 0.0, hi = 0.0;
    for (long long t = threadIdx.x; t < (long long)nx * nz; t += blockDim.x) {
        int i = (int)(t % nx), k = (int)(t / nx);
        lo += Fy[1 * n1 + ((long long)k * (ny + 1) + 0) * nx + i];
        hi += Fy[1 * n1 + ((long long)k * (ny + 1) + ny) * nx + i];
    }
    red[0][threadIdx.x] = lo;
    red[1][threadIdx.x] = hi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        int walls = 0;
        if (P.bc_lo[1] == 1) { s += -red[0][0]; walls++; }
        if (P.bc_hi[1] == 1) { s += red[1][0]; walls++; }
        ctl->wall_shear = walls ? s / (walls * lxlz) : 0.0;
    }
}
void launch_wall(const Params &P, const double *Fy, Ctl *ctl, double lxlz, cudaStream_t st)
{
    k_wall<<<1, 256, 0, st>>>(P, Fy, ctl, lxlz);
}

// ---------------------------------------------------------------------------
// interior <-> padded copies
// ---------------------------------------------------------------------------
__global__ void k_scatter(Params P, const double *in, double *q)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell) return;
    int i = (int)(t % P.n[0]);
    long long r = t / P.n[0];
    int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
    long long p = pidx(P, i, j, k);
#pragma unroll
    for (int c = 0; c < 5; c++) q[c * P.cs + p] = in[c * P.ncell + t];
}
__global__ void k_gather(Params P, const double *q, double *out)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell) return;
    int i = (int)(t % P.n[0]);
    long long r = t / P.n[0];
    int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
    long long p = pidx(P, i, j, k);
#pragma unroll
    for (int c = 0; c < 5; c++) out[c * P.ncell + t] = q[c * P.cs + p];
}
void launch_scatter(const Params &P, const double *in, double *q, cudaStream_t st)
{
    k_scatter<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, in, q);
}
void launch_gather(const Params &P, const double *q, double *out, cudaStream_t st)
{
    k_gather<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, q, out);
}

// ---------------------------------------------------------------------------
// diagnostics (Sec. 4.1): E_k, enstrophy, eps_com, totals, max Mach.
// Per-block partial sums in a fixed tree order, then one block folds the
// partials in block order: the result does not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int NSTAT = 10;  // vol, ek, ens, eps, mass, mx, my, mz, energy, max_mach
constexpr int STAT_BS = 256;

int stats_blocks(const Params &P) { return (int)grid_for(P.ncell, STAT_BS); }

__global__ void __launch_bounds__(STAT_BS) k_stats(Params P, const double *__restrict__ q, double *scratch)
{
    __shared__ double red[NSTAT][STAT_BS];
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; s++) v[s] = 0.0;
    if (t < P.ncell) {
        int i = (int)(t % P.n[0]);
        long long r = t / P.n[0];
        int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
        long long p = pidx(P, i, j, k);
        const double vol = P.h[0] * P.hy_cell[j] * P.h[2];
        double Q[5];
#pragma unroll
        for (int c = 0; c < 5; c++) Q[c] = q[c * P.cs + p];
        double ir = 1.0 / Q[0];
        double u[3] = { Q[1] * ir, Q[2] * ir, Q[3] * ir };
        double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double pr = (P.gamma - 1.0) * (Q[4] - 0.5 * Q[0] * u2);
        double T = pr * ir;
        double cs = sqrt(P.gamma * pr * ir);
        // velocity gradient by fourth-order central differences of cell-centre velocity
        double gr[3][3];
        const long long st3[3] = { 1, P.sy, P.sz };
        const double hb[3] = { P.h[0], P.my_cen[j], P.h[2] };
#pragma unroll
        for (int b = 0; b < 3; b++) {
            double uu[4][3];
            const int offs[4] = { -2, -1, 1, 2 };
#pragma unroll
            for (int s = 0; s < 4; s++) {
                long long ps = p + offs[s] * st3[b];
                double irs = 1.0 / q[ps];
#pragma unroll
                for (int a = 0; a < 3; a++) uu[s][a] = q[(1 + a) * P.cs + ps] * irs;
            }
#pragma unroll
            for (int a = 0; a < 3; a++)
                gr[a][b] = (uu[0][a] - 8.0 * uu[1][a] + 8.0 * uu[2][a] - uu[3][a]) / (12.0 * hb[b]);
        }
        double wx = gr[2][1] - gr[1][2], wy = gr[0][2] - gr[2][0], wz = gr[1][0] - gr[0][1];
        double w2 = wx * wx + wy * wy + wz * wz;
        double dv = gr[0][0] + gr[1][1] + gr[2][2];
        double mu = viscosity(P, T);
        v[0] = vol;
        v[1] = 0.5 * Q[0] * u2 * vol;
        v[2] = 0.5 * Q[0] * w2 * vol;
        v[3] = mu * (w2 + (4.0 / 3.0) * dv * dv) * vol;
        v[4] = Q[0] * vol;
        v[5] = Q[1] * vol;
        v[6] = Q[2] * vol;
        v[7] = Q[3] * vol;
        v[8] = Q[4] * vol;
        v[9] = sqrt(u2) / cs;
    }
#pragma unroll
    for (int s = 0; s < NSTAT; s++) red[s][threadIdx.x] = v[s];
    __syncthreads();
    for (int w = STAT_BS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int s = 0; s < NSTAT - 1; s++) red[s][threadIdx.x] += red[s][threadIdx.x + w];
            red[NSTAT - 1][threadIdx.x] = fmax(red[NSTAT - 1][threadIdx.x], red[NSTAT - 1][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < NSTAT) scratch[(long long)blockIdx.x * NSTAT + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(STAT_BS) k_stats_final(const double *scratch, int nblk, double *out, double rho_ref)
{
    __shared__ double red[NSTAT][STAT_BS];
    double v[NSTAT];
#pragma unroll
    for (int s = 0; s < NSTAT; s++) v[s] = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
        for (int s = 0; s < NSTAT - 1; s++) v[s] += scratch[(long long)b * NSTAT + s];
        v[NSTAT - 1] = fmax(v[NSTAT - 1], scratch[(long long)b * NSTAT + NSTAT - 1]);
    }
#pragma unroll
    for (int s = 0; s < NSTAT; s++) red[s][threadIdx.x] = v[s];
    __syncthreads();
    for (int w = STAT_BS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int s = 0; s < NSTAT - 1; s++) red[s][threadIdx.x] += red[s][threadIdx.x + w];
            red[NSTAT - 1][threadIdx.x] = fmax(red[NSTAT - 1][threadIdx.x], red[NSTAT - 1][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double vol = red[0][0];
        out[0] = red[1][0] / (rho_ref * vol);  // Ek
        out[1] = red[2][0] / (rho_ref * vol);  // enstrophy
        out[2] = red[3][0] / (rho_ref * vol);  // eps_com
        out[3] = red[4][0];                    // mass
        out[4] = red[5][0];
        out[5] = red[6][0];
        out[6] = red[7][0];
        out[7] = red[8][0];                    // energy
        out[8] = red[9][0];                    // max Mach
        out[9] = vol;
    }
}

void launch_stats(const Params &P, const double *q, double *scratch, double *out, double rho_ref, cudaStream_t st)
{
    int nb = stats_blocks(P);
    k_stats<<<nb, STAT_BS, 0, st>>>(P, q, scratch);
    k_stats_final<<<1, STAT_BS, 0, st>>>(scratch, nb, out, rho_ref);
}

// ---------------------------------------------------------------------------
// initial fields (Sec. 4.1 Taylor-Green vortex, Sec. 4.2 channel, smooth wave)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cell_of(const Params &P, long long t, int &i, int &j, int &k)
{
    i = (int)(t % P.n[0]);
    long long r = t / P.n[0];
    j = (int)(r % P.n[1]);
    k = (int)(r / P.n[1]);
}

__global__ void k_init_tgv(Params P, double *q, const double *yface, double x0, double z0, double Ma, double U0,
                           double rho0)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell) return;
    int i, j, k;
    cell_of(P, t, i, j, k);
    const double xl[3] = { x0 + i * P.h[0], yface[j], z0 + k * P.h[2] };
    const double xr[3] = { xl[0] + P.h[0], yface[j + 1], xl[2] + P.h[2] };
    // 1-D cell averages of sin, cos, cos 2x, sin^2, cos^2
    double S[3], C[3], C2[3], SS[3], CC[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double w = xr[d] - xl[d];
        S[d] = (cos(xl[d]) - cos(xr[d])) / w;
        C[d] = (sin(xr[d]) - sin(xl[d])) / w;
        C2[d] = (sin(2.0 * xr[d]) - sin(2.0 * xl[d])) / (2.0 * w);
        SS[d] = 0.5 - 0.5 * C2[d];
        CC[d] = 0.5 + 0.5 * C2[d];
    }
    const double p0 = rho0 * U0 * U0 / (P.gamma * Ma * Ma);
    const double pbar = p0 + rho0 * U0 * U0 / 16.0 * (C2[0] + C2[1]) * (C2[2] + 2.0);
    const long long p = pidx(P, i, j, k);
    q[p] = rho0;
    q[P.cs + p] = rho0 * U0 * S[0] * C[1] * C[2];
    q[2 * P.cs + p] = -rho0 * U0 * C[0] * S[1] * C[2];
    q[3 * P.cs + p] = 0.0;
    q[4 * P.cs + p] = pbar / (P.gamma - 1.0) + 0.5 * rho0 * U0 * U0 * (SS[0] * CC[1] * CC[2] + CC[0] * SS[1] * CC[2]);
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unit_pm1(unsigned long long x)
{
    return (double)(splitmix64(x) >> 11) * (1.0 / 4503599627370496.0) - 1.0;
}

__global__ void k_init_channel(Params P, double *q, const double *ycen, double ymid, double hh, double Ma_b, double amp,
                               unsigned long long seed)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell) return;
    int i, j, k;
    cell_of(P, t, i, j, k);
    const double Tw = 1.0 / (P.gamma * Ma_b * Ma_b), rho = 1.0, pr = rho * Tw;
    const double yn = (ycen[j] - ymid) / hh;
    const double U = 1.5 * (1.0 - yn * yn);
    const unsigned long long idx = (unsigned long long)t;
    const double u = U + amp * U * unit_pm1(seed ^ (3 * idx + 0));
    const double v = amp * unit_pm1(seed ^ (3 * idx + 1));
    const double w = amp * unit_pm1(seed ^ (3 * idx + 2));
    const long long p = pidx(P, i, j, k);
    q[p] = rho;
    q[P.cs + p] = rho * u;
    q[2 * P.cs + p] = rho * v;
    q[3 * P.cs + p] = rho * w;
    q[4 * P.cs + p] = pr / (P.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
}

__global__ void k_init_wave(Params P, double *q, double x0, double y0, double z0, double hy, double amp)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.ncell) return;
    int i, j, k;
    cell_of(P, t, i, j, k);
    const double kd[3] = { P.n[0] > 1 ? 1.0 : 0.0, P.n[1] > 1 ? 1.0 : 0.0, P.n[2] > 1 ? 1.0 : 0.0 };
    const double hs[3] = { P.h[0], hy, P.h[2] };
    const double pi = 3.14159265358979323846;
    double fac = 1.0;
#pragma unroll
    for (int d = 0; d < 3; d++)
        if (kd[d] > 0.0) fac *= sin(pi * hs[d] / 2.0) / (pi * hs[d] / 2.0);
    const double xc = x0 + (i + 0.5) * hs[0], yc = y0 + (j + 0.5) * hs[1], zc = z0 + (k + 0.5) * hs[2];
    const double rho = 1.0 + amp * sin(pi * (kd[0] * xc + kd[1] * yc + kd[2] * zc)) * fac;
    const long long p = pidx(P, i, j, k);
    q[p] = rho;
    q[P.cs + p] = rho * kd[0];
    q[2 * P.cs + p] = rho * kd[1];
    q[3 * P.cs + p] = rho * kd[2];
    q[4 * P.cs + p] = 1.0 / (P.gamma - 1.0) + 0.5 * rho * (kd[0] + kd[1] + kd[2]);
}

void launch_init_tgv(const Params &P, double *q, const double *yface, double x0, double z0, double Ma, double U0,
                     double rho0, cudaStream_t st)
{
    k_init_tgv<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, q, yface, x0, z0, Ma, U0, rho0);
}
void launch_init_channel(const Params &P, double *q, const double *ycen, double ymid, double hh, double Ma_b,
                         double amp, unsigned long long seed, cudaStream_t st)
{
    k_init_channel<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, q, ycen, ymid, hh, Ma_b, amp, seed);
}
void launch_init_wave(const Params &P, double *q, double x0, double y0, double z0, double hy, double amp,
                      cudaStream_t st)
{
    k_init_wave<<<grid_for(P.ncell, 256), 256, 0, st>>>(P, q, x0, y0, z0, hy, amp);
}

// ---------------------------------------------------------------------------
// FP64 throughput probe: eight independent FMA chains per thread, enough
// resident warps to keep the FP64 pipe busy, timed with CUDA events.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fp64_probe(double *out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += x[i];
    if (s == 1.2345) out[0] = s;  // keeps the chains live; never true for these inputs
}

cudaError_t fp64_probe(double *tflops)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    double *out = nullptr;
    e = cudaMalloc(&out, sizeof(double));
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    k_fp64_probe<<<blocks, threads>>>(out, 64, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(a);
    k_fp64_probe<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace hgks
