// hgks_passes.cuh -- the work of one position of each pass of the step
// (interface for the sweep passes, cell or ghost cell for the others), shared
// by the single-problem kernels and the batched work-list kernels.
#pragma once
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

// ---------------------------------------------------------------------------
// pass 1: normal reconstruction
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void pos_normal(const Params &P, int d, const Box &B, const double *__restrict__ q,
                                                  double *__restrict__ fq, long long t)
{
    const long long nq = box_count(B);
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
static __device__ __forceinline__ void pos_tan1(const Params &P, int d, const Box &Bt, const Box &Bq,
                                                const double *__restrict__ fq, double *__restrict__ t1, long long t)
{
    const long long nt = box_count(Bt), nq = box_count(Bq);
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
// The inputs of the two Gauss points of a line are staged in dynamic shared
// memory, one row of FLUX_STRIDE doubles per thread, laid out as the point
// flux reads them: for Gauss point n at n * 55: Ql (5), Qr (5), then the
// physical slopes dl[3][5], dr[3][5], d0[3][5] (normal, t1, t2).  Local arrays
// in their place were dynamically indexed and thrashed L1.  The odd row
// length keeps a half-warp's 8-byte accesses in distinct banks.
constexpr int FLUX_BLOCK = 128;
constexpr int FLUX_STRIDE = 111;
constexpr int FLUX_SMEM = FLUX_BLOCK * FLUX_STRIDE * (int)sizeof(double);

static __device__ __forceinline__ void pos_flux(const Params &P, int d, const Box &Bf, const Box &Bt,
                                                const double *__restrict__ t1, double *__restrict__ F, double dt,
                                                long long t, double *sm)
{
    const long long nf = box_count(Bf), nt = box_count(Bt);
    int p[3];
    box_pos(Bf, t, p);
    const int e1 = tdir(d, 0), e2 = tdir(d, 1);
    const int f = p[d], a = p[e1], b = p[e2];
    const long long base = box_lin(Bt, p), s2 = box_stride(Bt, e2);
    const FaceGeom G = face_geom(P, d, f, a, b);
    auto load = [&](int slot, int j) { return t1[slot * nt + base + (j - 2) * s2]; };
    double Fs[5], dFs[5];
    flux_body<double>(load, G, P, dt, sm + threadIdx.x * FLUX_STRIDE, Fs, dFs);
#pragma unroll
    for (int c = 0; c < 5; c++) {
        F[(long long)perm_of(d, c) * nf + t] = Fs[c];
        F[(long long)(5 + perm_of(d, c)) * nf + t] = dFs[c];
    }
}

static __device__ __forceinline__ void wall_ghost(const Params &P, const double s[5], double o[5])
{
    // mirror: U_g = -U_i, p_g = p_i, T_g = 2 T_w - T_i (floored at T_w / 2), rho_g = p_g / T_g
    double ir = 1.0 / s[0];
    double U = s[1] * ir, V = s[2] * ir, W = s[3] * ir;
    double p = (P.gamma - 1.0) * (s[4] - 0.5 * s[0] * (U * U + V * V + W * W));
    double T = p / s[0];
    double Tg = 2.0 * P.T_wall - T;
    if (Tg < 0.5 * P.T_wall) Tg = 0.5 * P.T_wall;
    double rho = p / Tg;
    o[0] = rho;
    o[1] = -rho * U;
    o[2] = -rho * V;
    o[3] = -rho * W;
    o[4] = p / (P.gamma - 1.0) + 0.5 * rho * (U * U + V * V + W * W);
}

// number of ghost cells filled by the pass of direction d
__host__ __device__ inline long long ghost_count(const Params &P, int d)
{
    const int ea = d == 0 ? 1 : 0, eb = d == 2 ? 1 : 2;
    const long long Ra = ea < d ? P.n[ea] + 2 * NG : P.n[ea];
    const long long Rb = eb < d ? P.n[eb] + 2 * NG : P.n[eb];
    return 2LL * NG * Ra * Rb;
}

static __device__ __forceinline__ void pos_ghost(const Params &P, double *q, int d, long long t)
{
    // the two other directions in increasing order; earlier directions span the padded range
    const int ea = d == 0 ? 1 : 0, eb = d == 2 ? 1 : 2;
    const int loa = ea < d ? -NG : 0, Ra = ea < d ? P.n[ea] + 2 * NG : P.n[ea];
    const int lob = eb < d ? -NG : 0;
    int g, ca, cb;
    if (d == 0) {  // ghost index fastest (x is the ghost direction)
        g = (int)(t % (2 * NG));
        long long r = t / (2 * NG);
        ca = (int)(r % Ra) + loa;
        cb = (int)(r / Ra) + lob;
    } else {       // x fastest
        ca = (int)(t % Ra) + loa;
        long long r = t / Ra;
        g = (int)(r % (2 * NG));
        cb = (int)(r / (2 * NG)) + lob;
    }
    const int side = g / NG, m = g % NG, n = P.n[d];
    const int gi = side == 0 ? -1 - m : n + m;
    const int bc = side == 0 ? P.bc_lo[d] : P.bc_hi[d];
    if (bc == 2) return;  // EXTERNAL: a neighbouring sub-domain's layers, set by the caller
    int si;
    if (bc == 0) si = ((gi % n) + n) % n;
    else si = side == 0 ? m : n - 1 - m;
    int ig[3], is[3];
    ig[d] = gi;
    is[d] = si;
    ig[ea] = is[ea] = ca;
    ig[eb] = is[eb] = cb;
    const long long pg = pidx(P, ig[0], ig[1], ig[2]), ps = pidx(P, is[0], is[1], is[2]);
    if (bc == 0) {
#pragma unroll
        for (int c = 0; c < 5; c++) q[c * P.cs + pg] = q[c * P.cs + ps];
    } else {
        double s[5], o[5];
#pragma unroll
        for (int c = 0; c < 5; c++) s[c] = q[c * P.cs + ps];
        wall_ghost(P, s, o);
#pragma unroll
        for (int c = 0; c < 5; c++) q[c * P.cs + pg] = o[c];
    }
}

// dx_d / (|u_d| + c) minimised over the directions of interior cell t
static __device__ __forceinline__ double pos_cfl(const Params &P, const double *__restrict__ q, long long t)
{
    int i = (int)(t % P.n[0]);
    long long r = t / P.n[0];
    int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
    long long p = pidx(P, i, j, k);
    double rho = q[p], ir = 1.0 / rho;
    double U = q[P.cs + p] * ir, V = q[2 * P.cs + p] * ir, W = q[3 * P.cs + p] * ir;
    double pr = (P.gamma - 1.0) * (q[4 * P.cs + p] - 0.5 * rho * (U * U + V * V + W * W));
    double c = sqrt(P.gamma * pr * ir);
    return fmin(P.h[0] / (fabs(U) + c), fmin(P.hy_cell[j] / (fabs(V) + c), P.h[2] / (fabs(W) + c)));
}

static __device__ __forceinline__ void cell_rhs(const Params &P, const double *q, const double *const F[3], int i, int j,
                                         int k, long long p, double L[5], double dL[5])
{
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const long long n0 = (long long)(nx + 1) * ny * nz, n1 = (long long)nx * (ny + 1) * nz,
                    n2 = (long long)nx * ny * (nz + 1);
    const long long l0 = ((long long)k * ny + j) * (nx + 1) + i;
    const long long l1 = ((long long)k * (ny + 1) + j) * nx + i;
    const long long l2 = ((long long)k * ny + j) * nx + i;
    // one reciprocal of the cell volume instead of ten FP64 divisions (the
    // update is FP64-bound; the results differ from division by <= 1 ulp)
    const double ivol = 1.0 / (P.h[0] * P.hy_cell[j] * P.h[2]);
#pragma unroll
    for (int c = 0; c < 5; c++) {
        double sx = F[0][c * n0 + l0 + 1] - F[0][c * n0 + l0];
        double sy = F[1][c * n1 + l1 + nx] - F[1][c * n1 + l1];
        double sz = F[2][c * n2 + l2 + (long long)nx * ny] - F[2][c * n2 + l2];
        L[c] = -((sx + sy) + sz) * ivol;
        double tx = F[0][(5 + c) * n0 + l0 + 1] - F[0][(5 + c) * n0 + l0];
        double ty = F[1][(5 + c) * n1 + l1 + nx] - F[1][(5 + c) * n1 + l1];
        double tz = F[2][(5 + c) * n2 + l2 + (long long)nx * ny] - F[2][(5 + c) * n2 + l2];
        dL[c] = -((tx + ty) + tz) * ivol;
    }
    if (P.has_force) {
        // source (0, rho G, rho u.G) and its time derivative (0, G L_rho, G.L_mom)
        const double rho = q[p], m0 = q[P.cs + p], m1 = q[2 * P.cs + p], m2 = q[3 * P.cs + p];
        L[1] += rho * P.G[0];
        L[2] += rho * P.G[1];
        L[3] += rho * P.G[2];
        L[4] += m0 * P.G[0] + m1 * P.G[1] + m2 * P.G[2];
        dL[1] += P.G[0] * L[0];
        dL[2] += P.G[1] * L[0];
        dL[3] += P.G[2] * L[0];
        dL[4] += P.G[0] * L[1] + P.G[1] * L[2] + P.G[2] * L[3];
    }
}

static __device__ __forceinline__ bool state_ok(const double Q[5])
{
    bool fin = isfinite(Q[0]) && isfinite(Q[1]) && isfinite(Q[2]) && isfinite(Q[3]) && isfinite(Q[4]);
    if (!fin || !(Q[0] > 0.0)) return false;
    double e = Q[4] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]) / Q[0];
    return e > 0.0;
}

// stage update of interior cell t; returns false for a bad new state
static __device__ __forceinline__ bool pos_update(const Params &P, int stage, const double *__restrict__ q,
                                                  const double *__restrict__ F0, const double *__restrict__ F1,
                                                  const double *__restrict__ F2, double *__restrict__ oa,
                                                  double *__restrict__ ob, double dt, long long t)
{
    int i = (int)(t % P.n[0]);
    long long r = t / P.n[0];
    int j = (int)(r % P.n[1]), k = (int)(r / P.n[1]);
    const long long p = pidx(P, i, j, k);
    const double *F[3] = { F0, F1, F2 };
    double L[5], dL[5], A[5];
    cell_rhs(P, q, F, i, j, k, p, L, dL);
    bool ok = true;
    const double dt2 = dt * dt;
    if (stage == 1) {
        double B[5];
        const double h1 = 0.5 * dt, h2 = 0.125 * dt2, s2 = dt2 * (1.0 / 6.0);
#pragma unroll
        for (int c = 0; c < 5; c++) {
            double Q = q[c * P.cs + p];
            A[c] = Q + h1 * L[c] + h2 * dL[c];
            B[c] = Q + dt * L[c] + s2 * dL[c];
            oa[c * P.cs + p] = A[c];
            ob[c * P.cs + p] = B[c];
        }
        ok = state_ok(A);
    } else {
        // oa = r + dt^2/3 dL(Q*), r = the stage-1 accumulator passed as ob
#pragma unroll
        for (int c = 0; c < 5; c++) {
            A[c] = ob[c * P.cs + p] + (dt2 * (1.0 / 3.0)) * dL[c];
            oa[c * P.cs + p] = A[c];
        }
        ok = state_ok(A);
    }
    return ok;
}

}  // namespace hgks
