// hgks_batch.cu -- many independent HGKS problems advanced together.
//
// A batch groups solver handles with their own grids (uneven sizes), gas
// parameters, precisions and state buffers.  Every pass of a step runs as one
// persistent kernel over a tile work-list that spans all problems: a tile is
// a contiguous range of positions (interfaces or cells) of one problem, and
// each block walks the tiles with a fixed stride, so small problems no longer
// leave most of the GPU idle.  The 30 to 51 launches of a step are captured
// once into a CUDA graph and replayed for every step.  Each problem keeps its own
// control block: its time step, its bad-state flag (a bad problem stops
// alone) and the index of its current state buffer, which the kernels read on
// the device, so the same graph serves every step.  The tile size is picked by
// a small autotuner (hgks_batch_tune) that times whole graph steps.
#include "../../include/hgks.h"
#include "hgks_passes.cuh"
#include "hgks_passes_mx.cuh"

#include "hgks_handle.h"

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

namespace hgks {

void set_global_error(const char *msg);  // hgks_api.cu

struct Inst {
    Params P;
    double *q[2], *qs, *r, *fq, *t1, *F[3];
    float2 *q2;  // mixed: the split state
    Ctl *ctl;
    int mixed, walls;
    double lxlz;
};

struct Tile {
    int inst;
    int pad;
    long long start, count;
};

// work-lists: ghost fill per direction, cells, then the three sweep passes
// per direction, once for the FP64 problems and once for the mixed ones (so
// each sweep kernel is compiled for one precision and keeps its registers)
enum { WL_GHOST = 0, WL_CELLS = 3, WL_SWEEP = 4, WL_PAD = 22, WL_N = 23 };  // WL_PAD: padded cells, mixed only
static inline int wl_sweep(int mixed, int pass, int d) { return WL_SWEEP + 9 * mixed + 3 * pass + d; }

// ---------------------------------------------------------------------------
// batched kernels: block b walks tiles b, b + gridDim.x, ...
// ---------------------------------------------------------------------------
__global__ void kb_ghost(const Inst *__restrict__ I, const Tile *__restrict__ T, int ntiles, int d, int stage)
{
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        double *q = stage == 0 ? in.q[in.ctl->good] : in.qs;
        for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x) pos_ghost(in.P, q, d, t);
    }
}

// mixed problems: split the state of this stage into hi / lo float planes
__global__ void __launch_bounds__(256) kb_split(const Inst *__restrict__ I, const Tile *__restrict__ T, int ntiles,
                                                int stage)
{
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        if (in.ctl->flag) continue;
        const double *q = stage == 0 ? in.q[in.ctl->good] : in.qs;
        for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x)
            pos_split_mx(in.P, q, in.q2, t);
    }
}

__global__ void kb_dt_reset(const Inst *__restrict__ I, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) I[i].ctl->dtmin_bits = 0x7FF0000000000000ull;
}

__global__ void __launch_bounds__(256) kb_cfl(const Inst *__restrict__ I, const Tile *__restrict__ T, int ntiles)
{
    __shared__ double red[8];
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        const double *q = in.q[in.ctl->good];
        double v = INFINITY;
        if (!in.ctl->flag)
            for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x)
                v = fmin(v, pos_cfl(in.P, q, t));
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : INFINITY;
            for (int o = 4; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
            if (threadIdx.x == 0 && v < INFINITY)
                atomicMin(&in.ctl->dtmin_bits, (unsigned long long)__double_as_longlong(v));
        }
        __syncthreads();
    }
}

__global__ void kb_dt_final(const Inst *__restrict__ I, int n, double cfl)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || I[i].ctl->flag) return;
    I[i].ctl->dt = cfl * __longlong_as_double((long long)I[i].ctl->dtmin_bits);
}

template <bool MX>
__global__ void __launch_bounds__(128) kb_normal(const Inst *__restrict__ I, const Tile *__restrict__ T, int ntiles,
                                                 int d, int stage)
{
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        if (in.ctl->flag) continue;
        const double *q = stage == 0 ? in.q[in.ctl->good] : in.qs;
        const Box B = box_fq(in.P, d);
        if constexpr (MX) {
            const FqMx o = fq_mx(in.fq, box_count(B));
            for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x)
                pos_normal_mx(in.P, d, B, in.q2, o, t);
        } else {
            for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x)
                pos_normal(in.P, d, B, q, in.fq, t);
        }
    }
}

__global__ void __launch_bounds__(128) kb_tan1(const Inst *__restrict__ I, const Tile *__restrict__ T, int ntiles,
                                               int d)
{
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        if (in.ctl->flag) continue;
        const Box Bt = box_t1(in.P, d), Bq = box_fq(in.P, d);
        for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x)
            pos_tan1(in.P, d, Bt, Bq, in.fq, in.t1, t);
    }
}

// The mixed tan1 pass, like the mixed flux pass, is not persistent: one block
// per tile of MX_TILE positions, one per thread, with the tile's problem
// constants read once into shared memory.  Under a persistent loop, or with
// the constants held in registers, its fully unrolled rows spilled 800-1000
// bytes per thread; this way they take 88 registers.
constexpr int MX_TILE = 128;

__global__ void __launch_bounds__(MX_TILE, 4) kb_tan1_mx(const Inst *__restrict__ I, const Tile *__restrict__ T,
                                                         int ntiles, int d)
{
    // the tile's problem constants, read once into shared memory
    struct TanArgs {
        Box Bt, Bq;
        FqMx in;
        T1Mx o;
        long long start, count;
        int flag;
    };
    __shared__ TanArgs a;
    const int k = blockIdx.x;
    if (k >= ntiles) return;
    if (threadIdx.x == 0) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        a.Bt = box_t1(in.P, d);
        a.Bq = box_fq(in.P, d);
        a.in = fq_mx(in.fq, box_count(a.Bq));
        a.o = t1_mx(in.t1, box_count(a.Bt));
        a.start = tl.start;
        a.count = tl.count;
        a.flag = in.ctl->flag;
    }
    __syncthreads();
    if (a.flag || (long long)threadIdx.x >= a.count) return;
    tan1_mx_rows(d, a.Bt, a.Bq, a.in.v, a.in.vs, a.o.th, a.o.tl, a.o.ts, a.start + threadIdx.x);
}

// The mixed flux pass is the one pass that is not persistent: it launches one
// block per flux tile of 32 x 4 faces (flux_mx_tile; a work-list entry per
// tile), and the hardware block scheduler hands out the tiles.  A persistent
// loop keeps its state live across the flux, which at the register budget of
// this latency-bound kernel raised the spills from 48 to 232 bytes and cost
// 40 %.
__global__ void __launch_bounds__(FLUX_MX_BLOCK, 3) kb_flux_mx(const Inst *__restrict__ I,
                                                               const Tile *__restrict__ T, int ntiles, int d)
{
    extern __shared__ float gp_sm[];
    const int k = blockIdx.x;
    if (k >= ntiles) return;
    const Tile tl = T[k];
    const Inst &in = I[tl.inst];
    if (in.ctl->flag) return;
    const Box Bf = box_face(in.P, d), Bt = box_t1(in.P, d);
    flux_mx_tile<false>(in.P, d, Bf, Bt, t1_mx(in.t1, box_count(Bt)), in.F[d], in.ctl->dt, tl.start, gp_sm);
}

__global__ void __launch_bounds__(FLUX_BLOCK, 2) kb_flux(const Inst *__restrict__ I, const Tile *__restrict__ T,
                                                         int ntiles, int d)
{
    extern __shared__ double flux_sm[];
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        if (in.ctl->flag) continue;
        const Box Bf = box_face(in.P, d), Bt = box_t1(in.P, d);
        const double dt = in.ctl->dt;
        for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x)
            pos_flux(in.P, d, Bf, Bt, in.t1, in.F[d], dt, t, flux_sm);
    }
}

__global__ void __launch_bounds__(256) kb_update(const Inst *__restrict__ I, const Tile *__restrict__ T, int ntiles,
                                                 int stage)
{
    for (int k = blockIdx.x; k < ntiles; k += gridDim.x) {
        const Tile tl = T[k];
        const Inst &in = I[tl.inst];
        if (in.ctl->flag) continue;
        const int cur = in.ctl->good;
        const double dt = in.ctl->dt;
        bool ok = true;
        for (long long t = tl.start + threadIdx.x; t < tl.start + tl.count; t += blockDim.x) {
            if (stage == 1) ok &= pos_update(in.P, 1, in.q[cur], in.F[0], in.F[1], in.F[2], in.qs, in.r, dt, t);
            else ok &= pos_update(in.P, 2, in.qs, in.F[0], in.F[1], in.F[2], in.q[1 - cur], in.r, dt, t);
        }
        if (!ok) atomicOr(&in.ctl->flag, 1);
    }
}

// mean wall stress of each problem with y walls (one block per problem)
__global__ void kb_wall(const Inst *__restrict__ I, int n)
{
    __shared__ double red[2][256];
    const Inst &in = I[blockIdx.x];
    if (!in.walls) return;
    const int nx = in.P.n[0], ny = in.P.n[1], nz = in.P.n[2];
    const long long n1 = (long long)nx * (ny + 1) * nz;
    const double *Fy = in.F[1];
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
    if (threadIdx.x == 0 && !in.ctl->flag) {
        double s = 0.0;
        int walls = 0;
        if (in.P.bc_lo[1] == 1) { s += -red[0][0]; walls++; }
        if (in.P.bc_hi[1] == 1) { s += red[1][0]; walls++; }
        in.ctl->wall_shear = walls ? s / (walls * in.lxlz) : 0.0;
    }
}

__global__ void kb_commit(const Inst *__restrict__ I, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Ctl *c = I[i].ctl;
    if (c->flag) return;
    c->t += c->dt;
    c->step += 1;
    c->last_dt = c->dt;
    c->good = 1 - c->good;
}

}  // namespace hgks

using namespace hgks;

struct hgks_batch_s {
    std::vector<hgks_t> h;
    cudaStream_t user = nullptr;  // the problems' stream
    cudaStream_t st = nullptr;    // the batch's own stream (graphs cannot be captured on the legacy stream)
    Inst *d_inst = nullptr;
    std::vector<Inst> inst;
    Tile *d_tiles = nullptr;
    int off[WL_N], cnt[WL_N];
    long long tile[WL_N];  // positions (or cells) per tile of each work-list
    int blocks_cells = 0, sms = 0;
    int bsweep[2][3] = {};  // resident blocks of the normal, tan1 and flux kernels, per precision
    bool any_walls = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double graph_cfl = -1.0;
    cudaEvent_t ev[2] = { nullptr, nullptr };
    double last_ms = 0.0;
    int last_steps = 0;
    std::vector<long long> steps;  // step counters read at the end of the last call
    std::string err;
};

static hgks_status berr(hgks_batch_t b, hgks_status s, const std::string &m)
{
    if (b) b->err = m;
    return s;
}

static void free_graph(hgks_batch_t b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_cfl = -1.0;
}

// tile work-lists of every pass for the current tile sizes
static hgks_status build_tiles(hgks_batch_t b)
{
    std::vector<Tile> all;
    auto add = [&](int, int i, long long total, long long ts) {
        for (long long s = 0; s < total; s += ts) all.push_back(Tile{ i, 0, s, std::min(ts, total - s) });
    };
    for (int w = 0; w < WL_N; w++) {
        b->off[w] = (int)all.size();
        for (int i = 0; i < (int)b->inst.size(); i++) {
            const Params &P = b->inst[i].P;
            if (w < 3) add(w, i, ghost_count(P, w), b->tile[w]);
            else if (w == WL_CELLS) add(w, i, P.ncell, b->tile[w]);
            else if (w == WL_PAD) {
                if (b->inst[i].mixed) add(w, i, P.cs, b->tile[w]);
            } else {
                const int mixed = (w - WL_SWEEP) / 9, pass = (w - WL_SWEEP) / 3 % 3, d = (w - WL_SWEEP) % 3;
                if (mixed != b->inst[i].mixed) continue;
                const Box B = pass == 0 ? box_fq(P, d) : pass == 1 ? box_t1(P, d) : box_face(P, d);
                if (mixed && pass == 2) add(w, i, flux_tiling(P, d).count, 1);  // one entry per flux tile
                else if (mixed && pass == 1) add(w, i, box_count(B), MX_TILE);   // one block per tile
                else add(w, i, box_count(B), b->tile[w]);
            }
        }
        b->cnt[w] = (int)all.size() - b->off[w];
    }
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    cudaError_t e = cudaMalloc(&b->d_tiles, all.size() * sizeof(Tile));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return berr(b, HGKS_ERR_CUDA, std::string("tile list: ") + cudaGetErrorString(e));
    free_graph(b);
    return HGKS_OK;
}

static unsigned pgrid(int ntiles, int blocks) { return (unsigned)std::max(1, std::min(ntiles, blocks)); }

static void enqueue_batch_step(hgks_batch_t b, double cfl)
{
    const Inst *I = b->d_inst;
    const int n = (int)b->inst.size();
    cudaStream_t st = b->st;
    const unsigned ib = (unsigned)((n + 127) / 128);
    auto T = [&](int w) { return b->d_tiles + b->off[w]; };
    for (int d = 0; d < 3; d++) kb_ghost<<<pgrid(b->cnt[WL_GHOST + d], b->blocks_cells), 256, 0, st>>>(
        I, T(WL_GHOST + d), b->cnt[WL_GHOST + d], d, 0);
    kb_dt_reset<<<ib, 128, 0, st>>>(I, n);
    kb_cfl<<<pgrid(b->cnt[WL_CELLS], b->blocks_cells), 256, 0, st>>>(I, T(WL_CELLS), b->cnt[WL_CELLS]);
    kb_dt_final<<<ib, 128, 0, st>>>(I, n, cfl);
    for (int stage = 0; stage < 2; stage++) {
        if (stage == 1)
            for (int d = 0; d < 3; d++) kb_ghost<<<pgrid(b->cnt[WL_GHOST + d], b->blocks_cells), 256, 0, st>>>(
                I, T(WL_GHOST + d), b->cnt[WL_GHOST + d], d, 1);
        if (b->cnt[WL_PAD])
            kb_split<<<pgrid(b->cnt[WL_PAD], b->blocks_cells), 256, 0, st>>>(I, T(WL_PAD), b->cnt[WL_PAD], stage);
        for (int d = 0; d < 3; d++) {
            for (int mx = 0; mx < 2; mx++) {
                const int wn = wl_sweep(mx, 0, d), wt = wl_sweep(mx, 1, d), wf = wl_sweep(mx, 2, d);
                if (!b->cnt[wn]) continue;  // no problem of this precision
                if (mx) {
                    kb_normal<true><<<pgrid(b->cnt[wn], b->bsweep[1][0]), 128, 0, st>>>(I, T(wn), b->cnt[wn], d,
                                                                                       stage);
                    kb_tan1_mx<<<(unsigned)b->cnt[wt], MX_TILE, 0, st>>>(I, T(wt), b->cnt[wt], d);
                    kb_flux_mx<<<(unsigned)b->cnt[wf], FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM, st>>>(I, T(wf), b->cnt[wf],
                                                                                              d);
                } else {
                    kb_normal<false><<<pgrid(b->cnt[wn], b->bsweep[0][0]), 128, 0, st>>>(I, T(wn), b->cnt[wn], d,
                                                                                        stage);
                    kb_tan1<<<pgrid(b->cnt[wt], b->bsweep[0][1]), 128, 0, st>>>(I, T(wt), b->cnt[wt], d);
                    kb_flux<<<pgrid(b->cnt[wf], b->bsweep[0][2]), FLUX_BLOCK, FLUX_SMEM, st>>>(I, T(wf), b->cnt[wf],
                                                                                              d);
                }
            }
            if (d == 1 && stage == 0 && b->any_walls) kb_wall<<<n, 256, 0, st>>>(I, n);
        }
        kb_update<<<pgrid(b->cnt[WL_CELLS], b->blocks_cells), 256, 0, st>>>(I, T(WL_CELLS), b->cnt[WL_CELLS],
                                                                              stage + 1);
    }
    kb_commit<<<ib, 128, 0, st>>>(I, n);
}

static hgks_status capture(hgks_batch_t b, double cfl)
{
    free_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return berr(b, HGKS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    enqueue_batch_step(b, cfl);
    e = cudaStreamEndCapture(b->st, &b->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        free_graph(b);
        return berr(b, HGKS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->graph_cfl = cfl;
    return HGKS_OK;
}

extern "C" hgks_status hgks_batch_create(hgks_t *handles, int n, hgks_batch_t *out)
{
    if (!handles || !out || n < 1) {
        set_global_error("hgks_batch_create: need handles, out and n >= 1");
        return HGKS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    hgks_batch_t b = new hgks_batch_s();
    b->user = handles[0] ? handles[0]->st : nullptr;
    for (int i = 0; i < n; i++) {
        hgks_t h = handles[i];
        if (!h || h->st != b->user) {
            delete b;
            set_global_error("hgks_batch_create: a NULL handle, or handles on different streams");
            return HGKS_ERR_INVALID_ARG;
        }
        for (int j = 0; j < i; j++)
            if (handles[j] == h) {
                delete b;
                set_global_error("hgks_batch_create: a handle appears twice");
                return HGKS_ERR_INVALID_ARG;
            }
        if (h->prec == HGKS_MIXED_T64) {
            delete b;
            set_global_error("hgks_batch_create: HGKS_MIXED_T64 handles are stepped alone (the batch runs "
                             "HGKS_FP64 and HGKS_MIXED problems)");
            return HGKS_ERR_INVALID_ARG;
        }
        if (h->P.bc_lo[2] == HGKS_BC_EXTERNAL || h->P.bc_hi[2] == HGKS_BC_EXTERNAL) {
            delete b;
            set_global_error("hgks_batch_create: a sub-domain handle (EXTERNAL sides) needs its halos set "
                             "between stages and cannot be stepped in a batch");
            return HGKS_ERR_INVALID_ARG;
        }
        b->h.push_back(h);
        Inst in;
        memset(&in, 0, sizeof in);
        in.P = h->P;
        in.q[0] = h->q[0];
        in.q[1] = h->q[1];
        in.qs = h->qs;
        in.r = h->r;
        in.fq = h->fq;
        in.t1 = h->t1;
        for (int d = 0; d < 3; d++) in.F[d] = h->F[d];
        in.ctl = h->ctl;
        in.mixed = h->prec == HGKS_MIXED;
        in.q2 = (float2 *)h->qf;
        in.walls = h->P.bc_lo[1] == HGKS_BC_ISOTHERMAL_WALL || h->P.bc_hi[1] == HGKS_BC_ISOTHERMAL_WALL;
        in.lxlz = h->grid.lx * h->grid.lz;
        b->any_walls |= in.walls != 0;
        b->inst.push_back(in);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        set_global_error("hgks_batch_create: no usable CUDA device");
        delete b;
        return HGKS_ERR_CUDA;
    }
    // persistent grids: as many blocks as stay resident (the dynamic shared
    // memory of the flux kernels needs the opt-in first)
    int nb[2][3] = {};
    cudaError_t e = cudaFuncSetAttribute((const void *)kb_flux, cudaFuncAttributeMaxDynamicSharedMemorySize, FLUX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)kb_flux_mx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 FLUX_MX_TILE_SMEM);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[0][0], kb_normal<false>, 128, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[0][1], kb_tan1, 128, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[0][2], kb_flux, FLUX_BLOCK, FLUX_SMEM);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[1][0], kb_normal<true>, 128, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[1][1], kb_tan1_mx, MX_TILE, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[1][2], kb_flux_mx, FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM);
    if (e != cudaSuccess) {
        set_global_error((std::string("hgks_batch_create: kernel set-up: ") + cudaGetErrorString(e)).c_str());
        delete b;
        return HGKS_ERR_CUDA;
    }
    for (int m = 0; m < 2; m++)
        for (int p = 0; p < 3; p++) b->bsweep[m][p] = std::max(1, nb[m][p]) * b->sms;
    b->blocks_cells = b->sms * 8;
    for (int w = 0; w < WL_N; w++) b->tile[w] = w < WL_SWEEP || w == WL_PAD ? 8192 : 2048;
    e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev[1]);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, n * sizeof(Inst));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_inst, b->inst.data(), n * sizeof(Inst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_global_error((std::string("hgks_batch_create: ") + cudaGetErrorString(e)).c_str());
        hgks_batch_destroy(b);
        return HGKS_ERR_CUDA;
    }
    hgks_status s = build_tiles(b);
    if (s) {
        hgks_batch_destroy(b);
        return s;
    }
    *out = b;
    return HGKS_OK;
}

extern "C" void hgks_batch_destroy(hgks_batch_t b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    free_graph(b);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_inst) cudaFree(b->d_inst);
    for (int i = 0; i < 2; i++)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

extern "C" const char *hgks_batch_last_error(hgks_batch_t b) { return b ? b->err.c_str() : "null batch"; }

// read every problem's control block: sync the host's buffer index, clear flags
static hgks_status batch_finish(hgks_batch_t b)
{
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return berr(b, HGKS_ERR_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
    int bad = -1;
    b->steps.assign(b->h.size(), 0);
    for (size_t i = 0; i < b->h.size(); i++) {
        Ctl c;
        e = cudaMemcpy(&c, b->h[i]->ctl, sizeof c, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return berr(b, HGKS_ERR_CUDA, cudaGetErrorString(e));
        b->h[i]->cur = c.good;
        b->steps[i] = (long long)c.step;
        if (c.flag) {
            if (bad < 0) bad = (int)i;
            c.flag = 0;
            e = cudaMemcpy(b->h[i]->ctl, &c, sizeof c, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return berr(b, HGKS_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    if (bad >= 0)
        return berr(b, HGKS_ERR_NONFINITE, "problem " + std::to_string(bad) +
                                               " produced a bad state; it (and any other) stayed at its last "
                                               "completed step, the others advanced");
    return HGKS_OK;
}

extern "C" hgks_status hgks_batch_step(hgks_batch_t b, int nsteps, double cfl)
{
    if (!b || nsteps < 0 || !(cfl > 0.0)) return berr(b, HGKS_ERR_INVALID_ARG, "need nsteps >= 0 and cfl > 0");
    // work already queued on the problems' stream comes first
    cudaError_t e0 = cudaStreamSynchronize(b->user);
    if (e0 != cudaSuccess) return berr(b, HGKS_ERR_CUDA, cudaGetErrorString(e0));
    if (!b->exec || b->graph_cfl != cfl) {
        hgks_status s = capture(b, cfl);
        if (s) return s;
    }
    cudaEventRecord(b->ev[0], b->st);
    for (int k = 0; k < nsteps; k++) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->st);
        if (e != cudaSuccess) return berr(b, HGKS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    }
    cudaEventRecord(b->ev[1], b->st);
    hgks_status s = batch_finish(b);
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess) {
        b->last_ms = ms;
        b->last_steps = nsteps;
    }
    return s;
}

extern "C" hgks_status hgks_batch_steps(hgks_batch_t b, long long *steps)
{
    if (!b || !steps) return berr(b, HGKS_ERR_INVALID_ARG, "need steps");
    if (b->steps.size() != b->h.size()) return berr(b, HGKS_ERR_STATE, "no hgks_batch_step call yet");
    for (size_t i = 0; i < b->h.size(); i++) steps[i] = b->steps[i];
    return HGKS_OK;
}

extern "C" hgks_status hgks_batch_info(hgks_batch_t b, hgks_batch_info_t *out)
{
    if (!b || !out) return HGKS_ERR_INVALID_ARG;
    out->problems = (int)b->h.size();
    out->tile_sweep = (int)b->tile[wl_sweep(0, 2, 0)];
    out->tile_cells = (int)b->tile[WL_CELLS];
    out->tile_normal = (int)b->tile[wl_sweep(0, 0, 0)];
    out->tile_tan1 = (int)b->tile[wl_sweep(0, 1, 0)];
    out->tile_normal_mx = (int)b->tile[wl_sweep(1, 0, 0)];
    // ghost 6, dt 3, update 2, commit 1, wall 0/1, split 2 when a mixed
    // problem is present, and 3 sweep passes x 3 directions x 2 stages for
    // each precision present
    int prec = 0;
    for (int mx = 0; mx < 2; mx++) prec += b->cnt[wl_sweep(mx, 0, 0)] ? 1 : 0;
    out->launches_per_step = 12 + 18 * prec + (b->cnt[WL_PAD] ? 2 : 0) + (b->any_walls ? 1 : 0);
    long long tiles = 0;
    for (int w = 0; w < WL_N; w++) tiles += b->cnt[w];
    out->tiles = tiles;
    out->last_ms = b->last_ms;
    out->last_steps = b->last_steps;
    return HGKS_OK;
}

// ---------------------------------------------------------------------------
// autotuner: the tile size of each tunable pass, chosen by timing that pass.
// Groups of work-lists share one tile size: the cell passes (ghost fill,
// CFL reduction, state split), and per precision the normal, first
// tangential and flux sweeps (the mixed first-tangential and flux passes run
// one block per tile of a fixed shape and are not tuned).  Each timing run
// enqueues the stage-1 ghost fill, CFL reduction and state split, then the
// sweep passes of direction x, with events between the groups.  These
// kernels write only ghost cells (with the values they already hold), the
// CFL minimum (reset at the start of every step) and scratch buffers, so the
// problems' states stay where they were and nothing needs to be copied.
// ---------------------------------------------------------------------------
enum { TG_CELLS = 0, TG_NORMAL64, TG_TAN64, TG_FLUX64, TG_NORMALMX, TG_N };

static void tg_lists(int g, std::vector<int> &w)
{
    w.clear();
    if (g == TG_CELLS) {
        for (int d = 0; d < 3; d++) w.push_back(WL_GHOST + d);
        w.push_back(WL_CELLS);
        w.push_back(WL_PAD);
    } else {
        const int mx = g == TG_NORMALMX, pass = g == TG_NORMAL64 || g == TG_NORMALMX ? 0 : g == TG_TAN64 ? 1 : 2;
        for (int d = 0; d < 3; d++) w.push_back(wl_sweep(mx, pass, d));
    }
}

// one timing run: ms[g] receives the device time of group g's kernels
static cudaError_t time_groups(hgks_batch_t b, cudaEvent_t *ev, float ms[TG_N])
{
    const Inst *I = b->d_inst;
    cudaStream_t st = b->st;
    auto T = [&](int w) { return b->d_tiles + b->off[w]; };
    int k = 0, mark[TG_N + 1];
    for (int g = 0; g <= TG_N; g++) mark[g] = -1;
    cudaEventRecord(ev[k++], st);
    for (int d = 0; d < 3; d++) kb_ghost<<<pgrid(b->cnt[WL_GHOST + d], b->blocks_cells), 256, 0, st>>>(
        I, T(WL_GHOST + d), b->cnt[WL_GHOST + d], d, 0);
    kb_cfl<<<pgrid(b->cnt[WL_CELLS], b->blocks_cells), 256, 0, st>>>(I, T(WL_CELLS), b->cnt[WL_CELLS]);
    if (b->cnt[WL_PAD])
        kb_split<<<pgrid(b->cnt[WL_PAD], b->blocks_cells), 256, 0, st>>>(I, T(WL_PAD), b->cnt[WL_PAD], 0);
    mark[TG_CELLS] = k;
    cudaEventRecord(ev[k++], st);
    const int d = 0;
    for (int mx = 0; mx < 2; mx++) {
        const int wn = wl_sweep(mx, 0, d), wt = wl_sweep(mx, 1, d), wf = wl_sweep(mx, 2, d);
        if (!b->cnt[wn]) continue;
        if (mx) {
            kb_normal<true><<<pgrid(b->cnt[wn], b->bsweep[1][0]), 128, 0, st>>>(I, T(wn), b->cnt[wn], d, 0);
            mark[TG_NORMALMX] = k;
            cudaEventRecord(ev[k++], st);
            kb_tan1_mx<<<(unsigned)b->cnt[wt], MX_TILE, 0, st>>>(I, T(wt), b->cnt[wt], d);
            kb_flux_mx<<<(unsigned)b->cnt[wf], FLUX_MX_BLOCK, FLUX_MX_TILE_SMEM, st>>>(I, T(wf), b->cnt[wf], d);
            cudaEventRecord(ev[k++], st);
        } else {
            kb_normal<false><<<pgrid(b->cnt[wn], b->bsweep[0][0]), 128, 0, st>>>(I, T(wn), b->cnt[wn], d, 0);
            mark[TG_NORMAL64] = k;
            cudaEventRecord(ev[k++], st);
            kb_tan1<<<pgrid(b->cnt[wt], b->bsweep[0][1]), 128, 0, st>>>(I, T(wt), b->cnt[wt], d);
            mark[TG_TAN64] = k;
            cudaEventRecord(ev[k++], st);
            kb_flux<<<pgrid(b->cnt[wf], b->bsweep[0][2]), FLUX_BLOCK, FLUX_SMEM, st>>>(I, T(wf), b->cnt[wf], d);
            mark[TG_FLUX64] = k;
            cudaEventRecord(ev[k++], st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[k - 1]);
    for (int g = 0; g < TG_N; g++) {
        ms[g] = 0.0f;
        if (e == cudaSuccess && mark[g] > 0) e = cudaEventElapsedTime(&ms[g], ev[mark[g] - 1], ev[mark[g]]);
    }
    return e;
}

extern "C" hgks_status hgks_batch_tune(hgks_batch_t b, double cfl, double *best_ms)
{
    if (!b || !(cfl > 0.0)) return berr(b, HGKS_ERR_INVALID_ARG, "need cfl > 0");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    constexpr int NEV = 8;
    cudaEvent_t ev[NEV] = {};
    for (int i = 0; i < NEV && e == cudaSuccess; i++) e = cudaEventCreate(&ev[i]);
    long long old[WL_N];
    for (int w = 0; w < WL_N; w++) old[w] = b->tile[w];
    const long long sweep_cand[] = { 256, 1024, 4096, 16384 }, cell_cand[] = { 2048, 8192, 32768 };
    std::vector<int> lists;
    double total = 0.0;
    for (int g = 0; g < TG_N && e == cudaSuccess; g++) {
        tg_lists(g, lists);
        bool present = false;
        for (int w : lists) present = present || (w != WL_PAD && b->cnt[w] > 0);
        if (!present) continue;
        const long long *cand = g == TG_CELLS ? cell_cand : sweep_cand;
        const int nc = g == TG_CELLS ? 3 : 4;
        long long best_t = b->tile[lists[0]];
        float best = 3e38f;
        for (int c = 0; c < nc && e == cudaSuccess; c++) {
            for (int w : lists) b->tile[w] = cand[c];
            if (build_tiles(b) != HGKS_OK) {
                e = cudaErrorUnknown;
                break;
            }
            float ms[TG_N];
            e = time_groups(b, ev, ms);  // warm-up
            if (e == cudaSuccess) e = time_groups(b, ev, ms);
            if (e == cudaSuccess && ms[g] < best) {
                best = ms[g];
                best_t = cand[c];
            }
        }
        for (int w : lists) b->tile[w] = best_t;
        total += best;
    }
    for (int i = 0; i < NEV; i++)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) {
        const std::string msg = std::string("tuning: ") + cudaGetErrorString(e);
        for (int w = 0; w < WL_N; w++) b->tile[w] = old[w];  // back to the tiling the batch had
        build_tiles(b);
        return berr(b, HGKS_ERR_CUDA, msg);
    }
    hgks_status s = build_tiles(b);
    if (s) return s;
    if (best_ms) *best_ms = total;
    return HGKS_OK;
}
