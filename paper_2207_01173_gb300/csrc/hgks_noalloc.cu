// hgks_noalloc.cu -- CFL time step of a caller-owned device state without any
// device allocation (hgks_cfl_dt_noalloc in include/hgks.h).
//
// Some callers cannot allocate device memory when they need a time step: an
// application whose memory manager reserved every byte of the device at
// start-up (a fixed arena), a solver embedded in another program's time loop
// that must not change the device footprint, or a time loop that cannot
// afford the implicit device-wide synchronisation of cudaMalloc/cudaFree.
// This entry point therefore keeps its scratch, one partial minimum per
// 256-cell block, in a fixed file-scope device array.
//
// The reduction has two passes: each block writes its minimum of
// dx_d / (|u_d| + c) into its own slot of the array, then one block folds
// the slots and writes cfl * min to the caller's output.  Every slot that the
// second pass reads is written by the first pass of the same call, so
// nothing has to be cleared between calls.  A cell with a non-positive
// density or pressure, or a non-finite value, makes its block's slot NaN and
// the result NaN (fmin alone would drop it and return a finite step).
#include "../../include/hgks.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

namespace hgks {
void set_global_error(const char *msg);  // hgks_api.cu
}

namespace {

constexpr int NA_BLOCK = 256;
// one partial minimum per block of 256 cells: 131072 doubles = 1 MiB, enough
// for grids up to 256 * 131072 = 33,554,432 cells (for example 320^3)
constexpr int NA_MAX_BLOCKS = HGKS_NOALLOC_MAX_CELLS / NA_BLOCK;
static_assert(HGKS_NOALLOC_MAX_CELLS % NA_BLOCK == 0, "cell limit must be a whole number of blocks");

// Lives on every device that loads the library, until the process exits.
// In host code this name is only a host-side stand-in for the device array:
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_cfl_partials[NA_MAX_BLOCKS];

struct NaGrid {
    int nx, ny, nz;
    double hx, hz;
    double ly, y0, b;  // y map (b = 0: uniform)
    double gamma;
    long long ncell;
};

// physical height of y cell j, from the map of include/hgks.h
__device__ double na_cell_height(const NaGrid &g, int j)
{
    if (!(g.b > 0.0)) return g.ly / g.ny;
    const double tb = tanh(g.b);
    const double s0 = 2.0 * j / g.ny, s1 = 2.0 * (j + 1) / g.ny;
    const double y0 = g.y0 + 0.5 * g.ly * (1.0 + tanh(g.b * (s0 - 1.0)) / tb);
    const double y1 = g.y0 + 0.5 * g.ly * (1.0 + tanh(g.b * (s1 - 1.0)) / tb);
    return y1 - y0;
}

// minimum that keeps a NaN (fmin returns the other operand)
__device__ __forceinline__ double na_min(double a, double b) { return (a != a || b != b) ? NAN : fmin(a, b); }

__global__ void __launch_bounds__(NA_BLOCK) k_na_cfl_partial(NaGrid g, const double *__restrict__ q,
                                                              double *__restrict__ partials)
{
    __shared__ double red[NA_BLOCK / 32];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = INFINITY;
    if (t < g.ncell) {
        const int j = (int)((t / g.nx) % g.ny);
        const double rho = q[t], ir = 1.0 / rho;
        const double U = q[g.ncell + t] * ir, V = q[2 * g.ncell + t] * ir, W = q[3 * g.ncell + t] * ir;
        const double p = (g.gamma - 1.0) * (q[4 * g.ncell + t] - 0.5 * rho * (U * U + V * V + W * W));
        const double c = sqrt(g.gamma * p * ir);
        v = fmin(g.hx / (fabs(U) + c), fmin(na_cell_height(g, j) / (fabs(V) + c), g.hz / (fabs(W) + c)));
        if (!(rho > 0.0) || !(p > 0.0) || !(v < INFINITY)) v = NAN;  // bad cell: no valid step
    }
    for (int o = 16; o > 0; o >>= 1) v = na_min(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < NA_BLOCK / 32 ? red[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = na_min(v, __shfl_down_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(NA_BLOCK) k_na_cfl_final(const double *__restrict__ partials, int nblocks,
                                                            double cfl, double *__restrict__ dt_out)
{
    __shared__ double red[NA_BLOCK / 32];
    double v = INFINITY;
    for (int b = threadIdx.x; b < nblocks; b += NA_BLOCK) v = na_min(v, partials[b]);
    for (int o = 16; o > 0; o >>= 1) v = na_min(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < NA_BLOCK / 32 ? red[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = na_min(v, __shfl_down_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) *dt_out = cfl * v;
    }
}

// Device address of g_cfl_partials, looked up with the device current, once
// per device and CUDA context.  The address belongs to the context that
// loaded this module: after cudaDeviceReset (or when a caller makes another
// context current) the module is loaded again, possibly at another address,
// so the cache is keyed by the context's unique id (cuCtxGetId; ids are never
// reused) and the lookup is repeated when the id changes.  The two driver
// calls are reached through the runtime's entry-point query, so the library
// does not link libcuda itself.
constexpr int NA_MAX_DEVICES = 64;
struct NaSlot {
    unsigned long long ctx_id;
    double *addr;
};
static NaSlot g_partials_slot[NA_MAX_DEVICES];
static std::mutex g_setup_mutex;

typedef CUresult (*NaCtxGetCurrent)(CUcontext *);
typedef CUresult (*NaCtxGetId)(CUcontext, unsigned long long *);
static NaCtxGetCurrent g_ctx_get_current = nullptr;
static NaCtxGetId g_ctx_get_id = nullptr;

// id of the context current on this thread (cudaErrorNotSupported if the
// driver does not offer the two calls; the address is then looked up anew on
// every call)
static cudaError_t current_context_id(int dev, unsigned long long *id)
{
    *id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        g_ctx_get_current = (NaCtxGetCurrent)f1;
        g_ctx_get_id = (NaCtxGetId)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    if (!ctx) {  // no runtime work on this thread yet: make the device's primary context current
        cudaError_t e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorUnknown;
    }
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

cudaError_t partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    e = current_context_id(dev, &id);
    const bool known = e == cudaSuccess;
    if (!known && e != cudaErrorNotSupported) return e;
    NaSlot &slot = g_partials_slot[dev];
    if (!known || !slot.addr || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cfl_partials);
        if (e != cudaSuccess) return e;
        slot.addr = (double *)p;
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return cudaSuccess;
}

}  // namespace

extern "C" hgks_status hgks_cfl_dt_noalloc(const hgks_grid *grid, double gamma, double cfl, const double *d_q,
                                           double *d_dt, void *cuda_stream)
{
    if (!grid || !d_q || !d_dt) {
        hgks::set_global_error("hgks_cfl_dt_noalloc: null argument");
        return HGKS_ERR_INVALID_ARG;
    }
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->lx > 0.0) || !(grid->ly > 0.0) ||
        !(grid->lz > 0.0) || !(gamma > 1.0) || !(cfl > 0.0)) {
        hgks::set_global_error("hgks_cfl_dt_noalloc: need positive sizes and lengths, gamma > 1, cfl > 0");
        return HGKS_ERR_INVALID_ARG;
    }
    const long long ncell = (long long)grid->nx * grid->ny * grid->nz;
    if (ncell > HGKS_NOALLOC_MAX_CELLS) {  // beyond the fixed scratch
        hgks::set_global_error("hgks_cfl_dt_noalloc: the grid has more than HGKS_NOALLOC_MAX_CELLS "
                               "(33554432) cells, the limit of its fixed scratch");
        return HGKS_ERR_INVALID_ARG;
    }
    char msg[256];
    // an error left by earlier, unrelated work: report it as such and leave it pending
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "hgks_cfl_dt_noalloc: a CUDA error from earlier work is pending: %s",
                 cudaGetErrorString(e));
        hgks::set_global_error(msg);
        return HGKS_ERR_CUDA;
    }
    double *partials = nullptr;
    e = partials_address(&partials);
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(msg, sizeof msg, "hgks_cfl_dt_noalloc: looking up the scratch array's device address failed: %s",
                 cudaGetErrorString(e));
        hgks::set_global_error(msg);
        return HGKS_ERR_CUDA;
    }
    NaGrid g;
    g.nx = grid->nx;
    g.ny = grid->ny;
    g.nz = grid->nz;
    g.hx = grid->lx / grid->nx;
    g.hz = grid->lz / grid->nz;
    g.ly = grid->ly;
    g.y0 = grid->y0;
    g.b = grid->y_stretch_b;
    g.gamma = gamma;
    g.ncell = ncell;
    const int nblocks = (int)((ncell + NA_BLOCK - 1) / NA_BLOCK);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_na_cfl_partial<<<nblocks, NA_BLOCK, 0, st>>>(g, d_q, partials);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_na_cfl_final<<<1, NA_BLOCK, 0, st>>>(partials, nblocks, cfl, d_dt);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "hgks_cfl_dt_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
        hgks::set_global_error(msg);
        return HGKS_ERR_CUDA;
    }
    return HGKS_OK;
}
