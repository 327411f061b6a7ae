// hgks_handle.h -- internals of a solver handle, shared by the C-ABI
// implementation (hgks_api.cu) and the batch module (hgks_batch.cu).
#pragma once
#include "../../include/hgks.h"
#include "hgks_kernels.cuh"

#include <string>

struct hgks_s {
    hgks::Params P;
    hgks_grid grid;
    hgks_bcs bcs;
    hgks_precision prec;
    cudaStream_t st;
    double *q[2] = { nullptr, nullptr };
    int cur = 0;
    double *qs = nullptr, *r = nullptr;
    double *fq = nullptr, *t1 = nullptr;
    double *qf = nullptr;  // mixed precision: the state split into hi / lo float planes
    double *F[3] = { nullptr, nullptr, nullptr };
    double *io[2] = { nullptr, nullptr };  // interior staging buffers [5][N]
    double *ytab = nullptr;                // y metric tables
    double *stat_scratch = nullptr, *stat_out = nullptr;
    hgks::Ctl *ctl = nullptr;
    double rho_ref = 1.0;
    bool stage1_done = false;  // hgks_stage: stage 1 of the step in progress has run
    std::string err;
};
