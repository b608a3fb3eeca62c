// k_sq.h -- argument blocks of the S(Q) kernels (passed by value as kernel parameters,
// so an exec enqueues no host-to-device copy and can be captured in a CUDA graph).
#pragma once

#include <cuda_runtime.h>

#include "epsr.h"

namespace epsr {

struct SqArgs {
    const float *g;        // [n_cols][n_bins]
    const float *Kt;       // [n_bins][nQ]
    float *S_partial;      // [n_cols][nQ]
    int nQ, n_bins, n_cols;
    double w[EPSR_SQ_MAX_COLS];
};

struct SqWeights {
    double flat[EPSR_SQ_MAX_COLS];
};

int sq_build_kt(const float *Q_dev, int nQ, int n_bins, double dr, float *Kt, cudaStream_t stream);
int sq_exec_fp32(const SqArgs &A, cudaStream_t stream);
int sq_exec_adjoint(const SqArgs &A, const float *dS, int cols_per_set, float *dg, cudaStream_t stream);
int sq_totals(const float *S_partial, int n_sets, int cols_per_set, int nQ, const SqWeights &W,
              float *S_total, cudaStream_t stream);

}  // namespace epsr
