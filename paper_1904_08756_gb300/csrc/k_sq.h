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

// tcgen05 split-precision contraction (k_sq_tc.cu)
struct TcArgs {
    const unsigned char *a_packed;   // [m_tiles][stages][np_a] packed blocks of the sine matrix
    unsigned char *b_packed;         // [stages][np_b] packed blocks of B = g - 1
    float *S_partial;                // [n_cols][nQ]
    int *status;                     // set to 1 if an MMA wait gave up
    int nQ, n_bins, n_cols, n_pad, m_tiles, stages, kt, np_a, np_b, fmt_bf16, tmem_cols, n_products;
    int prod_a[8], prod_b[8];
    double w[256];
};
int tc_pack_a(const float *Kt, int nQ, int n_bins, int m_tiles, int stages, int kt, int np, int fmt_bf16,
              unsigned char *out, cudaStream_t stream);
int tc_exec(const TcArgs &a, const float *g, cudaStream_t stream);

int sq_build_kt(const float *Q_dev, int nQ, int n_bins, double dr, float *Kt, cudaStream_t stream);
int sq_exec_fp32(const SqArgs &A, cudaStream_t stream);
int sq_exec_adjoint(const SqArgs &A, const float *dS, int cols_per_set, float *dg, cudaStream_t stream);
int sq_totals(const float *S_partial, int n_sets, int cols_per_set, int nQ, const SqWeights &W,
              float *S_total, cudaStream_t stream);

}  // namespace epsr
