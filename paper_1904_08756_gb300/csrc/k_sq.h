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

// tcgen05 split-precision contraction (k_sq_tc.cu). Passed as a __grid_constant__ kernel
// parameter (about 4 KB: the column weights and set backgrounds travel with the launch).
constexpr int kTcMaxKSplit = 8;     // CTAs of one cluster sharing an output tile (portable size)
constexpr int kTcMaxSlots = 8;      // K-unit buffers per CTA (copies of later units overlap MMAs)
struct TcArgs {
    const unsigned char *a_packed;   // [m_tiles][units][np_a] packed blocks of the sine matrix
    const float *g;                  // [n_cols][n_bins]; B = g - 1 is split and packed in the kernel
    float *S_partial;                // [n_cols][nQ] or NULL
    float *S_total;                  // [n_cols / cols_per_set][nQ] or NULL (fused sets only)
    int *status;                     // set to 1 if a copy or MMA wait gave up
    int nQ, n_bins, n_cols, m_tiles, units, ku, np_a, np_b, fmt_bf16, n_products;
    int n_chunk;                     // columns per CTA: a multiple of 16, <= 256
    int k_split;                     // CTAs per output tile (one cluster), <= kTcMaxKSplit
    int tmem_cols;                   // power of two >= max(32, n_chunk)
    int cols_per_set;                // S_total sets; n_chunk % cols_per_set == 0 when S_total != NULL
    int slots;                       // K-unit buffers per CTA, 2 .. kTcMaxSlots
    int recv_cols;                   // columns a cluster rank owns in the reduction, at most
    float w[EPSR_SQ_MAX_COLS];
    float flat[EPSR_SQ_MAX_COLS];
};
int tc_pack_a(const float *Kt, int nQ, int n_bins, int m_tiles, int stages, int kt, int np, int fmt_bf16,
              unsigned char *out, cudaStream_t stream);
// Shared memory of one CTA of the contraction (tc_smem_bytes: with two unit buffers, 0 if it
// does not fit), the unit buffers a CTA with units_per_cta units gets, and the columns one
// cluster rank owns in the reduction (grp: set size when the set totals are fused, else 1).
size_t tc_smem_need(int n_chunk, int np, int slots, int k_split, int grp);
size_t tc_smem_bytes(int n_chunk, int np, int k_split, int grp);
int tc_slots_for(int n_chunk, int np, int units_per_cta, int k_split, int grp, bool one_per_sm);
int tc_recv_cols(int n_chunk, int grp, int k_split);
int tc_exec(const TcArgs &a, cudaStream_t stream);

int sq_build_kt(const float *Q_dev, int nQ, int n_bins, double dr, float *Kt, cudaStream_t stream);
int sq_exec_fp32(const SqArgs &A, cudaStream_t stream);
int sq_exec_adjoint(const SqArgs &A, const float *dS, int cols_per_set, float *dg, cudaStream_t stream);
int sq_totals(const float *S_partial, int n_sets, int cols_per_set, int nQ, const SqWeights &W,
              float *S_total, cudaStream_t stream);

}  // namespace epsr
