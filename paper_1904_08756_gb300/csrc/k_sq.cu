// k_sq.cu -- S(Q) by Eq. (1) as a contraction of the sine-transform matrix
// K[i][k] = r_k^2 dr sin(Q_i r_k) / (Q_i r_k) (midpoint rule, r_k = (k + 1/2) dr) with the
// weighted columns G[c][k] = w_c (g_c(k) - 1).
//
// FP32 path (this file): K is built once per plan in FP64 and stored transposed,
// K_t[k][i], so that a warp reading one k row reads 32 consecutive Q values; the G
// columns of a block are staged in shared memory, each warp accumulates S_partial[c][i]
// over an interleaved subset of the bins with compensated (Kahan) FP32 summation, and the
// subsets are added in FP64 in a fixed order.
#include "epsr_device.cuh"
#include "epsr_internal.h"
#include "k_sq.h"

namespace epsr {

__global__ void build_sine_matrix_kernel(const float *Q, int nQ, int n_bins, double dr, float *Kt)
{
    const long long n = (long long)nQ * n_bins;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / nQ), i = (int)(e % nQ);
        const double r = ((double)k + 0.5) * dr;
        const double x = (double)Q[i] * r;
        Kt[e] = (float)(r * r * dr * sin(x) / x);
    }
}

int sq_build_kt(const float *Q_dev, int nQ, int n_bins, double dr, float *Kt, cudaStream_t stream)
{
    const long long n = (long long)nQ * n_bins;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    build_sine_matrix_kernel<<<grid, 256, 0, stream>>>(Q_dev, nQ, n_bins, dr, Kt);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "build_sine_matrix");
}

constexpr int kSqQ = 32;                       // Q values per block (one per lane)
constexpr int kSqSplit = 8;                    // interleaved bin subsets per Q (one warp each)
constexpr int kSqThreads = kSqQ * kSqSplit;
constexpr int kSqCols = 8;                     // columns per block

// S_partial[c][i] = w_c sum_k K_t[k][i] (g[c][k] - 1) for c in [c0, c0 + kSqCols). Warp p of a
// block sums the bins k = p (mod kSqSplit) for its 32 Q values with compensated (Kahan) FP32
// summation; the kSqSplit partial sums of a Q value are then added in FP64 in a fixed order.
__global__ void __launch_bounds__(kSqThreads) sq_fp32_kernel(SqArgs A)
{
    extern __shared__ float s_g[];      // [kSqCols][n_bins] of (g - 1)
    __shared__ double s_part[kSqSplit][kSqCols][kSqQ];
    const int c0 = blockIdx.y * kSqCols;
    const int nc = min(kSqCols, A.n_cols - c0);
    const int nb = A.n_bins;
    for (int e = threadIdx.x; e < nc * nb; e += kSqThreads)
        s_g[e] = A.g[(long long)(c0 + e / nb) * nb + e % nb] - 1.0f;
    __syncthreads();
    const int q = threadIdx.x % kSqQ, part = threadIdx.x / kSqQ;
    const int i = blockIdx.x * kSqQ + q;
    float sum[kSqCols], comp[kSqCols];
#pragma unroll
    for (int c = 0; c < kSqCols; ++c) sum[c] = comp[c] = 0.f;
    if (i < A.nQ) {
#pragma unroll 4
        for (int k = part; k < nb; k += kSqSplit) {
            const float kv = A.Kt[(long long)k * A.nQ + i];
#pragma unroll
            for (int c = 0; c < kSqCols; ++c) {
                if (c < nc) {
                    const float y = kv * s_g[c * nb + k] - comp[c];
                    const float t = sum[c] + y;
                    comp[c] = (t - sum[c]) - y;
                    sum[c] = t;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < kSqCols; ++c) s_part[part][c][q] = (double)sum[c] - (double)comp[c];
    __syncthreads();
    for (int e = threadIdx.x; e < nc * kSqQ; e += kSqThreads) {
        const int c = e / kSqQ, qq = e % kSqQ, ii = blockIdx.x * kSqQ + qq;
        if (ii >= A.nQ) continue;
        double t = 0.0;
        for (int p = 0; p < kSqSplit; ++p) t += s_part[p][c][qq];
        A.S_partial[(long long)(c0 + c) * A.nQ + ii] = (float)(t * A.w[c0 + c]);
    }
}

// S_total[s][i] = flat[s] + sum over the set's columns (in column order, FP64).
__global__ void sq_total_kernel(const float *S_partial, int n_sets, int cols_per_set, int nQ,
                                SqWeights W, float *S_total)
{
    const long long n = (long long)n_sets * nQ;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / nQ), i = (int)(e % nQ);
        double t = W.flat[s];
        for (int c = 0; c < cols_per_set; ++c)
            t += (double)S_partial[(long long)(s * cols_per_set + c) * nQ + i];
        S_total[e] = (float)t;
    }
}

int sq_exec_fp32(const SqArgs &A, cudaStream_t stream)
{
    dim3 grid((A.nQ + kSqQ - 1) / kSqQ, (A.n_cols + kSqCols - 1) / kSqCols);
    const size_t smem = (size_t)kSqCols * A.n_bins * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sq_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kSqCols * EPSR_MAX_BINS * sizeof(float)));
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(sq)");
        attr = true;
    }
    sq_fp32_kernel<<<grid, kSqThreads, smem, stream>>>(A);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "sq_fp32");
}

int sq_totals(const float *S_partial, int n_sets, int cols_per_set, int nQ, const SqWeights &W,
              float *S_total, cudaStream_t stream)
{
    const long long n = (long long)n_sets * nQ;
    const int grid = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
    sq_total_kernel<<<grid, 256, 0, stream>>>(S_partial, n_sets, cols_per_set, nQ, W, S_total);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "sq_total");
}

// Adjoint of the contraction: dg[c][k] = w_c sum_i K[i][k] dS_total[set(c)][i]. One warp per
// (c, k): lane l sums i = l (mod 32) with compensated (Kahan) FP32 summation, and the lanes'
// sums are added in FP64 by a fixed shuffle tree.
__global__ void sq_adjoint_kernel(SqArgs A, const float *dS, int cols_per_set, float *dg)
{
    const long long n = (long long)A.n_cols * A.n_bins;
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < n; e += warps) {
        const int c = (int)(e / A.n_bins), k = (int)(e % A.n_bins);
        const float *row = A.Kt + (long long)k * A.nQ;
        const float *d = dS + (long long)(c / cols_per_set) * A.nQ;
        float sum = 0.f, comp = 0.f;
#pragma unroll 4
        for (int i = lane; i < A.nQ; i += 32) {
            const float y = row[i] * d[i] - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        double v = (double)sum - (double)comp;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) dg[e] = (float)(v * A.w[c]);
    }
}

int sq_exec_adjoint(const SqArgs &A, const float *dS, int cols_per_set, float *dg, cudaStream_t stream)
{
    const long long n = (long long)A.n_cols * A.n_bins;                // one warp each
    const int grid = (int)((n + 3) / 4 < 8192 ? (n + 3) / 4 : 8192);    // 4 warps per block
    sq_adjoint_kernel<<<grid, 128, 0, stream>>>(A, dS, cols_per_set, dg);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "sq_adjoint");
}

}  // namespace epsr
