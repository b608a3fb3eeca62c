// k_ep.cu -- empirical-potential update (Sec. 2.1 and Eq. 2): the differences Delta S_i(Q)
// between measured and simulated structure factors are resolved into pair terms with the
// (pseudo-)inverse of the Eq. (1) weight matrix, fitted by a series of Poisson-shaped
// functions whose Q-space transform is known in closed form, and the fitted real-space
// series is added to the tabulated empirical potential:
//   U_EP[p][k] += -alpha kT sum_n C[p][n] p_n(r_k),  p_n(r) = (r/(n s))^n exp(n - r/s).
// The Poisson basis is nearly collinear (condition number ~1e10 for 20 functions), so the
// least-squares fit uses Householder QR in FP64, never normal equations. One CTA; this runs
// once per refinement iteration, off the Monte Carlo hot path.
#include <cuda_runtime.h>

#include "epsr_device.cuh"
#include "epsr_internal.h"

namespace epsr {

constexpr int kEpThreads = 512;

__device__ double block_sum_chi(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    return t;
}

__device__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < kEpThreads / 32; ++i) t += red[i];   // same order in every thread
    return t;
}

// 4 pi rho int_0^inf r^2 p_n(r) sin(Qr)/(Qr) dr in closed form:
// (4 pi rho / Q) e^n (n s)^-n Gamma(n+2) s^(n+2) sin((n+2) atan(Q s)) (1 + Q^2 s^2)^-((n+2)/2)
__device__ double poisson_F(int n, double s, double Q, double rho)
{
    const double m = n + 2.0;
    const double logc = n - n * log(n * s) + lgamma(m) + m * log(s);
    return 4.0 * 3.14159265358979323846 * rho / Q * exp(logc - 0.5 * m * log1p(Q * s * Q * s)) *
           sin(m * atan(Q * s));
}

__global__ void __launch_bounds__(kEpThreads, 1)
ep_update_kernel(EpArgs A)
{
    __shared__ double red[kEpThreads / 32];
    __shared__ double M[kEpMaxPairs][kEpMaxData];   // pair-resolving matrix
    __shared__ double Cf[kEpMaxPairs][kEpMaxBasis];  // fitted coefficients
    __shared__ double Rm[kEpMaxBasis][kEpMaxBasis];
    const int tid = threadIdx.x;
    const int nQ = A.nQ, nb = A.n_basis, P = A.n_pairs, nd = A.n_data;
    double *F = A.F;         // [nb][nQ] column-major by basis function
    double *Y = A.Y;         // [P][nQ] pair-resolved Delta S

    // 1. basis matrix
    for (int e = tid; e < nb * nQ; e += kEpThreads) {
        const int n = e / nQ, i = e % nQ;
        F[e] = poisson_F(n + 1, A.s, (double)A.Q[i], A.rho);
    }
    // 2. M = (A^T A)^-1 A^T restricted to the data rows, A = [w; gamma I] (P columns)
    if (tid == 0) {
        double G[kEpMaxPairs][2 * kEpMaxPairs];
        for (int a = 0; a < P; ++a)
            for (int b = 0; b < P; ++b) {
                double v = a == b ? A.gamma * A.gamma : 0.0;
                for (int d = 0; d < nd; ++d) v += A.w[d * P + a] * A.w[d * P + b];
                G[a][b] = v;
                G[a][P + b] = a == b ? 1.0 : 0.0;
            }
        for (int c = 0; c < P; ++c) {               // Gauss-Jordan with partial pivoting
            int piv = c;
            for (int r = c + 1; r < P; ++r)
                if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
            for (int k = 0; k < 2 * P; ++k) { double t = G[c][k]; G[c][k] = G[piv][k]; G[piv][k] = t; }
            const double inv = 1.0 / G[c][c];
            for (int k = 0; k < 2 * P; ++k) G[c][k] *= inv;
            for (int r = 0; r < P; ++r)
                if (r != c) {
                    const double f = G[r][c];
                    for (int k = 0; k < 2 * P; ++k) G[r][k] -= f * G[c][k];
                }
        }
        for (int p = 0; p < P; ++p)
            for (int d = 0; d < nd; ++d) {
                double v = 0.0;
                for (int b = 0; b < P; ++b) v += G[p][P + b] * A.w[d * P + b];
                M[p][d] = v;
            }
    }
    __syncthreads();
    // 3. pair-resolved differences
    for (int e = tid; e < P * nQ; e += kEpThreads) {
        const int p = e / nQ, i = e % nQ;
        double v = 0.0;
        for (int d = 0; d < nd; ++d) v += M[p][d] * (double)A.dS[(long long)d * nQ + i];
        Y[e] = v;
    }
    __syncthreads();
    // 4. Householder QR of F (nQ x nb), reflections applied to the P right-hand sides
    for (int j = 0; j < nb; ++j) {
        double *fj = F + (long long)j * nQ;
        double ss = 0.0;
        for (int i = j + tid; i < nQ; i += kEpThreads) ss += fj[i] * fj[i];
        const double norm = sqrt(block_sum(ss, red));
        const double x0 = fj[j];
        const double alpha = x0 > 0 ? -norm : norm;
        const double v0 = x0 - alpha;
        // v = (v0, f[j+1:]) ; beta = 2 / (v^T v) = 1 / (norm^2 - x0 alpha)
        const double vtv = norm * norm - x0 * x0 + v0 * v0;
        const double beta = vtv > 0 ? 2.0 / vtv : 0.0;
        __syncthreads();
        for (int k = j + 1; k < nb + P; ++k) {
            double *c = k < nb ? F + (long long)k * nQ : Y + (long long)(k - nb) * nQ;
            double dot = 0.0;
            for (int i = j + tid; i < nQ; i += kEpThreads) dot += (i == j ? v0 : fj[i]) * c[i];
            const double f = beta * block_sum(dot, red);
            for (int i = j + tid; i < nQ; i += kEpThreads) c[i] -= f * (i == j ? v0 : fj[i]);
            __syncthreads();
        }
        if (tid == 0) {
            Rm[j][j] = alpha;
            for (int k = j + 1; k < nb; ++k) Rm[j][k] = F[(long long)k * nQ + j];
        }
        __syncthreads();
    }
    // 5. back substitution R C_p = (Q^T y_p)[0:nb]
    if (tid < P) {
        const int p = tid;
        for (int j = nb - 1; j >= 0; --j) {
            double v = Y[(long long)p * nQ + j];
            for (int k = j + 1; k < nb; ++k) v -= Rm[j][k] * Cf[p][k];
            Cf[p][j] = v / Rm[j][j];
        }
    }
    __syncthreads();
    for (int e = tid; e < P * nb; e += kEpThreads) A.C_out[e] = Cf[e / nb][e % nb];
    // 6. table: U_EP[p][k] += -alpha kT sum_n C[p][n] p_n(r_k), r_k = (k + 1/2) dr
    for (int e = tid; e < P * A.n_bins; e += kEpThreads) {
        const int p = e / A.n_bins, k = e % A.n_bins;
        const double r = (k + 0.5) * A.dr;
        double v = 0.0;
        for (int n = 1; n <= nb; ++n)
            v += Cf[p][n - 1] * exp(n * log(r / (n * A.s)) + n - r / A.s);
        A.ep[e] = (float)((double)A.ep[e] - A.alpha * A.kT * v);
    }
}

// ---- chi^2 of the differentiable form: chi2 = sum_Q [S(Q) + sum_p W_p sum_n C_pn F_n(Q) - T(Q)]^2
// The basis values F_n(Q) (FP64 transcendentals, slow on GB300's narrow FP64 unit) are
// evaluated once per call by a grid-wide kernel; one CTA then forms the residuals and the
// sums in a fixed FP64 order (deterministic): dS = 2 res, dC_pn = 2 W_p sum_Q res F_n(Q).
constexpr int kChiThreads = 512;
constexpr int kChiMaxQ = 8192;

__global__ void chi2_basis_kernel(const float *Q, int nQ, int n_basis, double s, double rho, double *F)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_basis * nQ; e += gridDim.x * blockDim.x) {
        const int n = e / nQ, i = e % nQ;
        F[e] = poisson_F(n + 1, s, (double)Q[i], rho);
    }
}

__global__ void __launch_bounds__(kChiThreads, 1)
chi2_kernel(const float *S, const float *T, int nQ, ChiParams prm, const double *C, const double *F,
            double *chi2, float *dS, double *dC)
{
    __shared__ double red[kChiThreads / 32];
    double part = 0.0;
    for (int i = threadIdx.x; i < nQ; i += kChiThreads) {
        double img = 0.0;
        if (C)
            for (int p = 0; p < prm.P; ++p) {
                double v = 0.0;
                for (int n = 0; n < prm.n_basis; ++n) v += C[p * prm.n_basis + n] * F[n * nQ + i];
                img += prm.W[p] * v;
            }
        const double res = (double)S[i] + img - (double)T[i];
        dS[i] = (float)(2.0 * res);
        prm.res_scratch[i] = res;
        part += res * res;
    }
    const double tot = block_sum_chi(part, red);
    if (threadIdx.x == 0) *chi2 = tot;
    __syncthreads();
    if (dC)
        for (int e = threadIdx.x; e < prm.P * prm.n_basis; e += kChiThreads) {
            const int p = e / prm.n_basis, n = e % prm.n_basis;
            double v = 0.0;
            for (int i = 0; i < nQ; ++i) v += prm.res_scratch[i] * F[n * nQ + i];
            dC[e] = 2.0 * prm.W[p] * v;
        }
}

int launch_ep_update(const EpArgs &a, cudaStream_t stream)
{
    ep_update_kernel<<<1, kEpThreads, 0, stream>>>(a);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "ep_update");
}

int launch_chi2(const float *S, const float *target, const float *Q, int nQ, const ChiParams &prm,
                const double *C, double *chi2, float *dS, double *dC, cudaStream_t stream)
{
    if (nQ > kChiMaxQ) return set_error(EPSR_EINVAL, "chi2: nQ above %d", kChiMaxQ);
    if (C) {
        const int n = prm.n_basis * nQ;
        chi2_basis_kernel<<<(n + 255) / 256, 256, 0, stream>>>(Q, nQ, prm.n_basis, prm.s, prm.rho, prm.F_scratch);
        note_launch();
    }
    chi2_kernel<<<1, kChiThreads, 0, stream>>>(S, target, nQ, prm, C, prm.F_scratch, chi2, dS, dC);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "chi2");
}

}  // namespace epsr
