// k_smear.cu -- the differentiable form of the histogram: a Gaussian-smeared N_ab(r)
// (every pair spreads a Gaussian of width sigma, truncated at +-5 sigma, over the bins)
// and its adjoint, the gradient of sum_{p,k} lambda[p][k] Ht[p][k] with respect to the
// atom positions. Pair distances are recomputed in the adjoint, never stored.
//
//   w_k(r) = Phi(clip((r_{k+1} - r)/sigma)) - Phi(clip((r_k - r)/sigma)),  clip to [-5, 5]
//   dw_k/dr = (phi(a_k)[|a_k| < 5] - phi(a_{k+1})[|a_{k+1}| < 5]) / sigma,  a_k = (r_k - r)/sigma
//
// Same tiling as the pair histogram (persistent grid over (box, i-tile, j-tile) in
// spatial order, 2^32-periodic prefilter), with the cutoff r_max + 5 sigma. The forward
// accumulates every weight as an exact fixed-point integer (weight * 2^32, 64-bit integer
// atomics in shared then global memory): float atomics over ~10^4 additions per bin lose
// a systematic few 1e-6, which low-Q S(Q) (a cancellation of large terms) amplifies.
// Integer sums are also independent of the order, so the forward is deterministic.
#include "epsr_device.cuh"
#include "epsr_internal.h"

namespace epsr {

constexpr int kSmThreads = 256;
constexpr int kSmR = kGrTile / kSmThreads;

__device__ __forceinline__ unsigned smear_prefilter(const BoxDev &bx, double sigma)
{
    const double S = 1.0 / sqrt((double)bx.inv_s2);
    const double Rfx = ((double)bx.n_bins * bx.dr_A + 5.0 * sigma) * S + 2.0;
    const double Rs = ceil(Rfx * 4294967296.0 / (double)bx.L) + 2.0;
    return Rs >= 2147483647.0 ? 2147483647u : (unsigned)Rs;
}

template <bool kBackward>
__global__ void __launch_bounds__(kSmThreads, 2) smear_kernel(SmearArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    uint4 *s_scaled = reinterpret_cast<uint4 *>(dyn);
    int4 *s_true = reinterpret_cast<int4 *>(s_scaled + kGrTile);
    int *s_idx = reinterpret_cast<int *>(s_true + kGrTile);
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(s_idx + kGrTile);  // fwd
    float *s_buf = reinterpret_cast<float *>(s_idx + kGrTile);    // bwd: lambda
    float *s_gj = s_buf + A.max_pairs_bins;                       // bwd: j-tile gradients [3][tile]
    __shared__ BoxDev bx;
    __shared__ int cur_box;
    __shared__ unsigned pre;
    const int tid = threadIdx.x;
    const float sg = (float)A.sigma, inv_sg = 1.0f / sg;
    const float inv_sqrt2 = 0.70710678118654752f, inv_sqrt2pi = 0.39894228040143268f;
    if (tid == 0) cur_box = -1;
    if (!kBackward)
        for (int k = tid; k < A.max_pairs_bins; k += kSmThreads) s_acc[k] = 0ull;
    __syncthreads();
    for (long long w = blockIdx.x; w < A.n_tiles; w += gridDim.x) {
        const GrTile tl = A.tiles[w];
        __syncthreads();
        if (tl.box != cur_box) {
            if (!kBackward && cur_box >= 0) {
                const int n = bx.n_pairs * bx.n_bins;
                for (int k = tid; k < n; k += kSmThreads) {
                    const unsigned long long v = s_acc[k];
                    if (v) { atomicAdd(A.acc + bx.hist_off + k, v); s_acc[k] = 0ull; }
                }
            }
            __syncthreads();
            if (tid == 0) {
                bx = A.boxes[tl.box];
                cur_box = tl.box;
                pre = smear_prefilter(bx, A.sigma);
            }
            __syncthreads();
            if (kBackward)
                for (int k = tid; k < bx.n_pairs * bx.n_bins; k += kSmThreads)
                    s_buf[k] = A.lambda[bx.hist_off + k];
        }
        const int L = bx.L, N = bx.n_atoms, nb = bx.n_bins, nt = bx.n_types;
        const unsigned R = pre, R2 = 2u * pre;
        const float dr = (float)bx.dr_A, inv_dr = 1.0f / dr;
        const float S = 1.0f / sqrtf(bx.inv_s2);
        const float rcut = (float)nb * dr + 5.0f * sg;
        const int j0 = tl.tj * kGrTile, nj = min(kGrTile, N - j0);
        for (int j = tid; j < nj; j += kSmThreads) {
            s_scaled[j] = A.scaled[bx.atom0 + j0 + j];
            s_true[j] = A.coords[bx.atom0 + j0 + j];
            if (kBackward) {
                s_idx[j] = A.index[bx.atom0 + j0 + j];
                s_gj[j] = s_gj[kGrTile + j] = s_gj[2 * kGrTile + j] = 0.f;
            }
        }
        const int i0 = tl.ti * kGrTile;
        uint32_t xi[kSmR], yi[kSmR], zi[kSmR];
        int il[kSmR];
        float gi[kSmR][3];
#pragma unroll
        for (int r = 0; r < kSmR; ++r) {
            il[r] = tid + r * kSmThreads;
            gi[r][0] = gi[r][1] = gi[r][2] = 0.f;
            if (i0 + il[r] < N) {
                const uint4 s = A.scaled[bx.atom0 + i0 + il[r]];
                xi[r] = s.x + R; yi[r] = s.y + R; zi[r] = s.z + R;
            } else {
                il[r] = -1;
                xi[r] = yi[r] = zi[r] = 0u;
            }
        }
        const bool diag = tl.ti == tl.tj;
        __syncthreads();
        for (int j = 0; j < nj; ++j) {
            const uint4 sj = s_scaled[j];
#pragma unroll
            for (int r = 0; r < kSmR; ++r) {
                const bool hit = (xi[r] - sj.x < R2) & (yi[r] - sj.y < R2) & (zi[r] - sj.z < R2);
                if (!hit || il[r] < 0 || (diag && j <= il[r])) continue;
                const int4 pi = A.coords[bx.atom0 + i0 + il[r]];
                const int4 pj = s_true[j];
                int dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;   // signed minimum image
                if (2LL * dx > L) dx -= L; else if (2LL * dx <= -L) dx += L;
                if (2LL * dy > L) dy -= L; else if (2LL * dy <= -L) dy += L;
                if (2LL * dz > L) dz -= L; else if (2LL * dz <= -L) dz += L;
                const float fx = (float)dx / S, fy = (float)dy / S, fz = (float)dz / S;
                const float r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                const float rr = sqrtf(r2);
                if (!(rr < rcut) || rr == 0.f) continue;
                const int p = pair_index(pi.w, pj.w, nt);
                const int klo = max(0, (int)floorf((rr - 5.0f * sg) * inv_dr));
                const int khi = min(nb - 1, (int)floorf((rr + 5.0f * sg) * inv_dr));
                if (!kBackward) {
                    float a = fminf(5.f, fmaxf(-5.f, ((float)klo * dr - rr) * inv_sg));
                    float Pa = 0.5f * erff(a * inv_sqrt2);
                    for (int k = klo; k <= khi; ++k) {
                        const float b = fminf(5.f, fmaxf(-5.f, ((float)(k + 1) * dr - rr) * inv_sg));
                        const float Pb = 0.5f * erff(b * inv_sqrt2);
                        const float wk = fmaxf(0.f, Pb - Pa);
                        atomicAdd(&s_acc[p * nb + k], (unsigned long long)__float2ll_rn(wk * 4294967296.0f));
                        Pa = Pb;
                    }
                } else {
                    const float *lam = s_buf + p * nb;
                    float a = ((float)klo * dr - rr) * inv_sg;
                    float pa = fabsf(a) < 5.f ? expf(-0.5f * a * a) : 0.f;
                    float dEdr = 0.f;
                    for (int k = klo; k <= khi; ++k) {
                        const float b = ((float)(k + 1) * dr - rr) * inv_sg;
                        const float pb = fabsf(b) < 5.f ? expf(-0.5f * b * b) : 0.f;
                        dEdr = fmaf(lam[k], pa - pb, dEdr);
                        pa = pb;
                    }
                    const float f = dEdr * inv_sqrt2pi * inv_sg / rr;
                    gi[r][0] = fmaf(f, fx, gi[r][0]);
                    gi[r][1] = fmaf(f, fy, gi[r][1]);
                    gi[r][2] = fmaf(f, fz, gi[r][2]);
                    atomicAdd(&s_gj[j], -f * fx);
                    atomicAdd(&s_gj[kGrTile + j], -f * fy);
                    atomicAdd(&s_gj[2 * kGrTile + j], -f * fz);
                }
            }
        }
        if (kBackward) {
#pragma unroll
            for (int r = 0; r < kSmR; ++r) {
                if (il[r] < 0) continue;
                const int atom = A.index[bx.atom0 + i0 + il[r]];
                if (gi[r][0] != 0.f) atomicAdd(&A.grad[3 * atom], gi[r][0]);
                if (gi[r][1] != 0.f) atomicAdd(&A.grad[3 * atom + 1], gi[r][1]);
                if (gi[r][2] != 0.f) atomicAdd(&A.grad[3 * atom + 2], gi[r][2]);
            }
            __syncthreads();
            for (int j = tid; j < nj; j += kSmThreads) {
                const int atom = s_idx[j];
                for (int c = 0; c < 3; ++c) {
                    const float v = s_gj[c * kGrTile + j];
                    if (v != 0.f) atomicAdd(&A.grad[3 * atom + c], v);
                }
            }
        }
    }
    __syncthreads();
    if (!kBackward && cur_box >= 0) {
        const int n = bx.n_pairs * bx.n_bins;
        for (int k = tid; k < n; k += kSmThreads) {
            const unsigned long long v = s_acc[k];
            if (v) atomicAdd(A.acc + bx.hist_off + k, v);
        }
    }
}

int launch_smear(const SmearArgs &a, bool backward, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)kGrTile * (sizeof(uint4) + sizeof(int4) + sizeof(int)) +
                        (backward ? (size_t)a.max_pairs_bins * sizeof(float) + (size_t)3 * kGrTile * sizeof(float)
                                  : (size_t)a.max_pairs_bins * sizeof(unsigned long long));
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(smear_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(smear_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(smear)");
        attr = true;
    }
    if (smem > 200 * 1024) return set_error(EPSR_EINVAL, "smeared g: n_pairs*n_bins too large");
    if (backward) smear_kernel<true><<<grid, kSmThreads, smem, stream>>>(a);
    else smear_kernel<false><<<grid, kSmThreads, smem, stream>>>(a);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "smear launch");
}

// lambda[p][k] = dL/dgt[p][k] * V / (P_ab shell_k): the adjoint of the normalisation
__global__ void smear_lambda_kernel(const BoxDev *boxes, int n_boxes, const float *dgt, float *lam,
                                    long long hist_len, const long long *hist_box)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hist_len;
         i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_boxes;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (hist_box[mid] <= i) lo = mid; else hi = mid;
        }
        const BoxDev &b = boxes[lo];
        const long long e = i - b.hist_off;
        const int p = (int)(e / b.n_bins), k = (int)(e % b.n_bins);
        int a = 0, rem = p;
        while (rem >= b.n_types - a) { rem -= b.n_types - a; ++a; }
        const int c = a + rem;
        const double Pab = a == c ? 0.5 * (double)b.count[a] * (double)(b.count[a] - 1)
                                  : (double)b.count[a] * (double)b.count[c];
        const double r0 = (double)k * b.dr_A, r1 = (double)(k + 1) * b.dr_A;
        const double shell = 4.18879020478639098462 * (r1 * r1 * r1 - r0 * r0 * r0);
        lam[i] = Pab * shell > 0 ? (float)((double)dgt[i] * b.volume / (Pab * shell)) : 0.f;
    }
}

// Ht = acc 2^-32 and (optionally) gt = Ht V / (P_ab shell_k), normalised like g
__global__ void smear_norm_kernel(const BoxDev *boxes, int n_boxes, const unsigned long long *acc,
                                  double *Ht, float *gt, long long hist_len, const long long *hist_box)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hist_len;
         i += (long long)gridDim.x * blockDim.x) {
        const double h = (double)acc[i] * 0x1p-32;
        Ht[i] = h;
        if (!gt) continue;
        int lo = 0, hi = n_boxes;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (hist_box[mid] <= i) lo = mid; else hi = mid;
        }
        const BoxDev &b = boxes[lo];
        const long long e = i - b.hist_off;
        const int p = (int)(e / b.n_bins), k = (int)(e % b.n_bins);
        int a = 0, rem = p;
        while (rem >= b.n_types - a) { rem -= b.n_types - a; ++a; }
        const int c = a + rem;
        const double Pab = a == c ? 0.5 * (double)b.count[a] * (double)(b.count[a] - 1)
                                  : (double)b.count[a] * (double)b.count[c];
        const double r0 = (double)k * b.dr_A, r1 = (double)(k + 1) * b.dr_A;
        const double shell = 4.18879020478639098462 * (r1 * r1 * r1 - r0 * r0 * r0);
        gt[i] = Pab * shell > 0 ? (float)(h * b.volume / (Pab * shell)) : 0.f;
    }
}

int launch_smear_norm(const BoxDev *boxes, int n_boxes, const unsigned long long *acc, double *Ht,
                      float *gt, long long hist_len, const long long *hist_box, cudaStream_t stream)
{
    const int grid = (int)((hist_len + 255) / 256 < 2048 ? (hist_len + 255) / 256 : 2048);
    smear_norm_kernel<<<grid, 256, 0, stream>>>(boxes, n_boxes, acc, Ht, gt, hist_len, hist_box);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "smear_norm");
}

int launch_smear_lambda(const BoxDev *boxes, int n_boxes, const float *dgt, float *lam, long long hist_len,
                        const long long *hist_box, cudaStream_t stream)
{
    const int grid = (int)((hist_len + 255) / 256 < 2048 ? (hist_len + 255) / 256 : 2048);
    smear_lambda_kernel<<<grid, 256, 0, stream>>>(boxes, n_boxes, dgt, lam, hist_len, hist_box);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "smear_lambda");
}

}  // namespace epsr
