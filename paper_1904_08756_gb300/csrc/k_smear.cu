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
// accumulates every weight as an exact fixed-point integer (weight rounded to 2^-20, 32-bit
// integer atomics in shared memory, flushed into 64-bit global sums before they can wrap):
// float atomics over ~10^4 additions per bin lose a systematic few 1e-6, which low-Q S(Q) (a
// cancellation of large terms) amplifies, while rounding each weight to 2^-20 is unbiased.
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

// Per-warp queue of prefilter hits: the scan runs lane-parallel over pairs, and the costly
// smearing of a pair (about 17 bins, an erf or exp per bin edge) runs once 32 hits are queued,
// one hit per lane, so whole warps do it instead of single lanes.
constexpr int kSmWarps = kSmThreads / 32;
constexpr int kSmQueue = 32 + 32 * kSmR;    // holds a partial drain plus one j's worth of hits

// Smearing of one pair: the forward adds its clipped-Gaussian weights to the 32-bit shared
// accumulators (weight * 2^20; with kCarry a wrap carries 2^32 into the 64-bit global sum,
// otherwise the caller flushes before one can happen); the backward
// returns f = (dE/dr) / r with E = sum_k lambda_k w_k(r), so that the gradient of E is
// +f d for atom i and -f d for atom j (d = r_i - r_j in Angstrom, returned in fx, fy, fz).
template <bool kBackward, bool kCarry = true>
__device__ __forceinline__ float smear_core(const SmearArgs &A, const BoxDev &bx, int4 pi, int4 pj,
                                            unsigned *s_acc, const float *s_lam, float sg, float inv_sg,
                                            float S, float &fx, float &fy, float &fz)
{
    const float inv_sqrt2 = 0.70710678118654752f, inv_sqrt2pi = 0.39894228040143268f;
    const int L = bx.L, nb = bx.n_bins, nt = bx.n_types;
    const float dr = (float)bx.dr_A, inv_dr = 1.0f / dr;
    const float rcut = (float)nb * dr + 5.0f * sg;
    int dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;   // signed minimum image
    if (2LL * dx > L) dx -= L; else if (2LL * dx <= -L) dx += L;
    if (2LL * dy > L) dy -= L; else if (2LL * dy <= -L) dy += L;
    if (2LL * dz > L) dz -= L; else if (2LL * dz <= -L) dz += L;
    fx = (float)dx / S;
    fy = (float)dy / S;
    fz = (float)dz / S;
    const float r2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
    const float rr = sqrtf(r2);
    if (!(rr < rcut) || rr == 0.f) return 0.f;
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
            const unsigned v = (unsigned)__float2uint_rn(wk * 1048576.0f);
            if (kCarry) {
                const unsigned old = atomicAdd(&s_acc[p * nb + k], v);
                if (old > 0xFFFFFFFFu - v) atomicAdd(A.acc + bx.hist_off + p * nb + k, 1ull << 32);
            } else {
                atomicAdd(&s_acc[p * nb + k], v);          // the caller flushes before a wrap
            }
            Pa = Pb;
        }
        return 0.f;
    }
    const float *lam = s_lam + p * nb;
    float a = ((float)klo * dr - rr) * inv_sg;
    float pa = fabsf(a) < 5.f ? expf(-0.5f * a * a) : 0.f;
    float dEdr = 0.f;
    for (int k = klo; k <= khi; ++k) {
        const float b = ((float)(k + 1) * dr - rr) * inv_sg;
        const float pb = fabsf(b) < 5.f ? expf(-0.5f * b * b) : 0.f;
        dEdr = fmaf(lam[k], pa - pb, dEdr);
        pa = pb;
    }
    return dEdr * inv_sqrt2pi * inv_sg / rr;
}

template <bool kBackward>
__device__ __forceinline__ void smear_pair(const SmearArgs &A, const BoxDev &bx, int i_local, int i0, int j,
                                           const int4 *s_true, unsigned *s_acc, const float *s_lam,
                                           float *s_gi, float *s_gj, float sg, float inv_sg, float S)
{
    float fx, fy, fz;
    const float f = smear_core<kBackward>(A, bx, A.coords[bx.atom0 + i0 + i_local], s_true[j], s_acc, s_lam,
                                          sg, inv_sg, S, fx, fy, fz);
    if (kBackward && f != 0.f) {
        atomicAdd(&s_gi[i_local], f * fx);
        atomicAdd(&s_gi[kGrTile + i_local], f * fy);
        atomicAdd(&s_gi[2 * kGrTile + i_local], f * fz);
        atomicAdd(&s_gj[j], -f * fx);
        atomicAdd(&s_gj[kGrTile + j], -f * fy);
        atomicAdd(&s_gj[2 * kGrTile + j], -f * fz);
    }
}

template <bool kBackward>
__global__ void __launch_bounds__(kSmThreads, 2) smear_kernel(SmearArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    uint4 *s_scaled = reinterpret_cast<uint4 *>(dyn);
    int4 *s_true = reinterpret_cast<int4 *>(s_scaled + kGrTile);
    int *s_idx = reinterpret_cast<int *>(s_true + kGrTile);
    int2 *s_queue = reinterpret_cast<int2 *>(s_idx + kGrTile);                      // [warps][queue]
    unsigned *s_acc = reinterpret_cast<unsigned *>(s_queue + kSmWarps * kSmQueue);     // fwd
    float *s_buf = reinterpret_cast<float *>(s_queue + kSmWarps * kSmQueue);     // bwd: lambda
    float *s_gj = s_buf + A.max_pairs_bins;                                      // bwd: [3][tile]
    float *s_gi = s_gj + 3 * kGrTile;                                            // bwd: [3][tile]
    __shared__ BoxDev bx;
    __shared__ int cur_box;
    __shared__ unsigned pre;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int2 *q = s_queue + warp * kSmQueue;
    const float sg = (float)A.sigma, inv_sg = 1.0f / sg;
    if (tid == 0) cur_box = -1;
    if (!kBackward)
        for (int k = tid; k < A.max_pairs_bins; k += kSmThreads) s_acc[k] = 0u;
    __syncthreads();
    for (long long w = blockIdx.x; w < A.n_tiles; w += gridDim.x) {
        const GrTile tl = A.tiles[w];
        __syncthreads();
        if (tl.box != cur_box) {
            if (!kBackward && cur_box >= 0) {
                const int n = bx.n_pairs * bx.n_bins;
                for (int k = tid; k < n; k += kSmThreads) {
                    const unsigned v = s_acc[k];
                    if (v) { atomicAdd(A.acc + bx.hist_off + k, (unsigned long long)v); s_acc[k] = 0u; }
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
        const int N = bx.n_atoms;
        const unsigned R = pre, R2 = 2u * pre;
        const float S = 1.0f / sqrtf(bx.inv_s2);
        const int j0 = tl.tj * kGrTile, nj = min(kGrTile, N - j0);
        for (int j = tid; j < nj; j += kSmThreads) {
            s_scaled[j] = A.scaled[bx.atom0 + j0 + j];
            s_true[j] = A.coords[bx.atom0 + j0 + j];
            if (kBackward) {
                s_idx[j] = A.index[bx.atom0 + j0 + j];
                s_gj[j] = s_gj[kGrTile + j] = s_gj[2 * kGrTile + j] = 0.f;
            }
        }
        if (kBackward)
            for (int i = tid; i < kGrTile; i += kSmThreads) s_gi[i] = s_gi[kGrTile + i] = s_gi[2 * kGrTile + i] = 0.f;
        const int i0 = tl.ti * kGrTile;
        uint32_t xi[kSmR], yi[kSmR], zi[kSmR];
        int il[kSmR];
#pragma unroll
        for (int r = 0; r < kSmR; ++r) {
            il[r] = tid + r * kSmThreads;
            if (i0 + il[r] < N) {
                const uint4 sc = A.scaled[bx.atom0 + i0 + il[r]];
                xi[r] = sc.x + R; yi[r] = sc.y + R; zi[r] = sc.z + R;
            } else {
                il[r] = -1;
                xi[r] = yi[r] = zi[r] = 0u;
            }
        }
        const bool diag = tl.ti == tl.tj;
        __syncthreads();
        int qn = 0;                                       // entries in this warp's queue
        for (int j = 0; j < nj; ++j) {
            const uint4 sj = s_scaled[j];
#pragma unroll
            for (int r = 0; r < kSmR; ++r) {
                const bool hit = __vimax3_u32(xi[r] - sj.x, yi[r] - sj.y, zi[r] - sj.z) < R2 && il[r] >= 0 &&
                                 !(diag && j <= il[r]);
                const unsigned bal = __ballot_sync(0xffffffffu, hit);
                if (hit) q[qn + __popc(bal & ((1u << lane) - 1u))] = make_int2(il[r], j);
                qn += __popc(bal);
            }
            while (qn >= 32) {                            // drain 32 hits, one per lane
                __syncwarp();
                const int2 e = q[qn - 32 + lane];
                __syncwarp();
                smear_pair<kBackward>(A, bx, e.x, i0, e.y, s_true, s_acc, s_buf, s_gi, s_gj, sg, inv_sg, S);
                qn -= 32;
            }
        }
        __syncwarp();
        if (lane < qn) {
            const int2 e = q[lane];
            smear_pair<kBackward>(A, bx, e.x, i0, e.y, s_true, s_acc, s_buf, s_gi, s_gj, sg, inv_sg, S);
        }
        if (kBackward) {
            __syncthreads();
            for (int i = tid; i < kGrTile; i += kSmThreads) {
                if (i0 + i >= N) continue;
                const int atom = A.index[bx.atom0 + i0 + i];
                for (int c = 0; c < 3; ++c) {
                    const float v = s_gi[c * kGrTile + i];
                    if (v != 0.f) atomicAdd(&A.grad[3 * atom + c], v);
                }
            }
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
            const unsigned v = s_acc[k];
            if (v) atomicAdd(A.acc + bx.hist_off + k, (unsigned long long)v);
        }
    }
}

// ---- the same sums over cell lists -----------------------------------------------------------
// Cells of the cell-list histogram (at least r_max + 0.5 A + 2 grid units wide), valid for
// 5 sigma <= 0.5 A: every pair with r < r_max + 5 sigma lies in the same or a neighbouring
// cell. One work item per home cell; the home atoms (one per thread per pass) meet the home
// cell (later sorted positions only) and its 13 forward neighbours staged in shared memory,
// and pairs inside r_max + 5 sigma are queued per warp and smeared 32 at a time.
constexpr int kScThreads = 128;
constexpr int kScStage = 512;
constexpr int kScWarps = kScThreads / 32;
constexpr int kScQueue = 64;

__constant__ int c_sfwd[14][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 1, 0},  {0, 1, 0},   {1, 1, 0},
                                  {-1, -1, 1}, {0, -1, 1},  {1, -1, 1},  {-1, 0, 1},  {0, 0, 1},
                                  {1, 0, 1},  {-1, 1, 1},   {0, 1, 1},   {1, 1, 1}};

// One warp moves its 32-bit accumulators into the 64-bit global sums and clears them.
__device__ __forceinline__ void warp_flush(unsigned *acc, int n, unsigned long long *out, int lane)
{
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
        const unsigned v = acc[k];
        if (v) {
            atomicAdd(out + k, (unsigned long long)v);
            acc[k] = 0u;
        }
    }
    __syncwarp();
}

template <bool kBackward>
__global__ void __launch_bounds__(kScThreads) smear_cells_kernel(SmearArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    int4 *s_true = reinterpret_cast<int4 *>(dyn);
    int *s_idx = reinterpret_cast<int *>(s_true + kScStage);
    int2 *s_queue = reinterpret_cast<int2 *>(s_idx + kScStage);
    float *s_gj = reinterpret_cast<float *>(s_queue + kScWarps * kScQueue);     // bwd [3][stage]
    float *s_gi = s_gj + 3 * kScStage;                                        // bwd [3][threads]
    unsigned *s_acc_all = reinterpret_cast<unsigned *>(s_gi + 3 * kScThreads);  // fwd [warps][pairs*bins]
    float *s_lam = reinterpret_cast<float *>(s_gi + 3 * kScThreads);           // bwd
    __shared__ BoxDev bx;
    __shared__ int cur_box;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int2 *q = s_queue + warp * kScQueue;
    unsigned *s_acc = s_acc_all + warp * A.max_pairs_bins;   // this warp's accumulators
    int wcount = 0;                                          // pairs added since its last flush
    const float sg = (float)A.sigma, inv_sg = 1.0f / sg;
    if (tid == 0) cur_box = -1;
    if (!kBackward)
        for (int k = tid; k < kScWarps * A.max_pairs_bins; k += kScThreads) s_acc_all[k] = 0u;
    __syncthreads();
    for (long long w = blockIdx.x; w < A.n_items; w += gridDim.x) {
        const GcItem it = A.items[w];
        __syncthreads();
        if (it.box != cur_box) {
            if (!kBackward && cur_box >= 0)
                for (int k = tid; k < kScWarps * A.max_pairs_bins; k += kScThreads) {
                    const unsigned v = s_acc_all[k];
                    if (v) {
                        atomicAdd(A.acc + bx.hist_off + k % A.max_pairs_bins, (unsigned long long)v);
                        s_acc_all[k] = 0u;
                    }
                }
            __syncthreads();
            if (tid == 0) {
                bx = A.boxes[it.box];
                cur_box = it.box;
            }
            __syncthreads();
            if (kBackward)
                for (int k = tid; k < bx.n_pairs * bx.n_bins; k += kScThreads) s_lam[k] = A.lambda[bx.hist_off + k];
            __syncthreads();
        }
        const int n = bx.gc_n, L = bx.L;
        const float S = 1.0f / sqrtf(bx.inv_s2);
        const float rc = ((float)bx.n_bins * (float)bx.dr_A + 5.0f * sg) * S * 1.0001f + 2.0f;
        const float rc2 = rc * rc;                       // grid units^2, a superset test
        const int hc = it.cell, hx = hc % n, hy = (hc / n) % n, hz = hc / (n * n);
        const int hs = A.cell_start[bx.gc0 + hc], nh = A.cell_count[bx.gc0 + hc];
        for (int i0 = 0; i0 < nh; i0 += kScThreads) {
            const int ip = i0 + tid < nh ? hs + i0 + tid : -1;
            const int4 pi = ip >= 0 ? A.coords[ip] : make_int4(0, 0, 0, 0);
            if (kBackward) s_gi[tid] = s_gi[kScThreads + tid] = s_gi[2 * kScThreads + tid] = 0.f;
            for (int t = 0; t < 14; ++t) {
                const int cx = (hx + c_sfwd[t][0] + n) % n, cy = (hy + c_sfwd[t][1] + n) % n,
                          cz = (hz + c_sfwd[t][2] + n) % n;
                const int c = bx.gc0 + (cz * n + cy) * n + cx;
                const int cs = A.cell_start[c], nc = A.cell_count[c];
                for (int j0 = 0; j0 < nc; j0 += kScStage) {
                    const int nj = min(kScStage, nc - j0);
                    __syncthreads();
                    for (int j = tid; j < nj; j += kScThreads) {
                        s_true[j] = A.coords[cs + j0 + j];
                        if (kBackward) {
                            s_idx[j] = A.index[cs + j0 + j];
                            s_gj[j] = s_gj[kScStage + j] = s_gj[2 * kScStage + j] = 0.f;
                        }
                    }
                    __syncthreads();
                    const int jstart = ip < 0 ? nj : (t == 0 ? max(0, ip + 1 - (cs + j0)) : 0);
                    int qn = 0;
                    for (int jb = 0; jb < nj; jb += 32) {
                        // lane-parallel over this warp's home atoms x 32 staged atoms, in-range pairs queued
                        for (int jj = 0; jj < 32 && jb + jj < nj; ++jj) {
                            const int j = jb + jj;
                            bool hit = false;
                            if (j >= jstart) {
                                const Sep sp = sep(pi, s_true[j], L);
                                hit = g2_of(sp) < rc2;
                            }
                            const unsigned bal = __ballot_sync(0xffffffffu, hit);
                            if (hit) q[qn + __popc(bal & ((1u << lane) - 1u))] = make_int2(tid, j);
                            qn += __popc(bal);
                            if (qn >= 32) {
                                __syncwarp();
                                const int2 e = q[qn - 32 + lane];
                                __syncwarp();
                                float fx, fy, fz;
                                const int src = e.x & 31;
                                const int4 pe = make_int4(__shfl_sync(0xffffffffu, pi.x, src), __shfl_sync(0xffffffffu, pi.y, src),
                                                          __shfl_sync(0xffffffffu, pi.z, src), __shfl_sync(0xffffffffu, pi.w, src));
                                const float f = smear_core<kBackward, false>(A, bx, pe, s_true[e.y], s_acc, s_lam, sg, inv_sg, S, fx, fy, fz);
                                if (kBackward && f != 0.f) {
                                    atomicAdd(&s_gi[e.x], f * fx);
                                    atomicAdd(&s_gi[kScThreads + e.x], f * fy);
                                    atomicAdd(&s_gi[2 * kScThreads + e.x], f * fz);
                                    atomicAdd(&s_gj[e.y], -f * fx);
                                    atomicAdd(&s_gj[kScStage + e.y], -f * fy);
                                    atomicAdd(&s_gj[2 * kScStage + e.y], -f * fz);
                                }
                                qn -= 32;
                                if (!kBackward && (wcount += 32) > 4000) {
                                    warp_flush(s_acc, bx.n_pairs * bx.n_bins, A.acc + bx.hist_off, lane);
                                    wcount = 0;
                                }
                            }
                        }
                    }
                    // the rest of the queue before the stage is overwritten
                    if (!kBackward && wcount + qn > 4000) {
                        warp_flush(s_acc, bx.n_pairs * bx.n_bins, A.acc + bx.hist_off, lane);
                        wcount = 0;
                    }
                    wcount += qn;
                    __syncwarp();
                    {
                        const int2 e = lane < qn ? q[lane] : make_int2(warp * 32, 0);
                        const int src = e.x & 31;
                        const int4 pe = make_int4(__shfl_sync(0xffffffffu, pi.x, src), __shfl_sync(0xffffffffu, pi.y, src),
                                                  __shfl_sync(0xffffffffu, pi.z, src), __shfl_sync(0xffffffffu, pi.w, src));
                        if (lane < qn) {
                            float fx, fy, fz;
                            const float f = smear_core<kBackward, false>(A, bx, pe, s_true[e.y], s_acc, s_lam, sg, inv_sg, S, fx, fy, fz);
                            if (kBackward && f != 0.f) {
                                atomicAdd(&s_gi[e.x], f * fx);
                                atomicAdd(&s_gi[kScThreads + e.x], f * fy);
                                atomicAdd(&s_gi[2 * kScThreads + e.x], f * fz);
                                atomicAdd(&s_gj[e.y], -f * fx);
                                atomicAdd(&s_gj[kScStage + e.y], -f * fy);
                                atomicAdd(&s_gj[2 * kScStage + e.y], -f * fz);
                            }
                        }
                    }
                    if (kBackward) {
                        __syncthreads();
                        for (int j = tid; j < nj; j += kScThreads) {
                            const int atom = s_idx[j];
                            for (int cc = 0; cc < 3; ++cc) {
                                const float v = s_gj[cc * kScStage + j];
                                if (v != 0.f) atomicAdd(&A.grad[3 * atom + cc], v);
                            }
                        }
                    }
                }
            }
            if (kBackward) {
                __syncthreads();
                if (ip >= 0) {
                    const int atom = A.index[ip];
                    for (int cc = 0; cc < 3; ++cc) {
                        const float v = s_gi[cc * kScThreads + tid];
                        if (v != 0.f) atomicAdd(&A.grad[3 * atom + cc], v);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (!kBackward && cur_box >= 0)
        for (int k = tid; k < kScWarps * A.max_pairs_bins; k += kScThreads) {
            const unsigned v = s_acc_all[k];
            if (v) atomicAdd(A.acc + bx.hist_off + k % A.max_pairs_bins, (unsigned long long)v);
        }
}

int launch_smear_cells(const SmearArgs &a, bool backward, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)kScStage * (sizeof(int4) + sizeof(int)) + (size_t)kScWarps * kScQueue * sizeof(int2) +
                        (size_t)3 * (kScStage + kScThreads) * sizeof(float) +
                        (size_t)a.max_pairs_bins * (backward ? sizeof(float) : kScWarps * sizeof(unsigned));
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(smear_cells_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(smear_cells_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(smear cells)");
        attr = true;
    }
    if (smem > 200 * 1024) return set_error(EPSR_EINVAL, "smeared g: n_pairs*n_bins too large");
    if (backward) smear_cells_kernel<true><<<grid, kScThreads, smem, stream>>>(a);
    else smear_cells_kernel<false><<<grid, kScThreads, smem, stream>>>(a);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "smear cells launch");
}

int launch_smear(const SmearArgs &a, bool backward, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)kGrTile * (sizeof(uint4) + sizeof(int4) + sizeof(int)) +
                        (size_t)kSmWarps * kSmQueue * sizeof(int2) +
                        (backward ? (size_t)a.max_pairs_bins * sizeof(float) + (size_t)6 * kGrTile * sizeof(float)
                                  : (size_t)a.max_pairs_bins * sizeof(unsigned));
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

// Ht = acc 2^-20 and (optionally) gt = Ht V / (P_ab shell_k), normalised like g
__global__ void smear_norm_kernel(const BoxDev *boxes, int n_boxes, const unsigned long long *acc,
                                  double *Ht, float *gt, long long hist_len, const long long *hist_box)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hist_len;
         i += (long long)gridDim.x * blockDim.x) {
        const double h = (double)acc[i] * 0x1p-20;
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
