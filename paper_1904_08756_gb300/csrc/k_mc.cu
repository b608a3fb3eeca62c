// k_mc.cu -- Metropolis Monte Carlo sweep (Sec. 2.2 item III) with the per-move energy
// change of the moved molecule against all atoms (Sec. 2.3), as one cooperative
// persistent kernel on sm_103a.
//
// Layout: every box of the handle owns a contiguous group of CTAs; each CTA keeps a
// slice of its box's atoms (the "partners") resident in shared memory for the whole
// sweep, so a move reads no partner data from HBM.
//
// Batching without changing the chain: moves are taken in batches of up to K
// consecutive moves with distinct molecules (a batch ends before the first molecule that
// repeats). Warp k computes the partial dU of move k against the slice as the slice
// stood at the start of the batch. One grid barrier per batch gathers the per-CTA
// partials; every CTA then sums them in the same fixed order and resolves the batch
// sequentially: move k's dU is its batch-start value plus, for every earlier accepted
// move k' of the batch, the exact change of the pair energies between the two moved
// molecules, u(new,new') - u(old,new') - u(new,old') + u(old,old'). This is the energy
// change against the state after moves 0..k-1, i.e. the sequential Metropolis chain.
//
// Every device-side wait is bounded by a time limit and an iteration limit; on expiry
// the kernel records EPSR_ETIMEOUT in a status word and all CTAs return.
#include <cooperative_groups.h>

#include "epsr_device.cuh"
#include "epsr_internal.h"

namespace epsr {

constexpr int kMcThreads = 512;
constexpr int kMcWarps = kMcThreads / 32;
constexpr int kBatchMax = kMcWarps;            // one move per warp

struct McShared {
    BoxDev bx;
    uint32_t words[kBatchMax][12];
    int mol[kBatchMax];
    int natoms[kBatchMax];
    int a0[kBatchMax];                          // first atom (box-local) of the molecule
    double thr[kBatchMax];                      // -kT ln(u_acc)
    double u_acc[kBatchMax];
    int4 oldp[kBatchMax][kMaxMolAtoms];
    int4 newp[kBatchMax][kMaxMolAtoms];
    float part[kBatchMax];
    float base[kBatchMax];
    float corr[kBatchMax][kBatchMax];
    float dU[kBatchMax];
    int acc[kBatchMax];
    int n_batch;
    int abort_flag;
    // moves accepted in the previous batch (their global writes may not be visible yet)
    int pend_n;
    int pend_mol[kBatchMax];
    int pend_natoms[kBatchMax];
    int4 pend_new[kBatchMax][kMaxMolAtoms];
    // leader-only running statistics
    long long st_att, st_acc, st_nonfinite;
    double st_sum;
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kMcThreads, 1) mc_sweep_kernel(McArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ McShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cta = blockIdx.x;
    const int box = A.cta_box[cta];

    if (tid == 0) {
        sh.bx = A.boxes[box];
        sh.pend_n = 0;
        sh.abort_flag = 0;
        sh.st_att = sh.st_acc = sh.st_nonfinite = 0;
        sh.st_sum = 0.0;
    }
    __syncthreads();
    const BoxDev &bx = sh.bx;
    const int G = bx.n_cta;
    const int rank = cta - bx.cta0;
    const int L = bx.L;
    const int j_begin = min(bx.n_atoms, rank * bx.chunk);
    const int j_end = min(bx.n_atoms, j_begin + bx.chunk);
    const int n_slice = j_end - j_begin;

    // shared memory: partner slice, thresholds, empirical potential
    int4 *slice = reinterpret_cast<int4 *>(dyn);
    long long *T = reinterpret_cast<long long *>(slice + A.slice_cap);
    float *ep = reinterpret_cast<float *>(T + A.tbl_cap);
    for (int j = tid; j < n_slice; j += kMcThreads) slice[j] = A.coords[bx.atom0 + j_begin + j];
    for (int k = tid; k <= bx.n_bins; k += kMcThreads) T[k] = A.thresholds[bx.tbl_off + k];
    if (bx.has_ep)
        for (int k = tid; k < bx.n_pairs * bx.n_bins; k += kMcThreads) ep[k] = A.ep[bx.ep_off + k];
    __syncthreads();

    const int *mol_start = A.mol_start + bx.mol0;
    const uint32_t key0 = (uint32_t)A.seed, key1 = (uint32_t)(A.seed >> 32);
    unsigned seq = 0;

    for (long long t0 = 0; t0 < A.n_moves;) {
        const int kmax = (int)min((long long)A.batch_k, A.n_moves - t0);
        // ---- 1. random words and molecule of each move of the batch ----------------------
        if (warp < kmax) {
            const unsigned long long mv = A.move0 + (unsigned long long)(t0 + warp);
            if (lane < 3) {
                U32x4 w = philox4x32_10((uint32_t)mv, (uint32_t)(mv >> 32), (uint32_t)box,
                                        (uint32_t)lane, key0, key1);
                for (int i = 0; i < 4; ++i) sh.words[warp][4 * lane + i] = w.v[i];
            }
            __syncwarp();
            if (lane == 0)
                sh.mol[warp] = (int)(((unsigned long long)sh.words[warp][0] *
                                      (unsigned long long)bx.n_mol) >> 32);
        }
        __syncthreads();
        // ---- 2. the batch ends before the first repeated molecule ---------------------------
        if (tid == 0) {
            int n = kmax;
            for (int k = 1; k < kmax && n == kmax; ++k)
                for (int k2 = 0; k2 < k; ++k2)
                    if (sh.mol[k2] == sh.mol[k]) { n = k; break; }
            sh.n_batch = n;
        }
        __syncthreads();
        const int nb = sh.n_batch;
        // ---- 3. current and trial coordinates of each moved molecule -------------------------
        if (warp < nb) {
            const int mol = sh.mol[warp];
            const int a0 = mol_start[mol], m = mol_start[mol + 1] - a0;
            int pidx = -1;
            for (int p = 0; p < sh.pend_n; ++p)
                if (sh.pend_mol[p] == mol) pidx = p;
            if (lane < m) {
                int4 c;
                if (pidx >= 0) c = sh.pend_new[pidx][lane];
                else c = __ldcg(&A.coords[bx.atom0 + a0 + lane]);
                sh.oldp[warp][lane] = c;
            }
            __syncwarp();
            if (lane == 0) {
                const uint32_t *w = sh.words[warp];
                int shift[3];
                const unsigned span = 2u * (unsigned)bx.max_shift + 1u;
                for (int a = 0; a < 3; ++a) shift[a] = (int)(w[1 + a] % span) - bx.max_shift;
                if (bx.move_kind == EPSR_MOVE_RIGID_MOLECULE) {
                    const double vx = __dmul_rn(bx.h_rot, __dsub_rn(__dmul_rn(2.0, uniform53(w[4], w[5])), 1.0));
                    const double vy = __dmul_rn(bx.h_rot, __dsub_rn(__dmul_rn(2.0, uniform53(w[6], w[7])), 1.0));
                    const double vz = __dmul_rn(bx.h_rot, __dsub_rn(__dmul_rn(2.0, uniform53(w[8], w[9])), 1.0));
                    rigid_trial(sh.oldp[warp], m, vx, vy, vz, shift, L, sh.newp[warp]);
                } else {
                    for (int k = 0; k < m; ++k) {
                        const int4 o = sh.oldp[warp][k];
                        sh.newp[warp][k] = make_int4(wrap_coord((long long)o.x + shift[0], L),
                                                     wrap_coord((long long)o.y + shift[1], L),
                                                     wrap_coord((long long)o.z + shift[2], L), o.w);
                    }
                }
                const double u = uniform53(w[10], w[11]);
                sh.u_acc[warp] = u;
                sh.thr[warp] = -bx.kT * log(u);      // accept iff dU < -kT ln u  (u < e^{-dU/kT})
                sh.natoms[warp] = m;
                sh.a0[warp] = a0;
            }
        }
        __syncthreads();
        // ---- 4. partial dU of move `warp` against this CTA's slice ---------------------------
        if (warp < nb) {
            const int m = sh.natoms[warp];
            const int a0 = sh.a0[warp];
            float acc = 0.f;
            for (int j = lane; j < n_slice; j += 32) {
                const int jg = j_begin + j;
                if (jg >= a0 && jg < a0 + m) continue;
                const int4 pj = slice[j];
                for (int a = 0; a < m; ++a) {
                    const int4 pn = sh.newp[warp][a], po = sh.oldp[warp][a];
                    const PairRow pr = bx.row[pn.w * kMaxTypes + pj.w];
                    acc += pair_du(dist2(pn, pj, L), dist2(po, pj, L), pr, bx, T, ep);
                }
            }
            acc = warp_sum(acc);
            if (lane == 0) sh.part[warp] = acc;
        }
        __syncthreads();
        // ---- 5. gather the partials of the box's CTA group (one bounded grid barrier) -------
        ++seq;
        if (G > 1) {
            float *slot = A.slots + ((size_t)(seq & 1u) * A.grid + cta) * kBatchMax;
            if (tid == 0 && cta != A.skip_arrival_cta) {
                for (int k = 0; k < nb; ++k) slot[k] = sh.part[k];
                st_release_gpu(&A.flags[cta], seq);
            }
            if (warp == 0) {
                const uint64_t t_start = globaltimer_ns();
                long long it = 0;
                bool timed_out = false;
                for (;;) {
                    bool ready = true;
                    for (int r = lane; r < G; r += 32)
                        ready &= ld_acquire_gpu(&A.flags[bx.cta0 + r]) >= seq;
                    if (__all_sync(0xffffffffu, ready)) break;
                    if ((++it & 63) == 0) {
                        const bool stop = (globaltimer_ns() - t_start > A.timeout_ns) ||
                                          it > A.max_spin || ld_relaxed_gpu(A.status) != 0;
                        if (__any_sync(0xffffffffu, stop)) { timed_out = true; break; }
                    }
                }
                if (timed_out && lane == 0) {
                    atomicOr(A.status, kStatusTimeout);
                    sh.abort_flag = 1;
                }
            }
            __syncthreads();
            if (sh.abort_flag) return;
            if (warp < nb) {
                const float *base = A.slots + (size_t)(seq & 1u) * A.grid * kBatchMax;
                float v = 0.f;
                for (int r = lane; r < G; r += 32) v += __ldcg(&base[(size_t)(bx.cta0 + r) * kBatchMax + warp]);
                v = warp_sum(v);
                if (lane == 0) sh.base[warp] = v;
            }
        } else if (tid < nb) {
            sh.base[tid] = sh.part[tid];
        }
        // ---- 6. pair-energy corrections between the batch's moved molecules ------------------
        for (int pq = tid; pq < nb * nb; pq += kMcThreads) {
            const int k1 = pq / nb, k = pq % nb;       // k1 < k: earlier move k1 affects k
            if (k1 >= k) continue;
            float c = 0.f;
            for (int a = 0; a < sh.natoms[k]; ++a)
                for (int b = 0; b < sh.natoms[k1]; ++b) {
                    const int4 na = sh.newp[k][a], oa = sh.oldp[k][a];
                    const int4 nb_ = sh.newp[k1][b], ob = sh.oldp[k1][b];
                    const PairRow pr = bx.row[na.w * kMaxTypes + nb_.w];
                    c += pair_du(dist2(na, nb_, L), dist2(oa, nb_, L), pr, bx, T, ep) -
                         pair_du(dist2(na, ob, L), dist2(oa, ob, L), pr, bx, T, ep);
                }
            sh.corr[k1][k] = c;
        }
        __syncthreads();
        // ---- 7. sequential Metropolis decisions of the batch ----------------------------------
        if (tid == 0) {
            for (int k = 0; k < nb; ++k) {
                float d = sh.base[k];
                for (int k1 = 0; k1 < k; ++k1)
                    if (sh.acc[k1]) d += sh.corr[k1][k];
                sh.dU[k] = d;
                const double dd = (double)d;
                sh.acc[k] = (dd <= 0.0) || (dd < sh.thr[k]);
            }
        }
        __syncthreads();
        // ---- 8. apply accepted moves: shared slice, global coordinates, log, statistics ------
        for (int k = 0; k < nb; ++k) {
            if (!sh.acc[k]) continue;
            const int a0 = sh.a0[k], m = sh.natoms[k];
            if (tid < m) {
                const int ja = a0 + tid;
                if (ja >= j_begin && ja < j_end) slice[ja - j_begin] = sh.newp[k][tid];
                if (rank == 0) A.coords[bx.atom0 + ja] = sh.newp[k][tid];
            }
        }
        if (rank == 0) {
            if (A.log && tid < nb) {
                epsr_move_log *lg = A.log + (size_t)box * A.log_stride + (size_t)(t0 + tid);
                lg->mol = sh.mol[tid];
                lg->accepted = sh.acc[tid];
                lg->dU = sh.dU[tid];
                lg->n_atoms = sh.natoms[tid];
                lg->u_acc = sh.u_acc[tid];
                for (int a = 0; a < kMaxMolAtoms; ++a) {
                    const int4 p = a < sh.natoms[tid] ? sh.newp[tid][a] : make_int4(0, 0, 0, 0);
                    lg->trial[a][0] = p.x; lg->trial[a][1] = p.y; lg->trial[a][2] = p.z;
                }
            }
            if (tid == 0) {
                for (int k = 0; k < nb; ++k) {
                    sh.st_att += 1;
                    const float d = sh.dU[k];
                    if (!isfinite(d)) sh.st_nonfinite += 1;
                    if (sh.acc[k]) { sh.st_acc += 1; sh.st_sum += (double)d; }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int n = 0;
            for (int k = 0; k < nb; ++k)
                if (sh.acc[k]) {
                    sh.pend_mol[n] = sh.mol[k];
                    sh.pend_natoms[n] = sh.natoms[k];
                    for (int a = 0; a < sh.natoms[k]; ++a) sh.pend_new[n][a] = sh.newp[k][a];
                    ++n;
                }
            sh.pend_n = n;
        }
        __syncthreads();
        t0 += nb;
    }
    if (rank == 0 && tid == 0) {
        epsr_mc_stats *st = A.stats + box;
        st->attempted += sh.st_att;
        st->accepted += sh.st_acc;
        st->nonfinite += sh.st_nonfinite;
        st->sum_dU += sh.st_sum;
    }
}

int launch_mc_sweep(const McArgs &args, int grid, size_t smem, cudaStream_t stream)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(mc_sweep_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMcMaxDynSmem);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(mc)");
        attr_set = true;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mc_sweep_kernel,
                                                                  kMcThreads, smem);
    if (e != cudaSuccess) return set_cuda_error(e, "occupancy(mc)");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm * sms < grid)
        return set_error(EPSR_ELAUNCH, "mc sweep: %d CTAs cannot be co-resident (%d per SM x %d SMs)",
                         grid, per_sm, sms);
    McArgs a = args;
    void *params[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)mc_sweep_kernel, dim3(grid), dim3(kMcThreads),
                                    params, smem, stream);
    if (e == cudaErrorCooperativeLaunchTooLarge)
        return set_error(EPSR_ELAUNCH, "mc sweep: cooperative launch of %d CTAs refused", grid);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaLaunchCooperativeKernel(mc)");
    return EPSR_OK;
}

int mc_threads() { return kMcThreads; }
int mc_batch_max() { return kBatchMax; }

}  // namespace epsr
