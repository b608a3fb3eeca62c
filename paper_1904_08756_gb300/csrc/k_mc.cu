// k_mc.cu -- Metropolis Monte Carlo sweep (Sec. 2.2 item III) with the per-move energy
// change of the moved molecule against all atoms (Sec. 2.3), on sm_103a.
//
// Two kernels per chunk of moves:
//  1. mc_moves_kernel, one thread per (box, move): everything about a move that does not
//     depend on the configuration -- the Philox words, the molecule, the shift, the
//     rotation matrix (FP64, rounded to 2^-30 fixed point) and the Metropolis threshold
//     -kT ln u (rounded up to FP32, which makes `dU < threshold` in FP32 the same test
//     as in FP64). GB300's FP64 unit is narrow, so this runs once per move on the whole
//     GPU instead of once per move in every CTA.
//  2. mc_sweep_kernel, a cooperative persistent kernel: every box of the handle owns a
//     contiguous group of CTAs; each CTA keeps a slice of its box's atoms (the partners)
//     resident in shared memory for the whole sweep.
//
// Batching without changing the chain: moves are taken in batches of up to K
// consecutive moves with distinct molecules (a batch ends before the first molecule that
// repeats). Warp k computes the partial dU of move k against the slice as it stood at
// the start of the batch. One grid barrier per batch gathers the per-CTA partials; every
// CTA sums them in the same fixed order and resolves the batch in order: move k's dU is
// its batch-start value plus, for every earlier accepted move k' of the batch, the exact
// change of the pair energies between the two moved molecules,
// u(new,new') - u(old,new') - u(new,old') + u(old,old'). That is the energy change
// against the state after moves 0..k-1, i.e. the sequential Metropolis chain.
//
// Every device-side wait is bounded by a time limit and an iteration limit; on expiry
// the kernel records a timeout in the status word and all CTAs return.
#include "epsr_device.cuh"
#include "epsr_internal.h"

namespace epsr {

constexpr int kMcThreads = 512;
constexpr int kMcWarps = kMcThreads / 32;
constexpr int kBatchMax = kMcWarps;            // one move per warp

// ---- 1. configuration-independent part of each move ----------------------------------------
__global__ void mc_moves_kernel(const BoxDev *boxes, int n_boxes, long long chunk, long long n,
                                unsigned long long seed, unsigned long long move0, MoveRec *out)
{
    const long long total = (long long)n_boxes * chunk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / chunk);
        const long long t = e % chunk;
        if (t >= n) continue;
        const BoxDev &bx = boxes[b];
        const unsigned long long mv = move0 + (unsigned long long)t;
        uint32_t w[12];
#pragma unroll
        for (int lane = 0; lane < 3; ++lane) {
            const U32x4 r = philox4x32_10((uint32_t)mv, (uint32_t)(mv >> 32), (uint32_t)b,
                                          (uint32_t)lane, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
            for (int i = 0; i < 4; ++i) w[4 * lane + i] = r.v[i];
        }
        MoveRec m;
        m.mol = (int)(((unsigned long long)w[0] * (unsigned long long)bx.n_mol) >> 32);
        const unsigned span = 2u * (unsigned)bx.max_shift + 1u;
        for (int a = 0; a < 3; ++a) m.shift[a] = (int)(w[1 + a] % span) - bx.max_shift;
        if (bx.move_kind == EPSR_MOVE_RIGID_MOLECULE) {
            const double vx = __dmul_rn(bx.h_rot, __dsub_rn(__dmul_rn(2.0, uniform53(w[4], w[5])), 1.0));
            const double vy = __dmul_rn(bx.h_rot, __dsub_rn(__dmul_rn(2.0, uniform53(w[6], w[7])), 1.0));
            const double vz = __dmul_rn(bx.h_rot, __dsub_rn(__dmul_rn(2.0, uniform53(w[8], w[9])), 1.0));
            rotation_fixed(vx, vy, vz, m.R);
        } else {
            for (int i = 0; i < 9; ++i) m.R[i] = 0;
        }
        const double u = uniform53(w[10], w[11]);
        m.u_acc = u;
        // accept iff dU <= 0 or dU < -kT ln u; a float rounded up from the FP64 threshold
        // gives the identical comparison for FP32 dU
        m.thr = __double2float_ru(-bx.kT * log(u));
        out[e] = m;
    }
}

int launch_mc_moves(const BoxDev *boxes, int n_boxes, long long chunk, long long n,
                    unsigned long long seed, unsigned long long move0, MoveRec *out,
                    cudaStream_t stream)
{
    const long long total = (long long)n_boxes * chunk;
    const int grid = (int)((total + 127) / 128 < 8192 ? (total + 127) / 128 : 8192);
    mc_moves_kernel<<<grid, 128, 0, stream>>>(boxes, n_boxes, chunk, n, seed, move0, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "mc_moves");
}

// ---- 2. persistent sweep ----------------------------------------------------------------------
struct McShared {
    BoxDev bx;
    // batch records, double buffered by batch parity: the previous batch's accepted moves
    // are the "pending" updates whose global writes may not yet be visible
    int nb[2];
    int mol[2][kBatchMax];
    int acc[2][kBatchMax];
    int4 newp[2][kBatchMax][kMaxMolAtoms];
    // current batch
    int4 oldp[kBatchMax][kMaxMolAtoms];
    int natoms[kBatchMax];
    int a0[kBatchMax];
    float thr[kBatchMax];
    double u_acc[kBatchMax];
    float part[kBatchMax];
    float base[kBatchMax];
    float corr_part[kBatchMax][kBatchMax][kMaxMolAtoms];
    float corr[kBatchMax][kBatchMax];
    float dU[kBatchMax];
    int abort_flag;
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

__device__ __forceinline__ int floordiv32(int a, int b)   // b > 0
{
    int q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
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
        sh.nb[0] = sh.nb[1] = 0;
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
    const bool rigid = bx.move_kind == EPSR_MOVE_RIGID_MOLECULE;

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
    const MoveRec *moves = A.moves + (size_t)box * A.chunk;
    unsigned seq = 0;
    int par = 0;

    for (long long t0 = 0; t0 < A.n_moves; par ^= 1) {
        const int kmax = (int)min((long long)A.batch_k, A.n_moves - t0);
        // ---- A. molecules of the batch; it ends before the first repeated molecule -----------
        if (warp == 0) {
            const int my = lane < kmax ? moves[t0 + lane].mol : -1 - lane;
            bool dup = false;
#pragma unroll
            for (int k1 = 0; k1 < kBatchMax; ++k1) {
                const int o = __shfl_sync(0xffffffffu, my, k1);
                dup |= (k1 < lane) && (o == my);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, dup && lane < kmax);
            if (lane == 0) sh.nb[par] = bal ? __ffs(bal) - 1 : kmax;
            if (lane < kBatchMax) sh.mol[par][lane] = my;
        }
        __syncthreads();
        const int nb = sh.nb[par];
        // ---- B. current and trial coordinates of each moved molecule (integer arithmetic) ----
        if (warp < nb) {
            const int k = warp;
            const MoveRec &mr = moves[t0 + k];
            const int mol = sh.mol[par][k];
            const int a0 = mol_start[mol], m = mol_start[mol + 1] - a0;
            const int q = par ^ 1;
            int pidx = -1;
            for (int p = 0; p < sh.nb[q]; ++p)
                if (sh.acc[q][p] && sh.mol[q][p] == mol) pidx = p;
            if (lane < m)
                sh.oldp[k][lane] = pidx >= 0 ? sh.newp[q][pidx][lane]
                                             : __ldcg(&A.coords[bx.atom0 + a0 + lane]);
            __syncwarp();
            if (lane < 3 * m) {
                const int kk = lane / 3, a = lane - 3 * kk;
                const int4 *op = sh.oldp[k];
                int coord;
                if (rigid) {
                    const int base[3] = {op[0].x, op[0].y, op[0].z};
                    long long sum[3] = {0, 0, 0}, mine[3] = {0, 0, 0};
                    for (int i = 0; i < m; ++i) {
                        const int c[3] = {op[i].x, op[i].y, op[i].z};
                        for (int b = 0; b < 3; ++b) {
                            const long long o = mi_signed((long long)c[b] - base[b], L);
                            sum[b] += o;
                            if (i == kk) mine[b] = o;
                        }
                    }
                    long long num = sum[a] * 1073741824LL;
                    for (int b = 0; b < 3; ++b) num += (long long)mr.R[3 * a + b] * ((long long)m * mine[b] - sum[b]);
                    // floor((num + m 2^29) / 2^30) fits in 32 bits; then floor division by m
                    const int hi = (int)((num + (long long)m * 536870912LL) >> 30);
                    coord = wrap_coord((long long)base[a] + floordiv32(hi, m) + mr.shift[a], L);
                } else {
                    const int c[3] = {op[kk].x, op[kk].y, op[kk].z};
                    coord = wrap_coord((long long)c[a] + mr.shift[a], L);
                }
                int *dst = reinterpret_cast<int *>(&sh.newp[par][k][kk]);
                dst[a] = coord;
                if (a == 0) dst[3] = op[kk].w;
            }
            if (lane == 0) {
                sh.natoms[k] = m;
                sh.a0[k] = a0;
                sh.thr[k] = mr.thr;
                sh.u_acc[k] = mr.u_acc;
            }
        }
        __syncthreads();
        // ---- C. partial dU of move `warp` against this CTA's slice ---------------------------
        if (warp < nb) {
            const int m = sh.natoms[warp];
            const int a0 = sh.a0[warp];
            const int4 *np = sh.newp[par][warp];
            const int4 *op = sh.oldp[warp];
            float acc = 0.f;
            for (int j = lane; j < n_slice; j += 32) {
                const int jg = j_begin + j;
                if (jg >= a0 && jg < a0 + m) continue;
                const int4 pj = slice[j];
                for (int a = 0; a < m; ++a) {
                    const int4 pn = np[a], po = op[a];
                    const PairRow pr = bx.row[pn.w * kMaxTypes + pj.w];
                    acc += pair_du(sep(pn, pj, L), sep(po, pj, L), pr, bx, T, ep);
                }
            }
            acc = warp_sum(acc);
            if (lane == 0) sh.part[warp] = acc;
        }
        __syncthreads();
        // ---- D. gather the partials of the box's CTA group (one bounded grid barrier) -------
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
                const float *bs = A.slots + (size_t)(seq & 1u) * A.grid * kBatchMax;
                float v = 0.f;
                for (int r = lane; r < G; r += 32) v += __ldcg(&bs[(size_t)(bx.cta0 + r) * kBatchMax + warp]);
                v = warp_sum(v);
                if (lane == 0) sh.base[warp] = v;
            }
        } else if (tid < nb) {
            sh.base[tid] = sh.part[tid];
        }
        // ---- E. pair-energy corrections between the batch's moved molecules -----------------
        // item (k1, k, a): atom a of move k against the whole molecule of an earlier move k1
        for (int it = tid; it < nb * nb * kMaxMolAtoms; it += kMcThreads) {
            const int a = it % kMaxMolAtoms, pq = it / kMaxMolAtoms;
            const int k1 = pq / nb, k = pq % nb;
            if (k1 >= k || a >= sh.natoms[k]) continue;
            const int4 na = sh.newp[par][k][a], oa = sh.oldp[k][a];
            float c = 0.f;
            for (int b = 0; b < sh.natoms[k1]; ++b) {
                const int4 nb1 = sh.newp[par][k1][b], ob1 = sh.oldp[k1][b];
                const PairRow pr = bx.row[na.w * kMaxTypes + nb1.w];
                c += pair_du(sep(na, nb1, L), sep(oa, nb1, L), pr, bx, T, ep) -
                     pair_du(sep(na, ob1, L), sep(oa, ob1, L), pr, bx, T, ep);
            }
            sh.corr_part[k1][k][a] = c;
        }
        __syncthreads();
        for (int pq = tid; pq < nb * nb; pq += kMcThreads) {
            const int k1 = pq / nb, k = pq % nb;
            if (k1 >= k) continue;
            float c = 0.f;
            for (int a = 0; a < sh.natoms[k]; ++a) c += sh.corr_part[k1][k][a];
            sh.corr[k1][k] = c;
        }
        __syncthreads();
        // ---- F. Metropolis decisions of the batch, in order (warp 0, lane k = move k) -------
        if (warp == 0) {
            float d = lane < nb ? sh.base[lane] : 0.f;
            const float thr = lane < nb ? sh.thr[lane] : 0.f;
            int accepted = 0;
            for (int j = 0; j < nb; ++j) {
                const int aj = __shfl_sync(0xffffffffu, (d <= 0.f) || (d < thr), j);
                if (lane == j) accepted = aj;
                if (lane > j && lane < nb && aj) d += sh.corr[j][lane];
            }
            if (lane < nb) {
                sh.dU[lane] = d;
                sh.acc[par][lane] = accepted;
            }
            if (rank == 0) {
                const unsigned in = lane < nb ? 1u : 0u;
                const unsigned b_acc = __ballot_sync(0xffffffffu, in && accepted);
                const unsigned b_nf = __ballot_sync(0xffffffffu, in && !isfinite(d));
                double v = (in && accepted) ? (double)d : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) {
                    sh.st_att += nb;
                    sh.st_acc += __popc(b_acc);
                    sh.st_nonfinite += __popc(b_nf);
                    sh.st_sum += v;
                }
            }
        }
        __syncthreads();
        // ---- G. apply accepted moves: shared slice, global coordinates, log ------------------
        for (int it = tid; it < nb * kMaxMolAtoms; it += kMcThreads) {
            const int k = it / kMaxMolAtoms, a = it % kMaxMolAtoms;
            if (!sh.acc[par][k] || a >= sh.natoms[k]) continue;
            const int ja = sh.a0[k] + a;
            const int4 p = sh.newp[par][k][a];
            if (ja >= j_begin && ja < j_end) slice[ja - j_begin] = p;
            if (rank == 0) A.coords[bx.atom0 + ja] = p;
        }
        if (rank == 0 && A.log && tid < nb) {
            epsr_move_log *lg = A.log + (size_t)box * A.log_stride + (size_t)(A.log_off + t0 + tid);
            lg->mol = sh.mol[par][tid];
            lg->accepted = sh.acc[par][tid];
            lg->dU = sh.dU[tid];
            lg->n_atoms = sh.natoms[tid];
            lg->u_acc = sh.u_acc[tid];
            for (int a = 0; a < kMaxMolAtoms; ++a) {
                const int4 p = a < sh.natoms[tid] ? sh.newp[par][tid][a] : make_int4(0, 0, 0, 0);
                lg->trial[a][0] = p.x; lg->trial[a][1] = p.y; lg->trial[a][2] = p.z;
            }
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
