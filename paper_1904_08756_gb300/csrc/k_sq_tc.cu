// k_sq_tc.cu -- S(Q) by Eq. (1) on the 5th-generation tensor cores (tcgen05) with split
// precision: S_partial[c][i] = w_c sum_k K[i][k] B[c][k], B = g - 1, as D = A B^T with
// A = K [nQ x n_bins] and B [n_cols x n_bins], both K-major.
//
// Each operand is split into pieces x = x_0 + x_1 (+ x_2), x_0 = round(x) in the narrow
// type and x_1 = round(x - x_0), and the products x_i y_j with i + j below the split order
// are accumulated into one FP32 accumulator in tensor memory:
//   BF16X3: 2 x 2 pieces, products (0,0) (0,1) (1,0)      ~2^-16 relative per term
//   BF16X6: 3 x 3 pieces, products with i + j <= 2        ~2^-24
//   TF32X3: 2 x 2 pieces (TF32), products (0,0) (0,1) (1,0)  ~2^-22
//
// Layout: the sine matrix is pre-packed once per plan in the tensor core's canonical K-major
// layout without swizzle -- core matrices of 8 rows x 16 bytes, K-adjacent core matrices
// 128 bytes apart (leading byte offset), 8-row groups ku * esize / 16 * 128 bytes apart
// (stride byte offset) -- one contiguous block per (M tile, K unit of 128 bytes per row,
// piece), so one 1-D bulk copy (cp.async.bulk, completion counted on an mbarrier) stages a
// unit's pieces. The columns B = g - 1 are split and packed by the CTA's threads straight
// from g (no separate packing launch).
//
// Work split: grid (M tiles of 128 Q, column chunks of n_chunk, K split) with the k_split CTAs
// of one output tile launched as one thread-block cluster. Each CTA runs its range of K units
// through a two-slot pipeline (the bulk copy and the B packing of unit j+1 overlap the MMAs of
// unit j), then moves its FP32 partial accumulator from tensor memory into shared memory;
// after a cluster barrier, CTA r of the cluster sums the partials of every CTA of the cluster
// over distributed shared memory, in cluster-rank order (deterministic), for the column sets
// r, r + k_split, ..., applies w_c, writes S_partial and, when a chunk holds whole sets, the
// set totals flat + sum_c S_partial[c] (one launch for the whole contraction).
#include <cuda_bf16.h>

#include "epsr_device.cuh"
#include "epsr_internal.h"
#include "k_sq.h"

namespace epsr {

namespace {

constexpr int kTcThreads = 256;     // 8 warps: warps w and w + 4 share TMEM lane quarter w
constexpr int kTcM = 128;
constexpr unsigned long long kTcSpinLimit = 1ull << 26;
constexpr size_t kTcSmemMax = 220 * 1024;        // dynamic shared memory of one CTA, at most
constexpr size_t kTcSmemTwoPerSm = 110 * 1024;   // budget that leaves room for two CTAs per SM

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: no swizzle, K-major (version 1 for this architecture).
__device__ __forceinline__ unsigned long long make_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;                       // descriptor version
    return d;                              // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: D in FP32, A and B of format `fmt` (BF16 = 1, TF32 = 2), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned make_idesc(unsigned fmt, unsigned M, unsigned N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                         unsigned idesc, unsigned acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Split value x into `np` pieces of the narrow type (pieces returned as raw bits).
__device__ __forceinline__ void split_bf16(float x, int np, unsigned short *out)
{
    float r = x;
    for (int i = 0; i < np; ++i) {
        const __nv_bfloat16 h = __float2bfloat16_rn(r);
        out[i] = __bfloat16_as_ushort(h);
        r = r - __bfloat162float(h);
    }
}

__device__ __forceinline__ unsigned tf32_round(float x)
{
    // round to nearest (ties away) on the 10-bit mantissa; the low 13 bits are cleared
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

__device__ __forceinline__ void split_tf32(float x, int np, unsigned *out)
{
    float r = x;
    for (int i = 0; i < np; ++i) {
        const unsigned h = tf32_round(r);
        out[i] = h;
        r = r - __uint_as_float(h);
    }
}

}  // namespace

// Byte offset of element (row, k) inside one packed stage block of `rows` rows.
__host__ __device__ __forceinline__ size_t tc_elem_offset(int row, int kin, int esize, int kt)
{
    const int hk = kt * esize / 16;                 // 16-byte k-groups per row
    const int g = row >> 3, r = row & 7;
    const int h = kin * esize / 16, e = (kin * esize % 16) / esize;
    return ((size_t)(g * hk + h) * 128 + r * 16 + e * esize);
}

// Pack the split sine matrix A = K[Q][k] at plan creation:
// blocks [m_tile][stage][piece] of kTcM x kt elements.
__global__ void tc_pack_a_kernel(const float *Kt_, int nQ, int n_bins, int m_tiles, int stages, int kt,
                                 int np, int fmt_bf16, unsigned char *out)
{
    const int esize = fmt_bf16 ? 2 : 4;
    const size_t piece_bytes = (size_t)kTcM * kt * esize;
    const long long total = (long long)m_tiles * kTcM * stages * kt;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % ((long long)stages * kt));
        const int q = (int)(e / ((long long)stages * kt));
        const int mt = q / kTcM, row = q % kTcM, s = k / kt, kin = k % kt;
        const float v = (q < nQ && k < n_bins) ? Kt_[(long long)k * nQ + q] : 0.f;
        unsigned char *blk = out + ((size_t)mt * stages + s) * np * piece_bytes;
        const size_t off = tc_elem_offset(row, kin, esize, kt);
        if (fmt_bf16) {
            unsigned short p[3];
            split_bf16(v, np, p);
            for (int i = 0; i < np; ++i) *reinterpret_cast<unsigned short *>(blk + i * piece_bytes + off) = p[i];
        } else {
            unsigned p[3];
            split_tf32(v, np, p);
            for (int i = 0; i < np; ++i) *reinterpret_cast<unsigned *>(blk + i * piece_bytes + off) = p[i];
        }
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned addr, unsigned parity)
{
    for (unsigned long long spins = 0; !mbar_try_wait(addr, parity);)
        if (++spins > kTcSpinLimit) return false;
    return true;
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory address of the same variable in CTA `rank` of this cluster.
__device__ __forceinline__ unsigned map_rank(unsigned addr, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ float ld_cluster_f32(unsigned addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ int ld_cluster_s32(unsigned addr)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__host__ __device__ __forceinline__ size_t tc_a_unit_bytes(int np)
{
    return (size_t)np * kTcM * 128;                     // 128 bytes of K per row and piece
}

__host__ __device__ __forceinline__ size_t tc_b_unit_bytes(int n_chunk, int np)
{
    return (size_t)np * n_chunk * 128;
}

// Dynamic shared memory of one CTA: `slots` (A, B) unit buffers; the FP32 partial
// accumulator [n_chunk][128] reuses the A buffers once the MMAs are done.
// Columns of a chunk owned by cluster rank r for the reduction: the chunk's column groups
// (sets, or single columns) split into k_split contiguous ranges.
__host__ __device__ __forceinline__ void tc_owned_cols(int ncol, int grp, int k_split, int r, int *c_lo, int *c_hi)
{
    const int ng = (ncol + grp - 1) / grp;
    const int g_lo = (int)((long long)ng * r / k_split), g_hi = (int)((long long)ng * (r + 1) / k_split);
    *c_lo = g_lo * grp;
    *c_hi = min(ncol, g_hi * grp);
}

int tc_recv_cols(int n_chunk, int grp, int k_split)
{
    const int ng = (n_chunk + grp - 1) / grp;
    return (ng + k_split - 1) / k_split * grp;
}

// Dynamic shared memory of one CTA: `slots` (A, B) unit buffers; once the MMAs are done the A
// buffers hold this CTA's FP32 partial [n_chunk][128] and the B buffers the partials the other
// CTAs of the cluster push for the columns this CTA owns ([k_split][recv_cols][128]).
size_t tc_smem_need(int n_chunk, int np, int slots, int k_split, int grp)
{
    const size_t a = (size_t)slots * tc_a_unit_bytes(np);
    const size_t red = (size_t)n_chunk * kTcM * sizeof(float);
    const size_t b = (size_t)slots * tc_b_unit_bytes(n_chunk, np);
    const size_t recv = k_split > 1 ? (size_t)k_split * tc_recv_cols(n_chunk, grp, k_split) * kTcM * sizeof(float) : 0;
    return (a > red ? a : red) + (b > recv ? b : recv);
}

size_t tc_smem_bytes(int n_chunk, int np, int k_split, int grp)
{
    const size_t total = tc_smem_need(n_chunk, np, 2, k_split, grp);
    return total <= kTcSmemMax ? total : 0;
}

int tc_slots_for(int n_chunk, int np, int units_per_cta, int k_split, int grp, bool one_per_sm)
{
    // as many unit buffers as the CTA has units, within a budget that leaves room for two CTAs
    // per SM (unless the grid has at most one CTA per SM), at least two
    const size_t budget = one_per_sm ? kTcSmemMax : kTcSmemTwoPerSm;
    int s = 2;
    while (s < units_per_cta && s < kTcMaxSlots && tc_smem_need(n_chunk, np, s + 1, k_split, grp) <= budget) ++s;
    return s;
}

// K unit range [u0, u1) of split z out of k_split over `units` units (balanced).
__host__ __device__ __forceinline__ void tc_unit_range(int units, int k_split, int z, int *u0, int *u1)
{
    *u0 = (int)((long long)units * z / k_split);
    *u1 = (int)((long long)units * (z + 1) / k_split);
}

// Packs units u and u + 1 (n_units = 1 or 2) of B = g - 1 for this CTA's columns into slots
// sb0 and sb1: every thread takes 16-byte core-matrix rows (8 BF16 or 4 TF32 values), threads
// 8k..8k+7 the 8 rows of one core matrix (contiguous in shared memory), and the loads of both
// units are issued before any is used.
template <bool BF16, int NP>
__device__ __forceinline__ void tc_stage_b(const TcArgs &A, unsigned char *sb0, unsigned char *sb1, size_t b_piece,
                                           int u, int n_units, int c_base, int tid)
{
    constexpr int EPV = BF16 ? 8 : 4;              // values per 16-byte vector
    constexpr int KU = 8 * EPV;                    // K values per unit (128 bytes per row)
    constexpr int BATCH = 2;
    const int nvec = A.n_chunk * 8;
    for (int v0 = 0; v0 < nvec; v0 += kTcThreads * BATCH) {
        float x[2][BATCH][EPV];
#pragma unroll
        for (int uu = 0; uu < 2; ++uu)
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int v = v0 + i * kTcThreads + tid;
                const int r = v & 7, h = (v >> 3) & 7, g8 = v >> 6;
                const int c = c_base + g8 * 8 + r, k = (u + uu) * KU + h * EPV;
                const bool ok = uu < n_units && v < nvec && c < A.n_cols;
                const float *src = A.g + (size_t)(ok ? c : 0) * A.n_bins + k;
#pragma unroll
                for (int e = 0; e < EPV; ++e) x[uu][i][e] = (ok && k + e < A.n_bins) ? __ldg(src + e) : 1.0f;
            }
#pragma unroll
        for (int uu = 0; uu < 2; ++uu) {
            if (uu >= n_units) break;
            unsigned char *sb_s = uu ? sb1 : sb0;
#pragma unroll
            for (int i = 0; i < BATCH; ++i) {
                const int v = v0 + i * kTcThreads + tid;
                if (v >= nvec) break;
                const int r = v & 7, h = (v >> 3) & 7, g8 = v >> 6;
                const size_t off = (size_t)(g8 * 8 + h) * 128 + r * 16;
                float res[EPV];
#pragma unroll
                for (int e = 0; e < EPV; ++e) res[e] = x[uu][i][e] - 1.0f;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    unsigned wv[4];
                    if (BF16) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const __nv_bfloat16 lo = __float2bfloat16_rn(res[2 * e]);
                            const __nv_bfloat16 hi = __float2bfloat16_rn(res[2 * e + 1]);
                            wv[e] = (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
                            res[2 * e] -= __bfloat162float(lo);
                            res[2 * e + 1] -= __bfloat162float(hi);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            wv[e] = tf32_round(res[e]);
                            res[e] -= __uint_as_float(wv[e]);
                        }
                    }
                    *reinterpret_cast<uint4 *>(sb_s + p * b_piece + off) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                }
            }
        }
    }
}

template <bool BF16, int NP>
__global__ void __launch_bounds__(kTcThreads, 1) tc_sq_kernel(const __grid_constant__ TcArgs A)
{
    constexpr int ES = BF16 ? 2 : 4;
    constexpr int KU = 128 / ES;                            // K values per unit
    constexpr int KMMA = 32 / ES;                           // K per instruction: 16 BF16, 8 TF32
    constexpr size_t A_PIECE = (size_t)kTcM * 128;
    constexpr unsigned SBO = 8u * 128u;                     // stride between 8-row groups
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar_full[kTcMaxSlots];
    __shared__ __align__(8) unsigned long long mbar_empty[kTcMaxSlots];
    __shared__ __align__(8) unsigned long long mbar_red;
    __shared__ unsigned tmem_base_sh;
    __shared__ int err_sh;
    __shared__ float w_sh[256], flat_sh[256];              // this chunk's column weights, set backgrounds
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, chunk = blockIdx.y, z = blockIdx.z;
    const int S = A.slots;
    const size_t b_piece = (size_t)A.n_chunk * 128;
    const size_t a_slot = NP * A_PIECE, b_slot = NP * b_piece;
    const size_t red_bytes = (size_t)A.n_chunk * kTcM * sizeof(float);
    unsigned char *sa = smem;                               // [slot][piece] A blocks
    unsigned char *sb = smem + (S * a_slot > red_bytes ? S * a_slot : red_bytes);
    float *red = reinterpret_cast<float *>(smem);           // [n_chunk][128] partial, after the MMAs
    float *recv = reinterpret_cast<float *>(sb);            // [k_split][recv_cols][128], pushed partials
    const int c_base = chunk * A.n_chunk;
    int u0, u1;
    tc_unit_range(A.units, A.k_split, z, &u0, &u1);
    const int nu = u1 - u0;
    for (int c = tid; c < A.n_chunk; c += kTcThreads) {
        const int cc = min(c_base + c, A.n_cols - 1);
        w_sh[c] = A.w[cc];
        flat_sh[c] = A.S_total ? A.flat[cc / A.cols_per_set] : 0.f;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"((unsigned)A.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        err_sh = 0;
        for (int i = 0; i < S; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_empty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_red)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        // prologue: the copies of the first min(nu, S) units, all in flight at once
        for (int j = 0; j < nu && j < S; ++j) {
            const unsigned mb = smem_u32(&mbar_full[j]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"((unsigned)a_slot) : "memory");
            const unsigned char *src = A.a_packed + ((size_t)mt * A.units + u0 + j) * a_slot;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sa + j * a_slot)),
                "l"(src), "r"((unsigned)a_slot), "r"(mb)
                : "memory");
        }
    }
    for (int j = 0; j < nu && j < S; j += 2)
        tc_stage_b<BF16, NP>(A, sb + j * b_slot, sb + (j + 1) * b_slot, b_piece, u0 + j, min(2, min(nu, S) - j),
                             c_base, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem_d = tmem_base_sh;
    const unsigned idesc = make_idesc(BF16 ? 1u : 2u, kTcM, (unsigned)A.n_chunk);
    int pending_slot = -1;                                  // thread 0: a copy whose wait gave up
    unsigned pending_parity = 0;

    for (int j = 0; j < nu; ++j) {
        const int slot = j % S;
        unsigned char *sa_s = sa + slot * a_slot;
        unsigned char *sb_s = sb + slot * b_slot;
        if (j >= S) {
            // refill: the MMAs that last read this slot (unit j - S) must be complete
            if (!mbar_wait_bounded(smem_u32(&mbar_empty[slot]), (unsigned)((j / S - 1) & 1)))
                atomicOr(&err_sh, 1);
            __syncthreads();
            if (err_sh) break;
            if (tid == 0) {
                const unsigned mb = smem_u32(&mbar_full[slot]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"((unsigned)a_slot) : "memory");
                const unsigned char *src = A.a_packed + ((size_t)mt * A.units + u0 + j) * a_slot;
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sa_s)),
                    "l"(src), "r"((unsigned)a_slot), "r"(mb)
                    : "memory");
            }
            tc_stage_b<BF16, NP>(A, sb_s, sb_s, b_piece, u0 + j, 1, c_base, tid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (tid == 0 && !err_sh) {
            if (!mbar_wait_bounded(smem_u32(&mbar_full[slot]), (unsigned)((j / S) & 1))) {
                err_sh = 1;
                pending_slot = slot;
                pending_parity = (unsigned)((j / S) & 1);
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int kk = 0; kk < KU / KMMA; ++kk) {
                    const unsigned koff = (unsigned)kk * 256u;    // two 16-byte k-groups per MMA
#pragma unroll
                    for (int pa = 0; pa < NP; ++pa)
#pragma unroll
                        for (int pb = 0; pb < NP; ++pb) {
                            if (pa + pb >= NP) continue;        // products down to the split order
                            const unsigned long long da = make_desc(smem_u32(sa_s + pa * A_PIECE) + koff, 128u, SBO);
                            const unsigned long long db = make_desc(smem_u32(sb_s + pb * b_piece) + koff, 128u, SBO);
                            const unsigned acc = (j > 0 || kk > 0 || pa > 0 || pb > 0) ? 1u : 0u;
                            if (BF16) mma_bf16(tmem_d, da, db, idesc, acc);
                            else mma_tf32(tmem_d, da, db, idesc, acc);
                        }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&mbar_empty[slot])));
            }
        }
    }
    __syncthreads();
    if (!err_sh && nu > 0) {
        // the last commit covers every MMA this thread issued
        const int j = nu - 1;
        if (!mbar_wait_bounded(smem_u32(&mbar_empty[j % S]), (unsigned)((j / S) & 1))) atomicOr(&err_sh, 1);
    }
    if (tid == 0 && pending_slot >= 0) {
        // a copy wait gave up: let that copy land (bounded again) before the buffers go
        mbar_wait_bounded(smem_u32(&mbar_full[pending_slot]), pending_parity);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!err_sh) {
        // partial accumulator -> shared memory, red[c][row]: warp w reads TMEM lanes
        // 32 (w % 4) .. +31 (its lane quarter) for the 16-column blocks b = w / 4, w / 4 + 2, ...
        const int row = (warp & 3) * 32 + lane;
        for (int c0 = (warp >> 2) * 16; c0 < A.n_chunk; c0 += 32) {
            unsigned v[16];
            const unsigned taddr = tmem_d + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int t = 0; t < 16; ++t) red[(c0 + t) * kTcM + row] = __uint_as_float(v[t]);
        }
    }
    const int ks = A.k_split;
    const bool sets = A.S_total != nullptr;
    const int grp = sets ? A.cols_per_set : 1;
    const int ncol = min(A.n_chunk, A.n_cols - c_base);
    const unsigned my_rank = ks > 1 ? cluster_rank() : 0u;
    int c_lo, c_hi;
    tc_owned_cols(ncol, grp, ks, (int)my_rank, &c_lo, &c_hi);
    const unsigned recv_bytes = ks > 1 ? (unsigned)((ks - 1) * (c_hi - c_lo) * kTcM * sizeof(float)) : 0u;
    if (tid == 0 && recv_bytes > 0)      // before the barrier, so no pushed byte can come first
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar_red)), "r"(recv_bytes) : "memory");
    if (ks > 1) cluster_sync();
    else __syncthreads();
    // every CTA of the cluster must have a valid partial
    int any_err = 0;
    for (int r = 0; r < ks; ++r) any_err |= ks > 1 ? ld_cluster_s32(map_rank(smem_u32(&err_sh), (unsigned)r)) : err_sh;
    if (!any_err && ks > 1 && tid == 0) {
        // push this CTA's partial of every other CTA's owned columns into that CTA's receive
        // buffer (slot = this rank), one bulk copy over distributed shared memory each
        for (int d = 0; d < ks; ++d) {
            if (d == (int)my_rank) continue;
            int d_lo, d_hi;
            tc_owned_cols(ncol, grp, ks, d, &d_lo, &d_hi);
            if (d_hi <= d_lo) continue;
            const unsigned bytes = (unsigned)((d_hi - d_lo) * kTcM * sizeof(float));
            const unsigned src = smem_u32(red) + (unsigned)(d_lo * kTcM * sizeof(float));
            const unsigned dst = map_rank(smem_u32(recv) + (unsigned)(my_rank * A.recv_cols * kTcM * sizeof(float)), (unsigned)d);
            const unsigned mb = map_rank(smem_u32(&mbar_red), (unsigned)d);
            asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                         "r"(src), "r"(bytes), "r"(mb)
                         : "memory");
        }
    }
    int red_ok = !any_err;
    if (red_ok && recv_bytes > 0 && !mbar_wait_bounded(smem_u32(&mbar_red), 0u)) {
        red_ok = 0;
        atomicOr(A.status, 1);
    }
    if (red_ok) {
        // items (owned column group, row): each sums the k_split partials of its columns in rank
        // order (FP32, own partial from `red`, the others from `recv`), scales by w_c and, for
        // sets, adds the set's columns to its flat background
        const int items = (c_hi - c_lo + grp - 1) / grp * kTcM;
        for (int it = tid; it < items; it += kTcThreads) {
            const int gl = it / kTcM, row = it % kTcM;
            const int q = mt * kTcM + row;
            const int cl0 = c_lo + gl * grp;
            float tot = 0.f;
            for (int t = 0; t < grp && cl0 + t < ncol; ++t) {
                const int cl = cl0 + t, c = c_base + cl;
                float acc = 0.f;
                for (int r = 0; r < ks; ++r)
                    acc += r == (int)my_rank ? red[cl * kTcM + row]
                                             : recv[((size_t)r * A.recv_cols + (cl - c_lo)) * kTcM + row];
                const float sp = acc * w_sh[cl];
                if (q < A.nQ && A.S_partial) A.S_partial[(size_t)c * A.nQ + q] = sp;
                tot += sp;
            }
            if (sets && q < A.nQ) {
                const int set = (c_base + cl0) / grp;
                A.S_total[(size_t)set * A.nQ + q] = flat_sh[cl0] + tot;
            }
        }
    } else if (tid == 0 && err_sh) {
        atomicOr(A.status, 1);
    }
    // no CTA leaves while another may still read its shared memory
    if (ks > 1) cluster_sync();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d),
                     "r"((unsigned)A.tmem_cols));
}

int tc_pack_a(const float *Kt, int nQ, int n_bins, int m_tiles, int stages, int kt, int np, int fmt_bf16,
              unsigned char *out, cudaStream_t stream)
{
    const long long total = (long long)m_tiles * kTcM * stages * kt;
    const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    tc_pack_a_kernel<<<grid, 256, 0, stream>>>(Kt, nQ, n_bins, m_tiles, stages, kt, np, fmt_bf16, out);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "tc_pack_a");
}

int tc_exec(const TcArgs &a, cudaStream_t stream)
{
    const int np = a.np_a;
    const int grp = a.S_total ? a.cols_per_set : 1;
    const size_t smem = tc_smem_need(a.n_chunk, np, a.slots, a.k_split, grp);
    if (a.np_a != a.np_b || (np != 2 && np != 3) || (!a.fmt_bf16 && np != 2) || a.ku != (a.fmt_bf16 ? 64 : 32) ||
        smem > kTcSmemMax || a.n_chunk % 16 || a.n_chunk < 16 || a.n_chunk > 256 || a.k_split < 1 ||
        a.k_split > kTcMaxKSplit || a.k_split > a.units || a.slots < 2 || a.slots > kTcMaxSlots ||
        (a.k_split > 1 && a.recv_cols < tc_recv_cols(a.n_chunk, grp, a.k_split)) ||
        (a.S_total && (a.cols_per_set < 1 || a.n_chunk % a.cols_per_set)))
        return set_error(EPSR_EINVAL, "tc sq: tile configuration out of range");
    void (*kern)(const TcArgs) = a.fmt_bf16 ? (np == 3 ? tc_sq_kernel<true, 3> : tc_sq_kernel<true, 2>)
                                            : tc_sq_kernel<false, 2>;
    static bool attr[3] = {false, false, false};
    const int ki = a.fmt_bf16 ? (np == 3 ? 2 : 1) : 0;
    if (!attr[ki]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(tc_sq)");
        attr[ki] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.m_tiles, (unsigned)((a.n_cols + a.n_chunk - 1) / a.n_chunk), (unsigned)a.k_split);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr_cl[1];
    attr_cl[0].id = cudaLaunchAttributeClusterDimension;
    attr_cl[0].val.clusterDim.x = 1;
    attr_cl[0].val.clusterDim.y = 1;
    attr_cl[0].val.clusterDim.z = (unsigned)a.k_split;
    cfg.attrs = attr_cl;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
    note_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "tc_sq launch");
}

}  // namespace epsr
