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

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;
constexpr unsigned long long kTcSpinLimit = 1ull << 26;
constexpr int kTcMaxUnits = 64;     // K units of one CTA's range (n_bins <= 4096 at 64 per unit)
constexpr int kTcLoadBatch = 32;    // g values per thread loaded before any is packed

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
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ int ld_cluster_s32(unsigned addr)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__host__ __device__ __forceinline__ size_t tc_a_unit_bytes(int ku, int np, int esize)
{
    return (size_t)np * kTcM * ku * esize;
}

__host__ __device__ __forceinline__ size_t tc_b_unit_bytes(int n_chunk, int ku, int np, int esize)
{
    return (size_t)np * n_chunk * ku * esize;
}

size_t tc_smem_bytes(int n_chunk, int ku, int np_a, int np_b, int fmt_bf16)
{
    const int esize = fmt_bf16 ? 2 : 4;
    const size_t a = kTcSlots * tc_a_unit_bytes(ku, np_a, esize);
    const size_t red = (size_t)n_chunk * kTcM * sizeof(float);
    const size_t total = (a > red ? a : red) + kTcSlots * tc_b_unit_bytes(n_chunk, ku, np_b, esize);
    return total <= 220 * 1024 ? total : 0;
}

// K unit range [u0, u1) of split z out of k_split over `units` units (balanced).
__host__ __device__ __forceinline__ void tc_unit_range(int units, int k_split, int z, int *u0, int *u1)
{
    *u0 = (int)((long long)units * z / k_split);
    *u1 = (int)((long long)units * (z + 1) / k_split);
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_sq_kernel(const __grid_constant__ TcArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar_full[kTcSlots];
    __shared__ __align__(8) unsigned long long mbar_empty[kTcSlots];
    __shared__ unsigned tmem_base_sh;
    __shared__ int err_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, chunk = blockIdx.y, z = blockIdx.z;
    const int esize = A.fmt_bf16 ? 2 : 4;
    const int kmma = 32 / esize;                            // K per instruction: 16 BF16, 8 TF32
    const size_t a_piece = (size_t)kTcM * A.ku * esize;
    const size_t b_piece = (size_t)A.n_chunk * A.ku * esize;
    const size_t a_slot = A.np_a * a_piece, b_slot = A.np_b * b_piece;
    const size_t red_bytes = (size_t)A.n_chunk * kTcM * sizeof(float);
    unsigned char *sa = smem;                               // [slot][piece] A blocks
    unsigned char *sb = smem + (kTcSlots * a_slot > red_bytes ? kTcSlots * a_slot : red_bytes);
    float *red = reinterpret_cast<float *>(smem);           // [n_chunk][128] partial, after the MMAs
    const unsigned sbo = (unsigned)(A.ku * esize / 16) * 128u;   // stride between 8-row groups
    const int c_base = chunk * A.n_chunk;
    int u0, u1;
    tc_unit_range(A.units, A.k_split, z, &u0, &u1);
    const int nu = u1 - u0;
    const int ku_shift = __ffs(A.ku) - 1;                   // ku is a power of two

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"((unsigned)A.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        err_sh = 0;
        for (int i = 0; i < kTcSlots; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_empty[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem_d = tmem_base_sh;
    const unsigned idesc = make_idesc(A.fmt_bf16 ? 1u : 2u, kTcM, (unsigned)A.n_chunk);
    int pending_slot = -1;                                  // thread 0: a copy whose wait gave up
    unsigned pending_parity = 0;

    for (int j = 0; j < nu; ++j) {
        const int slot = j % kTcSlots;
        if (j >= kTcSlots) {
            // the MMAs that last read this slot (unit j - kTcSlots) must be complete
            if (!mbar_wait_bounded(smem_u32(&mbar_empty[slot]), (unsigned)((j / kTcSlots - 1) & 1)))
                atomicOr(&err_sh, 1);
        }
        __syncthreads();
        if (err_sh) break;
        const int u = u0 + j;
        unsigned char *sa_s = sa + slot * a_slot;
        unsigned char *sb_s = sb + slot * b_slot;
        if (tid == 0) {
            const unsigned bytes = (unsigned)a_slot;
            const unsigned mb = smem_u32(&mbar_full[slot]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
            const unsigned char *src = A.a_packed + ((size_t)mt * A.units + u) * a_slot;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(sa_s)),
                "l"(src), "r"(bytes), "r"(mb)
                : "memory");
        }
        // B = g - 1 for this CTA's columns and unit, split into pieces, packed K-major; the
        // loads of a batch are all issued before the first is used
        const int k0 = u * A.ku;
        const int n_el = A.n_chunk * A.ku;
        for (int e0 = 0; e0 < n_el; e0 += kTcThreads * kTcLoadBatch) {
            float v[kTcLoadBatch];
#pragma unroll
            for (int i = 0; i < kTcLoadBatch; ++i) {
                const int e = e0 + i * kTcThreads + tid;
                const int row = e >> ku_shift, kin = e & (A.ku - 1);
                const int c = c_base + row, k = k0 + kin;
                v[i] = (e < n_el && c < A.n_cols && k < A.n_bins) ? __ldg(A.g + (size_t)c * A.n_bins + k) : 1.0f;
            }
#pragma unroll
            for (int i = 0; i < kTcLoadBatch; ++i) {
                const int e = e0 + i * kTcThreads + tid;
                if (e >= n_el) break;
                const int row = e >> ku_shift, kin = e & (A.ku - 1);
                const size_t off = tc_elem_offset(row, kin, esize, A.ku);
                const float x = v[i] - 1.0f;
                if (A.fmt_bf16) {
                    float r = x;
                    for (int pc = 0; pc < A.np_b; ++pc) {
                        const __nv_bfloat16 h = __float2bfloat16_rn(r);
                        *reinterpret_cast<unsigned short *>(sb_s + pc * b_piece + off) = __bfloat16_as_ushort(h);
                        r = r - __bfloat162float(h);
                    }
                } else {
                    float r = x;
                    for (int pc = 0; pc < A.np_b; ++pc) {
                        const unsigned h = tf32_round(r);
                        *reinterpret_cast<unsigned *>(sb_s + pc * b_piece + off) = h;
                        r = r - __uint_as_float(h);
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait_bounded(smem_u32(&mbar_full[slot]), (unsigned)((j / kTcSlots) & 1))) {
                err_sh = 1;
                pending_slot = slot;
                pending_parity = (unsigned)((j / kTcSlots) & 1);
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int kk = 0; kk < A.ku / kmma; ++kk) {
                    const unsigned koff = (unsigned)kk * 256u;    // two 16-byte k-groups per MMA
                    for (int pr = 0; pr < A.n_products; ++pr) {
                        const int pa = A.prod_a[pr], pb = A.prod_b[pr];
                        const unsigned long long da = make_desc(smem_u32(sa_s + pa * a_piece) + koff, 128u, sbo);
                        const unsigned long long db = make_desc(smem_u32(sb_s + pb * b_piece) + koff, 128u, sbo);
                        const unsigned acc = (j > 0 || kk > 0 || pr > 0) ? 1u : 0u;
                        if (A.fmt_bf16) mma_bf16(tmem_d, da, db, idesc, acc);
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
        if (!mbar_wait_bounded(smem_u32(&mbar_empty[j % kTcSlots]), (unsigned)((j / kTcSlots) & 1)))
            atomicOr(&err_sh, 1);
    }
    if (tid == 0 && pending_slot >= 0) {
        // a copy wait gave up: let that copy land (bounded again) before the buffers go
        mbar_wait_bounded(smem_u32(&mbar_full[pending_slot]), pending_parity);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!err_sh) {
        // partial accumulator -> shared memory, red[c][row] (row = this thread's TMEM lane)
        const int row = warp * 32 + lane;
        for (int c0 = 0; c0 < A.n_chunk; c0 += 16) {
            unsigned v[16];
            const unsigned taddr = tmem_d + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            for (int t = 0; t < 16; ++t) red[(c0 + t) * kTcM + row] = __uint_as_float(v[t]);
        }
    }
    if (A.k_split > 1) cluster_sync();
    else __syncthreads();
    // every CTA of the cluster must have a valid partial
    const unsigned my_rank = A.k_split > 1 ? cluster_rank() : 0u;
    int any_err = 0;
    for (int r = 0; r < A.k_split; ++r)
        any_err |= A.k_split > 1 ? ld_cluster_s32(map_rank(smem_u32(&err_sh), (unsigned)r)) : err_sh;
    if (!any_err) {
        const int row = warp * 32 + lane;
        const int q = mt * kTcM + row;
        const bool sets = A.S_total != nullptr;
        const int grp = sets ? A.cols_per_set : 1;
        const unsigned red_addr = smem_u32(red);
        unsigned base[kTcMaxKSplit];
#pragma unroll
        for (int r = 0; r < kTcMaxKSplit; ++r)
            base[r] = (A.k_split > 1 && r < A.k_split) ? map_rank(red_addr, (unsigned)r) : red_addr;
        for (int gi = (int)my_rank; gi * grp < A.n_chunk; gi += A.k_split) {
            const int cg = c_base + gi * grp;
            if (cg >= A.n_cols) break;
            double tot = 0.0;
            for (int t = 0; t < grp; ++t) {
                const int cl = gi * grp + t, c = cg + t;
                const unsigned off = (unsigned)((cl * kTcM + row) * sizeof(float));
                // every CTA's partial of this element in flight at once, summed in rank order
                float p[kTcMaxKSplit];
#pragma unroll
                for (int r = 0; r < kTcMaxKSplit; ++r)
                    p[r] = r < A.k_split ? (A.k_split > 1 ? ld_cluster_f32(base[r] + off) : red[cl * kTcM + row]) : 0.f;
                double acc = 0.0;
#pragma unroll
                for (int r = 0; r < kTcMaxKSplit; ++r)
                    if (r < A.k_split) acc += (double)p[r];
                const float sp = (float)(acc * A.w[c]);
                if (q < A.nQ && A.S_partial) A.S_partial[(size_t)c * A.nQ + q] = sp;
                tot += (double)sp;
            }
            if (sets && q < A.nQ) A.S_total[(size_t)(cg / grp) * A.nQ + q] = (float)(A.flat[cg / grp] + tot);
        }
    } else if (tid == 0 && err_sh) {
        atomicOr(A.status, 1);
    }
    // no CTA leaves while another may still read its shared memory
    if (A.k_split > 1) cluster_sync();
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
    const size_t smem = tc_smem_bytes(a.n_chunk, a.ku, a.np_a, a.np_b, a.fmt_bf16);
    if (smem == 0 || a.n_chunk % 16 || a.n_chunk < 16 || a.n_chunk > 256 || a.k_split < 1 ||
        a.k_split > kTcMaxKSplit || a.k_split > a.units || (a.units + a.k_split - 1) / a.k_split > kTcMaxUnits)
        return set_error(EPSR_EINVAL, "tc sq: tile configuration out of range");
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_sq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(tc_sq)");
        attr = true;
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, tc_sq_kernel, a);
    note_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "tc_sq launch");
}

}  // namespace epsr
