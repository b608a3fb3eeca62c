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
// Layout: operands are pre-packed in global memory in the tensor core's canonical
// K-major layout without swizzle -- core matrices of 8 rows x 16 bytes, K-adjacent core
// matrices 128 bytes apart (leading byte offset), 8-row groups HK * 128 bytes apart
// (stride byte offset) -- one contiguous block per (M-tile or operand, K-stage, piece), so a
// stage is staged into shared memory by plain coalesced 16-byte copies.
//
// One CTA per 128-row tile of Q (M = 128, N = padded n_cols <= 256): per K-stage every thread
// copies its part of the tiles, a proxy fence publishes them to the tensor core, thread 0
// issues the MMAs and commits them to an mbarrier, and all threads wait (bounded) before
// the buffers are reused. The epilogue reads the accumulator with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31) and writes S_partial[c][i] coalesced along i.
#include <cuda_bf16.h>

#include "epsr_device.cuh"
#include "epsr_internal.h"
#include "k_sq.h"

namespace epsr {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;
constexpr unsigned long long kTcSpinLimit = 1ull << 26;

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

// Pack the split columns B[c][k] = g[c][k] - 1 per call: blocks [stage][piece] of n_pad x kt.
__global__ void tc_pack_b_kernel(const float *g, int n_cols, int n_bins, int n_pad, int stages, int kt,
                                 int np, int fmt_bf16, unsigned char *out)
{
    const int esize = fmt_bf16 ? 2 : 4;
    const size_t piece_bytes = (size_t)n_pad * kt * esize;
    const long long total = (long long)n_pad * stages * kt;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % ((long long)stages * kt));
        const int c = (int)(e / ((long long)stages * kt));
        const int s = k / kt, kin = k % kt;
        const float v = (c < n_cols && k < n_bins) ? g[(long long)c * n_bins + k] - 1.0f : 0.f;
        unsigned char *blk = out + (size_t)s * np * piece_bytes;
        const size_t off = tc_elem_offset(c, kin, esize, kt);
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

__global__ void __launch_bounds__(kTcThreads, 1) tc_sq_kernel(TcArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base_sh;
    __shared__ int err_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x;
    const int esize = A.fmt_bf16 ? 2 : 4;
    const int kmma = 32 / esize;                            // K per instruction: 16 BF16, 8 TF32
    const size_t a_piece = (size_t)kTcM * A.kt * esize;
    const size_t b_piece = (size_t)A.n_pad * A.kt * esize;
    unsigned char *sa = smem;
    unsigned char *sb = smem + A.np_a * a_piece;
    const unsigned hk_bytes = (unsigned)(A.kt * esize / 16) * 128u;   // stride between 8-row groups

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"((unsigned)A.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        err_sh = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem_d = tmem_base_sh;
    const unsigned idesc = make_idesc(A.fmt_bf16 ? 1u : 2u, kTcM, (unsigned)A.n_pad);

    for (int s = 0; s < A.stages; ++s) {
        // stage the A tile pieces of this M tile and the B pieces
        const int4 *ga = reinterpret_cast<const int4 *>(A.a_packed + ((size_t)mt * A.stages + s) * A.np_a * a_piece);
        const int4 *gb = reinterpret_cast<const int4 *>(A.b_packed + (size_t)s * A.np_b * b_piece);
        const int na4 = (int)(A.np_a * a_piece / 16), nb4 = (int)(A.np_b * b_piece / 16);
        for (int i = tid; i < na4; i += kTcThreads) reinterpret_cast<int4 *>(sa)[i] = ga[i];
        for (int i = tid; i < nb4; i += kTcThreads) reinterpret_cast<int4 *>(sb)[i] = gb[i];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int kk = 0; kk < A.kt / kmma; ++kk) {
                const unsigned koff = (unsigned)kk * 256u;    // two 16-byte k-groups per MMA
                for (int pr = 0; pr < A.n_products; ++pr) {
                    const int i = A.prod_a[pr], j = A.prod_b[pr];
                    const unsigned long long da =
                        make_desc(smem_u32(sa + i * a_piece) + koff, 128u, hk_bytes);
                    const unsigned long long db =
                        make_desc(smem_u32(sb + j * b_piece) + koff, 128u, hk_bytes);
                    const unsigned acc = (s > 0 || kk > 0 || pr > 0) ? 1u : 0u;
                    if (A.fmt_bf16) mma_bf16(tmem_d, da, db, idesc, acc);
                    else mma_tf32(tmem_d, da, db, idesc, acc);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        // wait until the MMAs reading this stage are done (bounded)
        unsigned long long spins = 0;
        while (!mbar_try_wait(smem_u32(&mbar), (unsigned)(s & 1))) {
            if (++spins > kTcSpinLimit) {
                atomicOr(&err_sh, 1);
                break;
            }
        }
        __syncthreads();
        if (err_sh) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!err_sh) {
        // epilogue: row i = 32 warp + lane of this tile, columns in chunks of 16
        const int q = mt * kTcM + warp * 32 + lane;
        for (int c0 = 0; c0 < A.n_pad; c0 += 16) {
            unsigned v[16];
            const unsigned taddr = tmem_d + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (q < A.nQ)
                for (int t = 0; t < 16; ++t) {
                    const int c = c0 + t;
                    if (c < A.n_cols)
                        A.S_partial[(size_t)c * A.nQ + q] = (float)((double)__uint_as_float(v[t]) * A.w[c]);
                }
        }
    } else if (tid == 0) {
        atomicOr(A.status, 1);
    }
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

int tc_exec(const TcArgs &a, const float *g, cudaStream_t stream)
{
    const long long total = (long long)a.n_pad * a.stages * a.kt;
    const int grid = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    tc_pack_b_kernel<<<grid, 256, 0, stream>>>(g, a.n_cols, a.n_bins, a.n_pad, a.stages, a.kt, a.np_b,
                                               a.fmt_bf16, a.b_packed);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e, "tc_pack_b");
    const int esize = a.fmt_bf16 ? 2 : 4;
    const size_t smem = (size_t)(a.np_a * kTcM + a.np_b * a.n_pad) * a.kt * esize;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(tc_sq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(tc_sq)");
        attr = true;
    }
    if (smem > 200 * 1024) return set_error(EPSR_EINVAL, "tc sq: stage does not fit in shared memory");
    tc_sq_kernel<<<a.m_tiles, kTcThreads, smem, stream>>>(a);
    note_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "tc_sq launch");
}

}  // namespace epsr
