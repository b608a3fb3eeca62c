// k_gr.cu -- all-pair partial histograms N_ab(r) (Sec. 2.3, O(N^2) per evaluation),
// g_ab(r) normalisation, and the O(N^2) total energy, on sm_103a.
//
// Work list: (box, i-tile, j-tile) with i-tile <= j-tile over tiles of kGrTile atoms,
// processed by a persistent grid. A CTA stages the j-tile in shared memory (coalesced
// 128-bit loads) and each thread keeps kGrR i-atoms in registers, so one broadcast
// shared load serves kGrR pair tests.
//
// Prefilter: a second copy of the coordinates is scaled so that the box side maps to
// 2^32 (x' = floor(x 2^32 / L)); its top 16 bits x16 = floor(x 2^16 / L) wrap modulo 2^16
// as minimum images wrap modulo L. Each thread packs the biased 16-bit coordinates of two
// of its i-atoms per axis in one word, so one 32-bit subtraction per axis gives both
// differences, a three-way halfword maximum (__vimax3_u16x2) the per-atom maxima over the
// axes, and two halfword minima and one compare decide whether any of the thread's four
// i-atoms is inside the cube around j. Four j are tested per step before one branch.
// Pairs that pass take the exact path: integer minimum image on the true grid coordinates;
// the bin from the FP32 squared distance, with the exact 64-bit squared distance and the
// threshold table only within the FP32 error of a bin edge or of the range. Counts go to a
// per-CTA shared-memory histogram (32-bit) and are flushed to the caller's 64-bit histogram
// with one atomic per non-empty bin.
#include "epsr_device.cuh"
#include "epsr_internal.h"

namespace epsr {

constexpr int kGrThreads = 256;
constexpr int kGrR = kGrTile / kGrThreads;   // i-atoms per thread

__global__ void scale_coords_kernel(const BoxDev *boxes, const int *atom_box, const int4 *coords,
                                    uint4 *scaled, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int4 c = coords[i];
        const unsigned long long L = (unsigned long long)boxes[atom_box[i]].L;
        uint4 s;
        s.x = (unsigned)(((unsigned long long)c.x << 32) / L);
        s.y = (unsigned)(((unsigned long long)c.y << 32) / L);
        s.z = (unsigned)(((unsigned long long)c.z << 32) / L);
        s.w = (unsigned)c.w;
        scaled[i] = s;
    }
}

int launch_scale_coords(const BoxDev *boxes, const int *atom_box, const int4 *coords,
                        uint4 *scaled, long long n, cudaStream_t stream)
{
    if (n == 0) return EPSR_OK;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    scale_coords_kernel<<<grid, 256, 0, stream>>>(boxes, atom_box, coords, scaled, n);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "scale_coords");
}

// ---- spatial order for the pair scan ---------------------------------------------------------
// Atoms are counting-sorted by the Morton code of their cell (up to 32 cells per side,
// about 3 A wide) so that the 32 i-atoms of a warp are neighbours in space: candidate
// pairs then come in dense runs instead of scattering single lanes into the exact path.
// Every pair is still tested; the order inside a cell is irrelevant to integer counts.
__device__ __forceinline__ unsigned spread5(unsigned v)
{
    v &= 31u;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Sort key: the Morton code of the atom's cell, offset by the box's first cell. With
// type_major the key space of a box is split into one block of cells per atom type, so
// the sorted order is type by type, each spatially ordered.
__global__ void cell_key_kernel(const BoxDev *boxes, const int *atom_box, const uint4 *scaled,
                                int *key, int *rank, int *count, long long n, int type_major)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const BoxDev &b = boxes[atom_box[i]];
        const uint4 s = scaled[i];
        const unsigned nc = (unsigned)b.cells;
        const unsigned cx = __umulhi(s.x, nc), cy = __umulhi(s.y, nc), cz = __umulhi(s.z, nc);
        int k;
        if (type_major == 2) {
            // cell-list order: cells of at least the histogram range per side, x fastest
            const unsigned n = (unsigned)(b.gc_n > 0 ? b.gc_n : 1);
            k = b.gc0 + (int)((__umulhi(s.z, n) * n + __umulhi(s.y, n)) * n + __umulhi(s.x, n));
        } else if (type_major) {
            // Monte Carlo partition: atom i of the box goes to CTA (i mod G) of its group;
            // inside a CTA's share of a type, atoms are ordered by an 8^3 Morton cell.
            const unsigned c8x = __umulhi(s.x, 8u), c8y = __umulhi(s.y, 8u), c8z = __umulhi(s.z, 8u);
            const int code8 = (int)(spread5(c8x) | (spread5(c8y) << 1) | (spread5(c8z) << 2));
            const int r = (int)((i - b.atom0) % b.n_cta);
            k = b.mc_cell0 + ((int)s.w * b.n_cta + r) * kMcCells + code8;
        } else {
            k = b.cell0 + (int)(spread5(cx) | (spread5(cy) << 1) | (spread5(cz) << 2));
        }
        key[i] = k;
        rank[i] = atomicAdd(&count[k], 1);
    }
}

// Exclusive scan of the cell counts in three passes over blocks of kScanBlock cells.
constexpr int kScanBlock = 1024;

__global__ void scan_block_sums_kernel(const int *count, int n, int *block_sum)
{
    __shared__ int red[32];
    const int b = blockIdx.x, i = b * kScanBlock + threadIdx.x;
    int v = i < n ? count[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) block_sum[b] = t;
    }
}

// Exclusive scan of the block sums in place by one CTA of 1024 threads, each owning a
// contiguous chunk.
__global__ void scan_block_offsets_kernel(int *block_sum, int nblocks)
{
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (nblocks + 1023) / 1024;
    const int b0 = min(nblocks, t * per), b1 = min(nblocks, b0 + per);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += block_sum[b];
    int x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = x - local + (w > 0 ? wsum[w - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        const int v = block_sum[b];
        block_sum[b] = run;
        run += v;
    }
}

__global__ void scan_finish_kernel(const int *count, int n, const int *block_off, int *offset)
{
    __shared__ int wsum[32];
    const int b = blockIdx.x, i = b * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? count[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    const int excl = x - v + (w > 0 ? wsum[w - 1] : 0) + block_off[b];
    if (i < n) offset[i] = excl;
}

__global__ void scatter_index_kernel(const int *key, const int *rank, const int *offset,
                                     int *sorted_index, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        sorted_index[offset[key[i]] + rank[i]] = (int)i;
}

// Makes the order deterministic: each cell's segment (a few atoms) is put in atom-index
// order, then (optionally) the coordinates are gathered in that order and the inverse map
// atom -> sorted position is written. Ranks from the counting pass depend on atomic timing;
// the final order depends only on the coordinates.
__global__ void cell_order_kernel(const int *count, const int *offset, int total_cells,
                                  int *idx, const uint4 *scaled, const int4 *coords,
                                  uint4 *s_scaled, int4 *s_coords, int *pos_of, int in_order)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < total_cells; c += gridDim.x * blockDim.x) {
        const int b = offset[c], n = in_order ? count[c] : 0;
        for (int a = 1; a < n; ++a) {
            const int v = idx[b + a];
            int k = a - 1;
            while (k >= 0 && idx[b + k] > v) {
                idx[b + k + 1] = idx[b + k];
                --k;
            }
            idx[b + k + 1] = v;
        }
        for (int a = 0, na = count[c]; a < na; ++a) {
            const int i = idx[b + a];
            if (s_scaled) s_scaled[b + a] = scaled[i];
            if (s_coords) s_coords[b + a] = coords[i];
            if (pos_of) pos_of[i] = b + a;
        }
    }
}

__global__ void gather_sorted_kernel(const int *idx, const uint4 *scaled, const int4 *coords,
                                     uint4 *s_scaled, int4 *s_coords, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = idx[p];
        if (s_scaled) s_scaled[p] = scaled[i];
        if (s_coords) s_coords[p] = coords[i];
    }
}

int launch_spatial_sort(const BoxDev *boxes, const int *atom_box, const uint4 *scaled,
                        const int4 *coords, long long n, int total_cells, int type_major,
                        SortScratch sc, uint4 *s_scaled, int4 *s_coords, int *pos_of,
                        cudaStream_t stream)
{
    if (n == 0) return EPSR_OK;
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    const int nblk = (total_cells + kScanBlock - 1) / kScanBlock;
    cudaError_t e = cudaMemsetAsync(sc.count, 0, (size_t)total_cells * sizeof(int), stream);
    if (e != cudaSuccess) return set_cuda_error(e, "sort memset");
    cell_key_kernel<<<grid, 256, 0, stream>>>(boxes, atom_box, scaled, sc.key, sc.rank, sc.count, n,
                                              type_major);
    note_launch();
    scan_block_sums_kernel<<<nblk, kScanBlock, 0, stream>>>(sc.count, total_cells, sc.block);
    note_launch();
    scan_block_offsets_kernel<<<1, 1024, 0, stream>>>(sc.block, nblk);
    note_launch();
    scan_finish_kernel<<<nblk, kScanBlock, 0, stream>>>(sc.count, total_cells, sc.block, sc.offset);
    note_launch();
    scatter_index_kernel<<<grid, 256, 0, stream>>>(sc.key, sc.rank, sc.offset, sc.index, n);
    note_launch();
    const int cgrid = (total_cells + 255) / 256 < 4096 ? (total_cells + 255) / 256 : 4096;
    if (type_major == 2) {
        // the cell-list order only feeds integer counts: the order inside a cell does not
        // matter there and its cells are large, so the scatter's order is kept and the
        // coordinates are gathered by position, in parallel
        gather_sorted_kernel<<<grid, 256, 0, stream>>>(sc.index, scaled, coords, s_scaled, s_coords, n);
    } else {
        cell_order_kernel<<<cgrid, 256, 0, stream>>>(sc.count, sc.offset, total_cells, sc.index, scaled,
                                                     coords, s_scaled, s_coords, pos_of, 1);
    }
    note_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "spatial sort");
}

__device__ __forceinline__ void flush_hist(unsigned *sh_hist, int n, unsigned long long *out)
{
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const unsigned v = sh_hist[k];
        if (v) {
            atomicAdd(out + k, (unsigned long long)v);
            sh_hist[k] = 0u;
        }
    }
}

// Bin of a pair from its FP32 squared distance g2 (relative error below 2^-21.7 from the
// int32 separations), falling back to the exact integer test only where that error could
// matter: the bin is floor(sqrt(d2) / w) exactly (d2 >= T[k] <=> d2 >= (k w)^2 for integer
// d2), and x = sqrt(g2) / w carries a relative error below 2^-21, so floor(x) is the bin
// unless x lies within x 2^-20 of an integer. Returns -1 outside the histogram range.
__device__ __forceinline__ int bin_of_fast(Sep sp, float g2, const long long *T, int nb, float inv,
                                           long long tmax, float tmax_lo, float tmax_hi)
{
    if (g2 >= tmax_hi) return -1;
    if (g2 >= tmax_lo && d2_of(sp) >= tmax) return -1;
    const float x = sqrtf(g2) * inv;
    const int k = (int)x;
    const float f = x - (float)k, eps = x * 0x1p-20f;
    if (f > eps && f < 1.f - eps && k < nb) return k;
    return bin_of(d2_of(sp), g2, T, nb, inv);
}

static_assert(kGrR == 4, "the prefilter packs the four i-atoms of a thread in pairs");
static_assert(kGrTile % 4 == 0, "four j per step");

__global__ void __launch_bounds__(kGrThreads, 4) partial_gr_kernel(GrArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    uint4 *s_pack = reinterpret_cast<uint4 *>(dyn);         // j: 16-bit x, y, z in both halfwords
    int4 *s_true = reinterpret_cast<int4 *>(s_pack + kGrTile);
    long long *s_T = reinterpret_cast<long long *>(s_true + kGrTile);
    unsigned *s_hist = reinterpret_cast<unsigned *>(s_T + A.max_bins1);
    __shared__ BoxDev bx;
    __shared__ int cur_box;

    const int tid = threadIdx.x;
    if (tid == 0) cur_box = -1;
    for (int k = tid; k < A.max_pairs_bins; k += kGrThreads) s_hist[k] = 0u;
    __syncthreads();

    for (long long w = A.tile_begin + blockIdx.x; w < A.tile_end; w += gridDim.x) {
        const GrTile tl = A.tiles[w];
        __syncthreads();   // the previous tile's counting is complete before any flush
        if (tl.box != cur_box) {
            // flush the previous box's counts, then load this box's parameters and table
            if (cur_box >= 0) {
                const BoxDev &pb = bx;
                flush_hist(s_hist, pb.n_pairs * pb.n_bins, A.hist + pb.hist_off);
            }
            __syncthreads();
            if (tid == 0) {
                bx = A.boxes[tl.box];
                cur_box = tl.box;
            }
            __syncthreads();
            for (int k = tid; k <= bx.n_bins; k += kGrThreads) s_T[k] = A.thresholds[bx.tbl_off + k];
        }
        const int L = bx.L;
        const int N = bx.n_atoms;
        const unsigned B = bx.pre16_bias, TT = bx.pre16_t, T = TT & 0xFFFFu;
        const bool all = bx.pre16_all != 0;
        const long long tmax = bx.tmax;
        const float tmax_hi = bx.tmax_hi, tmax_lo = bx.tmax_lo;
        const int nb = bx.n_bins, nt = bx.n_types;
        const float inv = bx.inv_dr_fx;
        // stage the j-tile: the 16-bit coordinate (top half of the 2^32-scaled one) in both
        // halfwords of a word per axis, and the true coordinates for the exact path
        const int j0 = tl.tj * kGrTile;
        const int nj = min(kGrTile, N - j0);
        __syncthreads();
        for (int j = tid; j < nj; j += kGrThreads) {
            const uint4 sc = A.scaled[bx.atom0 + j0 + j];
            s_pack[j] = make_uint4(__byte_perm(sc.x, 0u, 0x3232), __byte_perm(sc.y, 0u, 0x3232),
                                     __byte_perm(sc.z, 0u, 0x3232), 0u);
            s_true[j] = A.coords[bx.atom0 + j0 + j];
        }
        // i-atoms in registers: thread t holds tile rows t, t + 256, t + 512, t + 768, biased
        // 16-bit coordinates packed two rows per word (rows 0/2 low halfword, 1/3 high)
        const int i0 = tl.ti * kGrTile;
        int il[kGrR];
        unsigned bxr[kGrR], byr[kGrR], bzr[kGrR];
#pragma unroll
        for (int r = 0; r < kGrR; ++r) {
            il[r] = tid + r * kGrThreads;
            const int ig = i0 + il[r];
            bxr[r] = byr[r] = bzr[r] = 0u;
            if (ig < N) {
                const uint4 sc = A.scaled[bx.atom0 + ig];
                bxr[r] = ((sc.x >> 16) + B) & 0xFFFFu;
                byr[r] = ((sc.y >> 16) + B) & 0xFFFFu;
                bzr[r] = ((sc.z >> 16) + B) & 0xFFFFu;
            } else {
                il[r] = -1;
            }
        }
        const unsigned X01 = bxr[0] | (bxr[1] << 16), Y01 = byr[0] | (byr[1] << 16), Z01 = bzr[0] | (bzr[1] << 16);
        const unsigned X23 = bxr[2] | (bxr[3] << 16), Y23 = byr[2] | (byr[3] << 16), Z23 = bzr[2] | (bzr[3] << 16);
        const bool diag = tl.ti == tl.tj;
        __syncthreads();
        // four j per step: their tests are independent, and one branch covers all four
        for (int jb = 0; jb < nj; jb += 4) {
            unsigned msk[4], m01s[4], m23s[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint4 pj = s_pack[jb + u];   // jb + u < kGrTile; entries past nj are masked
                // one 32-bit subtraction per axis and row pair: the low halfword is exact
                // modulo 2^16, the high one may carry a borrow of one unit, which the bias absorbs;
                // per-row maxima over the axes, then the least of the four rows in both halfwords
                const unsigned m01 = __vimax3_u16x2(X01 - pj.x, Y01 - pj.y, Z01 - pj.z);
                const unsigned m23 = __vimax3_u16x2(X23 - pj.x, Y23 - pj.y, Z23 - pj.z);
                const unsigned x = __vimin3_u16x2(m01, m23, m23);
                const unsigned y = __vimin3_u16x2(x, __byte_perm(x, 0u, 0x1032), x);
                m01s[u] = m01; m23s[u] = m23;
                msk[u] = (jb + u < nj && (y <= TT || all)) ? 1u : 0u;
            }
            if (!(msk[0] | msk[1] | msk[2] | msk[3])) continue;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (!msk[u]) continue;
                const unsigned m01 = m01s[u], m23 = m23s[u];
                const unsigned mask = all ? 0xFu
                                          : ((m01 & 0xFFFFu) <= T ? 1u : 0u) | ((m01 >> 16) <= T ? 2u : 0u) |
                                                ((m23 & 0xFFFFu) <= T ? 4u : 0u) | ((m23 >> 16) <= T ? 8u : 0u);
                const int j = jb + u;
#pragma unroll
                for (int r = 0; r < kGrR; ++r) {
                    if ((mask >> r) & 1u) {
                        if (il[r] < 0 || (diag && j <= il[r])) continue;
                        const int4 pi = A.coords[bx.atom0 + i0 + il[r]];
                        const int4 pj = s_true[j];
                        const Sep sp = sep(pi, pj, L);
                        const int k = bin_of_fast(sp, g2_of(sp), s_T, nb, inv, tmax, tmax_lo, tmax_hi);
                        if (k >= 0) atomicAdd(&s_hist[pair_index(pi.w, pj.w, nt) * nb + k], 1u);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (cur_box >= 0) flush_hist(s_hist, bx.n_pairs * bx.n_bins, A.hist + bx.hist_off);
}

int launch_partial_gr(const GrArgs &args, int grid, cudaStream_t stream)
{
    if (args.tile_end <= args.tile_begin) return EPSR_OK;
    const size_t smem = (size_t)kGrTile * (sizeof(uint4) + sizeof(int4)) +
                        (size_t)args.max_bins1 * sizeof(long long) +
                        (size_t)args.max_pairs_bins * sizeof(unsigned);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(partial_gr_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(gr)");
        attr_set = true;
    }
    if (smem > 200 * 1024)
        return set_error(EPSR_EINVAL, "partial_gr: n_pairs*n_bins too large for shared memory");
    partial_gr_kernel<<<grid, kGrThreads, smem, stream>>>(args);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "partial_gr launch");
}

// ---- cell-list histogram (a counting order of the same pairs) ----------------------------------
// Every pair closer than the histogram range lies in the same cell or in neighbouring cells
// (cells are at least the range wide plus two grid units, and there are at least 3 per side,
// so the 13 forward offsets and their negatives reach 26 distinct cells). A work item counts
// the pairs of one home cell with itself (i < j in the sorted order) and with its 13 forward
// neighbours, each pair once; the pair test, bins and counts are those of partial_gr_kernel,
// so the histogram is the same integer array.
constexpr int kGcThreads = 128;
constexpr int kGcStage = 512;            // neighbour atoms staged in shared memory at once

__constant__ int c_fwd[14][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 1, 0},  {0, 1, 0},   {1, 1, 0},
                                 {-1, -1, 1}, {0, -1, 1},  {1, -1, 1},  {-1, 0, 1},  {0, 0, 1},
                                 {1, 0, 1},  {-1, 1, 1},   {0, 1, 1},   {1, 1, 1}};

__global__ void __launch_bounds__(kGcThreads) partial_gr_cells_kernel(GcArgs A)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    int4 *s_true = reinterpret_cast<int4 *>(dyn);
    long long *s_T = reinterpret_cast<long long *>(s_true + kGcStage);
    unsigned *s_hist = reinterpret_cast<unsigned *>(s_T + A.max_bins1);
    __shared__ BoxDev bx;
    __shared__ int cur_box;
    const int tid = threadIdx.x;
    if (tid == 0) cur_box = -1;
    for (int k = tid; k < A.max_pairs_bins; k += kGcThreads) s_hist[k] = 0u;
    __syncthreads();

    for (long long w = blockIdx.x; w < A.n_items; w += gridDim.x) {
        const GcItem it = A.items[w];
        __syncthreads();
        if (it.box != cur_box) {
            if (cur_box >= 0) flush_hist(s_hist, bx.n_pairs * bx.n_bins, A.hist + bx.hist_off);
            __syncthreads();
            if (tid == 0) {
                bx = A.boxes[it.box];
                cur_box = it.box;
            }
            __syncthreads();
            for (int k = tid; k <= bx.n_bins; k += kGcThreads) s_T[k] = A.thresholds[bx.tbl_off + k];
            __syncthreads();
        }
        const int n = bx.gc_n, L = bx.L, nb = bx.n_bins, nt = bx.n_types;
        const long long tmax = bx.tmax;
        const float tmax_lo = bx.tmax_lo, tmax_hi = bx.tmax_hi, inv = bx.inv_dr_fx;
        const int hc = it.cell, hx = hc % n, hy = (hc / n) % n, hz = hc / (n * n);
        const int hs = A.cell_start[bx.gc0 + hc], nh = A.cell_count[bx.gc0 + hc];
        for (int i0 = 0; i0 < nh; i0 += kGcThreads) {
            const int ip = i0 + tid < nh ? hs + i0 + tid : -1;        // sorted position of my atom
            const int4 pi = ip >= 0 ? A.coords[ip] : make_int4(0, 0, 0, 0);
            for (int t = 0; t < 14; ++t) {
                const int cx = (hx + c_fwd[t][0] + n) % n, cy = (hy + c_fwd[t][1] + n) % n,
                          cz = (hz + c_fwd[t][2] + n) % n;
                const int c = bx.gc0 + (cz * n + cy) * n + cx;
                const int cs = A.cell_start[c], nc = A.cell_count[c];
                for (int j0 = 0; j0 < nc; j0 += kGcStage) {
                    const int nj = min(kGcStage, nc - j0);
                    __syncthreads();
                    for (int j = tid; j < nj; j += kGcThreads) s_true[j] = A.coords[cs + j0 + j];
                    __syncthreads();
                    if (ip < 0) continue;
                    // own cell: only partners after me in the sorted order (each pair once)
                    const int jstart = t == 0 ? max(0, ip + 1 - (cs + j0)) : 0;
                    for (int j = jstart; j < nj; ++j) {
                        const int4 pj = s_true[j];
                        const Sep sp = sep(pi, pj, L);
                        const float g2 = g2_of(sp);
                        if (g2 < tmax_hi) {
                            const int k = bin_of_fast(sp, g2, s_T, nb, inv, tmax, tmax_lo, tmax_hi);
                            if (k >= 0) atomicAdd(&s_hist[pair_index(pi.w, pj.w, nt) * nb + k], 1u);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (cur_box >= 0) flush_hist(s_hist, bx.n_pairs * bx.n_bins, A.hist + bx.hist_off);
}

int launch_partial_gr_cells(const GcArgs &args, int grid, cudaStream_t stream)
{
    if (args.n_items <= 0) return EPSR_OK;
    const size_t smem = (size_t)kGcStage * sizeof(int4) + (size_t)args.max_bins1 * sizeof(long long) +
                        (size_t)args.max_pairs_bins * sizeof(unsigned);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(partial_gr_cells_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(gr cells)");
        attr_set = true;
    }
    if (smem > 200 * 1024)
        return set_error(EPSR_EINVAL, "partial_gr_cells: n_pairs*n_bins too large for shared memory");
    partial_gr_cells_kernel<<<grid, kGcThreads, smem, stream>>>(args);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "partial_gr_cells launch");
}

// g_ab(k) = H V / (n_configs P_ab (4 pi / 3)(r_{k+1}^3 - r_k^3)), r_k = k dr.
__global__ void normalize_g_kernel(const BoxDev *boxes, int n_boxes, const unsigned long long *hist,
                                   float *g, double inv_configs, long long hist_len,
                                   const long long *hist_box)
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
        int a = 0, rem = p;                      // pair index p -> types (a, c), a <= c
        while (rem >= b.n_types - a) { rem -= b.n_types - a; ++a; }
        const int c = a + rem;
        const double Pab = a == c ? 0.5 * (double)b.count[a] * (double)(b.count[a] - 1)
                                  : (double)b.count[a] * (double)b.count[c];
        const double r0 = (double)k * b.dr_A, r1 = (double)(k + 1) * b.dr_A;
        const double shell = 4.18879020478639098462 * (r1 * r1 * r1 - r0 * r0 * r0);
        const double denom = Pab * shell;
        g[i] = denom > 0.0 ? (float)((double)hist[i] * b.volume * inv_configs / denom) : 0.f;
    }
}

int launch_normalize_g(const BoxDev *boxes, int n_boxes, const unsigned long long *hist,
                       float *g, long long n_configs, long long hist_len, const long long *hist_box,
                       cudaStream_t stream)
{
    if (hist_len == 0) return EPSR_OK;
    const int grid = (int)((hist_len + 255) / 256 < 2048 ? (hist_len + 255) / 256 : 2048);
    normalize_g_kernel<<<grid, 256, 0, stream>>>(boxes, n_boxes, hist, g, 1.0 / (double)n_configs,
                                                 hist_len, hist_box);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "normalize_g");
}

// ---- total potential energy: pairs i < j in different molecules -----------------------------
constexpr int kUThreads = 256;
constexpr int kUR = kGrTile / kUThreads;

__global__ void __launch_bounds__(kUThreads, 2)
total_energy_kernel(const BoxDev *boxes, const int4 *coords, const int *atom_mol,
                    const long long *thresholds, const float *ep_all, const GrTile *tiles,
                    long long n_tiles, double *U)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    int4 *s_j = reinterpret_cast<int4 *>(dyn);
    int *s_mol = reinterpret_cast<int *>(s_j + kGrTile);
    long long *s_T = reinterpret_cast<long long *>(s_mol + kGrTile);
    __shared__ BoxDev bx;
    __shared__ int cur_box;
    __shared__ double s_red[kUThreads / 32];
    const int tid = threadIdx.x;
    if (tid == 0) cur_box = -1;
    __syncthreads();
    for (long long w = blockIdx.x; w < n_tiles; w += gridDim.x) {
        const GrTile tl = tiles[w];
        __syncthreads();
        if (tl.box != cur_box) {
            if (tid == 0) { bx = boxes[tl.box]; cur_box = tl.box; }
            __syncthreads();
            for (int k = tid; k <= bx.n_bins; k += kUThreads) s_T[k] = thresholds[bx.tbl_off + k];
        }
        const float *ep = ep_all + bx.ep_off;
        const int L = bx.L, N = bx.n_atoms;
        const int j0 = tl.tj * kGrTile, nj = min(kGrTile, N - j0);
        for (int j = tid; j < nj; j += kUThreads) {
            s_j[j] = coords[bx.atom0 + j0 + j];
            s_mol[j] = atom_mol[bx.atom0 + j0 + j];
        }
        const int i0 = tl.ti * kGrTile;
        int4 pi[kUR];
        int mi[kUR], il[kUR];
#pragma unroll
        for (int r = 0; r < kUR; ++r) {
            il[r] = tid + r * kUThreads;
            if (i0 + il[r] < N) {
                pi[r] = coords[bx.atom0 + i0 + il[r]];
                mi[r] = atom_mol[bx.atom0 + i0 + il[r]];
            } else {
                il[r] = -1;
                pi[r] = make_int4(0, 0, 0, 0);
                mi[r] = -1;
            }
        }
        const bool diag = tl.ti == tl.tj;
        __syncthreads();
        float acc = 0.f;
        for (int j = 0; j < nj; ++j) {
            const int4 pj = s_j[j];
            const int mj = s_mol[j];
#pragma unroll
            for (int r = 0; r < kUR; ++r) {
                if (il[r] < 0 || mi[r] == mj || (diag && j <= il[r])) continue;
                const PairRow pr = bx.row[pi[r].w * kMaxTypes + pj.w];
                acc += pair_u(sep(pi[r], pj, L), pr, bx, s_T, ep);
            }
        }
        double v = (double)acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int i = 0; i < kUThreads / 32; ++i) t += s_red[i];
            atomicAdd(&U[tl.box], t);
        }
    }
}

int launch_total_energy(const BoxDev *boxes, const int4 *coords, const int *atom_mol,
                        const long long *thresholds, const float *ep, const GrTile *tiles,
                        long long n_tiles, double *U, int grid, cudaStream_t stream)
{
    const size_t smem = (size_t)kGrTile * (sizeof(int4) + sizeof(int)) +
                        (size_t)(EPSR_MAX_BINS + 1) * sizeof(long long);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(total_energy_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(U)");
        attr_set = true;
    }
    total_energy_kernel<<<grid, kUThreads, smem, stream>>>(boxes, coords, atom_mol, thresholds, ep,
                                                           tiles, n_tiles, U);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "total_energy launch");
}

// Intra-molecular springs of flexible molecules (added to the total energy): one thread per
// molecule of box blockIdx.y, FP64.
__global__ void intra_energy_kernel(const BoxDev *boxes, const int4 *coords, const int *mol_start, double *U)
{
    const BoxDev &bx = boxes[blockIdx.y];
    if (bx.move_kind != EPSR_MOVE_FLEXIBLE_MOLECULE) return;
    double e = 0.0;
    for (int mol = blockIdx.x * blockDim.x + threadIdx.x; mol < bx.n_mol; mol += gridDim.x * blockDim.x) {
        const int a0 = mol_start[bx.mol0 + mol], a1 = mol_start[bx.mol0 + mol + 1];
        for (int i = a0; i < a1; ++i)
            for (int j = i + 1; j < a1; ++j) {
                const int4 pi = coords[bx.atom0 + i], pj = coords[bx.atom0 + j];
                const int t = pi.w * kMaxTypes + pj.w;
                if (bx.bond_k[t] == 0.0) continue;
                const double r = sqrt((double)dist2(pi, pj, bx.L) * (double)bx.inv_s2);
                e += bx.bond_k[t] * (r - bx.bond_d[t]) * (r - bx.bond_d[t]);
            }
    }
    if (e != 0.0) atomicAdd(&U[blockIdx.y], e);
}

int launch_intra_energy(const BoxDev *boxes, int n_boxes, const int4 *coords, const int *mol_start, double *U,
                        cudaStream_t stream)
{
    intra_energy_kernel<<<dim3(64, n_boxes), 256, 0, stream>>>(boxes, coords, mol_start, U);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "intra energy");
}

}  // namespace epsr
