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
// repeats; K <= 64). Warp w computes the partial dU of moves w, w + 16, w + 32 and w + 48
// against the slice as it stood at the start of the batch. One grid barrier per batch gathers the per-CTA partials; every
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
constexpr int kBatchMax = kMcBatchMax;         // moves per batch: warp w takes moves w, w + 16, w + 32, w + 48
constexpr int kPerWarp = kBatchMax / kMcWarps;  // moves per warp and batch
constexpr int kMoveBlock = 128;                // move records staged in shared memory at once
constexpr int kCorrItems = kMcCorrItems;       // >= 496 pairs x 8 atoms (coarse items at G = 1)
constexpr int kStageChunk = kMcStageChunk;     // partners per staged chunk (slices in global memory)
constexpr int kEscMax = 256;                   // escapee list capacity per CTA (at most)
constexpr int kEscFlag = (int)0x80000000u;     // bit 31 of a slice entry's .w: escapee
static_assert(kMcCorrPerCta == kBatchMax * (kBatchMax - 1) / 2 && kMcSlotStride == kBatchMax + kMcCorrPerCta,
              "barrier slot layout");
static_assert(kMcThreads == 8 * kBatchMax, "gather: 8 threads per move");
constexpr int kGatherLoads = 20;                // partials per gather thread in flight (CTA groups up to 160)
static_assert(kPerWarp == 4 && kBatchMax == 64, "phase A / F: two moves per lane of warp 0; phase B: the four moves of a warp in 8-lane groups");
static_assert(kMaxMolAtoms <= 8, "phase B: one lane per atom in 8-lane groups");

// ---- 1. configuration-independent part of each move ----------------------------------------
__global__ void mc_moves_kernel(const BoxDev *boxes, const int *mol_start, int n_boxes,
                                long long chunk, long long n, unsigned long long seed,
                                unsigned long long move0, MoveRec *out)
{
    const long long total = (long long)n_boxes * chunk;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / chunk);
        const long long t = e % chunk;
        if (t >= n) continue;
        const BoxDev &bx = boxes[b];
        const unsigned long long mv = move0 + (unsigned long long)t;
        const bool flex = bx.move_kind == EPSR_MOVE_FLEXIBLE_MOLECULE;
        uint32_t w[16];
#pragma unroll
        for (int lane = 0; lane < 4; ++lane) {
            if (lane == 3 && !flex) break;
            const U32x4 r = philox4x32_10((uint32_t)mv, (uint32_t)(mv >> 32), (uint32_t)b,
                                          (uint32_t)lane, (uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
            for (int i = 0; i < 4; ++i) w[4 * lane + i] = r.v[i];
        }
        MoveRec m;
        m.mol = (int)(((unsigned long long)w[0] * (unsigned long long)bx.n_mol) >> 32);
        m.a0 = mol_start[bx.mol0 + m.mol];
        m.m = mol_start[bx.mol0 + m.mol + 1] - m.a0;
        const unsigned span = 2u * (unsigned)bx.max_shift + 1u;
        for (int a = 0; a < 3; ++a) m.shift[a] = (int)(w[1 + a] % span) - bx.max_shift;
        // kind: 0 translate every atom, 1 rotate about the centre (then translate, for rigid
        // molecules), 2 translate one atom; flexible molecules draw the kind from w12 and the
        // atom from w13, and their rotations are not translated
        m.kind = flex ? (int)(w[12] % 3u) : (bx.move_kind == EPSR_MOVE_RIGID_MOLECULE ? 1 : 0);
        m.atom = flex ? (int)(w[13] % (uint32_t)m.m) : 0;
        if (flex && m.kind == 1) m.shift[0] = m.shift[1] = m.shift[2] = 0;
        if (m.kind == 1) {
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

int launch_mc_moves(const BoxDev *boxes, const int *mol_start, int n_boxes, long long chunk,
                    long long n, unsigned long long seed, unsigned long long move0, MoveRec *out,
                    cudaStream_t stream)
{
    const long long total = (long long)n_boxes * chunk;
    const int grid = (int)((total + 127) / 128 < 8192 ? (total + 127) / 128 : 8192);
    mc_moves_kernel<<<grid, 128, 0, stream>>>(boxes, mol_start, n_boxes, chunk, n, seed, move0, out);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EPSR_OK : set_cuda_error(e, "mc_moves");
}

// ---- 2. persistent sweep ----------------------------------------------------------------------
struct McShared {
    BoxDev bx;
    // batch records, double buffered by batch parity: the previous batch's accepted moves
    // are the "pending" updates whose global writes may not yet be visible
    int nb[2];
    int nb_min;                              // first move of the batch that repeats a molecule
    int mol[2][kBatchMax];
    int acc[2][kBatchMax];
    int4 newp[2][kBatchMax][kMaxMolAtoms];
    // current batch
    int4 oldp[kBatchMax][kMaxMolAtoms];
    int natoms[kBatchMax];
    int a0[kBatchMax];
    int spos[kBatchMax][kMaxMolAtoms];   // type-major sorted position of each moved atom
    int hw[kBatchMax];                   // half width of the near cube around old atom 0
    // first three atoms of each move on the 2^32-periodic grid, new and old: [move][atom][axis]
    unsigned scn[kBatchMax][3][3];
    unsigned sco[kBatchMax][3][3];
    // this CTA's partners: per type t, sorted positions [rs[t], rs[t] + rl[t]) held at
    // slice slots [blk[t], blk[t + 1])
    int rs[kMaxTypes];
    int rl[kMaxTypes];
    int blk[kMaxTypes + 1];
    float thr[kBatchMax];
    double u_acc[kBatchMax];
    float part[kBatchMax];
    float base[kBatchMax];
    float intra[kBatchMax];                 // flexible molecules: change of the springs
    int mm;                                  // largest molecule of the batch
    MoveRec mv[kMoveBlock];                  // staged move records [mv_base, mv_base + kMoveBlock)
    float acc_du[kMoveBlock];                // rank 0: dU of each decided move if accepted, else 0
    float dU[kBatchMax];
    int abort_flag;
    int cb[9];                               // cell boundaries ceil(j L / 8)
    int n_esc, cells_on;
    int esc[kEscMax];                        // escapee slots
    // leader-only running statistics
    long long st_att, st_acc, st_nonfinite;
    double st_sum;
};
static_assert(sizeof(McShared) + kMcMaxDynSmem <= 227 * 1024, "static plus dynamic shared memory per CTA");


__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp-wide FP64 sum of v[0..n) (lane-strided, then a fixed shuffle tree), added to acc by lane 0.
__device__ __forceinline__ void block_sum_du(const float *v, int n, int lane, double &acc)
{
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += (double)v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) acc += s;
}

// Correction of local pair u: the sum over atoms a of move k of the sum over atoms b of move
// k1 of [du(a; b new) - du(a; b old)], in that order. `fine` items hold each du separately;
// otherwise each item already holds the sum over b (same operations, same order).
// Metropolis test of a move with energy change d against its threshold thr = -kT ln u:
// accepted when d <= 0 or d < thr (Sec. 2.2); false for a NaN d.
__device__ __forceinline__ bool metropolis(float d, float thr) { return (d <= 0.f) || (d < thr); }

// Later move k of batch pair pq = k (k - 1) / 2 + k1 (0 <= k1 < k): a float estimate of
// the root of k (k - 1) / 2 = pq, corrected by one step either way.
__device__ __forceinline__ int pair_hi(int pq)
{
    int k = (int)((1.f + sqrtf(8.f * (float)pq + 1.f)) * 0.5f);
    if (k * (k - 1) / 2 > pq) --k;
    if ((k + 1) * k / 2 <= pq) ++k;
    return k;
}

__device__ __forceinline__ float corr_sum(const float *part, int u, int mm, bool fine)
{
    float c = 0.f;
    for (int a = 0; a < mm; ++a) {
        float ca = 0.f;
        if (fine)
            for (int b = 0; b < mm; ++b) {
                const float *v = part + ((u * mm + a) * mm + b) * 2;
                ca += v[0] - v[1];
            }
        else
            ca = part[u * mm + a];
        c += ca;
    }
    return c;
}

__device__ __forceinline__ int floordiv32(int a, int b)   // b > 0
{
    int q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

// ---- near-partner cells -------------------------------------------------------------------------
// A CTA's partners of each type are ordered by the cell of an 8^3 grid (cell k on an axis
// holds ceil(k L / 8) <= x < ceil((k + 1) L / 8)) as the sweep starts, so the partners
// inside a cube around a moved molecule lie in the slice ranges of the few cells the cube
// meets. Atoms move during the sweep: a partner that leaves its home cell widened by
// the cell margin is an escapee; it keeps its slot (flagged in bit 31 of .w) and joins a
// per-CTA list that every cell query scans in full. Cell queries cover the cube widened by
// the margin, so together with the escapees every partner inside the cube is found.

struct CellIndex {
    const unsigned *cst;         // [n_types][kMcCells + 1] first slot of each cell, relative to blk[t]
    const int *cb;               // [9] cell boundaries ceil(j L / 8), cb[8] = L
    const int *esc;              // escapee slots
    int n_esc;
    int margin;                  // drift (grid units) allowed before an atom becomes an escapee
    bool on;                     // cell queries allowed (escapee list not overflowed)
};

__device__ __forceinline__ int cell_of(int x, const int *cb)   // x in [0, L)
{
    int k = 0;
#pragma unroll
    for (int j = 1; j < 8; ++j) k += x >= cb[j] ? 1 : 0;
    return k;
}

// Cyclic run of cells [k0, k0 + n) (mod 8) meeting [c - w, c + w] on one axis.
__device__ __forceinline__ void cell_run(int c, long long w, int L, const int *cb, int &k0, int &n)
{
    if (8 * (2 * w + 1) >= 7LL * L) { k0 = 0; n = 8; return; }
    long long lo = c - w, hi = c + w;
    if (lo < 0) lo += L;
    if (hi >= L) hi -= L;
    k0 = cell_of((int)lo, cb);
    n = ((cell_of((int)hi, cb) - k0) & 7) + 1;
}

__device__ __forceinline__ unsigned spread3(unsigned v)   // bits 0..2 -> 0, 3, 6
{
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}

__device__ __forceinline__ unsigned compact3(unsigned v)  // bits 0, 3, 6 -> 0..2
{
    return (v & 1u) | ((v >> 2) & 2u) | ((v >> 4) & 4u);
}

__device__ __forceinline__ unsigned cell_code(int cx, int cy, int cz)
{
    return spread3((unsigned)cx) | (spread3((unsigned)cy) << 1) | (spread3((unsigned)cz) << 2);
}

// Is grid point x (one axis) within `margin` of cell k's interval (cyclically)?
__device__ __forceinline__ bool near_cell(int x, int k, const int *cb, int L, int margin)
{
    long long d = (long long)x - ((long long)cb[k] - margin);
    if (d < 0) d += L;
    if (d >= L) d -= L;
    return d < (long long)(cb[k + 1] - cb[k]) + 2LL * margin;
}

// Out-of-line copy of pair_du for code that runs once per batch (keeps the kernel small).
template <bool CUT>
__device__ __noinline__ float pair_du_cold(Sep sn, Sep so, const PairRow &pr, const BoxDev &bx,
                                           const long long *T, const float *ep)
{
    return pair_du<CUT>(sn, so, pr, bx, T, ep);
}

// Two FP32 values in one 64-bit register, operated on by the packed f32x2 instructions of
// sm_100 and later: one instruction for the same operation on the two partners of a lane.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Lennard-Jones change of two far partners (one f32x2 lane pair) from their packed separation
// components against a moved atom's new (XN, YN, ZN) and old (XO, YO, ZO) position, in units whose
// square S2 converts to A^2: the direct difference u(r') - u(r), and both squared distances of
// each partner in those units.
struct FarLJ {
    float d0, d1, g2n0, g2n1, g2o0, g2o1;
};
__device__ __forceinline__ FarLJ far_lj2_xyz(uint64_t XN, uint64_t YN, uint64_t ZN, uint64_t XO, uint64_t YO,
                                            uint64_t ZO, uint64_t S2, uint64_t C12, uint64_t NC6)
{
    const uint64_t G2N = f2_fma(XN, XN, f2_fma(YN, YN, f2_mul(ZN, ZN)));
    const uint64_t G2O = f2_fma(XO, XO, f2_fma(YO, YO, f2_mul(ZO, ZO)));
    FarLJ f;
    f2_unpack(G2N, f.g2n0, f.g2n1);
    f2_unpack(G2O, f.g2o0, f.g2o1);
    float r2n0, r2n1, r2o0, r2o1;
    f2_unpack(f2_mul(G2N, S2), r2n0, r2n1);
    f2_unpack(f2_mul(G2O, S2), r2o0, r2o1);
    const uint64_t AN = f2_pack(rsqrtf(r2n0), rsqrtf(r2n1)), AO = f2_pack(rsqrtf(r2o0), rsqrtf(r2o1));
    const uint64_t IN = f2_mul(AN, AN), IO = f2_mul(AO, AO);
    const uint64_t S6N = f2_mul(f2_mul(IN, IN), IN), S6O = f2_mul(f2_mul(IO, IO), IO);
    const uint64_t D = f2_sub(f2_mul(f2_fma(C12, S6N, NC6), S6N), f2_mul(f2_fma(C12, S6O, NC6), S6O));
    f2_unpack(D, f.d0, f.d1);
    return f;
}

// The same for two partners p and q on the 2^32-periodic grid (signed 32-bit differences).
__device__ __forceinline__ FarLJ far_lj2(uint4 p, uint4 q, unsigned nx, unsigned ny, unsigned nz, unsigned ox,
                                        unsigned oy, unsigned oz, uint64_t S2, uint64_t C12, uint64_t NC6)
{
    return far_lj2_xyz(f2_pack((float)(int)(p.x - nx), (float)(int)(q.x - nx)),
                       f2_pack((float)(int)(p.y - ny), (float)(int)(q.y - ny)),
                       f2_pack((float)(int)(p.z - nz), (float)(int)(q.z - nz)),
                       f2_pack((float)(int)(p.x - ox), (float)(int)(q.x - ox)),
                       f2_pack((float)(int)(p.y - oy), (float)(int)(q.y - oy)),
                       f2_pack((float)(int)(p.z - oz), (float)(int)(q.z - oz)), S2, C12, NC6);
}

// Lennard-Jones rows (bit a of lj: atom a of the move) against partners [j0, j1) of type t,
// added to acc in the order of a lane-strided scan, on the grid coordinates (integer minimum
// image). A lane takes two partners, j and j + 32, per step. A pair whose squared distances both
// exceed far2 has no Coulomb and no EP term, so its dU is the Lennard-Jones change alone, the
// direct difference computed for both partners at once in packed f32x2 arithmetic; a pair that
// is not that far takes the full pair_du (the cancellation-free form).
template <int M, bool CUT>
__device__ __forceinline__ float lj_rows(float acc, const int4 (&pn)[M], const int4 (&po)[M], unsigned lj, int a0,
                                         int m, const int4 *part, int j0, int j1, int t, const BoxDev &bx,
                                         const long long *T, const float *ep, int lane)
{
    const int L = bx.L;
    const float far2 = fmaxf(bx.rc2_hi, bx.has_ep ? bx.tmax_hi : 0.f);
    const uint64_t S2 = f2_pack(bx.inv_s2, bx.inv_s2);
    for (int j = j0 + lane; j < j1; j += 64) {
        const bool in1 = j + 32 < j1;
        const int4 p0 = part[j];
        const int4 p1 = part[in1 ? j + 32 : j];
        const int i0 = (p0.w & 0x7fffffff) >> 3, i1 = (p1.w & 0x7fffffff) >> 3;
        const bool v0 = !(i0 >= a0 && i0 < a0 + m);
        const bool v1 = in1 && !(i1 >= a0 && i1 < a0 + m);
#pragma unroll
        for (int a = 0; a < M; ++a) {
            if (a >= m || !((lj >> a) & 1u)) continue;
            const PairRow &r = bx.row[pn[a].w * kMaxTypes + t];
            const Sep n0 = sep(pn[a], p0, L), o0 = sep(po[a], p0, L);
            const Sep n1 = sep(pn[a], p1, L), o1 = sep(po[a], p1, L);
            const FarLJ f = far_lj2_xyz(f2_pack((float)n0.x, (float)n1.x), f2_pack((float)n0.y, (float)n1.y),
                                        f2_pack((float)n0.z, (float)n1.z), f2_pack((float)o0.x, (float)o1.x),
                                        f2_pack((float)o0.y, (float)o1.y), f2_pack((float)o0.z, (float)o1.z), S2,
                                        f2_pack(r.c12, r.c12), f2_pack(-r.c6, -r.c6));
            float d0 = f.d0, d1 = f.d1;
            const bool s0 = v0 && !(f.g2n0 > far2 && f.g2o0 > far2);
            const bool s1 = v1 && !(f.g2n1 > far2 && f.g2o1 > far2);
            if (s0 || s1) {
                if (s0) d0 = pair_du<CUT>(n0, o0, r, bx, T, ep);
                if (s1) d1 = pair_du<CUT>(n1, o1, r, bx, T, ep);
            }
            if (v0) acc += d0;
            if (v1) acc += d1;
        }
    }
    return acc;
}

// The Lennard-Jones rows of lj_rows on the 2^32-periodic copy of the slice (sx: {X, Y, Z,
// atom}, the moved atoms at qn/qo, [atom][axis]): a 32-bit difference wraps to the minimum
// image, so a separation component costs one subtraction and one conversion, and two
// partners share every FP32 instruction (f32x2). For single-atom moves a lane takes four
// partners per step (two independent packed pairs: the scan is latency-bound at 16 warps per
// SM), then two in the tail; for molecules (whose larger partner_sum the four-partner body
// slowed) two per step throughout. A far pair (both squared distances beyond the Coulomb
// cutoff and the EP table) has only the Lennard-Jones term, taken as the direct difference
// u(r') - u(r): its rounding is a few ulp of |u| there, where |u| is small. A pair that is not
// far takes pair_du on the exact grid slots (the cancellation-free form), one such partner of
// the lane after the other. The moved atoms with a Lennard-Jones row take the slice one after
// the other (water and single atoms have one such atom).
template <int M, bool CUT>
__device__ __forceinline__ float lj_rows_sc(float acc, const int4 *np, const int4 *op, const unsigned *qnp,
                                            const unsigned *qop, unsigned lj, int a0, int m, const int4 *slice,
                                            const uint4 *sx, int j0, int j1, int t, const BoxDev &bx,
                                            const long long *T, const float *ep, int lane)
{
    const int L = bx.L;
    const float far2 = fmaxf(bx.rc2_hi, bx.has_ep ? bx.tmax_hi : 0.f) * bx.sc_k2;
    const uint64_t S2 = f2_pack(bx.sc_s2, bx.sc_s2);
    for (int a = 0; a < m; ++a) {
        if (!((lj >> a) & 1u)) continue;
        const unsigned nx = qnp[3 * a], ny = qnp[3 * a + 1], nz = qnp[3 * a + 2];
        const unsigned ox = qop[3 * a], oy = qop[3 * a + 1], oz = qop[3 * a + 2];
        const PairRow &r = bx.row[np[a].w * kMaxTypes + t];
        const uint64_t C12 = f2_pack(r.c12, r.c12), NC6 = f2_pack(-r.c6, -r.c6);
        int j = j0 + lane;
        for (; M == 1 && j + 96 < j1; j += 128) {        // four partners: j, j + 32, j + 64, j + 96
            const uint4 p0 = sx[j], p1 = sx[j + 32], p2 = sx[j + 64], p3 = sx[j + 96];
            const FarLJ f = far_lj2(p0, p1, nx, ny, nz, ox, oy, oz, S2, C12, NC6);
            const FarLJ g = far_lj2(p2, p3, nx, ny, nz, ox, oy, oz, S2, C12, NC6);
            float d[4] = {f.d0, f.d1, g.d0, g.d1};
            const bool v0 = (unsigned)((int)p0.w - a0) >= (unsigned)m, v1 = (unsigned)((int)p1.w - a0) >= (unsigned)m;
            const bool v2 = (unsigned)((int)p2.w - a0) >= (unsigned)m, v3 = (unsigned)((int)p3.w - a0) >= (unsigned)m;
            unsigned nm = (v0 && !(f.g2n0 > far2 && f.g2o0 > far2) ? 1u : 0u) |
                          (v1 && !(f.g2n1 > far2 && f.g2o1 > far2) ? 2u : 0u) |
                          (v2 && !(g.g2n0 > far2 && g.g2o0 > far2) ? 4u : 0u) |
                          (v3 && !(g.g2n1 > far2 && g.g2o1 > far2) ? 8u : 0u);
            if (nm) {                                    // per lane: the loop's trip count differs by lane
                const int4 pn = np[a], po = op[a];
                while (nm) {
                    const int q = __ffs(nm) - 1;
                    nm &= nm - 1u;
                    const int4 pj = slice[j + 32 * q];
                    const float v = pair_du<CUT>(sep(pn, pj, L), sep(po, pj, L), r, bx, T, ep);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (u == q) d[u] = v;
                }
            }
            if (v0) acc += d[0];
            if (v1) acc += d[1];
            if (v2) acc += d[2];
            if (v3) acc += d[3];
        }
        for (; j < j1; j += 64) {                        // tail: two partners, j and j + 32
            const bool in1 = j + 32 < j1;
            const int jb = in1 ? j + 32 : j;
            const uint4 p0 = sx[j];
            const uint4 p1 = sx[jb];
            const bool v0 = (unsigned)((int)p0.w - a0) >= (unsigned)m;
            const bool v1 = in1 && (unsigned)((int)p1.w - a0) >= (unsigned)m;
            const FarLJ f = far_lj2(p0, p1, nx, ny, nz, ox, oy, oz, S2, C12, NC6);
            float d0 = f.d0, d1 = f.d1;
            const bool s0 = v0 && !(f.g2n0 > far2 && f.g2o0 > far2);
            const bool s1 = v1 && !(f.g2n1 > far2 && f.g2o1 > far2);
            if (s0 || s1) {
                const int4 pn = np[a], po = op[a];
                if (s0) {
                    const int4 pj = slice[j];
                    d0 = pair_du<CUT>(sep(pn, pj, L), sep(po, pj, L), r, bx, T, ep);
                }
                if (s1) {
                    const int4 pj = slice[jb];
                    d1 = pair_du<CUT>(sep(pn, pj, L), sep(po, pj, L), r, bx, T, ep);
                }
            }
            if (v0) acc += d0;
            if (v1) acc += d1;
        }
    }
    return acc;
}

// Near rows of one move against the partners of types ta (rows nra) and tb (rows nrb; tb < 0:
// none) found by a cell query: the ncell cells of the CTA's 8^3 grid that meet the cube around
// old atom 0 are taken one per lane, their runs for both types prefix-summed together (two
// independent shuffle chains), and the candidates of type ta, then of type tb, dealt out to the
// lanes; each candidate inside the cube (half width hw) adds its pair changes to acc.
template <int M, bool CUT>
__device__ __forceinline__ float cell_pairs(float acc, const int4 (&pn)[M], const int4 (&po)[M], int m, int a0,
                                            int hw, int4 o0, int ta, unsigned nra, int tb, unsigned nrb,
                                            const int4 *slice, const int *blk, const CellIndex &ci, int k0x, int nx,
                                            int k0y, int ny, int k0z, int ncell, const BoxDev &bx,
                                            const long long *T, const float *ep, int lane)
{
    const int L = bx.L;
    int fa = 0, na = 0, fb = 0, nb = 0;
    if (lane < ncell) {
        const int ix = lane % nx, iy = (lane / nx) % ny, iz = lane / (nx * ny);
        const unsigned code = cell_code((k0x + ix) & 7, (k0y + iy) & 7, (k0z + iz) & 7);
        const unsigned *ca = ci.cst + ta * (kMcCells + 1);
        fa = ca[code];
        na = ca[code + 1] - fa;
        if (tb >= 0) {
            const unsigned *cb = ci.cst + tb * (kMcCells + 1);
            fb = cb[code];
            nb = cb[code + 1] - fb;
        }
    }
    int ia = na, ib = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ya = __shfl_up_sync(0xffffffffu, ia, o);
        const int yb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ya;
            ib += yb;
        }
    }
    const int ea = ia - na, eb = ib - nb;
    const int tota = __shfl_sync(0xffffffffu, ia, 31), totb = __shfl_sync(0xffffffffu, ib, 31);
    const int total = tota + totb;
    for (int q0 = 0; q0 < total; q0 += 32) {
        const int q = q0 + lane;
        const bool isb = q >= tota;
        const int qq = isb ? q - tota : q;
        int c = 0;                                       // last cell whose run starts at or before qq
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int xa = __shfl_sync(0xffffffffu, ea, c + step);
            const int xb = __shfl_sync(0xffffffffu, eb, c + step);
            if (c + step < ncell && (isb ? xb : xa) <= qq) c += step;
        }
        const int cfa = __shfl_sync(0xffffffffu, fa, c), cea = __shfl_sync(0xffffffffu, ea, c);
        const int cfb = __shfl_sync(0xffffffffu, fb, c), ceb = __shfl_sync(0xffffffffu, eb, c);
        if (q < total) {
            const int t = isb ? tb : ta;
            const unsigned nr = isb ? nrb : nra;
            const int4 pj = slice[blk[t] + (isb ? cfb + (qq - ceb) : cfa + (qq - cea))];
            const int jatom = (pj.w & 0x7fffffff) >> 3;
            const bool take = pj.w >= 0 && !(jatom >= a0 && jatom < a0 + m) && mi_abs(pj.x - o0.x, L) < hw &&
                              mi_abs(pj.y - o0.y, L) < hw && mi_abs(pj.z - o0.z, L) < hw;
            if (take) {
#pragma unroll
                for (int a = 0; a < M; ++a)
                    if (a < m && ((nr >> a) & 1u))
                        acc += pair_du<CUT>(sep(pn[a], pj, L), sep(po[a], pj, L), bx.row[pn[a].w * kMaxTypes + t], bx,
                                            T, ep);
            }
        }
    }
    return acc;
}

// Partial dU of one move (atoms np/op, m <= M) against the partners of this CTA, lane-
// strided. Per partner type the kind of each moved atom's pair row is uniform across the
// warp: a Lennard-Jones row (LJ is not cut) is evaluated against every partner of the type;
// a row without LJ has Coulomb or empirical-potential terms only inside the near cube
// around old atom 0 (half width hw), so its partners come from a cell query when the cube
// meets at most 32 cells, else from the full scan with the cube test. M is a compile-time
// bound so the atom loop unrolls into independent dependency chains. SC: the slice has its
// 2^32-periodic copy sx and the moved atoms theirs (qn, qo), used by the Lennard-Jones rows.
template <int M, bool CELLS, bool CUT, bool SKIP_LJ = false, bool SC = false>
__device__ __forceinline__ float partner_sum(const int4 *np, const int4 *op, int m, int a0, int hw,
                                             const int4 *slice, const int *blk, const CellIndex &ci,
                                             const BoxDev &bx, const long long *T, const float *ep,
                                             int lane, const uint4 *sx = nullptr, const unsigned *qn = nullptr,
                                             const unsigned *qo = nullptr)
{
    const int L = bx.L;
    const int4 o0 = op[0];
    int4 pn[M], po[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        pn[a] = a < m ? np[a] : make_int4(0, 0, 0, 0);
        po[a] = a < m ? op[a] : make_int4(0, 0, 0, 0);
    }
    int k0x = 0, nx = 8, k0y = 0, ny = 8, k0z = 0, nz = 8;
    if (CELLS && ci.on) {
        const long long w = (long long)hw + ci.margin;
        cell_run(o0.x, w, L, ci.cb, k0x, nx);
        cell_run(o0.y, w, L, ci.cb, k0y, ny);
        cell_run(o0.z, w, L, ci.cb, k0z, nz);
    }
    const int ncell = nx * ny * nz;
    const bool use_cells = CELLS && ci.on && ncell <= 32;
    unsigned cell_types = 0u;
    int pend_t = -1;                                     // a type whose cell query waits for a second
    unsigned pend_nr = 0u;
    float acc = 0.f;
    for (int t = 0; t < bx.n_types; ++t) {
        unsigned lj = 0u, nr = 0u;
        const PairRow *pr[M];
#pragma unroll
        for (int a = 0; a < M; ++a) {
            pr[a] = &bx.row[pn[a].w * kMaxTypes + t];
            if (a >= m) continue;
            if (lj_full_row<CUT>(*pr[a], bx)) lj |= 1u << a;
            else if (near_row<CUT>(*pr[a], bx)) nr |= 1u << a;
        }
        if (SKIP_LJ) lj = 0u;                            // Lennard-Jones rows done by the caller
        if (!(lj | nr)) continue;
        const bool cells = nr && use_cells;
        const unsigned scan_nr = cells ? 0u : nr;
        if (lj && !scan_nr) {
            if (SC)
                acc = lj_rows_sc<M, CUT>(acc, np, op, qn, qo, lj, a0, m, slice, sx, blk[t], blk[t + 1], t, bx, T, ep,
                                         lane);
            else
                acc = lj_rows<M, CUT>(acc, pn, po, lj, a0, m, slice, blk[t], blk[t + 1], t, bx, T, ep, lane);
        } else if (lj | scan_nr) {
            const int jb = blk[t + 1];
#pragma unroll 2
            for (int j = blk[t] + lane; j < jb; j += 32) {
                int4 pj = slice[j];
                const int jatom = (pj.w & 0x7fffffff) >> 3;
                const bool self = jatom >= a0 && jatom < a0 + m;
                const bool near = scan_nr && mi_abs(pj.x - o0.x, L) < hw &&
                                  mi_abs(pj.y - o0.y, L) < hw && mi_abs(pj.z - o0.z, L) < hw;
#pragma unroll
                for (int a = 0; a < M; ++a) {
                    if (a < m && !self && (((lj >> a) & 1u) || (((scan_nr >> a) & 1u) && near)))
                        acc += pair_du<CUT>(sep(pn[a], pj, L), sep(po[a], pj, L), *pr[a], bx, T, ep);
                }
            }
        }
        if (CELLS && cells) {
            // cell queries of two partner types share one enumeration of the cells
            cell_types |= 1u << t;
            if (pend_t < 0) {
                pend_t = t;
                pend_nr = nr;
            } else {
                acc = cell_pairs<M, CUT>(acc, pn, po, m, a0, hw, o0, pend_t, pend_nr, t, nr, slice, blk, ci, k0x, nx,
                                         k0y, ny, k0z, ncell, bx, T, ep, lane);
                pend_t = -1;
            }
        }
    }
    if (CELLS && pend_t >= 0)
        acc = cell_pairs<M, CUT>(acc, pn, po, m, a0, hw, o0, pend_t, pend_nr, -1, 0u, slice, blk, ci, k0x, nx, k0y,
                                 ny, k0z, ncell, bx, T, ep, lane);
    // escapees of the types answered by cell queries (their LJ rows were in the full scans)
    if (CELLS && cell_types)
        for (int e = lane; e < ci.n_esc; e += 32) {
            const int4 pj = slice[ci.esc[e]];
            const int t = pj.w & 7;
            const int jatom = (pj.w & 0x7fffffff) >> 3;
            if (!((cell_types >> t) & 1u) || (jatom >= a0 && jatom < a0 + m)) continue;
            if (!(mi_abs(pj.x - o0.x, L) < hw && mi_abs(pj.y - o0.y, L) < hw && mi_abs(pj.z - o0.z, L) < hw))
                continue;
            for (int a = 0; a < m; ++a) {
                const PairRow &r = bx.row[np[a].w * kMaxTypes + t];
                if (near_row<CUT>(r, bx))
                    acc += pair_du_cold<CUT>(sep(np[a], pj, L), sep(op[a], pj, L), r, bx, T, ep);
            }
        }
    return acc;
}

// Lennard-Jones rows of one move against a staged chunk of partners of type t (the chunk
// is shared by all warps of the CTA; used when the slices live in global memory).
template <int M, bool CUT>
__device__ __forceinline__ float lj_chunk(const int4 *np, const int4 *op, int m, int a0, const int4 *stage,
                                          int nc, int t, const BoxDev &bx, const long long *T, const float *ep,
                                          int lane)
{
    unsigned lj = 0u;
    int4 pn[M], po[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
        pn[a] = a < m ? np[a] : make_int4(0, 0, 0, 0);
        po[a] = a < m ? op[a] : make_int4(0, 0, 0, 0);
        if (a < m) {
            const PairRow &r = bx.row[pn[a].w * kMaxTypes + t];
            if (lj_full_row<CUT>(r, bx)) lj |= 1u << a;
        }
    }
    if (!lj) return 0.f;
    return lj_rows<M, CUT>(0.f, pn, po, lj, a0, m, stage, 0, nc, t, bx, T, ep, lane);
}

// The same for any molecule size (atoms read from shared memory; out-of-line pair function).
template <bool CUT>
__device__ __noinline__ float partner_sum_any(const int4 *np, const int4 *op, int m, int a0, int hw,
                                              const int4 *slice, const int *blk, const BoxDev &bx,
                                              const long long *T, const float *ep, int lane)
{
    const int L = bx.L;
    const int4 o0 = op[0];
    float acc = 0.f;
    for (int t = 0; t < bx.n_types; ++t) {
        unsigned lj = 0u, nr = 0u;
        for (int a = 0; a < m; ++a) {
            const PairRow &pr = bx.row[np[a].w * kMaxTypes + t];
            if (lj_full_row<CUT>(pr, bx)) lj |= 1u << a;
            else if (near_row<CUT>(pr, bx)) nr |= 1u << a;
        }
        if (!(lj | nr)) continue;
        for (int j = blk[t] + lane; j < blk[t + 1]; j += 32) {
            int4 pj = slice[j];
            const int jatom = (pj.w & 0x7fffffff) >> 3;
            if (jatom >= a0 && jatom < a0 + m) continue;
            pj.w = t;
            const bool near = nr && mi_abs(pj.x - o0.x, L) < hw && mi_abs(pj.y - o0.y, L) < hw &&
                              mi_abs(pj.z - o0.z, L) < hw;
            const unsigned todo = lj | (near ? nr : 0u);
            for (int a = 0; a < m; ++a) {
                if ((todo >> a) & 1u) {
                    const int4 pn = np[a], po = op[a];
                    acc += pair_du_cold<CUT>(sep(pn, pj, L), sep(po, pj, L), bx.row[pn.w * kMaxTypes + t], bx, T, ep);
                }
            }
        }
    }
    return acc;
}

// GSLICE: the partner slices live in global memory ([grid][slice_cap], read through L1/L2)
// because they do not fit in shared memory; the thresholds, EP table and cell index stay
// in shared memory either way.
template <bool GSLICE, bool CUT>
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
        sh.nb_min = 1 << 30;
        sh.abort_flag = 0;
        sh.st_att = sh.st_acc = sh.st_nonfinite = 0;
        sh.st_sum = 0.0;
    }
    __syncthreads();
    const BoxDev &bx = sh.bx;

    const int G = bx.n_cta;
    const int rank = cta - bx.cta0;
    const int L = bx.L;
    const int nt = bx.n_types;
    // Partners of this CTA: the atoms i of the box with i mod G == rank (an even share of
    // every region and type), grouped by type and ordered in space within each type.
    if (tid == 0) {
        int b = 0;
        for (int t = 0; t < nt; ++t) {
            const int key0 = bx.mc_cell0 + (t * G + rank) * kMcCells;
            const int s0 = A.mc_offset[key0] - (int)bx.atom0;
            const int s1 = A.mc_offset[key0 + kMcCells] - (int)bx.atom0;
            sh.rs[t] = s0;
            sh.rl[t] = s1 - s0;
            sh.blk[t] = b;
            b += s1 - s0;
        }
        sh.blk[nt] = b;
    }
    __syncthreads();

    // shared memory: partner slice {x, y, z, type | atom << 3}, thresholds, empirical potential
    // (shared-memory slices: the slice, then its 2^32-periodic copy {X, Y, Z, atom})
    int4 *slice = GSLICE ? A.slice_g + (size_t)cta * A.slice_cap : reinterpret_cast<int4 *>(dyn);
    uint4 *sx = GSLICE ? nullptr : reinterpret_cast<uint4 *>(slice + A.slice_cap);
    long long *T = GSLICE ? reinterpret_cast<long long *>(dyn) : reinterpret_cast<long long *>(sx + A.slice_cap);
    float *ep = reinterpret_cast<float *>(T + A.tbl_cap);
    for (int t = 0; t < nt; ++t)
        for (int i = tid; i < sh.rl[t]; i += kMcThreads) {
            const int atom = A.sorted_index[bx.atom0 + sh.rs[t] + i] - (int)bx.atom0;
            int4 c = A.coords[bx.atom0 + atom];
            c.w = c.w | (atom << 3);
            slice[sh.blk[t] + i] = c;
            if (!GSLICE)
                sx[sh.blk[t] + i] = make_uint4(scale32(c.x, L, bx.sc_rcp), scale32(c.y, L, bx.sc_rcp),
                                               scale32(c.z, L, bx.sc_rcp), (unsigned)atom);
        }
    for (int k = tid; k <= bx.n_bins; k += kMcThreads) T[k] = A.thresholds[bx.tbl_off + k];
    if (bx.has_ep)
        for (int k = tid; k < bx.n_pairs * bx.n_bins; k += kMcThreads) ep[k] = A.ep[bx.ep_off + k];
    // cell index: first slot of each cell per type (relative to the type's block), the
    // home cell of every slot, cell boundaries; cell queries only where some pair row has
    // no Lennard-Jones term but a Coulomb or empirical-potential one
    unsigned *cst = reinterpret_cast<unsigned *>(ep + A.ep_cap);
    float (*corr)[kBatchMax] = reinterpret_cast<float (*)[kBatchMax]>(cst + A.types_cap * (kMcCells + 1));
    float *corr_part = &corr[kBatchMax][0];                                              // [kCorrItems]
    // GSLICE: staged chunk of partners [kStageChunk], on the next 16-byte boundary (the host
    // sizes the dynamic shared memory as the 16-byte-rounded tables plus the chunk)
    int4 *stage = reinterpret_cast<int4 *>((reinterpret_cast<uintptr_t>(corr_part + kCorrItems) + 15) &
                                           ~static_cast<uintptr_t>(15));
    unsigned short *home = GSLICE ? A.home_g + (size_t)cta * A.slice_cap
                                  : reinterpret_cast<unsigned short *>(corr_part + kCorrItems);
    for (int t = 0; t < nt; ++t) {
        const int key0 = bx.mc_cell0 + (t * G + rank) * kMcCells;
        for (int c = tid; c <= kMcCells; c += kMcThreads)
            cst[t * (kMcCells + 1) + c] = (unsigned)(A.mc_offset[key0 + c] - A.mc_offset[key0]);
    }
    if (tid <= 8) sh.cb[tid] = (int)(((long long)tid * L + 7) / 8);
    if (tid == 0) {
        bool near_rows = false;
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < nt; ++b) {
                const PairRow &r = bx.row[a * kMaxTypes + b];
                near_rows |= near_row<CUT>(r, bx);
            }
        sh.n_esc = 0;
        sh.cells_on = near_rows && A.esc_cap > 0 ? 1 : 0;
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
        const unsigned *ct = cst + t * (kMcCells + 1);
        for (int i = tid; i < sh.rl[t]; i += kMcThreads) {
            int c = 0;                                   // last cell starting at or before i
            for (int step = kMcCells / 2; step > 0; step >>= 1)
                if (ct[c + step] <= (unsigned)i) c += step;
            home[sh.blk[t] + i] = (unsigned short)c;
        }
    }
    __syncthreads();

    // moves per batch: as set, else 64 for large CTA groups (the per-batch phases amortise
    // over more moves), 32 for middling and 16 for small ones (corrections grow with the
    // square of the batch); above 32 only with 8 or more CTAs per box, so that a CTA's share
    // of the batch-pair corrections fits its item buffer
    const int batch_k = min(A.batch_k > 0 ? A.batch_k : (G >= 64 ? 64 : G >= 32 ? 32 : 16), G >= 8 ? kBatchMax : 32);
    const MoveRec *moves = A.moves + (size_t)box * A.chunk;
    unsigned seq = 0;
    int par = 0;

    long long mv_base = 0, mv_end = 0;
    for (long long t0 = 0; t0 < A.n_moves; par ^= 1) {
        const int kmax = (int)min((long long)batch_k, A.n_moves - t0);
        if (t0 + kmax > mv_end) {           // stage the next block of move records
            if (rank == 0 && warp == 0) block_sum_du(sh.acc_du, (int)(t0 - mv_base), lane, sh.st_sum);
            mv_base = t0;
            mv_end = min(A.n_moves, t0 + kMoveBlock);
            const int4 *src = reinterpret_cast<const int4 *>(moves + mv_base);
            int4 *dst = reinterpret_cast<int4 *>(sh.mv);
            const int n4 = (int)(mv_end - mv_base) * (int)(sizeof(MoveRec) / sizeof(int4));
            for (int i = tid; i < n4; i += kMcThreads) dst[i] = src[i];
            __syncthreads();
        }
        // ---- A. molecules of the batch; it ends before the first repeated molecule -----------
        // (every pair of the batch's candidate moves tested once, across the CTA)
        {
            const MoveRec *mv = sh.mv + (t0 - mv_base);
            for (int pq = tid; pq < kmax * (kmax - 1) / 2; pq += kMcThreads) {
                const int k = pair_hi(pq), k1 = pq - k * (k - 1) / 2;
                if (mv[k].mol == mv[k1].mol) atomicMin(&sh.nb_min, k);
            }
            if (tid < kBatchMax) sh.mol[par][tid] = tid < kmax ? mv[tid].mol : -1 - tid;
            if (tid == 0) sh.mm = 0;
        }
        __syncthreads();
        const int nb = min(kmax, sh.nb_min);
        if (tid == 0) sh.nb[par] = nb;
        // ---- B. current and trial coordinates of each moved molecule (integer arithmetic) ----
        // Current coordinates of a warp's four molecules: from the previous batch's accepted move
        // of the molecule if there is one (its global update may not be visible yet), else from
        // the global coordinates. The global loads of all four go out first (one round trip;
        // a value that a pending move replaces is loaded and dropped).
        {
            int4 gc[kPerWarp];
            int gp[kPerWarp];
            const int q = par ^ 1;
#pragma unroll
            for (int h = 0; h < kPerWarp; ++h) {
                const int k = warp + h * kMcWarps;
                gc[h] = make_int4(0, 0, 0, 0);
                gp[h] = 0;
                if (k < nb) {
                    const MoveRec &mr = sh.mv[t0 + k - mv_base];
                    if (lane < mr.m) {
                        gc[h] = __ldcg(&A.coords[bx.atom0 + mr.a0 + lane]);
                        gp[h] = A.pos_of[bx.atom0 + mr.a0 + lane];
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < kPerWarp; ++h) {
                const int k = warp + h * kMcWarps;
                if (k < nb) {
                    const MoveRec &mr = sh.mv[t0 + k - mv_base];
                    const int mol = sh.mol[par][k];
                    const bool hit0 = lane < sh.nb[q] && sh.acc[q][lane] && sh.mol[q][lane] == mol;
                    const bool hit1 = lane + 32 < sh.nb[q] && sh.acc[q][lane + 32] && sh.mol[q][lane + 32] == mol;
                    const unsigned h0 = __ballot_sync(0xffffffffu, hit0), h1 = __ballot_sync(0xffffffffu, hit1);
                    // molecules of a batch are distinct: at most one hit
                    const int pidx = h1 ? 63 - __clz(h1) : h0 ? 31 - __clz(h0) : -1;
                    if (lane < mr.m) {
                        sh.oldp[k][lane] = pidx >= 0 ? sh.newp[q][pidx][lane] : gc[h];
                        sh.spos[k][lane] = gp[h] - (int)bx.atom0;
                    }
                }
            }
            __syncwarp();
        }
        // Trial coordinates: the four moves of a warp at once, one per 8-lane group, one lane per
        // atom of the molecule (all three axes in the lane).
        {
            const int k = warp + (lane >> 3) * kMcWarps;
            const int kk = lane & 7;
            const bool act = k < nb;
            const MoveRec &mr = sh.mv[t0 + (act ? k : 0) - mv_base];
            const int a0 = mr.a0, m = act ? mr.m : 0;
            int4 np4 = make_int4(0, 0, 0, 0), op4 = make_int4(0, 0, 0, 0);
            if (kk < m) {
                const int4 *op = sh.oldp[k];
                op4 = op[kk];
                int nx, ny, nz;
                if (mr.kind == 1) {
                    // minimum-image offsets from atom 0, summed over the molecule, and this atom's own
                    const int4 b0 = op[0];
                    long long sx = 0, sy = 0, sz = 0, ox = 0, oy = 0, oz = 0;
                    for (int i = 0; i < m; ++i) {
                        const int4 c = op[i];
                        const long long dx = mi_signed((long long)c.x - b0.x, L);
                        const long long dy = mi_signed((long long)c.y - b0.y, L);
                        const long long dz = mi_signed((long long)c.z - b0.z, L);
                        sx += dx; sy += dy; sz += dz;
                        if (i == kk) { ox = dx; oy = dy; oz = dz; }
                    }
                    const long long ux = (long long)m * ox - sx, uy = (long long)m * oy - sy,
                                    uz = (long long)m * oz - sz;
                    const int *R = mr.R;
                    // per axis: s 2^30 + R (m o - s), then floor((. + m 2^29) / 2^30) (32 bits) and
                    // floor division by m
                    const long long numx = sx * 1073741824LL + (long long)R[0] * ux + (long long)R[1] * uy +
                                           (long long)R[2] * uz;
                    const long long numy = sy * 1073741824LL + (long long)R[3] * ux + (long long)R[4] * uy +
                                           (long long)R[5] * uz;
                    const long long numz = sz * 1073741824LL + (long long)R[6] * ux + (long long)R[7] * uy +
                                           (long long)R[8] * uz;
                    const long long half = (long long)m * 536870912LL;
                    nx = wrap_coord((long long)b0.x + floordiv32((int)((numx + half) >> 30), m) + mr.shift[0], L);
                    ny = wrap_coord((long long)b0.y + floordiv32((int)((numy + half) >> 30), m) + mr.shift[1], L);
                    nz = wrap_coord((long long)b0.z + floordiv32((int)((numz + half) >> 30), m) + mr.shift[2], L);
                } else {
                    const bool moved = mr.kind != 2 || kk == mr.atom;
                    nx = wrap_coord((long long)op4.x + (moved ? mr.shift[0] : 0), L);
                    ny = wrap_coord((long long)op4.y + (moved ? mr.shift[1] : 0), L);
                    nz = wrap_coord((long long)op4.z + (moved ? mr.shift[2] : 0), L);
                }
                np4 = make_int4(nx, ny, nz, op4.w);
                sh.newp[par][k][kk] = np4;
                if (!GSLICE && kk < 3) {
                    sh.scn[k][kk][0] = scale32(nx, L, bx.sc_rcp);
                    sh.scn[k][kk][1] = scale32(ny, L, bx.sc_rcp);
                    sh.scn[k][kk][2] = scale32(nz, L, bx.sc_rcp);
                    sh.sco[k][kk][0] = scale32(op4.x, L, bx.sc_rcp);
                    sh.sco[k][kk][1] = scale32(op4.y, L, bx.sc_rcp);
                    sh.sco[k][kk][2] = scale32(op4.z, L, bx.sc_rcp);
                }
            }
            __syncwarp();
            if (act && kk == 0) {
                // flexible molecules: change of the intra-molecular springs, written without
                // cancellation: k[(r' - d)^2 - (r - d)^2] = k (r' - r)(r' + r - 2d), with
                // r' - r = (r'^2 - r^2) / (r' + r) from the exact integer squared distances
                float di = 0.f;
                if (bx.move_kind == EPSR_MOVE_FLEXIBLE_MOLECULE)
                    for (int i = 0; i < m; ++i)
                        for (int j = i + 1; j < m; ++j) {
                            const int4 ni = sh.newp[par][k][i], nj = sh.newp[par][k][j];
                            const int t = ni.w * kMaxTypes + nj.w;
                            if (bx.bond_k[t] == 0.0) continue;
                            const long long d2n = dist2(ni, nj, L), d2o = dist2(sh.oldp[k][i], sh.oldp[k][j], L);
                            if (d2n == d2o) continue;
                            const float rn = sqrtf((float)d2n * bx.inv_s2), ro = sqrtf((float)d2o * bx.inv_s2);
                            const float dr = (float)(d2n - d2o) * bx.inv_s2 / (rn + ro);
                            di = fmaf((float)bx.bond_k[t] * dr, rn + ro - 2.f * (float)bx.bond_d[t], di);
                        }
                sh.intra[k] = di;
                atomicMax(&sh.mm, m);
                sh.natoms[k] = m;
                sh.a0[k] = a0;
                sh.thr[k] = mr.thr;
                sh.u_acc[k] = mr.u_acc;
            }
            // near cube: every old and new atom position lies within `reach` of old atom 0
            int reach = 0;
            if (kk < m) {
                const int4 o = sh.oldp[k][0];
                reach = max(max(mi_abs(op4.x - o.x, L), max(mi_abs(op4.y - o.y, L), mi_abs(op4.z - o.z, L))),
                            max(mi_abs(np4.x - o.x, L), max(mi_abs(np4.y - o.y, L), mi_abs(np4.z - o.z, L))));
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) reach = max(reach, __shfl_xor_sync(0xffffffffu, reach, o));
            if (act && kk == 0) sh.hw[k] = bx.near_fx + reach + 2;
        }
        __syncthreads();
        // ---- E. pair-energy corrections between the batch's moved molecules -----------------
        // Pair pq = (k1 < k) is computed by CTA pq mod G of the box's group, as items (pq, atom
        // a of move k) against the whole molecule of move k1, spread one per warp before the
        // partner sums; the per-pair sums travel with the partials through the grid barrier.
        // Items are (pair, a, b, side): atom a of move k (old and new) against atom b of
        // move k1 at its new (side 0) or old (side 1) position, one pair_du each, so a CTA's
        // share (18 items for water with G >= 120) runs as one warp's lanes in parallel.
        const int npq = nb * (nb - 1) / 2;
        const int mm = sh.mm;
        const int n_local = npq > rank ? (npq - rank + G - 1) / G : 0;
        const int n_items = n_local * mm * mm * 2;
        if (n_items <= kCorrItems) {
            for (int it = tid; it < n_items; it += kMcThreads) {
                const int side = it & 1, b = (it >> 1) % mm, a = ((it >> 1) / mm) % mm;
                const int pq = rank + ((it >> 1) / mm / mm) * G;
                const int k = pair_hi(pq);
                const int k1 = pq - k * (k - 1) / 2;
                float v = 0.f;
                if (a < sh.natoms[k] && b < sh.natoms[k1]) {
                    const int4 na = sh.newp[par][k][a], oa = sh.oldp[k][a];
                    const int4 p1 = side ? sh.oldp[k1][b] : sh.newp[par][k1][b];
                    v = pair_du<CUT>(sep(na, p1, L), sep(oa, p1, L), bx.row[na.w * kMaxTypes + p1.w], bx, T, ep);
                }
                corr_part[it] = v;
            }
        } else {                                  // large molecules and few CTAs: items (pair, a)
            for (int it = tid; it < n_local * mm; it += kMcThreads) {
                const int a = it % mm, pq = rank + (it / mm) * G;
                const int k = pair_hi(pq);
                const int k1 = pq - k * (k - 1) / 2;
                float ca = 0.f;
                if (a < sh.natoms[k]) {
                    const int4 na = sh.newp[par][k][a], oa = sh.oldp[k][a];
                    for (int b = 0; b < sh.natoms[k1]; ++b) {
                        const int4 nb1 = sh.newp[par][k1][b], ob1 = sh.oldp[k1][b];
                        const PairRow &pr = bx.row[na.w * kMaxTypes + nb1.w];
                        ca += pair_du_cold<CUT>(sep(na, nb1, L), sep(oa, nb1, L), pr, bx, T, ep) -
                              pair_du_cold<CUT>(sep(na, ob1, L), sep(oa, ob1, L), pr, bx, T, ep);
                    }
                }
                corr_part[it] = ca;
            }
        }
        const bool fine = n_items <= kCorrItems;
        // ---- C. partial dU of move `warp` against this CTA's slice ---------------------------
        if (GSLICE && sh.mm <= 3) {
            // slices in global memory: the Lennard-Jones partners are staged chunk by chunk in
            // shared memory and every warp scans each chunk for its moves, so a batch reads the
            // slice once instead of once per move; then each move's near-only rows
            float accL[kPerWarp];
#pragma unroll
            for (int q = 0; q < kPerWarp; ++q) accL[q] = 0.f;
            for (int t = 0; t < nt; ++t) {
                for (int c0 = sh.blk[t]; c0 < sh.blk[t + 1]; c0 += kStageChunk) {
                    const int nc = min(kStageChunk, sh.blk[t + 1] - c0);
                    __syncthreads();
                    for (int i = tid; i < nc; i += kMcThreads) stage[i] = __ldcg(&slice[c0 + i]);
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < kPerWarp; ++q) {
                        const int k = warp + q * kMcWarps;
                        if (k >= nb) continue;
                        const int m = sh.natoms[k];
                        accL[q] += m == 1 ? lj_chunk<1, CUT>(sh.newp[par][k], sh.oldp[k], 1, sh.a0[k], stage, nc, t, bx, T, ep, lane)
                                          : lj_chunk<3, CUT>(sh.newp[par][k], sh.oldp[k], m, sh.a0[k], stage, nc, t, bx, T, ep, lane);
                    }
                }
            }
            CellIndex ci;
            ci.cst = cst;
            ci.cb = sh.cb;
            ci.esc = sh.esc;
            ci.n_esc = min(sh.n_esc, A.esc_cap);
            ci.margin = A.cell_margin;
            ci.on = sh.cells_on != 0;
#pragma unroll
            for (int q = 0; q < kPerWarp; ++q) {
                const int k = warp + q * kMcWarps;
                if (k >= nb) continue;
                const int m = sh.natoms[k];
                float acc = accL[q];
                if (m == 1)
                    acc += ci.on ? partner_sum<1, true, CUT, true>(sh.newp[par][k], sh.oldp[k], 1, sh.a0[k], sh.hw[k],
                                                              slice, sh.blk, ci, bx, T, ep, lane)
                                 : partner_sum<1, false, CUT, true>(sh.newp[par][k], sh.oldp[k], 1, sh.a0[k], sh.hw[k],
                                                               slice, sh.blk, ci, bx, T, ep, lane);
                else
                    acc += ci.on ? partner_sum<3, true, CUT, true>(sh.newp[par][k], sh.oldp[k], m, sh.a0[k], sh.hw[k],
                                                              slice, sh.blk, ci, bx, T, ep, lane)
                                 : partner_sum<3, false, CUT, true>(sh.newp[par][k], sh.oldp[k], m, sh.a0[k], sh.hw[k],
                                                               slice, sh.blk, ci, bx, T, ep, lane);
                acc = warp_sum(acc);
                if (lane == 0) sh.part[k] = acc;
            }
        } else
        for (int k = warp; k < nb; k += kMcWarps) {
            const int m = sh.natoms[k];
            float acc;
            CellIndex ci;
            ci.cst = cst;
            ci.cb = sh.cb;
            ci.esc = sh.esc;
            ci.n_esc = min(sh.n_esc, A.esc_cap);
            ci.margin = A.cell_margin;
            ci.on = sh.cells_on != 0;
            const unsigned *qn = &sh.scn[k][0][0], *qo = &sh.sco[k][0][0];
            if (m == 1)
                acc = ci.on ? partner_sum<1, true, CUT, false, !GSLICE>(sh.newp[par][k], sh.oldp[k], 1, sh.a0[k],
                                                                      sh.hw[k], slice, sh.blk, ci, bx, T, ep, lane,
                                                                      sx, qn, qo)
                            : partner_sum<1, false, CUT, false, !GSLICE>(sh.newp[par][k], sh.oldp[k], 1, sh.a0[k],
                                                                       sh.hw[k], slice, sh.blk, ci, bx, T, ep, lane,
                                                                       sx, qn, qo);
            else if (m <= 3)
                acc = ci.on ? partner_sum<3, true, CUT, false, !GSLICE>(sh.newp[par][k], sh.oldp[k], m, sh.a0[k],
                                                                      sh.hw[k], slice, sh.blk, ci, bx, T, ep, lane,
                                                                      sx, qn, qo)
                            : partner_sum<3, false, CUT, false, !GSLICE>(sh.newp[par][k], sh.oldp[k], m, sh.a0[k],
                                                                       sh.hw[k], slice, sh.blk, ci, bx, T, ep, lane,
                                                                       sx, qn, qo);
            else
                acc = partner_sum_any<CUT>(sh.newp[par][k], sh.oldp[k], m, sh.a0[k], sh.hw[k],
                                      slice, sh.blk, bx, T, ep, lane);
            acc = warp_sum(acc);
            if (lane == 0) sh.part[k] = acc;
        }
        __syncthreads();
        // ---- D. gather the partials of the box's CTA group (one bounded grid barrier) -------
        // Slot buffer, per parity: partials [kBatchMax][grid] (one move's partials of the group
        // are contiguous), then corrections, the box's pair pq at cta0 * kMcCorrPerCta + pq.
        // Arrival: warp 0 writes the CTA's partials and corrections in parallel, then lane 0
        // makes a release add on the group's counter and polls it with acquire loads (the warp
        // barrier orders the other lanes' writes before the release, which is cumulative; the
        // CTA barrier after the poll orders every thread's reads after the acquire).
        ++seq;
        const int gk = tid >> 3, gsub = tid & 7;     // gather group: move gk, member gsub
        const bool gin = gk < nb;
        float cv[8];                                  // corrections (j, gk), j = gsub + 8 i < gk
        float gv = 0.f, gw = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) cv[i] = 0.f;
        if (G > 1) {
            float *ps = A.slots + (size_t)(seq & 1u) * A.grid * kMcSlotStride;
            float *cs = ps + (size_t)kBatchMax * A.grid + (size_t)bx.cta0 * kMcCorrPerCta;
            if (warp == 0) {
                const bool arrive = cta != A.skip_arrival_cta;
                if (arrive) {
                    for (int k = lane; k < nb; k += 32) ps[(size_t)k * A.grid + cta] = sh.part[k];
                    for (int u = lane; u < n_local; u += 32) cs[rank + u * G] = corr_sum(corr_part, u, mm, fine);
                }
                __syncwarp();
                if (lane == 0) {
                    if (arrive) red_add_release_gpu(&A.flags[box], 1u);
                    const unsigned target = seq * (unsigned)G;
                    const uint64_t t_start = globaltimer_ns();
                    long long it = 0;
                    bool timed_out = false;
                    while (ld_acquire_gpu(&A.flags[box]) < target) {
                        if ((++it & 255) == 0 &&
                            ((globaltimer_ns() - t_start > A.timeout_ns) || it > A.max_spin ||
                             ld_relaxed_gpu(A.status) != 0)) {
                            timed_out = true;
                            break;
                        }
                    }
                    if (timed_out) {
                        atomicOr(A.status, kStatusTimeout);
                        sh.abort_flag = 1;
                    }
                }
            }
            __syncthreads();
            if (sh.abort_flag) return;
            // 8 threads per move k: every 8th CTA's partial and every 8th correction (j, k),
            // j < k, all loads in flight at once (one L2 round trip)
            if (gin) {
                const float *pk = ps + (size_t)gk * A.grid + bx.cta0;
                const float *ck = cs + gk * (gk - 1) / 2;
                float pv[kGatherLoads];
#pragma unroll
                for (int i = 0; i < kGatherLoads; ++i) {
                    const int r = gsub + 8 * i;
                    pv[i] = r < G ? __ldcg(&pk[r]) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int j = gsub + 8 * i;
                    cv[i] = j < gk ? __ldcg(&ck[j]) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < kGatherLoads; ++i) gv += pv[i];
                for (int r = gsub + 8 * kGatherLoads; r < G; r += 8) gv += __ldcg(&pk[r]);
            }
        } else if (gin) {
            gv = gsub == 0 ? sh.part[gk] : 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int j = gsub + 8 * i;
                cv[i] = j < gk ? corr_sum(corr_part, gk * (gk - 1) / 2 + j, mm, fine) : 0.f;
            }
        }
        // the group's sums in a fixed shuffle tree (the same order in every run): the move's
        // partial dU and the magnitude sum of its corrections
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int j = gsub + 8 * i;
            if (gin && j < gk) corr[j][gk] = cv[i];
            gw += fabsf(cv[i]);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            gv += __shfl_xor_sync(0xffffffffu, gv, o);
            gw += __shfl_xor_sync(0xffffffffu, gw, o);
        }
        // ---- F. Metropolis decisions of the batch, in order: move k's dU includes the
        // corrections of every earlier accepted move. Fast path: when no move's decision can
        // change with any subset of its earlier corrections (|dU - threshold| beyond the sum of
        // their magnitudes plus the FP32 rounding of that many additions), every group decides
        // its move at once and then adds its accepted corrections (fixed tree order); otherwise
        // warp 0 decides one move after the other (lane l holds moves l and l + 32) and adds
        // the corrections in the chain's order. Both give the same decisions.
        {
            const float d = gin ? gv + sh.intra[gk] : 0.f;
            const float thr = gin ? sh.thr[gk] : 0.f;
            const float wv = gw + (fabsf(d) + gw) * 0x1p-16f;
            const bool sure = !gin || metropolis(d + wv, thr) || !metropolis(d - wv, thr);
            if (gin && gsub == 0) sh.base[gk] = gv;
            if (__syncthreads_and(sure)) {
                const bool acc = gin && metropolis(d, thr);
                if (gin && gsub == 0) sh.acc[par][gk] = acc;
                __syncthreads();
                float c = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int j = gsub + 8 * i;
                    if (j < gk && sh.acc[par][j]) c += cv[i];
                }
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                if (gin && gsub == 0) sh.dU[gk] = d + c;
            } else if (warp == 0) {
                const bool in0 = lane < nb, in1 = lane + 32 < nb;
                float d0 = in0 ? sh.base[lane] + sh.intra[lane] : 0.f;
                float d1 = in1 ? sh.base[lane + 32] + sh.intra[lane + 32] : 0.f;
                const float thr0 = in0 ? sh.thr[lane] : 0.f, thr1 = in1 ? sh.thr[lane + 32] : 0.f;
                int acc0 = 0, acc1 = 0;
#pragma unroll 8
                for (int j = 0; j < 32; ++j) {
                    if (j < nb) {
                        const float c0 = corr[j][lane], c1 = corr[j][lane + 32];
                        const int aj = __shfl_sync(0xffffffffu, metropolis(d0, thr0), j);
                        if (lane == j) acc0 = aj;
                        if (aj) {
                            if (lane > j) d0 += c0;
                            d1 += c1;
                        }
                    }
                }
#pragma unroll 8
                for (int j = 32; j < kBatchMax; ++j) {
                    if (j < nb) {
                        const float c1 = corr[j][lane + 32];
                        const int aj = __shfl_sync(0xffffffffu, metropolis(d1, thr1), j - 32);
                        if (lane == j - 32) acc1 = aj;
                        if (aj && lane + 32 > j) d1 += c1;
                    }
                }
                if (in0) {
                    sh.dU[lane] = d0;
                    sh.acc[par][lane] = acc0;
                }
                if (in1) {
                    sh.dU[lane + 32] = d1;
                    sh.acc[par][lane + 32] = acc1;
                }
            }
        }
        __syncthreads();
        if (rank == 0 && warp == 0) {
            // counts now; the FP64 sum of accepted dU once per staged block of moves
            const bool in0 = lane < nb, in1 = lane + 32 < nb;
            const bool acc0 = in0 && sh.acc[par][lane], acc1 = in1 && sh.acc[par][lane + 32];
            const float d0 = in0 ? sh.dU[lane] : 0.f, d1 = in1 ? sh.dU[lane + 32] : 0.f;
            const unsigned b_acc = __ballot_sync(0xffffffffu, acc0), b_acc1 = __ballot_sync(0xffffffffu, acc1);
            const unsigned b_nf = __ballot_sync(0xffffffffu, in0 && !isfinite(d0)),
                           b_nf1 = __ballot_sync(0xffffffffu, in1 && !isfinite(d1));
            if (in0) sh.acc_du[t0 - mv_base + lane] = acc0 ? d0 : 0.f;
            if (in1) sh.acc_du[t0 - mv_base + lane + 32] = acc1 ? d1 : 0.f;
            if (lane == 0) {
                sh.st_att += nb;
                sh.st_acc += __popc(b_acc) + __popc(b_acc1);
                sh.st_nonfinite += __popc(b_nf) + __popc(b_nf1);
            }
        }
        // ---- G. apply accepted moves: shared slice, global coordinates, log ------------------
        for (int it = tid; it < nb * kMaxMolAtoms; it += kMcThreads) {
            const int k = it / kMaxMolAtoms, a = it % kMaxMolAtoms;
            if (!sh.acc[par][k] || a >= sh.natoms[k]) continue;
            const int ja = sh.a0[k] + a;
            const int4 p = sh.newp[par][k][a];
            const int t = p.w, sp = sh.spos[k][a] - sh.rs[t];
            if (sp >= 0 && sp < sh.rl[t]) {
                const int slot = sh.blk[t] + sp;
                int w = t | (ja << 3);
                if (sh.cells_on) {
                    bool esc = slice[slot].w < 0;
                    if (!esc) {
                        const unsigned h = home[slot];
                        esc = !(near_cell(p.x, (int)compact3(h), sh.cb, L, A.cell_margin) &&
                                near_cell(p.y, (int)compact3(h >> 1), sh.cb, L, A.cell_margin) &&
                                near_cell(p.z, (int)compact3(h >> 2), sh.cb, L, A.cell_margin));
                        if (esc) {
                            const int e = atomicAdd(&sh.n_esc, 1);
                            if (e < A.esc_cap) sh.esc[e] = slot;
                            else sh.cells_on = 0;            // too many: full scans from now on
                        }
                    }
                    if (esc) w |= kEscFlag;
                }
                slice[slot] = make_int4(p.x, p.y, p.z, w);
                if (!GSLICE)
                    sx[slot] = make_uint4(scale32(p.x, L, bx.sc_rcp), scale32(p.y, L, bx.sc_rcp),
                                          scale32(p.z, L, bx.sc_rcp), (unsigned)ja);
            }
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
        if (tid == 0) sh.nb_min = 1 << 30;      // every thread read it before phase B
        __syncthreads();
        t0 += nb;
    }

    if (rank == 0 && warp == 0) block_sum_du(sh.acc_du, (int)(A.n_moves - mv_base), lane, sh.st_sum);
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
    // instantiations: partner slices in shared or global memory x Lennard-Jones uncut or cut
    const void *fns[2][2] = {{(const void *)mc_sweep_kernel<false, false>, (const void *)mc_sweep_kernel<false, true>},
                             {(const void *)mc_sweep_kernel<true, false>, (const void *)mc_sweep_kernel<true, true>}};
    static bool attr_set = false;
    if (!attr_set) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                cudaError_t e = cudaFuncSetAttribute(fns[i][j], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)kMcMaxDynSmem);
                if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute(mc)");
            }
        attr_set = true;
    }
    const void *fn = fns[args.slice_g ? 1 : 0][args.lj_cut ? 1 : 0];
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMcThreads, smem);
    if (e != cudaSuccess) return set_cuda_error(e, "occupancy(mc)");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm * sms < grid)
        return set_error(EPSR_ELAUNCH, "mc sweep: %d CTAs cannot be co-resident (%d per SM x %d SMs)",
                         grid, per_sm, sms);
    McArgs a = args;
    void *params[] = {&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kMcThreads), params, smem, stream);
    if (e == cudaErrorCooperativeLaunchTooLarge)
        return set_error(EPSR_ELAUNCH, "mc sweep: cooperative launch of %d CTAs refused", grid);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaLaunchCooperativeKernel(mc)");
    note_launch();
    return EPSR_OK;
}

int mc_threads() { return kMcThreads; }
int mc_escapee_max() { return kEscMax; }
int mc_batch_max() { return kBatchMax; }

}  // namespace epsr
