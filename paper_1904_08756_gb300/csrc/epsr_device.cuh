// epsr_device.cuh -- device-side data layout and helpers of libepsr (sm_103a).
//
// Box state lives in HBM as one int4 per atom {x, y, z, type} on the fixed-point grid
// (16 B/atom, coalesced 128-bit loads); per-box parameters are a POD struct that each
// CTA copies into shared memory. Squared distances are exact 64-bit integers; histogram
// bins come from a float estimate corrected against an exact integer threshold table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "epsr.h"

namespace epsr {

constexpr int kMaxTypes = EPSR_MAX_TYPES;
constexpr int kMaxPairs = kMaxTypes * (kMaxTypes + 1) / 2;
constexpr int kMaxMolAtoms = EPSR_MAX_MOL_ATOMS;

// Per-type-pair force-field row, indexed [ta * kMaxTypes + tb]: LJ 12 and 6 coefficients
// (4 eps sigma^12, 4 eps sigma^6 in kJ/mol A^12 / A^6), Coulomb k_e q_a q_b (kJ A/mol) and
// the pair index (upper-triangle order) as an int in the last lane.
struct __align__(16) PairRow {
    float c12, c6, kqq;
    int pair;
};

struct BoxDev {
    int64_t atom0;        // first atom of this box in the concatenated arrays
    int64_t mol0;         // first entry of this box's mol_start block
    int64_t hist_off;     // first element of this box's histogram block
    int64_t rc2;          // (llround(r_coul * S))^2, grid units^2
    int64_t tmax;         // threshold of bin n_bins: d2 < tmax <=> inside the table
    int32_t n_atoms, n_mol;
    int32_t L;            // box side, grid units
    int32_t n_types, n_pairs, n_bins;
    int32_t move_kind, max_shift;
    int32_t tbl_off;      // offset of the n_bins+1 thresholds
    int32_t ep_off;       // offset of the n_pairs * n_bins empirical potential
    int32_t has_ep;       // 0 while the empirical potential is identically zero
    int32_t cta0, n_cta;  // CTA group of the Monte Carlo kernel
    int32_t chunk;        // partner atoms per CTA of the group
    double h_rot;         // tan(max_rotation / 2) / sqrt(3)
    double kT;            // kJ/mol
    double volume;        // A^3
    double dr_A;          // bin width in Angstrom (bin_p / bin_q)
    float inv_s2;         // 2^(-2 scale_log2): grid units^2 -> A^2
    float inv_dr_fx;      // 1 / (bin width in grid units)
    uint32_t pre_r;       // g(r) prefilter half width on the 2^32-periodic scaled grid
    uint32_t pre16_bias;  // all-pairs histogram prefilter on the 2^16-periodic grid: bias B = R16 + 1
    uint32_t pre16_t;     // threshold T = 2 R16 + 1 in both halfwords
    int32_t pre16_all;    // 1: the cube covers the whole period (every pair takes the exact path)
    int32_t cells;        // spatial-sort cells per side (g(r) work order)
    float rc2_lo, rc2_hi; // rc2 * (1 -/+ 2^-20) as floats: the exact test runs only between
    float tmax_lo, tmax_hi;   // tmax * (1 -/+ 2^-20)
    int32_t cell0;        // first global cell of this box (spatial sort)
    int32_t cells_p3;     // cells per box in the sort key space (power of two cubed)
    int32_t mc_cell0;     // first key of this box in the type-major sort
    int32_t near_fx;      // ceil(sqrt(max(rc2, tmax if an EP is set, lj2 if LJ is cut))), grid units
    int32_t lj_cut;       // 1: Lennard-Jones truncated at d2 < lj2; 0: over every pair
    int64_t lj2;          // (llround(r_lj * S))^2, grid units^2
    float lj2_lo, lj2_hi; // lj2 * (1 -/+ 2^-20)
    int32_t gc_n;         // cell-list histogram: cells per side (>= 3, each at least the
                          // histogram range wide), or 0 when the box is too small for it
    int32_t gc0;          // first key of this box in the cell-list sort
    uint64_t sc_rcp;      // floor((2^64 - 1) / L): grid coordinate -> 2^32-periodic coordinate
    float sc_s2;          // A^2 per squared unit of the 2^32-periodic grid, (L / 2^32)^2 inv_s2
    float sc_k2;          // squared units of the 2^32-periodic grid per grid unit^2, (2^32 / L)^2
    int32_t type_start[kMaxTypes];  // first type-major sorted position of each type (box-local)
    int64_t count[kMaxTypes];   // atoms per type
    PairRow row[kMaxTypes * kMaxTypes];
    // flexible molecules: intra-molecular spring constant and reference distance per type pair
    double bond_k[kMaxTypes * kMaxTypes];
    double bond_d[kMaxTypes * kMaxTypes];
};

__host__ __device__ __forceinline__ int pair_index(int a, int b, int n_types)
{
    if (a > b) { int t = a; a = b; b = t; }
    return a * n_types - a * (a - 1) / 2 + (b - a);
}

// |minimum image| of a coordinate difference d in (-L, L): min(|d|, L - |d|).
__device__ __forceinline__ int mi_abs(int d, int L)
{
    int a = abs(d);
    return min(a, L - a);
}

// Non-negative minimum-image separation components of two grid points (exact int32).
struct Sep {
    int x, y, z;
};

__device__ __forceinline__ Sep sep(int4 a, int4 b, int L)
{
    Sep s;
    s.x = mi_abs(a.x - b.x, L);
    s.y = mi_abs(a.y - b.y, L);
    s.z = mi_abs(a.z - b.z, L);
    return s;
}

// floor(x 2^32 / L) for 0 <= x < L: the coordinate on the 2^32-periodic grid, on which the
// 32-bit difference of two coordinates wraps to the minimum image by itself. The product with
// rcp = floor((2^64 - 1) / L) is that quotient or one less; one exact test corrects it.
__device__ __forceinline__ unsigned scale32(int x, int L, uint64_t rcp)
{
    const uint64_t n = (uint64_t)(unsigned)x << 32;
    uint64_t q = __umul64hi(n, rcp);
    if ((q + 1) * (uint64_t)(unsigned)L <= n) ++q;
    return (unsigned)q;
}

// Exact squared distance (grid units^2); 64-bit products, used only off the fast path.
__device__ __forceinline__ long long d2_of(Sep s)
{
    return (long long)s.x * s.x + (long long)s.y * s.y + (long long)s.z * s.z;
}

// Squared distance in grid units^2 as FP32 from the int32 components (32-bit conversions
// only: a 64-bit integer conversion would run on the FP64 unit). Relative error < 2^-22.
__device__ __forceinline__ float g2_of(Sep s)
{
    const float fx = (float)s.x, fy = (float)s.y, fz = (float)s.z;
    return fmaf(fx, fx, fmaf(fy, fy, fz * fz));
}

__device__ __forceinline__ long long dist2(int4 a, int4 b, int L) { return d2_of(sep(a, b, L)); }

// Exact d2 < lim, decided from the FP32 estimate g2 unless it lies within a relative
// 2^-20 of the limit (lo, hi are lim * (1 -/+ 2^-20)).
__device__ __forceinline__ bool below(float g2, Sep s, long long lim, float lo, float hi)
{
    if (g2 < lo) return true;
    if (g2 > hi) return false;
    return d2_of(s) < lim;
}

// Largest k with T[k] <= d2, for d2 < T[n_bins]: a float guess from g2 ~ d2, corrected
// against the exact threshold table.
__device__ __forceinline__ int bin_of(long long d2, float g2, const long long *T, int n_bins,
                                      float inv_dr_fx)
{
    int k = (int)(sqrtf(g2) * inv_dr_fx);
    k = max(0, min(k, n_bins - 1));
    while (k > 0 && T[k] > d2) --k;
    while (T[k + 1] <= d2) ++k;
    return k;
}

// A pair row whose Lennard-Jones term reaches every partner (LJ not cut): evaluated against
// the whole slice. Any other row with a term is "near": non-zero only within near_fx of the
// moved atom, so its partners can come from cell queries. CUT = false compiles the form
// without a cutoff (boxes with r_lj = 0); CUT = true reads the box's setting.
template <bool CUT = true>
__device__ __forceinline__ bool lj_full_row(const PairRow &r, const BoxDev &bx)
{
    return (r.c12 != 0.f || r.c6 != 0.f) && !(CUT && bx.lj_cut);
}

template <bool CUT = true>
__device__ __forceinline__ bool near_row(const PairRow &r, const BoxDev &bx)
{
    return !lj_full_row<CUT>(r, bx) && (r.c12 != 0.f || r.c6 != 0.f || r.kqq != 0.f || bx.has_ep);
}

// Pair energy of a separation (FP32; Sec. 2.1: reference potential + empirical
// potential). Coincident points have +inf energy.
__device__ __forceinline__ float pair_u(Sep s, const PairRow &pr, const BoxDev &bx,
                                        const long long *T, const float *ep)
{
    const float g2 = g2_of(s);
    if (g2 == 0.f) return __int_as_float(0x7f800000);
    const float r2 = g2 * bx.inv_s2;
    const float a = rsqrtf(r2);
    float u = 0.f;
    if ((pr.c12 != 0.f || pr.c6 != 0.f) && (!bx.lj_cut || below(g2, s, bx.lj2, bx.lj2_lo, bx.lj2_hi))) {
        const float i2 = a * a;
        const float s6 = i2 * i2 * i2;
        u = fmaf(pr.c12, s6, -pr.c6) * s6;
    }
    if (below(g2, s, bx.rc2, bx.rc2_lo, bx.rc2_hi)) u = fmaf(pr.kqq, a, u);
    if (bx.has_ep && g2 < bx.tmax_hi && below(g2, s, bx.tmax, bx.tmax_lo, bx.tmax_hi))
        u += ep[pr.pair * bx.n_bins + bin_of(d2_of(s), g2, T, bx.n_bins, bx.inv_dr_fx)];
    return u;
}

// The part of u(r') - u(r) shared by every term: squared distances in grid units, r^2 and
// r'^2 in A^2, their difference r^2 - r'^2 from the exact integer factors, and 1/r, 1/r'.
struct DuCore {
    float g2n, g2o, r2n, r2o, dr2, an, ao;
};

__device__ __forceinline__ DuCore du_core(Sep sn, Sep so, float inv_s2)
{
    const float fxn = (float)sn.x, fyn = (float)sn.y, fzn = (float)sn.z;
    const float fxo = (float)so.x, fyo = (float)so.y, fzo = (float)so.z;
    DuCore c;
    c.g2n = fmaf(fxn, fxn, fmaf(fyn, fyn, fzn * fzn));
    c.g2o = fmaf(fxo, fxo, fmaf(fyo, fyo, fzo * fzo));
    c.r2n = c.g2n * inv_s2;
    c.r2o = c.g2o * inv_s2;
    c.dr2 = fmaf(fxo - fxn, fxo + fxn, fmaf(fyo - fyn, fyo + fyn, (fzo - fzn) * (fzo + fzn))) * inv_s2;
    c.an = rsqrtf(c.r2n);
    c.ao = rsqrtf(c.r2o);
    return c;
}

// Lennard-Jones change c12 (s'^2 - s^2) - c6 (s' - s), s = r^-6, without cancellation.
__device__ __forceinline__ float lj_du(const DuCore &c, float c12, float c6)
{
    const float in = c.an * c.an, io = c.ao * c.ao;
    const float s6n = in * in * in, s6o = io * io * io;
    const float poly = fmaf(c.r2o, c.r2o, fmaf(c.r2o, c.r2n, c.r2n * c.r2n));
    const float ds = ((c.dr2 * poly) * s6n) * s6o;
    return ds * fmaf(c12, s6n + s6o, -c6);
}

// u(r') - u(r) for one partner seen from a moved atom's new (sn) and old (so) positions,
// written so that neither the Lennard-Jones nor the Coulomb difference cancels: both are
// proportional to r^2 - r'^2 = sum over axes (|do| - |dn|)(|do| + |dn|), whose factors are
// exact small integers.
//   Coulomb: 1/r' - 1/r = (r^2 - r'^2) (a a')^2 / (a + a'),        a = 1/r, a' = 1/r'
//   LJ:      s' - s = (r^2 - r'^2)(r^4 + r^2 r'^2 + r'^4) s s',      s = r^-6, s' = r'^-6
//            c12 (s'^2 - s^2) - c6 (s' - s) = (s' - s)(c12 (s' + s) - c6)
// so the FP32 error is a few ulp of |u(r') - u(r)|, not of |u|. With CUT, a box whose LJ is
// truncated (lj_cut) takes the LJ term only where r' or r is inside r_lj.
template <bool CUT = false>
__device__ __forceinline__ float pair_du(Sep sn, Sep so, const PairRow &pr, const BoxDev &bx,
                                         const long long *T, const float *ep)
{
    const DuCore c = du_core(sn, so, bx.inv_s2);
    const float g2n = c.g2n, g2o = c.g2o, an = c.an, ao = c.ao, dr2 = c.dr2;
    if (g2n == 0.f) return __int_as_float(0x7f800000);
    float du = 0.f;
    if (pr.c12 != 0.f || pr.c6 != 0.f) {
        if (!CUT || !bx.lj_cut) {
            du = lj_du(c, pr.c12, pr.c6);
        } else {
            // truncated LJ: the difference where both sides are inside, else the one term
            const bool ln = below(g2n, sn, bx.lj2, bx.lj2_lo, bx.lj2_hi);
            const bool lo = below(g2o, so, bx.lj2, bx.lj2_lo, bx.lj2_hi);
            if (ln && lo) {
                du = lj_du(c, pr.c12, pr.c6);
            } else if (ln || lo) {
                const float a2 = ln ? an * an : ao * ao;
                const float s6 = a2 * a2 * a2;
                const float u = fmaf(pr.c12, s6, -pr.c6) * s6;
                du = ln ? u : -u;
            }
        }
    }
    const bool cn = below(g2n, sn, bx.rc2, bx.rc2_lo, bx.rc2_hi);
    const bool co = below(g2o, so, bx.rc2, bx.rc2_lo, bx.rc2_hi);
    if (cn && co) {
        const float p = an * ao;
        du = fmaf(pr.kqq * dr2, __fdividef(p * p, an + ao), du);   // 2 ulp; an + ao ~ 0.1..10
    } else if (cn) {
        du = fmaf(pr.kqq, an, du);
    } else if (co) {
        du = fmaf(-pr.kqq, ao, du);
    }
    if (bx.has_ep && (g2n < bx.tmax_hi || g2o < bx.tmax_hi)) {
        const float *row = ep + pr.pair * bx.n_bins;
        if (below(g2n, sn, bx.tmax, bx.tmax_lo, bx.tmax_hi))
            du += row[bin_of(d2_of(sn), g2n, T, bx.n_bins, bx.inv_dr_fx)];
        if (below(g2o, so, bx.tmax, bx.tmax_lo, bx.tmax_hi))
            du -= row[bin_of(d2_of(so), g2o, T, bx.n_bins, bx.inv_dr_fx)];
    }
    return du;
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ------------------------------------------------
struct U32x4 { uint32_t v[4]; };

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    U32x4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// FP64 uniform on [0, 1) from two words, 53 random bits (exact).
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b)
{
    return __dmul_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)),
                     0x1p-53);
}

__device__ __forceinline__ int wrap_coord(long long x, int L)
{
    if (x >= 0 && x < L) return (int)x;                  // trial coordinates land within one
    if (x < 0 && x >= -(long long)L) return (int)(x + L); // box side of [0, L): no division
    if (x >= L && x < 2LL * L) return (int)(x - L);
    const long long r = x % L;
    return (int)(r < 0 ? r + L : r);
}

// Signed minimum image with the tie rule: result in (-L/2, L/2].
__device__ __forceinline__ long long mi_signed(long long d, long long L)
{
    if (2 * d > L) return d - L;
    if (2 * d <= -L) return d + L;
    return d;
}

// Rotation matrix of the unit quaternion (1, v)/|(1, v)| in FP64, rounded to 2^-30 fixed
// point. Explicit round-to-nearest operations (no contraction) make the sequence exact:
// any implementation performing the same IEEE operations in this order gets the same
// integers.
__device__ inline void rotation_fixed(double vx, double vy, double vz, int *Rq)
{
    const double ss = __dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(vx, vx)), __dmul_rn(vy, vy)),
                                __dmul_rn(vz, vz));
    const double nn = __dsqrt_rn(ss);
    const double qw = __ddiv_rn(1.0, nn), qx = __ddiv_rn(vx, nn);
    const double qy = __ddiv_rn(vy, nn), qz = __ddiv_rn(vz, nn);
    const double xx = __dmul_rn(qx, qx), yy = __dmul_rn(qy, qy), zz = __dmul_rn(qz, qz);
    const double xy = __dmul_rn(qx, qy), xz = __dmul_rn(qx, qz), yz = __dmul_rn(qy, qz);
    const double wx = __dmul_rn(qw, qx), wy = __dmul_rn(qw, qy), wz = __dmul_rn(qw, qz);
    double R[9];
    R[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(yy, zz)));
    R[1] = __dmul_rn(2.0, __dsub_rn(xy, wz));
    R[2] = __dmul_rn(2.0, __dadd_rn(xz, wy));
    R[3] = __dmul_rn(2.0, __dadd_rn(xy, wz));
    R[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, zz)));
    R[5] = __dmul_rn(2.0, __dsub_rn(yz, wx));
    R[6] = __dmul_rn(2.0, __dsub_rn(xz, wy));
    R[7] = __dmul_rn(2.0, __dadd_rn(yz, wx));
    R[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, yy)));
    for (int i = 0; i < 9; ++i) Rq[i] = (int)__double2ll_rn(__dmul_rn(R[i], 1073741824.0));
}

// Configuration-independent part of one Monte Carlo move (80 bytes).
struct __align__(16) MoveRec {
    int mol;
    int shift[3];
    int R[9];        // rotation matrix * 2^30, rounded
    float thr;       // FP32 rounded up from -kT ln u_acc
    double u_acc;
    int a0, m;       // first atom (box-local) and atom count of the molecule
    int kind;        // 0 translate every atom, 1 rotate (and translate), 2 translate atom `atom`
    int atom;
};

// ---- device status word ------------------------------------------------------------------
constexpr int kStatusTimeout = 1;
constexpr int kStatusNonfinite = 2;

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Host side: prefilter half widths of the all-pairs histogram. Every counted pair has
// |dx| < R = ceil(sqrt(tmax)) + 1 grid units on each axis. On the 2^32-periodic grid
// (x' = floor(x 2^32 / L)) that is |dx'| < R' = ceil(R 2^32 / L) + 2; on the 2^16-periodic
// grid (x16 = x' >> 16) |dx16| <= R16 = ceil(R 2^16 / L) + 1, tested as the biased value
// (x16_i + R16 + 1 - x16_j) mod 2^16 <= 2 R16 + 1. A pair at exactly |dx16| = R16 has
// |dx| > R and is never counted.
inline void set_prefilter(BoxDev &bx)
{
    const double R = std::ceil(std::sqrt((double)bx.tmax)) + 1.0;
    const double Rs = std::ceil(R * 4294967296.0 / (double)bx.L) + 2.0;
    bx.pre_r = Rs >= 2147483647.0 ? 2147483647u : (unsigned)Rs;
    const double R16 = std::ceil(R * 65536.0 / (double)bx.L) + 1.0;
    if (2.0 * R16 + 1.0 <= 65534.0) {
        const uint32_t r16 = (uint32_t)R16, t = 2u * r16 + 1u;
        bx.pre16_bias = r16 + 1u;
        bx.pre16_t = t | (t << 16);
        bx.pre16_all = 0;
    } else {
        bx.pre16_bias = 0u;
        bx.pre16_t = 0xFFFFFFFFu;
        bx.pre16_all = 1;
    }
}

}  // namespace epsr
