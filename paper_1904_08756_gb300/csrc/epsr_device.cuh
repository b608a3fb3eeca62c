// epsr_device.cuh -- device-side data layout and helpers of libepsr (sm_103a).
//
// Box state lives in HBM as one int4 per atom {x, y, z, type} on the fixed-point grid
// (16 B/atom, coalesced 128-bit loads); per-box parameters are a POD struct that each
// CTA copies into shared memory. Squared distances are exact 64-bit integers; histogram
// bins come from a float estimate corrected against an exact integer threshold table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
    int32_t pad0;
    int64_t count[kMaxTypes];   // atoms per type
    PairRow row[kMaxTypes * kMaxTypes];
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

__device__ __forceinline__ long long dist2(int4 a, int4 b, int L)
{
    const long long dx = mi_abs(a.x - b.x, L);
    const long long dy = mi_abs(a.y - b.y, L);
    const long long dz = mi_abs(a.z - b.z, L);
    return dx * dx + dy * dy + dz * dz;
}

// Largest k with T[k] <= d2, for d2 < T[n_bins] (exact; the float guess is corrected).
__device__ __forceinline__ int bin_of(long long d2, const long long *T, int n_bins,
                                      float inv_dr_fx)
{
    int k = (int)(sqrtf((float)d2) * inv_dr_fx);
    k = min(k, n_bins - 1);
    while (k > 0 && T[k] > d2) --k;
    while (T[k + 1] <= d2) ++k;
    return k;
}

// Pair energy at squared distance d2 (grid units^2), FP32 (Sec. 2.1: reference
// potential + empirical potential). Coincident points have +inf energy.
__device__ __forceinline__ float pair_u(long long d2, const PairRow &pr, const BoxDev &bx,
                                        const long long *T, const float *ep)
{
    if (d2 == 0) return __int_as_float(0x7f800000);
    const float r2 = (float)d2 * bx.inv_s2;
    const float a = rsqrtf(r2);
    float u = 0.f;
    if (pr.c12 != 0.f || pr.c6 != 0.f) {
        const float i2 = a * a;
        const float s6 = i2 * i2 * i2;
        u = fmaf(pr.c12, s6, -pr.c6) * s6;
    }
    if (d2 < bx.rc2) u = fmaf(pr.kqq, a, u);
    if (bx.has_ep && d2 < bx.tmax)
        u += ep[pr.pair * bx.n_bins + bin_of(d2, T, bx.n_bins, bx.inv_dr_fx)];
    return u;
}

// u(d2n) - u(d2o) for one partner seen from a moved atom's new and old positions,
// written so that neither the Lennard-Jones nor the Coulomb difference cancels: both
// are proportional to the exact integer difference r^2 - r'^2 = (d2o - d2n) S^-2.
//   Coulomb: 1/r' - 1/r = (r^2 - r'^2) (a a')^2 / (a + a'),        a = 1/r, a' = 1/r'
//   LJ:      s' - s = (r^2 - r'^2)(r^4 + r^2 r'^2 + r'^4) s s',      s = r^-6, s' = r'^-6
//            c12 (s'^2 - s^2) - c6 (s' - s) = (s' - s)(c12 (s' + s) - c6)
// so the FP32 error is a few ulp of |u(r') - u(r)|, not of |u|.
__device__ __forceinline__ float pair_du(long long d2n, long long d2o, const PairRow &pr,
                                         const BoxDev &bx, const long long *T, const float *ep)
{
    if (d2n == 0) return __int_as_float(0x7f800000);
    const float r2n = (float)d2n * bx.inv_s2;
    const float r2o = (float)d2o * bx.inv_s2;
    const float dr2 = (float)(d2o - d2n) * bx.inv_s2;       // r^2 - r'^2 (exact integer)
    const float an = rsqrtf(r2n), ao = rsqrtf(r2o);
    float du = 0.f;
    if (pr.c12 != 0.f || pr.c6 != 0.f) {
        const float in = an * an, io = ao * ao;
        const float sn = in * in * in, so = io * io * io;
        const float poly = fmaf(r2o, r2o, fmaf(r2o, r2n, r2n * r2n));
        const float ds = ((dr2 * poly) * sn) * so;
        du = ds * fmaf(pr.c12, sn + so, -pr.c6);
    }
    const bool cn = d2n < bx.rc2, co = d2o < bx.rc2;
    if (cn && co) {
        const float p = an * ao;
        du = fmaf(pr.kqq * dr2, p * p / (an + ao), du);
    } else if (cn) {
        du = fmaf(pr.kqq, an, du);
    } else if (co) {
        du = fmaf(-pr.kqq, ao, du);
    }
    if (bx.has_ep && (d2n < bx.tmax || d2o < bx.tmax)) {
        const float *row = ep + pr.pair * bx.n_bins;
        if (d2n < bx.tmax) du += row[bin_of(d2n, T, bx.n_bins, bx.inv_dr_fx)];
        if (d2o < bx.tmax) du -= row[bin_of(d2o, T, bx.n_bins, bx.inv_dr_fx)];
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
    long long r = x % L;
    return (int)(r < 0 ? r + L : r);
}

// Signed minimum image with the tie rule: result in (-L/2, L/2].
__device__ __forceinline__ long long mi_signed(long long d, long long L)
{
    if (2 * d > L) return d - L;
    if (2 * d <= -L) return d + L;
    return d;
}

// Trial coordinates of a rigid-molecule move: rotation by the unit quaternion (1, v)/|(1, v)|
// about the centre of the molecule (unwrapped around its first atom), then the integer
// shift, wrapped into the box. Explicit round-to-nearest FP64 operations (no contraction)
// make the sequence exact and reproducible: the same IEEE operations in the same order.
__device__ inline void rigid_trial(const int4 *old, int m, double vx, double vy, double vz,
                                   const int *shift, int L, int4 *out)
{
    const double ss = __dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(vx, vx)), __dmul_rn(vy, vy)),
                                __dmul_rn(vz, vz));
    const double nn = __dsqrt_rn(ss);
    const double qw = __ddiv_rn(1.0, nn), qx = __ddiv_rn(vx, nn);
    const double qy = __ddiv_rn(vy, nn), qz = __ddiv_rn(vz, nn);
    const double xx = __dmul_rn(qx, qx), yy = __dmul_rn(qy, qy), zz = __dmul_rn(qz, qz);
    const double xy = __dmul_rn(qx, qy), xz = __dmul_rn(qx, qz), yz = __dmul_rn(qy, qz);
    const double wx = __dmul_rn(qw, qx), wy = __dmul_rn(qw, qy), wz = __dmul_rn(qw, qz);
    double R[3][3];
    R[0][0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(yy, zz)));
    R[0][1] = __dmul_rn(2.0, __dsub_rn(xy, wz));
    R[0][2] = __dmul_rn(2.0, __dadd_rn(xz, wy));
    R[1][0] = __dmul_rn(2.0, __dadd_rn(xy, wz));
    R[1][1] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, zz)));
    R[1][2] = __dmul_rn(2.0, __dsub_rn(yz, wx));
    R[2][0] = __dmul_rn(2.0, __dsub_rn(xz, wy));
    R[2][1] = __dmul_rn(2.0, __dadd_rn(yz, wx));
    R[2][2] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, yy)));
    long long off[kMaxMolAtoms][3];
    long long sum[3] = {0, 0, 0};
    const int base[3] = {old[0].x, old[0].y, old[0].z};
    for (int k = 0; k < m; ++k) {
        const int c[3] = {old[k].x, old[k].y, old[k].z};
        for (int a = 0; a < 3; ++a) {
            off[k][a] = mi_signed((long long)c[a] - base[a], L);
            sum[a] += off[k][a];
        }
    }
    double cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = __ddiv_rn((double)sum[a], (double)m);
    for (int k = 0; k < m; ++k) {
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = __dsub_rn((double)off[k][a], cen[a]);
        int o[3];
        for (int a = 0; a < 3; ++a) {
            const double p = __dadd_rn(cen[a], __dadd_rn(__dadd_rn(__dmul_rn(R[a][0], d[0]),
                                                                   __dmul_rn(R[a][1], d[1])),
                                                         __dmul_rn(R[a][2], d[2])));
            o[a] = wrap_coord((long long)base[a] + __double2ll_rn(p) + shift[a], L);
        }
        out[k] = make_int4(o[0], o[1], o[2], old[k].w);
    }
}

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

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace epsr
