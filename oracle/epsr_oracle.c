/*
 * epsr_oracle.c -- plain FP64 CPU oracle for the EPSR hot path.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the package smoke check and the
 * benchmark's CPU-baseline arm; never by the CUDA library or its binding. It shares
 * no code with the CUDA path. Build: gcc -O2 -fopenmp -ffp-contract=off (contraction
 * off so that the move proposal's FP64 arithmetic is exactly the stated sequence).
 *
 * Method: NeuDATool (arXiv:1904.08756). Metropolis MC over a reference plus empirical
 * potential (Sec. 2.1, Sec. 2.2 item III), the all-pair histograms N(r) -> g_ab(r)
 * (Sec. 2.3) and the structure factor of Eq. (1). Where the paper is silent the
 * reading used is stated at the function.
 */
#include "epsr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11). Each round multiplies counter words 0 and 2 by the Philox
 * multipliers, takes 64-bit products apart into high and low halves and mixes the
 * high halves with the other two counter words and the round key; the key is bumped
 * by the Weyl constants between rounds.
 * ---------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * c0;
        uint64_t p1 = (uint64_t)mul1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Coulomb constant from SI: e = 1.602176634e-19 C (exact), N_A = 6.02214076e23 (exact),
 * eps0 = 8.8541878128e-12 F/m (CODATA 2018). Converted J m -> kJ A. */
double orc_coulomb_constant(void)
{
    const double e = 1.602176634e-19, NA = 6.02214076e23, eps0 = 8.8541878128e-12;
    const double pi = 3.14159265358979323846;
    return e * e * NA / (4.0 * pi * eps0) * 1e10 * 1e-3;
}

/* Molar gas constant k_B N_A (both exact in SI), in kJ / mol / K. */
double orc_gas_constant(void)
{
    return 1.380649e-23 * 6.02214076e23 * 1e-3;
}

/* Minimum image of a coordinate difference dx in (-L, L): result in (-L/2, L/2]. */
int64_t orc_min_image(int64_t dx, int64_t L)
{
    if (2 * dx > L) dx -= L;
    else if (2 * dx <= -L) dx += L;
    return dx;
}

/* Exact squared minimum-image distance between two grid points (grid units^2). */
int64_t orc_dist2_points(const int32_t *a, const int32_t *b, int64_t L)
{
    int64_t d2 = 0;
    for (int c = 0; c < 3; ++c) {
        int64_t d = orc_min_image((int64_t)a[c] - (int64_t)b[c], L);
        d2 += d * d;
    }
    return d2;
}

static uint64_t isqrt_u128(unsigned __int128 x)
{
    uint64_t r = (uint64_t)sqrt((double)x);
    while ((unsigned __int128)r * r > x) --r;
    while ((unsigned __int128)(r + 1) * (r + 1) <= x) ++r;
    return r;
}

/* Histogram bin of a squared distance for bins of width p/q Angstrom:
 * k = floor(r / dr) = floor(sqrt(d2) q / (p S)) = isqrt(floor(d2 q^2 / (p^2 S^2))).
 * (Sec. 2.3: N(r) is the count of pairs per distance bin.) */
int64_t orc_bin_index(int64_t d2, int32_t bin_p, int32_t bin_q, int32_t scale_log2)
{
    unsigned __int128 num = (unsigned __int128)(uint64_t)d2 * (uint64_t)bin_q * (uint64_t)bin_q;
    unsigned __int128 den = ((unsigned __int128)(uint64_t)bin_p * (uint64_t)bin_p)
                            << (2 * scale_log2);
    return (int64_t)isqrt_u128(num / den);
}

/* Pair index of types a, b in the upper triangle, row major: (0,0),(0,1),..,(1,1),..
 * M types give M(M+1)/2 partials (Sec. 1, after Eq. 1). */
int32_t orc_pair_index(int32_t a, int32_t b, int32_t n_types)
{
    if (a > b) { int32_t t = a; a = b; b = t; }
    return a * n_types - a * (a - 1) / 2 + (b - a);
}

/* Pair energy of types ta, tb at squared distance d2 (grid units^2).
 * Reference potential (Sec. 2.1 names MD force fields only; reading c1): Lennard-Jones
 * 12-6 with Lorentz-Berthelot mixing over all minimum-image pairs, plus Coulomb
 * k_e q_a q_b / r for r < r_coul (plain truncation). Empirical potential (Sec. 2.1,
 * reading c4): the tabulated value of the pair's distance bin, zero beyond the table.
 * Coincident atoms (d2 == 0) have infinite energy (reading c8). */
double orc_pair_energy(const orc_system *s, int32_t ta, int32_t tb, int64_t d2)
{
    if (d2 == 0) return INFINITY;
    const double S = ldexp(1.0, s->scale_log2);
    const double r = sqrt((double)d2) / S;
    double u = 0.0;
    const double eps = sqrt(s->eps[ta] * s->eps[tb]);
    const int64_t rl_fx = llround(s->r_lj * S);
    if (eps > 0.0 && (s->r_lj <= 0.0 || d2 < rl_fx * rl_fx)) {
        const double sig = 0.5 * (s->sigma[ta] + s->sigma[tb]);
        const double x = sig / r;
        const double x6 = x * x * x * x * x * x;
        u += 4.0 * eps * (x6 * x6 - x6);
    }
    const int64_t rc_fx = llround(s->r_coul * S);
    if (d2 < rc_fx * rc_fx)
        u += orc_coulomb_constant() * s->q[ta] * s->q[tb] / r;
    if (s->ep) {
        int64_t k = orc_bin_index(d2, s->bin_p, s->bin_q, s->scale_log2);
        if (k < s->n_bins)
            u += s->ep[(int64_t)orc_pair_index(ta, tb, s->n_types) * s->n_bins + k];
    }
    return u;
}

static int64_t mol_of_atom(const orc_system *s, int64_t i)
{
    int64_t lo = 0, hi = s->n_mol;      /* mol_start[lo] <= i < mol_start[hi] */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (s->mol_start[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

/* Intra-molecular energy of a flexible molecule (Sec. 3.1: the molecule is held together
 * by harmonic potentials between every two of its atoms; reading r6 for the form):
 * sum over atom pairs a < b of k_ab (r_ab - d_ab)^2, r_ab the minimum-image distance of
 * the coordinates xyz_mol [m][3]. Zero for boxes without flexible molecules. */
double orc_intra_energy(const orc_system *s, int64_t mol, const int32_t *xyz_mol)
{
    if (!s->flexible) return 0.0;
    const int64_t a0 = s->mol_start[mol], m = s->mol_start[mol + 1] - a0;
    const double inv_S = ldexp(1.0, -s->scale_log2);
    double U = 0.0;
    for (int64_t a = 0; a < m; ++a)
        for (int64_t b = a + 1; b < m; ++b) {
            const int t = s->type[a0 + a] * ORC_MAX_TYPES + s->type[a0 + b];
            if (s->bond_k[t] == 0.0) continue;
            const double r = sqrt((double)orc_dist2_points(&xyz_mol[3 * a], &xyz_mol[3 * b], s->L_fx)) * inv_S;
            U += s->bond_k[t] * (r - s->bond_d[t]) * (r - s->bond_d[t]);
        }
    return U;
}

/* Total potential energy: sum over all pairs of atoms in different molecules (the
 * intra-molecular terms of rigid molecules are constant and left out, reading c2), plus
 * the intra-molecular springs of flexible molecules. */
double orc_total_energy(const orc_system *s)
{
    double U = 0.0;
    for (int64_t i = 0; i < s->n_atoms; ++i) {
        int64_t mi = mol_of_atom(s, i);
        int64_t j0 = s->mol_start[mi + 1];
        for (int64_t j = j0; j < s->n_atoms; ++j)
            U += orc_pair_energy(s, s->type[i], s->type[j],
                                 orc_dist2_points(&s->xyz[3 * i], &s->xyz[3 * j], s->L_fx));
    }
    if (s->flexible)
        for (int64_t mol = 0; mol < s->n_mol; ++mol)
            U += orc_intra_energy(s, mol, &s->xyz[3 * s->mol_start[mol]]);
    return U;
}

static double u53(uint32_t a, uint32_t b)
{
    /* Two words -> an FP64 uniform on [0, 1) with 53 random bits (reading c12). */
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * 0x1p-53;
}

static int64_t wrap(int64_t x, int64_t L)
{
    int64_t r = x % L;
    return r < 0 ? r + L : r;
}

static int64_t floordiv64(int64_t a, int64_t b)    /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

/* Move proposal (Sec. 2.2 item III: molecules or atoms moved at random; Sec. 3.1:
 * molecule translation and rotation). Random words: three Philox4x32-10 blocks with
 * counter (move lo, move hi, box index, lane), lane = 0, 1, 2, key (seed lo, seed hi).
 *   mol   = floor(w0 * n_mol / 2^32)
 *   shift = (w_{1+a} mod (2M+1)) - M per axis, M = llround(max_translation * S)
 *   v_c   = h (2 u_c - 1), u_c from the word pairs (w4,w5), (w6,w7), (w8,w9),
 *           h = tan(max_rotation / 2) / sqrt(3) (reading c10)
 *   u_acc from (w10, w11)
 * Rotation (rigid molecules): R is the matrix of the unit quaternion (1, v) / |(1, v)|,
 * evaluated in FP64 in the order written below and rounded to Rq = rint(R 2^30). It is
 * applied exactly, in integers, about the geometric centre of the molecule unwrapped
 * around its first atom: with offsets o_k (minimum image of X_k - X_0), Sum = sum_k o_k,
 * and e_k = m o_k - Sum, the new offset is the nearest integer (halves rounded up) to
 * (Sum 2^30 + Rq e_k) / (m 2^30) = c + (Rq / 2^30)(o_k - c), c = Sum / m, computed as
 * floor(floor((Sum 2^30 + Rq e_k + m 2^29) / 2^30) / m). New position = X_0 + that
 * offset + shift, wrapped into the box. Atom moves: X + shift, wrapped. Everything
 * after the FP64 matrix is integer arithmetic, so an independent implementation of the
 * same definition reproduces the trial coordinates bit for bit. */
void orc_rotation_fixed(double vx, double vy, double vz, int32_t Rq[9])
{
    const double ss = ((1.0 + vx * vx) + vy * vy) + vz * vz;
    const double nn = sqrt(ss);
    const double qw = 1.0 / nn, qx = vx / nn, qy = vy / nn, qz = vz / nn;
    const double xx = qx * qx, yy = qy * qy, zz = qz * qz;
    const double xy = qx * qy, xz = qx * qz, yz = qy * qz;
    const double wx = qw * qx, wy = qw * qy, wz = qw * qz;
    const double R[9] = {1.0 - 2.0 * (yy + zz), 2.0 * (xy - wz), 2.0 * (xz + wy),
                         2.0 * (xy + wz), 1.0 - 2.0 * (xx + zz), 2.0 * (yz - wx),
                         2.0 * (xz - wy), 2.0 * (yz + wx), 1.0 - 2.0 * (xx + yy)};
    for (int i = 0; i < 9; ++i) Rq[i] = (int32_t)llrint(R[i] * 1073741824.0);
}

void orc_propose(const orc_system *s, uint64_t seed, uint64_t move, uint32_t box_index,
                 int64_t *mol_out, int32_t *trial, double *u_acc)
{
    uint32_t w[16];
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t lane = 0; lane < (s->flexible ? 4u : 3u); ++lane) {
        const uint32_t ctr[4] = {(uint32_t)move, (uint32_t)(move >> 32), box_index, lane};
        orc_philox4x32_10(ctr, key, &w[4 * lane]);
    }
    const int64_t mol = (int64_t)(((uint64_t)w[0] * (uint64_t)s->n_mol) >> 32);
    const double S = ldexp(1.0, s->scale_log2);
    const int64_t M = llround(s->max_translation * S);
    int64_t shift[3];
    for (int a = 0; a < 3; ++a)
        shift[a] = (int64_t)(w[1 + a] % (uint32_t)(2 * M + 1)) - M;
    const int64_t a0 = s->mol_start[mol], m = s->mol_start[mol + 1] - a0;
    const int64_t L = s->L_fx;
    /* Flexible molecules (Sec. 3.1: molecule translation, molecule rotation, or the
     * translation of one atom): kind = w12 mod 3, the atom = w13 mod m (reading r6). */
    const int kind = s->flexible ? (int)(w[12] % 3u) : -1;
    if (kind == 0 || kind == 2) {
        for (int64_t k = 0; k < m; ++k) {
            const int moved = kind == 0 || k == (int64_t)(w[13] % (uint32_t)m);
            for (int a = 0; a < 3; ++a)
                trial[3 * k + a] = (int32_t)wrap((int64_t)s->xyz[3 * (a0 + k) + a] + (moved ? shift[a] : 0), L);
        }
    } else if (s->rigid || kind == 1) {
        if (kind == 1) shift[0] = shift[1] = shift[2] = 0;
        const double pi = 3.14159265358979323846;
        const double h = tan(0.5 * s->max_rotation_deg * pi / 180.0) / sqrt(3.0);
        int32_t Rq[9];
        orc_rotation_fixed(h * (2.0 * u53(w[4], w[5]) - 1.0), h * (2.0 * u53(w[6], w[7]) - 1.0),
                           h * (2.0 * u53(w[8], w[9]) - 1.0), Rq);
        int64_t off[ORC_MAX_MOL_ATOMS][3];
        int64_t sum[3] = {0, 0, 0};
        for (int64_t k = 0; k < m; ++k)
            for (int a = 0; a < 3; ++a) {
                off[k][a] = orc_min_image((int64_t)s->xyz[3 * (a0 + k) + a] -
                                          (int64_t)s->xyz[3 * a0 + a], L);
                sum[a] += off[k][a];
            }
        for (int64_t k = 0; k < m; ++k) {
            int64_t e[3];
            for (int b = 0; b < 3; ++b) e[b] = m * off[k][b] - sum[b];
            for (int a = 0; a < 3; ++a) {
                const int64_t num = sum[a] * 1073741824LL + (int64_t)Rq[3 * a] * e[0] +
                                    (int64_t)Rq[3 * a + 1] * e[1] + (int64_t)Rq[3 * a + 2] * e[2];
                const int64_t p = floordiv64(floordiv64(num + m * 536870912LL, 1073741824LL), m);
                trial[3 * k + a] = (int32_t)wrap((int64_t)s->xyz[3 * a0 + a] + p + shift[a], L);
            }
        }
    } else {
        for (int64_t k = 0; k < m; ++k)
            for (int a = 0; a < 3; ++a)
                trial[3 * k + a] = (int32_t)wrap((int64_t)s->xyz[3 * (a0 + k) + a] + shift[a], L);
    }
    *mol_out = mol;
    *u_acc = u53(w[10], w[11]);
}

/* Energy change of moving molecule `mol` to `trial` (Sec. 2.2 item III:
 * dU = U_after - U_before; Sec. 2.3: it needs the moved molecule against all atoms).
 * Non-bonded pairs inside the molecule are left out (reading c2); for flexible molecules
 * the change of the intra-molecular springs is added (Sec. 3.1, reading r6). cond (optional) receives the
 * condition scale sum |u(new) - u(old)| over the same pairs. */
double orc_delta_u(const orc_system *s, int64_t mol, const int32_t *trial, double *cond)
{
    const int64_t a0 = s->mol_start[mol], a1 = s->mol_start[mol + 1];
    double dU = 0.0, C = 0.0;
    for (int64_t k = 0; k < a1 - a0; ++k) {
        const int32_t ti = s->type[a0 + k];
        const int32_t *old = &s->xyz[3 * (a0 + k)];
        const int32_t *nw = &trial[3 * k];
        for (int64_t j = 0; j < s->n_atoms; ++j) {
            if (j >= a0 && j < a1) continue;
            const int32_t tj = s->type[j];
            const double un = orc_pair_energy(s, ti, tj, orc_dist2_points(nw, &s->xyz[3 * j], s->L_fx));
            const double uo = orc_pair_energy(s, ti, tj, orc_dist2_points(old, &s->xyz[3 * j], s->L_fx));
            dU += un - uo;
            C += fabs(un - uo);
        }
    }
    if (s->flexible) {
        const double di = orc_intra_energy(s, mol, trial) - orc_intra_energy(s, mol, &s->xyz[3 * a0]);
        dU += di;
        C += fabs(di);
    }
    if (cond) *cond = C;
    return dU;
}

/* Metropolis rule (Sec. 2.2 item III): accept if dU < 0, else with probability
 * exp(-dU / kT); dU == 0 is accepted (reading c3). NaN is rejected. */
int orc_accept(double dU, double u_acc, double temperature)
{
    if (dU <= 0.0) return 1;
    return u_acc < exp(-dU / (orc_gas_constant() * temperature));
}

/* Sequential Metropolis sweep of n_moves moves, move indices move0 .. move0+n-1. */
void orc_mc_sweep(orc_system *s, int64_t n_moves, uint64_t seed, uint64_t move0,
                  uint32_t box_index, orc_mc_stats *stats)
{
    int32_t trial[3 * ORC_MAX_MOL_ATOMS];
    for (int64_t t = 0; t < n_moves; ++t) {
        int64_t mol;
        double u_acc;
        orc_propose(s, seed, move0 + (uint64_t)t, box_index, &mol, trial, &u_acc);
        const double dU = orc_delta_u(s, mol, trial, NULL);
        stats->attempted += 1;
        if (orc_accept(dU, u_acc, s->temperature)) {
            const int64_t a0 = s->mol_start[mol], m = s->mol_start[mol + 1] - a0;
            memcpy(&s->xyz[3 * a0], trial, sizeof(int32_t) * 3 * (size_t)m);
            stats->accepted += 1;
            stats->sum_dU += dU;
        }
    }
}

/* Partial pair histograms N_ab(k) (Sec. 2.3, the O(N^2) N(r)): every unordered pair
 * i < j with i in [i0, i1), intra-molecular pairs included (reading c5), counted in
 * bin k of its type pair when k < n_bins. H [n_pairs][n_bins] is accumulated. */
void orc_histogram(const orc_system *s, int64_t i0, int64_t i1, uint64_t *H)
{
    for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = i + 1; j < s->n_atoms; ++j) {
            int64_t d2 = orc_dist2_points(&s->xyz[3 * i], &s->xyz[3 * j], s->L_fx);
            int64_t k = orc_bin_index(d2, s->bin_p, s->bin_q, s->scale_log2);
            if (k < s->n_bins)
                H[(int64_t)orc_pair_index(s->type[i], s->type[j], s->n_types) * s->n_bins + k] += 1;
        }
}

/* The same count split over host threads (OpenMP), each thread with its own
 * histogram, summed at the end. Integer sums: identical to orc_histogram. */
void orc_histogram_omp(const orc_system *s, uint64_t *H, int nthreads)
{
    const int64_t P = (int64_t)s->n_types * (s->n_types + 1) / 2;
    const int64_t nb = P * s->n_bins;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    uint64_t *priv = calloc((size_t)(nb * nthreads), sizeof(uint64_t));
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < s->n_atoms; ++i)
            orc_histogram(s, i, i + 1, priv + tid * nb);
    }
    for (int t = 0; t < nthreads; ++t)
        for (int64_t k = 0; k < nb; ++k) H[k] += priv[t * nb + k];
    free(priv);
}

/* g_ab(k) = N_ab(k) V / (n_configs P_ab (4 pi / 3)(r_{k+1}^3 - r_k^3)), r_k = k dr,
 * P_ab = N_a N_b (a != b), N_a (N_a - 1) / 2 (a == b) unordered pairs (reading c7). */
void orc_normalize_g(const orc_system *s, const uint64_t *H, int64_t n_configs, double *g)
{
    const double pi = 3.14159265358979323846;
    const double S = ldexp(1.0, s->scale_log2);
    const double Lb = (double)s->L_fx / S;
    const double V = Lb * Lb * Lb;
    const double dr = (double)s->bin_p / (double)s->bin_q;
    int64_t count[ORC_MAX_TYPES] = {0};
    for (int64_t i = 0; i < s->n_atoms; ++i) count[s->type[i]]++;
    for (int32_t a = 0; a < s->n_types; ++a)
        for (int32_t b = a; b < s->n_types; ++b) {
            const int32_t p = orc_pair_index(a, b, s->n_types);
            const double Pab = (a == b) ? 0.5 * (double)count[a] * (double)(count[a] - 1)
                                        : (double)count[a] * (double)count[b];
            for (int32_t k = 0; k < s->n_bins; ++k) {
                const double r0 = k * dr, r1 = (k + 1) * dr;
                const double shell = 4.0 * pi / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0);
                const double denom = (double)n_configs * Pab * shell;
                g[(int64_t)p * s->n_bins + k] =
                    denom > 0.0 ? (double)H[(int64_t)p * s->n_bins + k] * V / denom : 0.0;
            }
        }
}

/* Eq. (1), discretised by the midpoint rule on bin centres r_k = (k + 1/2) dr up to
 * the last bin (reading c6):
 *   S_partial[c](Q) = w_c sum_k r_k^2 dr (g_c(k) - 1) sin(Q r_k) / (Q r_k)
 * with w_c = 4 pi rho (2 - delta_ab) c_a c_b b_a b_b given per column, and
 *   S_total[s](Q) = flat[s] + sum of the cols_per_set columns of set s,
 * flat = sum_a c_a b_a^2 (the flat background of Eq. 1). Compensated summation. */
void orc_sq(const double *g, int32_t n_cols, int32_t n_bins, double dr, const double *Q,
            int32_t nQ, const double *w, int32_t cols_per_set, const double *flat,
            double *S_partial, double *S_total)
{
    const int32_t n_sets = n_cols / cols_per_set;
    for (int32_t s = 0; s < n_sets; ++s)
        for (int32_t i = 0; i < nQ; ++i) {
            double tot = flat[s], tc = 0.0;
            for (int32_t cc = 0; cc < cols_per_set; ++cc) {
                const int32_t c = s * cols_per_set + cc;
                double acc = 0.0, comp = 0.0;
                for (int32_t k = 0; k < n_bins; ++k) {
                    const double r = (k + 0.5) * dr;
                    const double x = Q[i] * r;
                    const double term = r * r * dr * (g[(int64_t)c * n_bins + k] - 1.0) * sin(x) / x;
                    const double y = term - comp;
                    const double t = acc + y;
                    comp = (t - acc) - y;
                    acc = t;
                }
                const double part = w[c] * acc;
                if (S_partial) S_partial[(int64_t)c * nQ + i] = part;
                const double y = part - tc;
                const double t = tot + y;
                tc = (t - tot) - y;
                tot = t;
            }
            if (S_total) S_total[(int64_t)s * nQ + i] = tot;
        }
}

/* ---- Gaussian-smeared histogram and its adjoint (differentiable form) -------------
 * Each unordered pair at distance r adds to bin k the mass in the bin of a Gaussian
 * of width sigma centred on r and truncated at +-5 sigma:
 *   w_k(r) = Phi(clip((r_{k+1} - r)/sigma)) - Phi(clip((r_k - r)/sigma)),
 *   clip(x) = min(max(x, -5), 5),  r_k = k dr,  Phi the standard normal CDF.
 * Bins outside [r - 5 sigma, r + 5 sigma] get exactly zero, so w_k is continuous in r;
 * only bins k in [floor((r - 5 sigma)/dr), floor((r + 5 sigma)/dr)] within [0, n_bins)
 * need evaluating. This is a smooth stand-in for the counts N(r) of Sec. 2.3. */
static double clip5(double x) { return x < -5.0 ? -5.0 : (x > 5.0 ? 5.0 : x); }

static void smear_window(double r, double sigma, double dr, int32_t n_bins,
                         int64_t *k_lo, int64_t *k_hi)
{
    int64_t lo = (int64_t)floor((r - 5.0 * sigma) / dr);
    int64_t hi = (int64_t)floor((r + 5.0 * sigma) / dr);
    if (lo < 0) lo = 0;
    if (hi > n_bins - 1) hi = n_bins - 1;
    *k_lo = lo;
    *k_hi = hi;
}

static void smeared_range(const orc_system *s, double sigma, int64_t i0, int64_t i1,
                          double *Ht)
{
    const double S = ldexp(1.0, s->scale_log2);
    const double dr = (double)s->bin_p / (double)s->bin_q;
    const double rmax = s->n_bins * dr + 5.0 * sigma;
    const double is2 = 1.0 / sqrt(2.0);
    for (int64_t i = i0; i < i1; ++i)
        for (int64_t j = i + 1; j < s->n_atoms; ++j) {
            const double r = sqrt((double)orc_dist2_points(&s->xyz[3 * i], &s->xyz[3 * j], s->L_fx)) / S;
            if (r >= rmax) continue;
            int64_t lo, hi;
            smear_window(r, sigma, dr, s->n_bins, &lo, &hi);
            const int64_t p = orc_pair_index(s->type[i], s->type[j], s->n_types);
            for (int64_t k = lo; k <= hi; ++k) {
                const double a = clip5((k * dr - r) / sigma), b = clip5(((k + 1) * dr - r) / sigma);
                Ht[p * s->n_bins + k] += 0.5 * (erf(b * is2) - erf(a * is2));
            }
        }
}

void orc_smeared_hist(const orc_system *s, double sigma, double *Ht)
{
    const int64_t P = (int64_t)s->n_types * (s->n_types + 1) / 2;
    const int64_t nb = P * s->n_bins;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *priv = calloc((size_t)(nb * nthreads), sizeof(double));
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < s->n_atoms; ++i)
            smeared_range(s, sigma, i, i + 1, priv + tid * nb);
    }
    for (int t = 0; t < nthreads; ++t)
        for (int64_t k = 0; k < nb; ++k) Ht[k] += priv[t * nb + k];
    free(priv);
}

/* Gradient of sum_{p,k} lambda[p][k] Ht[p][k] with respect to the position of atom i
 * (in Angstrom): for every pair, dw_k/dr = (phi(a_k) [|a_k| < 5] - phi(a_{k+1})
 * [|a_{k+1}| < 5]) / sigma with a_k = (r_k - r)/sigma and phi the standard normal
 * density, times the unit vector of the minimum-image separation x_i - x_j. */
static void smeared_grad_atom(const orc_system *s, double sigma, const double *lambda,
                              int64_t i, double *gi)
{
    const double S = ldexp(1.0, s->scale_log2);
    const double dr = (double)s->bin_p / (double)s->bin_q;
    const double rmax = s->n_bins * dr + 5.0 * sigma;
    const double inv_sqrt_2pi = 0.39894228040143267794;
    gi[0] = gi[1] = gi[2] = 0.0;
    for (int64_t j = 0; j < s->n_atoms; ++j) {
        if (j == i) continue;
        int64_t d[3];
        int64_t d2 = 0;
        for (int c = 0; c < 3; ++c) {
            d[c] = orc_min_image((int64_t)s->xyz[3 * i + c] - (int64_t)s->xyz[3 * j + c], s->L_fx);
            d2 += d[c] * d[c];
        }
        const double r = sqrt((double)d2) / S;
        if (r >= rmax || d2 == 0) continue;
        int64_t lo, hi;
        smear_window(r, sigma, dr, s->n_bins, &lo, &hi);
        const int64_t p = orc_pair_index(s->type[i], s->type[j], s->n_types);
        double dEdr = 0.0;
        for (int64_t k = lo; k <= hi; ++k) {
            const double a = (k * dr - r) / sigma, b = ((k + 1) * dr - r) / sigma;
            const double pa = fabs(a) < 5.0 ? exp(-0.5 * a * a) : 0.0;
            const double pb = fabs(b) < 5.0 ? exp(-0.5 * b * b) : 0.0;
            const double dw = (pa - pb) * inv_sqrt_2pi / sigma;
            dEdr += lambda[p * s->n_bins + k] * dw;
        }
        for (int c = 0; c < 3; ++c) gi[c] += dEdr * ((double)d[c] / S) / r;
    }
}

/* grad [n_atoms][3] is overwritten with the gradient for every atom. */
void orc_smeared_grad(const orc_system *s, double sigma, const double *lambda, double *grad)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < s->n_atoms; ++i)
        smeared_grad_atom(s, sigma, lambda, i, &grad[3 * i]);
}

/* The same for a sample of atoms idx[0..n_idx): grad [n_idx][3]. */
void orc_smeared_grad_atoms(const orc_system *s, double sigma, const double *lambda,
                            const int64_t *idx, int64_t n_idx, double *grad)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < n_idx; ++t)
        smeared_grad_atom(s, sigma, lambda, idx[t], &grad[3 * t]);
}
