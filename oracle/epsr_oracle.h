/*
 * epsr_oracle.h -- plain FP64 CPU oracle for the EPSR hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path (the CUDA library and its
 * Python binding) may include, link, load or call this code; only the tests, the
 * package-level smoke check and the benchmark's CPU-baseline arm use it. It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Every function states the passage of the paper (NeuDATool, arXiv:1904.08756) it
 * follows, or the reading taken where the paper is silent. Units: Angstrom, kJ/mol,
 * elementary charge, fm (scattering lengths), K. Coordinates are integers on a grid
 * of 2^-scale_log2 Angstrom.
 *
 * Parity pins: every function here is pinned by a CPU test against a closed form,
 * brute force, a published value or an invariant; none is "parity unpinned".
 */
#ifndef EPSR_ORACLE_H
#define EPSR_ORACLE_H
#include <stdint.h>

#define ORC_MAX_TYPES 8
#define ORC_MAX_MOL_ATOMS 64

typedef struct {
    int64_t n_atoms;
    int64_t n_mol;
    int64_t L_fx;              /* cubic box side in grid units */
    int32_t n_types;
    int32_t scale_log2;        /* grid: 2^-scale_log2 Angstrom */
    int32_t *xyz;              /* [n_atoms][3], each in [0, L_fx); updated by orc_mc_sweep */
    const int32_t *type;       /* [n_atoms] */
    const int64_t *mol_start;  /* [n_mol + 1] contiguous molecules */
    double q[ORC_MAX_TYPES];
    double sigma[ORC_MAX_TYPES];
    double eps[ORC_MAX_TYPES];
    double r_coul;             /* Coulomb cutoff (A) */
    int32_t bin_p, bin_q;      /* bin width p/q Angstrom */
    int32_t n_bins;
    int32_t rigid;             /* 1: molecule rotation + translation, 0: translation only */
    int32_t flexible;          /* 1: flexible molecules (Sec. 3.1): springs between every two
                                  atoms of a molecule, moves = translation, rotation or one atom */
    double bond_k[ORC_MAX_TYPES * ORC_MAX_TYPES];  /* spring constant k_ab, kJ/mol/A^2 */
    double bond_d[ORC_MAX_TYPES * ORC_MAX_TYPES];  /* reference distance d_ab, A */
    double temperature;        /* K */
    double max_translation;    /* A */
    double max_rotation_deg;
    const double *ep;          /* [n_pairs][n_bins] empirical potential (kJ/mol) or NULL */
    double r_lj;               /* Lennard-Jones cutoff (A): 0 = every pair (reading c1), > 0 =
                                  plainly truncated at r_lj (d^2 < llround(r_lj S)^2) */
} orc_system;

typedef struct {
    int64_t attempted;
    int64_t accepted;
    double sum_dU;             /* sum of accepted dU */
} orc_mc_stats;

/* Salmon et al., SC'11: Philox4x32 with 10 rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Physical constants (CODATA/SI exact where exact). */
double orc_coulomb_constant(void);   /* e^2 N_A / (4 pi eps0), kJ A / mol / e^2 */
double orc_gas_constant(void);       /* k_B N_A, kJ / mol / K */

int64_t orc_min_image(int64_t dx, int64_t L);
int64_t orc_dist2_points(const int32_t *a, const int32_t *b, int64_t L);
int64_t orc_bin_index(int64_t d2, int32_t bin_p, int32_t bin_q, int32_t scale_log2);
int32_t orc_pair_index(int32_t a, int32_t b, int32_t n_types);

double orc_pair_energy(const orc_system *s, int32_t ta, int32_t tb, int64_t d2);
double orc_total_energy(const orc_system *s);
double orc_intra_energy(const orc_system *s, int64_t mol, const int32_t *xyz_mol);
void orc_rotation_fixed(double vx, double vy, double vz, int32_t Rq[9]);
void orc_propose(const orc_system *s, uint64_t seed, uint64_t move, uint32_t box_index,
                 int64_t *mol, int32_t *trial /* [m][3] */, double *u_acc);
double orc_delta_u(const orc_system *s, int64_t mol, const int32_t *trial, double *cond);
int orc_accept(double dU, double u_acc, double temperature);
void orc_mc_sweep(orc_system *s, int64_t n_moves, uint64_t seed, uint64_t move0,
                  uint32_t box_index, orc_mc_stats *stats);

void orc_histogram(const orc_system *s, int64_t i0, int64_t i1, uint64_t *H);
void orc_histogram_omp(const orc_system *s, uint64_t *H, int nthreads);
void orc_normalize_g(const orc_system *s, const uint64_t *H, int64_t n_configs, double *g);

void orc_sq(const double *g, int32_t n_cols, int32_t n_bins, double dr, const double *Q,
            int32_t nQ, const double *w, int32_t cols_per_set, const double *flat,
            double *S_partial, double *S_total);

void orc_smeared_hist(const orc_system *s, double sigma, double *Ht);
void orc_smeared_grad(const orc_system *s, double sigma, const double *lambda, double *grad);
void orc_smeared_grad_atoms(const orc_system *s, double sigma, const double *lambda,
                            const int64_t *idx, int64_t n_idx, double *grad);

#endif
