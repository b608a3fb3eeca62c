/*
 * epsr.h -- C ABI of libepsr, the GB300 (sm_103a) implementation of the data-parallel
 * hot path of empirical potential structure refinement (EPSR) as described in
 * NeuDATool (arXiv:1904.08756):
 *
 *   - Metropolis Monte Carlo moves of molecules or atoms, each decided by the energy
 *     change dU of the moved molecule against all atoms of a periodic box
 *     (Sec. 2.2 item III, Sec. 2.3);
 *   - the all-pair partial histograms N_ab(r) and the pair distribution functions
 *     g_ab(r) (Sec. 2.3);
 *   - the structure factor S(Q) of Eq. (1), the weighted sine transform of g_ab(r);
 *   - the empirical-potential update from Delta S(Q) with a Poisson basis (Sec. 2.1,
 *     Eq. 2).
 *
 * Conventions (apply to every call):
 *   - Every function returns an int status (EPSR_OK on success). No C++ exception
 *     crosses this boundary. epsr_strerror() names a status; epsr_last_error_detail()
 *     copies a one-line description of the last failure on the calling host thread.
 *   - Work is enqueued on the caller's CUDA stream (`stream`, NULL = legacy default
 *     stream) and is asynchronous unless a function says it synchronises.
 *   - Device pointers are caller-owned device memory (for example torch tensors);
 *     host pointers are ordinary host memory. The library owns the opaque handles and
 *     the device memory behind them.
 *   - Coordinates are integers on a grid of 2^-scale_log2 Angstrom (scale_log2 = 20
 *     in all shipped workloads), in [0, L_fx) for a cubic box of side L_fx grid units.
 *     Squared distances are exact 64-bit integers, so histogram bins are exact.
 *   - Units: Angstrom, kJ/mol, elementary charge, fm (scattering lengths), K, 1/A (Q).
 *     S(Q) is in barn per steradian per atom.
 *   - A handle must not be used from two streams at the same time.
 */
#ifndef EPSR_H
#define EPSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *epsr_stream_t; /* same object as cudaStream_t */

/* ---- status codes ------------------------------------------------------------------ */
#define EPSR_OK 0
#define EPSR_EINVAL 1   /* an argument is out of range or inconsistent */
#define EPSR_ENOMEM 2   /* a device or host allocation failed */
#define EPSR_ECUDA 3    /* a CUDA runtime call failed */
#define EPSR_ELAUNCH 4  /* the persistent kernel's CTAs cannot all be resident at once */
#define EPSR_ETIMEOUT 5 /* a device-side wait gave up (the kernel exited cleanly) */
#define EPSR_ENUMERIC 6 /* a non-finite energy or structure factor was produced */

#define EPSR_MAX_TYPES 8       /* atom types per box */
#define EPSR_MAX_MOL_ATOMS 8   /* atoms per molecule moved as a rigid body */
#define EPSR_MAX_BINS 4096     /* histogram bins per pair */
#define EPSR_SQ_MAX_COLS 512   /* partial g(r) columns in one S(Q) call */

#define EPSR_MOVE_ATOM 0            /* translate one atom (single-atom molecules) */
#define EPSR_MOVE_RIGID_MOLECULE 1  /* rotate then translate one rigid molecule */
#define EPSR_MOVE_FLEXIBLE_MOLECULE 2  /* Sec. 3.1: springs k_ab (r - d_ab)^2 between every two atoms
                                          of a molecule; each move translates the molecule, rotates
                                          it, or translates one of its atoms (one third each) */

#define EPSR_SQ_FP32 0    /* CUDA-core FP32 contraction */
#define EPSR_SQ_TF32X3 1  /* tensor cores (tcgen05), TF32 hi/lo split, 3 products */
#define EPSR_SQ_BF16X3 2  /* tensor cores (tcgen05), BF16 hi/lo split, 3 products */
#define EPSR_SQ_BF16X6 3  /* tensor cores (tcgen05), BF16 three-way split, 6 products */

/* ---- box description ------------------------------------------------------------------
 * One periodic cubic box. Force field (Sec. 2.1 reference potential; the paper names
 * MD force fields only, this library takes): Lennard-Jones 12-6 with Lorentz-Berthelot
 * mixing over every minimum-image pair, plus Coulomb k_e q_a q_b / r for
 * r < r_coul (plain truncation, k_e from SI constants), plus the empirical potential
 * table (per type pair, piecewise constant on the histogram bins, zero beyond).
 * Bins have width bin_p / bin_q Angstrom (an exact rational) and there are n_bins.  */
typedef struct {
    int64_t n_atoms;
    int64_t n_mol;            /* molecules are contiguous atom ranges (mol_start) */
    int64_t L_fx;             /* box side in grid units, < 2^31 */
    int32_t scale_log2;       /* grid is 2^-scale_log2 Angstrom; 10 .. 24 */
    int32_t n_types;          /* 1 .. EPSR_MAX_TYPES */
    double q[EPSR_MAX_TYPES];      /* charge per type (e) */
    double sigma[EPSR_MAX_TYPES];  /* LJ sigma per type (A) */
    double eps[EPSR_MAX_TYPES];    /* LJ epsilon per type (kJ/mol); 0 = no LJ */
    double b[EPSR_MAX_TYPES];      /* coherent scattering length per type (fm) */
    double r_coul;            /* Coulomb cutoff (A) */
    int32_t bin_p, bin_q;     /* bin width = bin_p / bin_q Angstrom */
    int32_t n_bins;           /* 1 .. EPSR_MAX_BINS */
    int32_t move_kind;        /* EPSR_MOVE_ATOM, _RIGID_MOLECULE or _FLEXIBLE_MOLECULE */
    double temperature;       /* K */
    double max_translation;   /* A, per axis */
    double max_rotation_deg;  /* rigid-molecule rotation limit */
    /* EPSR_MOVE_FLEXIBLE_MOLECULE only: spring constant (kJ/mol/A^2) and reference distance
     * (A) of the intra-molecular spring between atoms of types a and b, at [a * EPSR_MAX_TYPES
     * + b] (symmetric; k = 0: no spring). Non-bonded terms inside a molecule are left out. */
    double bond_k[EPSR_MAX_TYPES * EPSR_MAX_TYPES];
    double bond_d[EPSR_MAX_TYPES * EPSR_MAX_TYPES];
    /* Lennard-Jones cutoff (A). 0, the form the paper's dU takes (every atom of the box):
     * LJ over every minimum-image pair. > 0: LJ plainly truncated at r_lj (the exact integer
     * test d^2 < llround(r_lj S)^2, no shift), so every partner beyond max(r_lj, r_coul, the
     * EP table) contributes nothing and the sweep finds the others by cell queries: the cost
     * of a move is O(neighbours) instead of O(N) (Sec. 2.3's cost statement). */
    double r_lj;
} epsr_box_desc;

typedef struct epsr_box epsr_box;   /* opaque: one box or a batch of boxes */
typedef struct epsr_sq_plan epsr_sq_plan;   /* opaque: cached sine-transform matrix */

/* Running Monte Carlo statistics of one box, accumulated over every sweep since the
 * box was created. */
typedef struct {
    int64_t attempted;
    int64_t accepted;
    int64_t nonfinite;   /* moves whose dU was not finite (rejected) */
    double sum_dU;       /* sum of accepted dU (kJ/mol), FP64 */
} epsr_mc_stats;

/* One logged move (for replay against an independent implementation). */
typedef struct {
    int32_t mol;         /* moved molecule (index within its box) */
    int32_t accepted;
    float dU;            /* the FP32 energy change that decided the move */
    int32_t n_atoms;     /* atoms of the molecule (rows of trial used) */
    double u_acc;        /* the uniform variate of the Metropolis test */
    int32_t trial[EPSR_MAX_MOL_ATOMS][3];  /* trial grid coordinates */
    int32_t pad[2];
} epsr_move_log;         /* 128 bytes */

/* ---- errors ------------------------------------------------------------------------- */
const char *epsr_strerror(int status);
/* Copies the last failure message of this host thread into buf (NUL-terminated,
 * truncated to len). Returns the status of that failure (EPSR_OK if none). */
int epsr_last_error_detail(char *buf, size_t len);
int epsr_version(void);   /* major * 10000 + minor * 100 + patch */

/* ---- boxes ---------------------------------------------------------------------------
 * epsr_box_create: one box. Host inputs are copied (the caller keeps ownership):
 *   xyz       int32 [n_atoms][3] grid coordinates in [0, L_fx)
 *   type      int32 [n_atoms], 0 .. n_types-1
 *   mol_start int64 [n_mol+1], mol_start[0] = 0, strictly increasing,
 *             mol_start[n_mol] = n_atoms; with EPSR_MOVE_RIGID_MOLECULE each molecule
 *             has at most EPSR_MAX_MOL_ATOMS atoms, with EPSR_MOVE_ATOM exactly one;
 *             every atom lies within 2^25 grid units (32 A at scale_log2 = 20) of its
 *             molecule's first atom on each axis.
 * Builds the exact bin-threshold table, the pair-parameter table and a zero empirical
 * potential. Synchronises `stream` before returning. Errors: EINVAL (any inconsistent
 * field or array), ENOMEM, ECUDA.
 *
 * epsr_batch_create: n_boxes independent boxes (replicas) advanced together by one
 * persistent kernel. descs[n_boxes]; xyz and type concatenated over the boxes in
 * order; mol_start concatenated as n_boxes arrays of n_mol_b+1 entries, each starting
 * at 0 (box-local atom indices).                                                       */
int epsr_box_create(const epsr_box_desc *desc, const int32_t *xyz, const int32_t *type,
                    const int64_t *mol_start, epsr_stream_t stream, epsr_box **out);
int epsr_batch_create(const epsr_box_desc *descs, int32_t n_boxes, const int32_t *xyz,
                      const int32_t *type, const int64_t *mol_start, epsr_stream_t stream,
                      epsr_box **out);
/* Frees the handle and its device memory (synchronises the device). NULL is a no-op. */
int epsr_box_destroy(epsr_box *box);

/* Sizes: number of boxes, total atoms, and the length in elements of the histogram
 * buffer epsr_partial_gr expects (sum over boxes of n_pairs_b * n_bins_b). Any output
 * pointer may be NULL. Host only, no CUDA call. */
int epsr_box_info(const epsr_box *box, int32_t *n_boxes, int64_t *n_atoms_total,
                  int64_t *hist_len);
/* Offset (elements) of box b's block in the histogram / g buffers, and of its first
 * atom in the coordinate arrays. Host only. */
int epsr_box_offsets(const epsr_box *box, int32_t b, int64_t *hist_offset, int64_t *atom_offset);

/* Copies the current coordinates to host int32 [n_atoms_total][3] (synchronises). */
int epsr_box_get_coords(epsr_box *box, int32_t *xyz, epsr_stream_t stream);
/* Replaces the coordinates from host int32 [n_atoms_total][3] (validated, in [0, L)).
 * Enqueued on `stream`; the host array must stay valid until the stream reaches it. */
int epsr_box_set_coords(epsr_box *box, const int32_t *xyz, epsr_stream_t stream);
/* Same from a device int32 [n_atoms_total][3] (not validated; caller guarantees range). */
int epsr_box_set_coords_device(epsr_box *box, const int32_t *xyz_dev, epsr_stream_t stream);
/* Copies the current coordinates to device int32 [n_atoms_total][3]. */
int epsr_box_get_coords_device(epsr_box *box, int32_t *xyz_dev, epsr_stream_t stream);

/* Replaces box b's empirical potential from host FP32 [n_pairs][n_bins] (kJ/mol),
 * pair order (0,0),(0,1),..,(1,1),.. (synchronises). */
int epsr_box_set_ep(epsr_box *box, int32_t b, const float *ep, epsr_stream_t stream);
int epsr_box_get_ep(epsr_box *box, int32_t b, float *ep, epsr_stream_t stream);

/* Total potential energy of every box from scratch (Sec. 2.2 item III defines dU as
 * U_after - U_before; this is U): sum over all pairs of atoms in different molecules
 * of the pair energy, FP32 per pair, FP64 accumulation, plus (flexible molecules) the
 * intra-molecular springs in FP64. U_host [n_boxes]. Synchronises. */
int epsr_box_total_energy(epsr_box *box, double *U_host, epsr_stream_t stream);

/* ---- Monte Carlo (Sec. 2.2 item III; Sec. 2.3: dU from the moved molecule against
 * all atoms after every step) ----------------------------------------------------------
 * Runs moves move0 .. move0+n_moves-1 on every box of the handle. Move t of box b
 * draws three Philox4x32-10 blocks with counter (t lo, t hi, b, lane 0..2) and key
 * (seed lo, seed hi): the molecule, a translation of at most max_translation per axis
 * and (rigid molecules) a rotation of at most max_rotation_deg about the molecule's
 * centre, then accepts with the Metropolis rule (dU <= 0, else with probability
 * exp(-dU/kT)). The result is a deterministic function of (coordinates, seed, move0).
 *   stats  host [n_boxes] or NULL: overwritten with the running totals.
 *   log    device [n_boxes][n_moves] or NULL: one epsr_move_log per move.
 * One cooperative persistent launch; synchronises `stream` to read its status.
 * Errors: EINVAL, ELAUNCH (the CTAs cannot be co-resident), ETIMEOUT (a grid barrier
 * wait exceeded its limit; coordinates are then unspecified), ECUDA.                 */
int epsr_mc_sweep(epsr_box *box, int64_t n_moves, uint64_t seed, uint64_t move0,
                  epsr_mc_stats *stats, epsr_move_log *log, epsr_stream_t stream);
/* The same sweep enqueued without synchronising and without reading the status back:
 * it allocates nothing and can be captured in a CUDA graph. Read the status of the last
 * sweep later with epsr_mc_status (EPSR_OK or EPSR_ETIMEOUT in *status). */
int epsr_mc_sweep_async(epsr_box *box, int64_t n_moves, uint64_t seed, uint64_t move0,
                        epsr_move_log *log, epsr_stream_t stream);
int epsr_mc_status(epsr_box *box, int32_t *status, epsr_stream_t stream);
/* Reads the running statistics without running moves (synchronises). */
int epsr_mc_stats_get(epsr_box *box, epsr_mc_stats *stats, epsr_stream_t stream);
/* Moves per speculative batch (1 .. 64; 0, the default: 64 for boxes swept by at least 64
 * CTAs, 32 for at least 32, else 16; a box swept by fewer than 8 CTAs takes at most 32):
 * the sweep evaluates up to this many
 * consecutive moves with distinct molecules per grid barrier and resolves them in order
 * with exact pairwise corrections, so every value gives the sequential Metropolis chain
 * (up to FP32 rounding of dU). Host only. */
int epsr_mc_set_batch(epsr_box *box, int32_t batch_k);
/* CTAs per box of the sweep (0 = automatic). For a batch of boxes, a total budget split
 * in proportion to the atom counts. Host only; takes effect at the next sweep. */
int epsr_mc_set_ctas(epsr_box *box, int32_t ctas);
/* Cell queries of the sweep (a performance device, no effect on results): partners whose
 * pair rows have no Lennard-Jones term are looked up in the 8^3 cells of each CTA's slice
 * that meet the cube around the moved molecule widened by margin_fx grid units; a partner
 * that drifts more than margin_fx out of its cell during a launch joins a per-CTA escapee
 * list of escapee_cap entries (-1: the maximum, 256; 0: no cell queries, every partner is
 * scanned) and, when that list is full, the CTA scans every partner for the rest of the
 * launch. Defaults: 2^20 (1 A), -1. EPSR_EINVAL for margin_fx < 0, margin_fx >= L_fx / 4
 * of a box, or escapee_cap outside [-1, 256]. Host only; takes effect at the next sweep. */
int epsr_mc_set_cells(epsr_box *box, int32_t margin_fx, int32_t escapee_cap);
/* Persistent CTAs per SM of the all-pair histogram kernel (1 .. 4; 0 restores the default, 4).
 * A performance setting: the integer counts do not depend on it. Host only. */
int epsr_gr_set_ctas_per_sm(epsr_box *box, int32_t ctas_per_sm);
/* The current launch settings: moves per barrier and CTA budget of the sweep (0 = automatic),
 * CTAs per SM of the histogram. Any pointer may be NULL. Host only. */
int epsr_box_get_launch(const epsr_box *box, int32_t *mc_batch, int32_t *mc_ctas, int32_t *gr_ctas_per_sm);

/* ---- autotuner (no counterpart in the paper, whose GPU and MPI versions fix their own
 * decomposition; here the launch shapes are chosen by timing) ------------------------------
 * epsr_autotune times, on this handle, the sweep at CTA budgets {SMs, 3/4, 1/2 of the SMs}
 * x {16, 32, 64} moves per barrier (probe_moves moves each, 0 = 2048, after a warm-up run)
 * and the all-pair histogram at {2, 3, 4} CTAs per SM, and applies the fastest. The
 * handle's coordinates, empirical potentials and running statistics are saved to a host
 * checkpoint before and restored after, so the handle continues from the state it had; every
 * candidate computes the same chain and the same counts. The choice is cached per shape
 * (every box's atoms, molecules, types, move kind and bins, and the SM count) for the life of
 * the process: a later call on a handle of the same shape applies it without timing
 * (out->from_cache = 1). Synchronises; allocates a scratch histogram while timing.
 * Errors: those of the calls it makes (a probe sweep that times out returns ETIMEOUT and
 * leaves the handle's previous settings).
 *
 * epsr_sq_plan_autotune times the tensor-core tilings (n_chunk in {16, 32, 64} and, with
 * S_total, the least multiple of 16 and cols_per_set and its double; k_split in
 * {1, 2, 4, 8}) of epsr_sq_exec with these arguments (which it writes, three times per
 * candidate), sets the fastest on the plan (epsr_sq_plan_set_tiles) and caches it per (Q
 * grid size, bins, mode, columns, set size, totals or not, SM count). Reports the tiling and
 * its time per call in microseconds (pointers may be NULL). An FP32 plan has nothing to tune
 * (zeros, EPSR_OK). Synchronises. */
typedef struct {
    int32_t mc_batch;        /* moves per grid barrier chosen for the sweep */
    int32_t mc_ctas;         /* CTA budget of the sweep over the handle */
    int32_t gr_ctas_per_sm;  /* persistent CTAs per SM of the all-pair histogram */
    int32_t from_cache;      /* 1: applied from the process's cache, nothing timed */
    double mc_us_per_move;   /* measured at the chosen setting (per move of every box) */
    double gr_ms;            /* measured at the chosen setting, one full histogram */
} epsr_tuning;
int epsr_autotune(epsr_box *box, uint64_t seed, int32_t probe_moves, epsr_tuning *out, epsr_stream_t stream);
int epsr_sq_plan_autotune(epsr_sq_plan *plan, const float *g, int32_t n_cols, const double *w,
                          int32_t cols_per_set, const double *flat, float *S_partial, float *S_total,
                          int32_t *n_chunk, int32_t *k_split, double *us, epsr_stream_t stream);

/* Test hook: CTA `cta` of the following sweeps skips its barrier arrival and every
 * barrier wait is limited to timeout_ms, so the bounded wait expires and the sweep
 * returns EPSR_ETIMEOUT with the GPU context intact. cta = -1 restores normal operation
 * and the default limit (2000 ms). Host only. */
int epsr_debug_barrier_fault(epsr_box *box, int32_t cta, double timeout_ms);

/* Number of kernels this library has enqueued, on any stream and device, since it was
 * loaded (a host-side counter, one per kernel launch; a launch recorded into a CUDA graph
 * counts once when it is captured, not at each replay). No counterpart in the paper: it
 * lets a caller state how many of the library's kernels ran inside a timed region. */
int epsr_launch_count(uint64_t *count);

/* ---- checkpoint / resume ----------------------------------------------------------------
 * A checkpoint is the coordinates, the empirical-potential tables and the running MC
 * statistics of every box, in a host buffer of epsr_checkpoint_size() bytes. The move
 * stream is counter-based (Philox), so a run resumed from a checkpoint at move index t with
 * move0 = t continues bit for bit as if it had not stopped. epsr_checkpoint_load accepts
 * only a checkpoint of a handle with the same boxes, atoms and tables (else EPSR_EINVAL).
 * Both synchronise. */
int epsr_checkpoint_size(const epsr_box *box, size_t *bytes);
int epsr_checkpoint_save(epsr_box *box, void *buf, size_t len, epsr_stream_t stream);
int epsr_checkpoint_load(epsr_box *box, const void *buf, size_t len, epsr_stream_t stream);

/* ---- pair histograms and g(r) (Sec. 2.3: N(r), O(N^2) per evaluation) -----------------
 * For every unordered pair i < j of each box (intra-molecular pairs included), the
 * exact squared minimum-image distance selects bin k = floor(r / dr); if k < n_bins the
 * pair's count hist[pair(t_i, t_j)][k] is incremented. Pair order is (0,0), (0,1), ..,
 * (1,1), ... (upper triangle, row major); boxes are concatenated (epsr_box_offsets).
 *   hist  device uint64 [hist_len], ACCUMULATED (not cleared), so repeated calls
 *         accumulate statistics over configurations (Sec. 2.2 item VI).
 *   g     device float [hist_len] or NULL: g_ab(k) = hist V / (n_configs P_ab shell_k),
 *         P_ab = N_a N_b (a != b) or N_a (N_a - 1)/2, shell_k = 4 pi/3 (r_{k+1}^3 - r_k^3).
 *   n_configs  number of configurations accumulated in hist (>= 1) for g.
 * Bins beyond half the box side are only partly sampled (minimum-image distances cover a
 * shell of radius r > L/2 only in part), so g falls below 1 there; the counts are still
 * the exact minimum-image counts. Asynchronous. Errors: EINVAL, ECUDA.                   */
int epsr_partial_gr(epsr_box *box, uint64_t *hist, float *g, int64_t n_configs,
                    epsr_stream_t stream);
/* The same histogram counted over cell lists: cells at least the histogram range wide
 * (at least 3 per side), each pair counted from its home cell against itself and the 13
 * forward neighbour cells, so the work is O(N * rho * r_max^3) instead of O(N^2) while
 * the integer counts are identical to epsr_partial_gr's. Boxes with fewer than three cells
 * per side are counted with the all-pairs kernel. Same arguments, accumulation and errors
 * as epsr_partial_gr. No counterpart in the paper, whose kernel is the O(N^2) scan. */
int epsr_partial_gr_cells(epsr_box *box, uint64_t *hist, float *g, int64_t n_configs,
                          epsr_stream_t stream);
/* The same over a sub-range [pair_begin, pair_end) of the handle's pair-tile work list
 * (for splitting one evaluation across devices or calls; the union of disjoint ranges
 * covering [0, n_tiles) equals one full call). epsr_partial_gr_tiles reports n_tiles. */
int epsr_partial_gr_tiles(const epsr_box *box, int64_t *n_tiles);
int epsr_partial_gr_range(epsr_box *box, int64_t tile_begin, int64_t tile_end, uint64_t *hist,
                          epsr_stream_t stream);
/* g from an accumulated histogram only (no pair scan). */
int epsr_normalize_g(epsr_box *box, const uint64_t *hist, float *g, int64_t n_configs,
                     epsr_stream_t stream);

/* Eq. (1) weight factors of box b: w[p] = 4 pi rho (2 - delta_ab) c_a c_b b_a b_b per
 * pair (b in 1e-12 cm so S is in barn) and flat = sum_a c_a b_a^2. Host only. */
int epsr_sq_weights(const epsr_box *box, int32_t b, double *w, double *flat);

/* ---- differentiable form: Gaussian-smeared histogram, its adjoint, chi^2 ------------------
 * A smooth stand-in for the counts N(r) of Sec. 2.3: every unordered pair at distance r
 * adds to bin k the mass of a Gaussian of width sigma centred on r, truncated at +-5 sigma,
 *   w_k(r) = Phi(clip((r_{k+1} - r)/sigma)) - Phi(clip((r_k - r)/sigma)),  clip to [-5, 5].
 * epsr_gr_smeared_fwd: Ht device double [hist_len] (overwritten); gt device float [hist_len]
 *   or NULL: the smeared g~ = Ht V / (P_ab shell_k), normalised like epsr_partial_gr's g.
 * epsr_gr_smeared_bwd: given dL/dg~ (device float [hist_len]) writes dL/dx, device float
 *   [n_atoms_total][3] per Angstrom (overwritten). Pair distances are recomputed.
 * epsr_sq_exec_adjoint: dg[c][k] = w_c sum_i K[i][k] dS_total[set(c)][i], the adjoint of
 *   epsr_sq_exec with respect to g (dS_total device [n_sets][nQ], dg device [n_cols][n_bins]).
 * epsr_chi2: chi2 = sum_Q [S(Q) + sum_p W[p] sum_n C[p][n] F_n(Q) - target(Q)]^2 on the plan's
 *   Q grid, F_n the closed-form transform of the Poisson function p_n (4 pi rho included);
 *   writes chi2 (device double [1]), dS = dchi2/dS (device float [nQ]) and, if C is given,
 *   dC = dchi2/dC (device double [P][n_basis]). W host double [P] (barn); C device or NULL.
 * All asynchronous on `stream`. */
int epsr_gr_smeared_fwd(epsr_box *box, double sigma, double *Ht, float *gt, epsr_stream_t stream);
int epsr_gr_smeared_bwd(epsr_box *box, double sigma, const float *dgt, float *grad,
                        epsr_stream_t stream);
int epsr_sq_exec_adjoint(epsr_sq_plan *plan, const float *dS_total, int32_t n_cols, const double *w,
                         int32_t cols_per_set, float *dg, epsr_stream_t stream);
int epsr_chi2(epsr_sq_plan *plan, const float *S, const float *target, const double *W, int32_t P,
              const double *C, int32_t n_basis, double s_basis, double rho, double *chi2, float *dS,
              double *dC, epsr_stream_t stream);

/* ---- empirical-potential update (Sec. 2.1: the EMP is a Poisson series fitted in Q space
 * to Delta S(Q); Eq. (2): pair terms through the inverse of the weight matrix) ----------------
 * For box b with P = n_types (n_types + 1)/2 pairs:
 *   1. pair-resolve: Delta S_p = sum_d M[p][d] dS[d], M = pinv([w; gamma I]) restricted to the
 *      data rows (w [n_data][P] host: the Eq. (1) weights (2 - delta) c_a c_b b_a b_b of each
 *      dataset, barn; gamma = 0 with n_data == P inverts w; fewer datasets need gamma > 0);
 *   2. fit: C_p = argmin || Delta S_p - F C_p || by Householder QR in FP64, where
 *      F[Q][n] = 4 pi rho int r^2 p_n(r) sin(Qr)/(Qr) dr in closed form, p_n(r) =
 *      (r/(n s))^n exp(n - r/s) (peak 1 at r = n s), n = 1..n_basis;
 *   3. table: U_EP[p][k] += -alpha kT sum_n C[p][n] p_n((k + 1/2) dr).
 *   dS      device float [n_data][nQ];  Q host float [nQ] (> 0)
 *   C_out   host double [P][n_basis] or NULL
 * Limits: n_data <= 16, n_basis <= 40, nQ >= n_basis. Synchronises. The basis is nearly
 * collinear (condition ~1e10 for 20 functions): C carries that conditioning, the fitted
 * Delta S and the table do not. */
int epsr_ep_update(epsr_box *box, int32_t b, const float *dS, int32_t n_data, const double *w,
                   const float *Q, int32_t nQ, int32_t n_basis, double s_basis, double gamma,
                   double alpha, double *C_out, epsr_stream_t stream);

/* ---- the refinement loop (Sec. 2.2 items III-VI; Sec. 2.1; Eq. 2) ------------------------
 * A refiner drives the loop of the method on a one-box handle: each epsr_refine_step runs
 *   III  moves_per_pass Metropolis moves (epsr_mc_sweep; moves continue from move0 on),
 *   VI   the pair histograms, accumulated over the passes (accumulate = 1, Sec. 2.2 item VI)
 *        or of this configuration alone (0), and g_ab(r),
 *   IV   S_d(Q) of every dataset d by Eq. (1): flat_d + sum_p 4 pi rho w[d][p] sum_k K (g_p - 1),
 *        then Delta S_d = target_d - S_d and chi^2 = sum_d sum_Q Delta S_d^2,
 *   V    epsr_ep_update(Delta S, w, n_basis, s_basis, gamma, alpha): the Poisson fit of the
 *        pair-resolved Delta S added to the empirical potential.
 * The loop is repeated by the caller until ep_change_max (the largest change the pass made to
 * the table, kJ/mol) or chi^2 is small enough (Sec. 2.1).
 *   plan    an S(Q) plan on the datasets' Q grid (nQ points, the box's bins, at least
 *           n_data * n_pairs columns), any mode
 *   target  device float [n_data][nQ], the measured S(Q) (barn/sr/atom); caller-owned, read at
 *           every step
 *   w       host double [n_data][n_pairs], Eq. (1) weights (2 - delta) c_a c_b b_a b_b of each
 *           dataset (barn), copied; flat host double [n_data], sum_a c_a b_a^2; Q host float [nQ]
 *   n_data  1 .. 16; fewer datasets than pairs need gamma > 0
 * epsr_refiner_get copies the accumulated histogram (device uint64 [n_pairs][n_bins]), g, S and
 * Delta S of the last step (device float) and its fitted coefficients (host double
 * [n_pairs][n_basis]); any pointer may be NULL. Steps synchronise; create and destroy
 * allocate and free the refiner's device buffers. */
typedef struct epsr_refiner epsr_refiner;
typedef struct {
    int64_t moves_per_pass;   /* Metropolis moves per step (0: no moves) */
    uint64_t seed;            /* Philox key of the moves */
    uint64_t move0;           /* index of the first move of the first step */
    int32_t accumulate;       /* 1: histograms accumulate over steps; 0: each step alone */
    int32_t n_basis;          /* Poisson functions per pair, 1 .. 40 */
    double s_basis;           /* Poisson width s (A) */
    double gamma;             /* pair-resolution regulariser */
    double alpha;             /* feedback factor of the update */
} epsr_refine_params;
typedef struct {
    int64_t iteration;        /* steps done */
    int64_t attempted, accepted;  /* running Monte Carlo totals of the box */
    int64_t n_configs;        /* configurations in the histogram */
    uint64_t next_move;       /* move index the next step starts at */
    double chi2;              /* sum over datasets and Q of Delta S^2 before this step's update */
    double ep_change_max;     /* largest |change| of the empirical-potential table (kJ/mol) */
} epsr_refine_result;
int epsr_refiner_create(epsr_box *box, epsr_sq_plan *plan, const float *target, int32_t n_data,
                        const double *w, const double *flat, const float *Q, int32_t nQ,
                        const epsr_refine_params *params, epsr_stream_t stream, epsr_refiner **out);
int epsr_refine_step(epsr_refiner *r, epsr_move_log *log, epsr_refine_result *res, epsr_stream_t stream);
int epsr_refiner_get(const epsr_refiner *r, uint64_t *hist, float *g, float *S, float *dS, double *C,
                     epsr_stream_t stream);
int epsr_refiner_destroy(epsr_refiner *r);

/* ---- pair histogram without device allocation -----------------------------------------
 * The paper has no counterpart: this entry point exists for callers that must not
 * allocate device memory when they need the counts -- plug-ins whose host framework's
 * caching allocator owns the device memory and hands them none, or real-time loops that
 * may not call cudaMalloc/cudaFree (which can synchronise the device) after start-up.
 *
 * epsr_partial_gr_noalloc adds to hist the same counts epsr_partial_gr adds for a
 * one-box handle with the same coordinates, types and bins, and allocates nothing: all
 * working memory is one fixed __device__ array of epsr_noalloc_scratch_bytes() bytes
 * (about 12.6 MB) that every GPU loading the library holds until the process exits.
 *   xyz, type   HOST int32 [n_atoms][3] in [0, L_fx) and [n_atoms] in [0, n_types)
 *               (validated; staged by the copy calls before they return, so they may be
 *               reused on return)
 *   n_atoms     1 .. EPSR_NOALLOC_MAX_ATOMS; larger boxes are rejected with EPSR_EINVAL
 *   hist        device uint64 [n_types (n_types + 1) / 2][n_bins], accumulated
 * The first call on a device, made while that device is current, looks the array's
 * address up (cudaGetSymbolAddress) and caches it for the life of that device's primary
 * context: after cudaDeviceReset the cached address is stale, so do not call this entry
 * point after a reset. Make the first call on a device before any stream capture.
 * Every call shares the array, so calls whose GPU work overlaps (other streams, other
 * host threads on the same device) race and corrupt each other's counts: serialise them.
 * Work is enqueued on `stream`. */
#define EPSR_NOALLOC_MAX_ATOMS 131072
size_t epsr_noalloc_scratch_bytes(void);
int epsr_partial_gr_noalloc(const int32_t *xyz, const int32_t *type, int64_t n_atoms,
                            int64_t L_fx, int32_t scale_log2, int32_t n_types, int32_t bin_p,
                            int32_t bin_q, int32_t n_bins, uint64_t *hist, epsr_stream_t stream);

/* ---- S(Q) by Eq. (1) ---------------------------------------------------------------------
 * Midpoint rule on bin centres r_k = (k + 1/2) dr:
 *   S_partial[c](Q_i) = w[c] sum_k K[i][k] (g[c][k] - 1),  K[i][k] = r_k^2 dr sin(Q_i r_k)/(Q_i r_k)
 *   S_total[s](Q_i)   = flat[s] + sum_{c in set s} S_partial[c](Q_i),
 * sets being consecutive groups of cols_per_set columns. A plan caches K for one
 * (Q grid, n_bins, dr, mode). mode EPSR_SQ_FP32 contracts on CUDA cores in FP32; the
 * split modes contract on tcgen05 tensor cores with FP32 accumulation in TMEM, K and G
 * split into hi + lo parts (lo = residual of hi) and the small cross terms kept.
 *   Q          host float [nQ] (> 0)
 *   g          device float [n_cols][n_bins]
 *   w, flat    host double [n_cols], [n_cols / cols_per_set]
 *   S_partial  device float [n_cols][nQ] or NULL;  S_total device float [n_sets][nQ] or NULL
 * epsr_sq_plan_create synchronises; epsr_sq_exec is asynchronous and allocates nothing
 * (graph-capturable). epsr_sq is a one-shot convenience (plan, exec, free).
 * Every tensor-core completion wait is bounded; one that gives up skips its tile and sets
 * the plan's status word, which epsr_sq_plan_status reads (synchronising `stream`; status
 * EPSR_OK or EPSR_ETIMEOUT, and the word is cleared) and epsr_sq checks before returning. */
int epsr_sq_plan_create(const float *Q, int32_t nQ, int32_t n_bins, double dr, int32_t mode,
                        int32_t max_cols, epsr_stream_t stream, epsr_sq_plan **out);
int epsr_sq_plan_destroy(epsr_sq_plan *plan);
int epsr_sq_plan_status(epsr_sq_plan *plan, int32_t *status, epsr_stream_t stream);
int epsr_sq_exec(epsr_sq_plan *plan, const float *g, int32_t n_cols, const double *w,
                 int32_t cols_per_set, const double *flat, float *S_partial, float *S_total,
                 epsr_stream_t stream);
int epsr_sq(const float *g, int32_t n_cols, int32_t n_bins, double dr, const float *Q,
            int32_t nQ, const double *w, int32_t cols_per_set, const double *flat,
            float *S_partial, float *S_total, int32_t mode, epsr_stream_t stream);
/* Tiling of the tensor-core modes (no counterpart in the paper; a performance setting that
 * does not change which products are summed, only how the K sum is split): n_chunk columns
 * of g per CTA (a multiple of 16, at most 256; when it is a multiple of cols_per_set the set
 * totals are formed in the same launch) and k_split CTAs per output tile along the bins (one
 * thread-block cluster, at most 8, at most the number of 128-byte K units), whose FP32
 * partials are added in a fixed order. 0 selects the built-in rule. EPSR_EINVAL for the FP32
 * mode (unless both are 0) or a tiling whose buffers do not fit in shared memory. Host only.
 * epsr_sq_plan_get_tiles reports the tiling an epsr_sq_exec of n_cols columns would use. */
int epsr_sq_plan_set_tiles(epsr_sq_plan *plan, int32_t n_chunk, int32_t k_split);
int epsr_sq_plan_get_tiles(const epsr_sq_plan *plan, int32_t n_cols, int32_t cols_per_set,
                           int32_t with_totals, int32_t *n_chunk, int32_t *k_split);

#ifdef __cplusplus
}
#endif
#endif /* EPSR_H */
