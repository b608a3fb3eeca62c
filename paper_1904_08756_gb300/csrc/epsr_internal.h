// epsr_internal.h -- host-side declarations shared by libepsr's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "epsr.h"

namespace epsr {

struct BoxDev;
struct MoveRec;

// ---- errors (thread-local last error, see epsr_last_error_detail) -------------------------
int set_error(int status, const char *fmt, ...);
int set_cuda_error(cudaError_t e, const char *what);

// ---- launch accounting (epsr_launch_count): called once after every kernel enqueue ----------
void note_launch();

// ---- autotuner support (epsr_tune.cu): the shape a tuning is cached under --------------------
std::string box_shape_key(const epsr_box *box);
struct BoxSummary {
    int n_boxes, n_pairs, n_bins;
    double kT, rho, dr;     // kJ/mol, atoms per A^3, A
};
int box_summary(const epsr_box *box, int b, BoxSummary *out);
int box_sms(const epsr_box *box);
std::string sq_plan_key(const epsr_sq_plan *p, int n_cols, int cols_per_set, bool totals);
int sq_plan_mode(const epsr_sq_plan *p);
void sq_plan_dims(const epsr_sq_plan *p, int *nQ, int *n_bins, int *max_cols);
int sq_plan_stages(const epsr_sq_plan *p);

// ---- Monte Carlo kernel ----------------------------------------------------------------------
constexpr size_t kMcMaxDynSmem = 176 * 1024;   // with about 44 KB of static shared memory, under the 227 KB per CTA
// exchange buffer of the sweep, per parity: the partial dU of every move of a batch from every
// CTA ([kMcBatchMax][grid]), then kMcSlotStride - kMcBatchMax = kMcCorrPerCta floats per CTA of
// which a box group uses its first CTA's share onwards for the batch-pair corrections
constexpr int kMcBatchMax = 64;           // moves per batch of the sweep, at most
constexpr int kMcCorrPerCta = kMcBatchMax * (kMcBatchMax - 1) / 2;   // batch-pair corrections
constexpr int kMcSlotStride = kMcBatchMax + kMcCorrPerCta;
// correction items of one batch in shared memory (>= 496 pairs x 8 atoms: batches above 32 moves
// need 8 or more CTAs per box)
constexpr int kMcCorrItems = 4096;
// partners staged per chunk in shared memory when the slices live in global memory
constexpr int kMcStageChunk = 2048;

struct McArgs {
    const BoxDev *boxes;
    int4 *coords;                 // [n_atoms_total] {x, y, z, type}
    const int *mol_start;         // concatenated box-local molecule starts
    const long long *thresholds;  // concatenated [n_bins + 1] per box
    const float *ep;              // concatenated [n_pairs * n_bins] per box
    const int *cta_box;           // [grid]
    float *slots;                 // [2][grid * kMcSlotStride]: partials [kBatchMax][grid], then corrections
                                  // [grid][kMcCorrPerCta] (a box group uses cta0 * kMcCorrPerCta onwards)
    unsigned *flags;              // [grid] arrival sequence numbers (zeroed per launch)
    epsr_mc_stats *stats;         // [n_boxes] running totals (device)
    epsr_move_log *log;           // nullable [n_boxes][log_stride]
    const MoveRec *moves;         // [n_boxes][chunk] this launch's moves
    const int *sorted_index;      // [n_atoms_total] atom at each type-major sorted position
    const int *pos_of;            // [n_atoms_total] sorted position of each atom
    const int *mc_offset;         // [total keys + 1] first sorted position of each key
    long long chunk;              // move-table stride per box
    long long log_off;            // log index of this launch's first move
    int *status;                  // device status word
    long long n_moves;
    unsigned long long seed, move0;
    long long log_stride;
    long long max_spin;           // iteration limit of one barrier wait
    unsigned long long timeout_ns;// time limit of one barrier wait
    int grid;
    int lj_cut;                   // 1: some box truncates Lennard-Jones (the cut instantiation runs)
    int batch_k;
    int slice_cap;                // int4 capacity of the shared partner slice
    int tbl_cap;                  // capacity (entries) of the shared threshold table
    int ep_cap;                   // capacity (entries) of the shared empirical-potential table
    int types_cap;                // largest number of atom types of the handle's boxes
    int4 *slice_g;                // [grid][slice_cap] partner slices in global memory, or NULL
    unsigned short *home_g;       // [grid][slice_cap] home cells of those slots, or NULL
    int cell_margin;              // drift (grid units) before a partner leaves its cell's queries
    int esc_cap;                  // escapee list capacity (0: no cell queries)
    int skip_arrival_cta;         // test hook: this CTA never arrives (-1: none)
};

int launch_mc_sweep(const McArgs &args, int grid, size_t smem, cudaStream_t stream);
int launch_mc_moves(const BoxDev *boxes, const int *mol_start, int n_boxes, long long chunk,
                    long long n, unsigned long long seed, unsigned long long move0, MoveRec *out,
                    cudaStream_t stream);
int launch_intra_energy(const BoxDev *boxes, int n_boxes, const int4 *coords, const int *mol_start, double *U,
                        cudaStream_t stream);
int mc_threads();
int mc_escapee_max();
int mc_batch_max();

// ---- pair histogram kernels ---------------------------------------------------------------
struct GrTile {           // one (i-tile, j-tile) pair of one box
    int box;
    int ti, tj;
    int pad;
};

struct GrArgs {
    const BoxDev *boxes;
    const int4 *coords;          // [n_atoms_total]
    const uint4 *scaled;         // [n_atoms_total] {x', y', z', type} on the 2^32-periodic grid
    const long long *thresholds;
    const GrTile *tiles;
    long long tile_begin, tile_end;
    unsigned long long *hist;    // accumulated output
    int max_pairs_bins;          // max over boxes of n_pairs * n_bins (shared histogram size)
    int max_bins1;               // max over boxes of n_bins + 1
};

constexpr int kGrTile = 1024;    // atoms per tile (both sides)

// Cell-list histogram: one work item per (box, home cell); pairs of the home cell with itself
// and with its 13 forward neighbours.
struct GcItem {
    int box, cell;
};

struct GcArgs {
    const BoxDev *boxes;
    const int4 *coords;          // [n_atoms_total] in cell-list order
    const uint4 *scaled;         // [n_atoms_total] in cell-list order
    const int *cell_start;       // [total cells + 1] first sorted position of each cell
    const int *cell_count;       // [total cells]
    const long long *thresholds;
    const GcItem *items;
    long long n_items;
    unsigned long long *hist;
    int max_pairs_bins, max_bins1;
};

int launch_partial_gr_cells(const GcArgs &args, int grid, cudaStream_t stream);
constexpr int kMcCells = 512;    // cells per (type, CTA) block of the Monte Carlo order

int launch_scale_coords(const BoxDev *boxes, const int *atom_box, const int4 *coords,
                        uint4 *scaled, long long n, cudaStream_t stream);
int launch_partial_gr(const GrArgs &args, int grid, cudaStream_t stream);

struct SortScratch {      // device scratch of the spatial sort
    int *count;           // [total_cells]
    int *offset;          // [total_cells]
    int *block;           // [ceil(total_cells / 1024)]
    int *key, *rank;      // [n_atoms_total]
    int *index;           // [n_atoms_total] atom index at each sorted position
};
int launch_spatial_sort(const BoxDev *boxes, const int *atom_box, const uint4 *scaled,
                        const int4 *coords, long long n, int total_cells, int type_major,
                        SortScratch sc, uint4 *s_scaled, int4 *s_coords, int *pos_of,
                        cudaStream_t stream);
int launch_normalize_g(const BoxDev *boxes, int n_boxes, const unsigned long long *hist,
                       float *g, long long n_configs, long long hist_len, const long long *hist_box,
                       cudaStream_t stream);
int launch_total_energy(const BoxDev *boxes, const int4 *coords, const int *atom_mol,
                        const long long *thresholds, const float *ep, const GrTile *tiles,
                        long long n_tiles, double *U, int grid, cudaStream_t stream);

// ---- smeared histogram and adjoint -----------------------------------------------------------
struct SmearArgs {
    const BoxDev *boxes;
    const int4 *coords;        // spatially sorted
    const uint4 *scaled;       // spatially sorted, 2^32-periodic copy
    const int *index;          // atom at each sorted position
    const GrTile *tiles;
    long long n_tiles;
    double sigma;
    unsigned long long *acc;   // forward output: weights * 2^24, accumulated
    const float *lambda;       // backward input: dL/dHt [hist_len]
    float *grad;               // backward output [n_atoms_total][3] (accumulated)
    int max_pairs_bins;
    // cell-list form (coords, index in cell order): items and cell ranges
    const GcItem *items;
    long long n_items;
    const int *cell_start, *cell_count;
};
int launch_smear(const SmearArgs &a, bool backward, int grid, cudaStream_t stream);
int launch_smear_cells(const SmearArgs &a, bool backward, int grid, cudaStream_t stream);
// cell-list cells are widened by this margin so that smearing with 5 sigma up to it fits
constexpr double kCellSmearMarginA = 0.5;
int launch_smear_norm(const BoxDev *boxes, int n_boxes, const unsigned long long *acc, double *Ht,
                      float *gt, long long hist_len, const long long *hist_box, cudaStream_t stream);
int launch_smear_lambda(const BoxDev *boxes, int n_boxes, const float *dgt, float *lam, long long hist_len,
                        const long long *hist_box, cudaStream_t stream);

// ---- empirical-potential update -------------------------------------------------------------
constexpr int kEpMaxData = 16;     // measured datasets
constexpr int kEpMaxBasis = 40;    // Poisson functions per pair
constexpr int kEpMaxPairs = EPSR_MAX_TYPES * (EPSR_MAX_TYPES + 1) / 2;

struct EpArgs {
    const float *dS;     // [n_data][nQ] device
    const float *Q;      // [nQ] device
    int nQ, n_data, n_pairs, n_basis, n_bins;
    double w[kEpMaxData * kEpMaxPairs];   // [n_data][n_pairs] Eq. (1) weights (barn)
    double s, gamma, alpha, kT, rho, dr;
    double *F;           // [n_basis][nQ] scratch
    double *Y;           // [n_pairs][nQ] scratch
    double *C_out;       // [n_pairs][n_basis] device
    float *ep;           // [n_pairs][n_bins] the box's table, updated in place
};
int launch_ep_update(const EpArgs &a, cudaStream_t stream);

struct ChiParams {
    int P, n_basis;
    double s, rho;
    double W[kEpMaxPairs];     // Eq. (1) weights (2 - delta) c_a c_b b_a b_b, barn
    double *res_scratch;       // [nQ] residuals
    double *F_scratch;         // [n_basis][nQ] basis values F_n(Q)
};
int launch_chi2(const float *S, const float *target, const float *Q, int nQ, const ChiParams &prm,
                const double *C, double *chi2, float *dS, double *dC, cudaStream_t stream);

// ---- S(Q) --------------------------------------------------------------------------------
int sq_build_kernel_matrix(const float *Q, int nQ, int n_bins, double dr, int mode, float *K32,
                           void *Ksplit, int ld_split, cudaStream_t stream);

}  // namespace epsr
