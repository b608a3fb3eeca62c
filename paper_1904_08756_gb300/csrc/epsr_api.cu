// epsr_api.cu -- host side of the libepsr C ABI: validation, exact tables, work lists,
// device buffers and kernel launches. No exception crosses the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "epsr.h"
#include "epsr_device.cuh"
#include "epsr_internal.h"
#include "k_sq.h"

using namespace epsr;

// ---- errors ------------------------------------------------------------------------------
static thread_local int g_last_status = EPSR_OK;
static thread_local char g_last_msg[512] = "";

int epsr::set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_msg, sizeof(g_last_msg), fmt, ap);
    va_end(ap);
    g_last_status = status;
    return status;
}

int epsr::set_cuda_error(cudaError_t e, const char *what)
{
    return set_error(EPSR_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

static std::atomic<unsigned long long> g_launches{0};

void epsr::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" int epsr_launch_count(uint64_t *count)
{
    if (!count) return set_error(EPSR_EINVAL, "NULL argument");
    *count = g_launches.load(std::memory_order_relaxed);
    return EPSR_OK;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return set_cuda_error(e_, #call);   \
    } while (0)

extern "C" const char *epsr_strerror(int status)
{
    switch (status) {
    case EPSR_OK: return "success";
    case EPSR_EINVAL: return "invalid argument";
    case EPSR_ENOMEM: return "out of memory";
    case EPSR_ECUDA: return "CUDA runtime error";
    case EPSR_ELAUNCH: return "persistent kernel cannot be co-resident";
    case EPSR_ETIMEOUT: return "device-side wait timed out";
    case EPSR_ENUMERIC: return "non-finite result";
    default: return "unknown status";
    }
}

extern "C" int epsr_last_error_detail(char *buf, size_t len)
{
    if (buf && len) {
        strncpy(buf, g_last_msg, len - 1);
        buf[len - 1] = '\0';
    }
    return g_last_status;
}

extern "C" int epsr_version(void) { return 10000; }

// ---- physical constants (SI exact values; eps0 CODATA 2018) --------------------------------
static double coulomb_k()   // e^2 N_A / (4 pi eps0), kJ A / mol / e^2
{
    const double e = 1.602176634e-19, NA = 6.02214076e23, eps0 = 8.8541878128e-12;
    const double pi = 3.14159265358979323846;
    return e * e * NA / (4.0 * pi * eps0) * 1e10 * 1e-3;
}

static double gas_r() { return 1.380649e-23 * 6.02214076e23 * 1e-3; }   // kJ / mol / K

// ---- handle -------------------------------------------------------------------------------
template <class T>
static int dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(EPSR_ENOMEM, "cudaMalloc of %zu bytes failed", n * sizeof(T));
    }
    return EPSR_OK;
}

struct epsr_box {
    int n_boxes = 0;
    long long n_atoms = 0;
    long long hist_len = 0;
    std::vector<epsr_box_desc> desc;
    std::vector<BoxDev> hb;              // host copy of per-box parameters
    std::vector<long long> hist_box_h;   // hist_off per box (ascending)
    std::vector<int> mol_h;              // concatenated mol_start (box-local, int32)
    std::vector<int> type_h;
    std::vector<GrTile> tiles_h;
    int sms = 0;
    int mc_batch = 0;                         // 0: chosen per box by the kernel
    int cell_margin = 1 << 20;                // 1 A on the 2^20 grid
    int esc_cap = -1;                         // -1: the kernel's maximum
    int mc_ctas = 0;
    int gr_ctas_per_sm = 4;                   // persistent CTAs per SM of the all-pairs histogram
    int fault_cta = -1;
    double timeout_ms = 2000.0;
    // device
    BoxDev *boxes = nullptr;
    int4 *coords = nullptr;
    uint4 *scaled = nullptr;
    int *mol_start = nullptr;
    int *atom_box = nullptr;
    int *atom_mol = nullptr;
    long long *thresholds = nullptr;
    float *ep = nullptr;
    GrTile *tiles = nullptr;
    long long *hist_box = nullptr;
    int *cta_box = nullptr;
    int cta_box_len = 0;
    float *slots = nullptr;
    unsigned *flags = nullptr;
    epsr_mc_stats *stats = nullptr;
    int *status = nullptr;
    double *U = nullptr;
    int tbl_cap = 0, ep_cap = 0;
    // spatial sort of the pair scan
    int total_cells = 0;
    SortScratch sort{};
    uint4 *sorted_scaled = nullptr;
    int4 *sorted_coords = nullptr;
    // Monte Carlo move table and type-major spatial partition
    MoveRec *moves = nullptr;
    long long moves_cap = 0;
    int total_mc_cells = 0;
    SortScratch mc_sort{};
    int *pos_of = nullptr;
    // empirical-potential update scratch (allocated on first use)
    double *ep_F = nullptr, *ep_Y = nullptr, *ep_C = nullptr;
    float *ep_Q = nullptr;
    long long ep_cap_Q = 0;
    float *lambda = nullptr;     // adjoint of the smeared normalisation [hist_len]
    unsigned long long *smear_acc = nullptr;   // fixed-point smeared counts [hist_len]
    // cell-list histogram: keys, items, per-box tile ranges of the all-pairs list (fallback)
    int total_gcells = 0;
    std::vector<GcItem> gc_items_h;
    GcItem *gc_items = nullptr;
    int *gc_count = nullptr, *gc_offset = nullptr, *gc_block = nullptr;
    uint4 *gc_scaled = nullptr;
    int4 *gc_coords = nullptr;
    std::vector<long long> tile_lo, tile_hi;
    // partner slices in global memory, for boxes whose slices do not fit in shared memory
    int4 *slice_g = nullptr;
    unsigned short *home_g = nullptr;
    size_t slice_g_cap = 0;

    ~epsr_box()
    {
        void *ptrs[] = {boxes, coords, scaled, mol_start, atom_box, atom_mol, thresholds, ep,
                        tiles, hist_box, cta_box, slots, flags, stats, status, U,
                        sort.count, sort.offset, sort.block, sort.key, sort.rank, sort.index,
                        sorted_scaled, sorted_coords, moves, mc_sort.count, mc_sort.offset,
                        mc_sort.block, mc_sort.key, mc_sort.rank, mc_sort.index, pos_of,
                        ep_F, ep_Y, ep_C, ep_Q, lambda, smear_acc, slice_g, home_g,
                        gc_items, gc_count, gc_offset, gc_block, gc_scaled, gc_coords};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
};

static int validate_desc(const epsr_box_desc &d, int b)
{
    if (d.n_atoms < 1 || d.n_atoms > (1LL << 28))
        return set_error(EPSR_EINVAL, "box %d: n_atoms %lld out of range", b, (long long)d.n_atoms);
    if (d.n_mol < 1 || d.n_mol > d.n_atoms)
        return set_error(EPSR_EINVAL, "box %d: n_mol %lld out of range", b, (long long)d.n_mol);
    if (d.L_fx < 2 || d.L_fx >= (1LL << 31))
        return set_error(EPSR_EINVAL, "box %d: L_fx %lld out of range", b, (long long)d.L_fx);
    if (d.scale_log2 < 10 || d.scale_log2 > 24)
        return set_error(EPSR_EINVAL, "box %d: scale_log2 %d out of range", b, d.scale_log2);
    if (d.n_types < 1 || d.n_types > EPSR_MAX_TYPES)
        return set_error(EPSR_EINVAL, "box %d: n_types %d out of range", b, d.n_types);
    if (d.bin_p < 1 || d.bin_q < 1 || d.n_bins < 1 || d.n_bins > EPSR_MAX_BINS)
        return set_error(EPSR_EINVAL, "box %d: bins (%d/%d, %d) invalid", b, d.bin_p, d.bin_q, d.n_bins);
    if (d.move_kind != EPSR_MOVE_ATOM && d.move_kind != EPSR_MOVE_RIGID_MOLECULE &&
        d.move_kind != EPSR_MOVE_FLEXIBLE_MOLECULE)
        return set_error(EPSR_EINVAL, "box %d: move_kind %d invalid", b, d.move_kind);
    if (d.move_kind == EPSR_MOVE_FLEXIBLE_MOLECULE)
        for (int a = 0; a < d.n_types; ++a)
            for (int c = 0; c < d.n_types; ++c) {
                const double k = d.bond_k[a * EPSR_MAX_TYPES + c], r0 = d.bond_d[a * EPSR_MAX_TYPES + c];
                if (!(k >= 0) || !std::isfinite(k) || !(r0 >= 0) || !std::isfinite(r0) ||
                    k != d.bond_k[c * EPSR_MAX_TYPES + a] || r0 != d.bond_d[c * EPSR_MAX_TYPES + a])
                    return set_error(EPSR_EINVAL, "box %d: spring of types %d-%d invalid or not symmetric", b, a, c);
            }
    if (!(d.temperature > 0) || !(d.max_translation >= 0) || !(d.max_rotation_deg >= 0) ||
        !(d.max_rotation_deg < 180) || !(d.r_coul >= 0) || !(d.r_lj >= 0) || !(d.r_lj < 1e6))
        return set_error(EPSR_EINVAL, "box %d: temperature/move/cutoff parameters invalid", b);
    const double S = std::ldexp(1.0, d.scale_log2);
    if (d.max_translation * S > 0.25 * (double)d.L_fx)
        return set_error(EPSR_EINVAL, "box %d: max_translation too large for the box", b);
    for (int t = 0; t < d.n_types; ++t)
        if (!std::isfinite(d.q[t]) || !std::isfinite(d.sigma[t]) || !(d.eps[t] >= 0) ||
            !std::isfinite(d.eps[t]) || !(d.sigma[t] >= 0) || !std::isfinite(d.b[t]))
            return set_error(EPSR_EINVAL, "box %d: force field of type %d invalid", b, t);
    // the table edge r_max must map to a 63-bit squared distance
    const double rmax_fx = (double)d.n_bins * d.bin_p / d.bin_q * S;
    if (rmax_fx * rmax_fx > 4.0e18)
        return set_error(EPSR_EINVAL, "box %d: bin range too large", b);
    return EPSR_OK;
}

// Exact threshold table: T[k] = ceil((k p S / q)^2), k = 0..n_bins, so that
// d2 >= T[k] <=> sqrt(d2) >= k dr (d2 integer).
static void build_thresholds(const epsr_box_desc &d, long long *T)
{
    const unsigned __int128 q2 = (unsigned __int128)d.bin_q * d.bin_q;
    for (int k = 0; k <= d.n_bins; ++k) {
        const unsigned __int128 num = ((unsigned __int128)k * k * d.bin_p * d.bin_p) << (2 * d.scale_log2);
        T[k] = (long long)((num + q2 - 1) / q2);
    }
}

static void fill_boxdev(const epsr_box_desc &d, const int *type, BoxDev &b)
{
    memset(&b, 0, sizeof(b));
    const double S = std::ldexp(1.0, d.scale_log2);
    b.n_atoms = (int)d.n_atoms;
    b.n_mol = (int)d.n_mol;
    b.L = (int)d.L_fx;
    b.n_types = d.n_types;
    b.n_pairs = d.n_types * (d.n_types + 1) / 2;
    b.n_bins = d.n_bins;
    b.move_kind = d.move_kind;
    b.max_shift = (int)std::llround(d.max_translation * S);
    const long long rc = std::llround(d.r_coul * S);
    b.rc2 = rc * rc;
    b.lj_cut = d.r_lj > 0.0 ? 1 : 0;
    const long long rl = b.lj_cut ? std::llround(d.r_lj * S) : 0;
    b.lj2 = rl * rl;
    b.lj2_lo = (float)((double)b.lj2 * (1.0 - 0x1p-20));
    b.lj2_hi = (float)((double)b.lj2 * (1.0 + 0x1p-20));
    const double pi = 3.14159265358979323846;
    b.h_rot = std::tan(0.5 * d.max_rotation_deg * pi / 180.0) / std::sqrt(3.0);
    if (d.move_kind == EPSR_MOVE_FLEXIBLE_MOLECULE)
        for (int i = 0; i < EPSR_MAX_TYPES * EPSR_MAX_TYPES; ++i) {
            b.bond_k[i] = d.bond_k[i];
            b.bond_d[i] = d.bond_d[i];
        }
    b.kT = gas_r() * d.temperature;
    const double LA = (double)d.L_fx / S;
    b.volume = LA * LA * LA;
    b.dr_A = (double)d.bin_p / (double)d.bin_q;
    b.inv_s2 = (float)std::ldexp(1.0, -2 * d.scale_log2);
    b.sc_rcp = UINT64_MAX / (uint64_t)d.L_fx;
    const double unit = (double)d.L_fx * 0x1p-32;                  // grid units per 2^32-grid unit
    b.sc_s2 = (float)(unit * unit * std::ldexp(1.0, -2 * d.scale_log2));
    b.sc_k2 = (float)(1.0 / (unit * unit));
    b.inv_dr_fx = (float)((double)d.bin_q / ((double)d.bin_p * S));
    for (long long i = 0; i < d.n_atoms; ++i) b.count[type[i]]++;
    const double ke = coulomb_k();
    for (int a = 0; a < kMaxTypes; ++a)
        for (int c = 0; c < kMaxTypes; ++c) {
            PairRow &r = b.row[a * kMaxTypes + c];
            r.c12 = r.c6 = r.kqq = 0.f;
            r.pair = 0;
            if (a >= d.n_types || c >= d.n_types) continue;
            const double eps = std::sqrt(d.eps[a] * d.eps[c]);
            const double sig = 0.5 * (d.sigma[a] + d.sigma[c]);
            if (eps > 0.0) {
                const double s6 = std::pow(sig, 6.0);
                r.c12 = (float)(4.0 * eps * s6 * s6);
                r.c6 = (float)(4.0 * eps * s6);
            }
            r.kqq = (float)(ke * d.q[a] * d.q[c]);
            r.pair = pair_index(a, c, d.n_types);
        }
}

// Radius (grid units) beyond which a pair has no Coulomb, no empirical-potential and, when the
// Lennard-Jones term is cut, no Lennard-Jones term.
static void set_near(BoxDev &bx)
{
    const long long lim = std::max<long long>(std::max<long long>(bx.rc2, bx.has_ep ? bx.tmax : 0LL),
                                              bx.lj_cut ? bx.lj2 : 0LL);
    bx.near_fx = (int)std::ceil(std::sqrt((double)lim)) + 1;
}

static void plan_mc_groups(epsr_box *h)
{
    // CTAs per box: a single box uses up to one CTA per SM, at least ~512 partner atoms
    // per CTA; a batch gives each box one CTA, then the rest greedily to the largest slices.
    const int nb = h->n_boxes;
    const int budget = h->mc_ctas > 0 ? h->mc_ctas : h->sms;
    h->total_mc_cells = 0;
    std::vector<int> G(nb, 1);
    if (nb == 1) {
        long long want = (h->hb[0].n_atoms + 511) / 512;
        G[0] = (int)std::max(1LL, std::min<long long>(want, budget));
    } else {
        // every box starts with one CTA; each further CTA goes to the box whose per-CTA
        // slice is largest (the slowest group of the persistent kernel)
        int used = nb;
        while (used < budget) {
            int imax = 0;
            long long worst = -1;
            for (int i = 0; i < nb; ++i) {
                const long long c = (h->hb[i].n_atoms + G[i] - 1) / G[i];
                if (c > worst) { worst = c; imax = i; }
            }
            if (worst <= 512) break;          // small slices gain nothing from another CTA
            ++G[imax];
            ++used;
        }
    }
    int c0 = 0;
    for (int i = 0; i < nb; ++i) {
        BoxDev &b = h->hb[i];
        b.cta0 = c0;
        b.n_cta = G[i];
        // slice capacity: the most atoms any CTA gets (atom j goes to CTA j mod G)
        const long long cap = (b.n_atoms + G[i] - 1) / G[i];
        b.chunk = (int)cap;
        b.mc_cell0 = h->total_mc_cells;
        h->total_mc_cells += b.n_types * G[i] * kMcCells;
        c0 += G[i];
    }
    h->cta_box_len = c0;
}

// Shared-memory layout of the sweep for the current CTA split: thresholds, EP table, cell
// index [types][513] (uint32), correction items, and, when they fit, the partner slice (int4 per
// slot, and its copy on the 2^32-periodic grid) and the home cell of every slot (uint16); otherwise the slices and home cells live in
// global memory and a chunk of partners is staged.
struct McLayout {
    int slice_cap = 0, types_cap = 1;
    size_t smem = 0;
    bool gslice = false;
};

static int mc_layout(const epsr_box *h, McLayout *L)
{
    for (auto &b : h->hb) L->slice_cap = std::max(L->slice_cap, b.chunk);
    for (auto &b : h->hb) L->types_cap = std::max(L->types_cap, b.n_types);
    const size_t tables = (size_t)h->tbl_cap * sizeof(long long) + (size_t)h->ep_cap * sizeof(float) +
                          (size_t)L->types_cap * (kMcCells + 1) * sizeof(unsigned) +
                          (size_t)kMcBatchMax * kMcBatchMax * sizeof(float) + (size_t)kMcCorrItems * sizeof(float);
    const size_t per_slot = 2 * sizeof(int4) + sizeof(unsigned short);   // slot, its 2^32-grid copy, home cell
    L->smem = (((size_t)L->slice_cap * per_slot + tables) + 15) & ~(size_t)15;
    L->gslice = L->smem > kMcMaxDynSmem;
    if (L->gslice) {
        L->smem = ((tables + 15) & ~(size_t)15) + (size_t)kMcStageChunk * sizeof(int4);
        if (L->smem > kMcMaxDynSmem)
            return set_error(EPSR_EINVAL, "mc sweep: %zu bytes of tables per CTA (limit %zu)", L->smem, kMcMaxDynSmem);
    }
    return EPSR_OK;
}

// Global-memory slices of the partners when the layout needs them (allocated here, outside
// any sweep, so that a sweep can be captured in a CUDA graph).
static int alloc_mc_slices(epsr_box *h)
{
    McLayout L;
    int rc = mc_layout(h, &L);
    if (rc) return rc;
    if (!L.gslice) return EPSR_OK;
    const size_t slots = (size_t)h->cta_box_len * L.slice_cap;
    if (h->slice_g_cap >= slots) return EPSR_OK;
    if (h->slice_g) cudaFree(h->slice_g);
    if (h->home_g) cudaFree(h->home_g);
    h->slice_g = nullptr;
    h->home_g = nullptr;
    h->slice_g_cap = 0;
    rc = dalloc(&h->slice_g, slots);
    if (!rc) rc = dalloc(&h->home_g, slots);
    if (rc) return rc;
    h->slice_g_cap = slots;
    return EPSR_OK;
}

static int upload_mc_groups(epsr_box *h)
{
    std::vector<int> cb;
    for (int i = 0; i < h->n_boxes; ++i)
        for (int k = 0; k < h->hb[i].n_cta; ++k) cb.push_back(i);
    if (h->cta_box) cudaFree(h->cta_box);
    if (h->slots) cudaFree(h->slots);
    if (h->flags) cudaFree(h->flags);
    h->cta_box = nullptr; h->slots = nullptr; h->flags = nullptr;
    int rc;
    if ((rc = dalloc(&h->cta_box, cb.size())) || (rc = dalloc(&h->slots, 2 * cb.size() * kMcSlotStride)) ||
        (rc = dalloc(&h->flags, cb.size())))
        return rc;
    if (h->mc_sort.count) cudaFree(h->mc_sort.count);
    if (h->mc_sort.offset) cudaFree(h->mc_sort.offset);
    if (h->mc_sort.block) cudaFree(h->mc_sort.block);
    h->mc_sort.count = h->mc_sort.offset = h->mc_sort.block = nullptr;
    if ((rc = dalloc(&h->mc_sort.count, h->total_mc_cells + 1)) ||
        (rc = dalloc(&h->mc_sort.offset, h->total_mc_cells + 1)) ||
        (rc = dalloc(&h->mc_sort.block, (h->total_mc_cells + 1 + 1023) / 1024)))
        return rc;
    CK(cudaMemcpy(h->cta_box, cb.data(), cb.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->boxes, h->hb.data(), h->hb.size() * sizeof(BoxDev), cudaMemcpyHostToDevice));
    return alloc_mc_slices(h);
}

static int create_impl(const epsr_box_desc *descs, int n_boxes, const int32_t *xyz,
                       const int32_t *type, const int64_t *mol_start, cudaStream_t stream,
                       epsr_box **out)
{
    if (!out) return set_error(EPSR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs || !xyz || !type || !mol_start || n_boxes < 1 || n_boxes > 65536)
        return set_error(EPSR_EINVAL, "NULL array or n_boxes out of range");
    epsr_box *h = new (std::nothrow) epsr_box();
    if (!h) return set_error(EPSR_ENOMEM, "host allocation failed");
    h->n_boxes = n_boxes;
    h->desc.assign(descs, descs + n_boxes);
    h->hb.resize(n_boxes);
    long long atom0 = 0, mol0 = 0, hist0 = 0;
    int tbl0 = 0, ep0 = 0;
    for (int b = 0; b < n_boxes; ++b) {
        const epsr_box_desc &d = descs[b];
        int rc = validate_desc(d, b);
        if (rc) { delete h; return rc; }
        const int32_t *ty = type + atom0;
        for (long long i = 0; i < d.n_atoms; ++i)
            if (ty[i] < 0 || ty[i] >= d.n_types) { delete h; return set_error(EPSR_EINVAL, "box %d: type[%lld] = %d out of range", b, i, ty[i]); }
        for (long long i = 0; i < 3 * d.n_atoms; ++i) {
            const int32_t v = xyz[3 * atom0 + i];
            if (v < 0 || v >= d.L_fx) { delete h; return set_error(EPSR_EINVAL, "box %d: coordinate %lld = %d outside [0, L_fx)", b, i, v); }
        }
        const int64_t *ms = mol_start + mol0;
        if (ms[0] != 0 || ms[d.n_mol] != d.n_atoms) { delete h; return set_error(EPSR_EINVAL, "box %d: mol_start must run from 0 to n_atoms", b); }
        for (long long m = 0; m < d.n_mol; ++m) {
            const long long sz = ms[m + 1] - ms[m];
            if (sz < 1) { delete h; return set_error(EPSR_EINVAL, "box %d: mol_start not strictly increasing at %lld", b, m); }
            if (d.move_kind == EPSR_MOVE_ATOM && sz != 1) { delete h; return set_error(EPSR_EINVAL, "box %d: atom moves need single-atom molecules", b); }
            if (sz > EPSR_MAX_MOL_ATOMS) { delete h; return set_error(EPSR_EINVAL, "box %d: molecule %lld has %lld > %d atoms", b, m, sz, EPSR_MAX_MOL_ATOMS); }
            // rigid rotations use 32-bit intermediates: molecule extent below 2^25 grid units
            for (long long i = ms[m]; i < ms[m + 1]; ++i)
                for (int c = 0; c < 3; ++c) {
                    long long dd = (long long)xyz[3 * (atom0 + i) + c] - xyz[3 * (atom0 + ms[m]) + c];
                    if (2 * dd > d.L_fx) dd -= d.L_fx;
                    else if (2 * dd <= -d.L_fx) dd += d.L_fx;
                    if (dd >= (1LL << 25) || dd <= -(1LL << 25)) { delete h; return set_error(EPSR_EINVAL, "box %d: molecule %lld wider than 2^25 grid units", b, m); }
                }
        }
        BoxDev &bx = h->hb[b];
        fill_boxdev(d, ty, bx);
        bx.atom0 = atom0;
        bx.mol0 = mol0;
        bx.hist_off = hist0;
        bx.tbl_off = tbl0;
        bx.ep_off = ep0;
        h->hist_box_h.push_back(hist0);
        for (long long m = 0; m <= d.n_mol; ++m) h->mol_h.push_back((int)ms[m]);
        atom0 += d.n_atoms;
        mol0 += d.n_mol + 1;
        hist0 += (long long)bx.n_pairs * bx.n_bins;
        tbl0 += bx.n_bins + 1;
        ep0 += bx.n_pairs * bx.n_bins;
        h->tbl_cap = std::max(h->tbl_cap, bx.n_bins + 1);
        h->ep_cap = std::max(h->ep_cap, bx.n_pairs * bx.n_bins);
    }
    h->n_atoms = atom0;
    h->hist_len = hist0;
    // thresholds, prefilter widths
    std::vector<long long> T(tbl0);
    for (int b = 0; b < n_boxes; ++b) {
        BoxDev &bx = h->hb[b];
        build_thresholds(descs[b], &T[bx.tbl_off]);
        bx.tmax = T[bx.tbl_off + bx.n_bins];
        bx.tmax_lo = (float)((double)bx.tmax * (1.0 - 0x1p-20));
        bx.tmax_hi = (float)((double)bx.tmax * (1.0 + 0x1p-20));
        bx.rc2_lo = (float)((double)bx.rc2 * (1.0 - 0x1p-20));
        bx.rc2_hi = (float)((double)bx.rc2 * (1.0 + 0x1p-20));
        const double LA = (double)bx.L / std::ldexp(1.0, descs[b].scale_log2);
        int nc = (int)std::floor(LA / 3.0);
        nc = std::max(1, std::min(nc, 32));
        int p2 = 1;
        while (p2 < nc) p2 <<= 1;
        bx.cells = nc;
        bx.cells_p3 = p2 * p2 * p2;
        bx.cell0 = h->total_cells;
        h->total_cells += p2 * p2 * p2;
        long long ts = 0;
        for (int t = 0; t < bx.n_types; ++t) {
            bx.type_start[t] = (int)ts;
            ts += bx.count[t];
        }
        set_near(bx);
        set_prefilter(bx);
        // cell-list histogram: cells at least the histogram range plus two grid units wide
        const long long rcut = (long long)std::ceil(std::sqrt((double)bx.tmax)) + 2 +
                               (long long)std::ceil(kCellSmearMarginA * std::ldexp(1.0, descs[b].scale_log2));
        long long side = 1;                       // more cells than atoms gain nothing
        while (side * side * side < bx.n_atoms) ++side;
        const long long gn = std::min<long long>(std::min<long long>(bx.L / rcut, side), 512);
        bx.gc_n = gn >= 3 ? (int)gn : 0;
        bx.gc0 = h->total_gcells;
        h->total_gcells += bx.gc_n ? bx.gc_n * bx.gc_n * bx.gc_n : 1;
        for (int c = 0; c < bx.gc_n * bx.gc_n * bx.gc_n; ++c) h->gc_items_h.push_back(GcItem{b, c});
    }
    // g(r) work list: upper triangle of tile pairs per box
    for (int b = 0; b < n_boxes; ++b) {
        const int nt = (h->hb[b].n_atoms + kGrTile - 1) / kGrTile;
        h->tile_lo.push_back((long long)h->tiles_h.size());
        for (int i = 0; i < nt; ++i)
            for (int j = i; j < nt; ++j) h->tiles_h.push_back(GrTile{b, i, j, 0});
        h->tile_hi.push_back((long long)h->tiles_h.size());
    }
    // per-atom arrays
    std::vector<int4> c4(atom0);
    std::vector<int> abox(atom0), amol(atom0);
    long long a = 0, mo = 0;
    for (int b = 0; b < n_boxes; ++b) {
        const epsr_box_desc &d = descs[b];
        for (long long m = 0; m < d.n_mol; ++m)
            for (long long i = mol_start[mo + m]; i < mol_start[mo + m + 1]; ++i) amol[a + i] = (int)m;
        for (long long i = 0; i < d.n_atoms; ++i, ++a) {
            c4[a] = make_int4(xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2], type[a]);
            abox[a] = b;
        }
        mo += d.n_mol + 1;
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
    int rc;
    if ((rc = dalloc(&h->boxes, n_boxes)) || (rc = dalloc(&h->coords, atom0)) ||
        (rc = dalloc(&h->scaled, atom0)) || (rc = dalloc(&h->mol_start, h->mol_h.size())) ||
        (rc = dalloc(&h->atom_box, atom0)) || (rc = dalloc(&h->atom_mol, atom0)) ||
        (rc = dalloc(&h->thresholds, T.size())) || (rc = dalloc(&h->ep, (size_t)ep0)) ||
        (rc = dalloc(&h->tiles, h->tiles_h.size())) || (rc = dalloc(&h->hist_box, n_boxes)) ||
        (rc = dalloc(&h->stats, n_boxes)) || (rc = dalloc(&h->status, 1)) ||
        (rc = dalloc(&h->U, n_boxes)) || (rc = dalloc(&h->sort.count, h->total_cells)) ||
        (rc = dalloc(&h->sort.offset, h->total_cells)) ||
        (rc = dalloc(&h->sort.block, (h->total_cells + 1023) / 1024)) ||
        (rc = dalloc(&h->sort.key, atom0)) || (rc = dalloc(&h->sort.rank, atom0)) ||
        (rc = dalloc(&h->sort.index, atom0)) ||
        (rc = dalloc(&h->sorted_scaled, atom0)) || (rc = dalloc(&h->sorted_coords, atom0)) ||
        (rc = dalloc(&h->mc_sort.key, atom0)) || (rc = dalloc(&h->mc_sort.rank, atom0)) ||
        (rc = dalloc(&h->mc_sort.index, atom0)) || (rc = dalloc(&h->pos_of, atom0)) ||
        (rc = dalloc(&h->lambda, (size_t)hist0)) || (rc = dalloc(&h->smear_acc, (size_t)hist0)) ||
        (rc = dalloc(&h->gc_items, std::max<size_t>(1, h->gc_items_h.size()))) ||
        (rc = dalloc(&h->gc_count, (size_t)h->total_gcells + 1)) ||
        (rc = dalloc(&h->gc_offset, (size_t)h->total_gcells + 1)) ||
        (rc = dalloc(&h->gc_block, ((size_t)h->total_gcells + 1 + 1023) / 1024)) ||
        (rc = dalloc(&h->gc_scaled, atom0)) || (rc = dalloc(&h->gc_coords, atom0))) {
        delete h;
        return rc;
    }
#define CKD(call)                                                            \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) { int r_ = set_cuda_error(e_, #call); delete h; return r_; } \
    } while (0)
    CKD(cudaMemcpyAsync(h->coords, c4.data(), atom0 * sizeof(int4), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemcpyAsync(h->mol_start, h->mol_h.data(), h->mol_h.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemcpyAsync(h->atom_box, abox.data(), atom0 * sizeof(int), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemcpyAsync(h->atom_mol, amol.data(), atom0 * sizeof(int), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemcpyAsync(h->thresholds, T.data(), T.size() * sizeof(long long), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemsetAsync(h->ep, 0, (size_t)std::max(ep0, 1) * sizeof(float), stream));
    CKD(cudaMemcpyAsync(h->tiles, h->tiles_h.data(), h->tiles_h.size() * sizeof(GrTile), cudaMemcpyHostToDevice, stream));
    if (!h->gc_items_h.empty())
        CKD(cudaMemcpyAsync(h->gc_items, h->gc_items_h.data(), h->gc_items_h.size() * sizeof(GcItem), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemcpyAsync(h->hist_box, h->hist_box_h.data(), n_boxes * sizeof(long long), cudaMemcpyHostToDevice, stream));
    CKD(cudaMemsetAsync(h->stats, 0, n_boxes * sizeof(epsr_mc_stats), stream));
    CKD(cudaMemsetAsync(h->status, 0, sizeof(int), stream));
    CKD(cudaStreamSynchronize(stream));
    plan_mc_groups(h);
    if ((rc = upload_mc_groups(h))) { delete h; return rc; }
    // move table: up to 65,536 moves per box and launch, at most 2^22 moves in total
    h->moves_cap = std::max<long long>(1024, std::min<long long>(65536, (1LL << 22) / n_boxes)) * n_boxes;
    if ((rc = dalloc(&h->moves, (size_t)h->moves_cap))) { delete h; return rc; }
    *out = h;
    return EPSR_OK;
}

extern "C" int epsr_box_create(const epsr_box_desc *desc, const int32_t *xyz, const int32_t *type,
                               const int64_t *mol_start, epsr_stream_t stream, epsr_box **out)
{
    return create_impl(desc, 1, xyz, type, mol_start, (cudaStream_t)stream, out);
}

extern "C" int epsr_batch_create(const epsr_box_desc *descs, int32_t n_boxes, const int32_t *xyz,
                                 const int32_t *type, const int64_t *mol_start, epsr_stream_t stream,
                                 epsr_box **out)
{
    return create_impl(descs, n_boxes, xyz, type, mol_start, (cudaStream_t)stream, out);
}

extern "C" int epsr_box_destroy(epsr_box *box)
{
    if (!box) return EPSR_OK;
    cudaDeviceSynchronize();
    delete box;
    return EPSR_OK;
}

extern "C" int epsr_box_info(const epsr_box *box, int32_t *n_boxes, int64_t *n_atoms_total,
                             int64_t *hist_len)
{
    if (!box) return set_error(EPSR_EINVAL, "box is NULL");
    if (n_boxes) *n_boxes = box->n_boxes;
    if (n_atoms_total) *n_atoms_total = box->n_atoms;
    if (hist_len) *hist_len = box->hist_len;
    return EPSR_OK;
}

extern "C" int epsr_box_offsets(const epsr_box *box, int32_t b, int64_t *hist_offset,
                                int64_t *atom_offset)
{
    if (!box || b < 0 || b >= box->n_boxes) return set_error(EPSR_EINVAL, "bad box or index");
    if (hist_offset) *hist_offset = box->hb[b].hist_off;
    if (atom_offset) *atom_offset = box->hb[b].atom0;
    return EPSR_OK;
}

// int4 {x,y,z,type} <-> int32 [n][3]
__global__ static void pack_xyz_kernel(const int4 *c, int *xyz, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int4 v = c[i];
        xyz[3 * i] = v.x; xyz[3 * i + 1] = v.y; xyz[3 * i + 2] = v.z;
    }
}

__global__ static void unpack_xyz_kernel(const int *xyz, int4 *c, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int4 v = c[i];
        v.x = xyz[3 * i]; v.y = xyz[3 * i + 1]; v.z = xyz[3 * i + 2];
        c[i] = v;
    }
}

static int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

extern "C" int epsr_box_get_coords_device(epsr_box *box, int32_t *xyz_dev, epsr_stream_t stream)
{
    if (!box || !xyz_dev) return set_error(EPSR_EINVAL, "NULL argument");
    pack_xyz_kernel<<<grid_for(box->n_atoms), 256, 0, (cudaStream_t)stream>>>(box->coords, xyz_dev, box->n_atoms);
    note_launch();
    CK(cudaGetLastError());
    return EPSR_OK;
}

extern "C" int epsr_box_set_coords_device(epsr_box *box, const int32_t *xyz_dev, epsr_stream_t stream)
{
    if (!box || !xyz_dev) return set_error(EPSR_EINVAL, "NULL argument");
    unpack_xyz_kernel<<<grid_for(box->n_atoms), 256, 0, (cudaStream_t)stream>>>(xyz_dev, box->coords, box->n_atoms);
    note_launch();
    CK(cudaGetLastError());
    return EPSR_OK;
}

extern "C" int epsr_box_get_coords(epsr_box *box, int32_t *xyz, epsr_stream_t stream)
{
    if (!box || !xyz) return set_error(EPSR_EINVAL, "NULL argument");
    std::vector<int4> c(box->n_atoms);
    CK(cudaMemcpyAsync(c.data(), box->coords, box->n_atoms * sizeof(int4), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    for (long long i = 0; i < box->n_atoms; ++i) {
        xyz[3 * i] = c[i].x; xyz[3 * i + 1] = c[i].y; xyz[3 * i + 2] = c[i].z;
    }
    return EPSR_OK;
}

extern "C" int epsr_box_set_coords(epsr_box *box, const int32_t *xyz, epsr_stream_t stream)
{
    if (!box || !xyz) return set_error(EPSR_EINVAL, "NULL argument");
    std::vector<int4> c(box->n_atoms);
    CK(cudaMemcpyAsync(c.data(), box->coords, box->n_atoms * sizeof(int4), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    for (int b = 0; b < box->n_boxes; ++b) {
        const BoxDev &bx = box->hb[b];
        for (long long i = bx.atom0; i < bx.atom0 + bx.n_atoms; ++i)
            for (int a = 0; a < 3; ++a) {
                const int v = xyz[3 * i + a];
                if (v < 0 || v >= bx.L) return set_error(EPSR_EINVAL, "coordinate %lld outside [0, L_fx)", 3 * i + a);
            }
    }
    for (long long i = 0; i < box->n_atoms; ++i) {
        c[i].x = xyz[3 * i]; c[i].y = xyz[3 * i + 1]; c[i].z = xyz[3 * i + 2];
    }
    CK(cudaMemcpyAsync(box->coords, c.data(), box->n_atoms * sizeof(int4), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return EPSR_OK;
}

extern "C" int epsr_box_set_ep(epsr_box *box, int32_t b, const float *ep, epsr_stream_t stream)
{
    if (!box || !ep || b < 0 || b >= box->n_boxes) return set_error(EPSR_EINVAL, "bad argument");
    BoxDev &bx = box->hb[b];
    const int n = bx.n_pairs * bx.n_bins;
    int nz = 0;
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(ep[i])) return set_error(EPSR_EINVAL, "empirical potential not finite");
        nz |= ep[i] != 0.f;
    }
    CK(cudaMemcpyAsync(box->ep + bx.ep_off, ep, n * sizeof(float), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    bx.has_ep = nz;
    set_near(bx);
    CK(cudaMemcpyAsync(box->boxes + b, &bx, sizeof(BoxDev), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return EPSR_OK;
}

extern "C" int epsr_box_get_ep(epsr_box *box, int32_t b, float *ep, epsr_stream_t stream)
{
    if (!box || !ep || b < 0 || b >= box->n_boxes) return set_error(EPSR_EINVAL, "bad argument");
    const BoxDev &bx = box->hb[b];
    CK(cudaMemcpyAsync(ep, box->ep + bx.ep_off, bx.n_pairs * bx.n_bins * sizeof(float), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return EPSR_OK;
}

extern "C" int epsr_box_total_energy(epsr_box *box, double *U_host, epsr_stream_t stream)
{
    if (!box || !U_host) return set_error(EPSR_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(box->U, 0, box->n_boxes * sizeof(double), s));
    int rc = launch_total_energy(box->boxes, box->coords, box->atom_mol, box->thresholds, box->ep,
                                 box->tiles, (long long)box->tiles_h.size(), box->U, box->sms * 2, s);
    if (rc) return rc;
    bool flexible = false;
    for (const auto &b : box->hb) flexible |= b.move_kind == EPSR_MOVE_FLEXIBLE_MOLECULE;
    if (flexible && (rc = launch_intra_energy(box->boxes, box->n_boxes, box->coords, box->mol_start, box->U, s)))
        return rc;
    CK(cudaMemcpyAsync(U_host, box->U, box->n_boxes * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return EPSR_OK;
}

// ---- Monte Carlo ------------------------------------------------------------------------------
extern "C" int epsr_mc_set_batch(epsr_box *box, int32_t batch_k)
{
    if (!box || batch_k < 0 || batch_k > mc_batch_max()) return set_error(EPSR_EINVAL, "batch_k out of range");
    box->mc_batch = batch_k;
    return EPSR_OK;
}

extern "C" int epsr_gr_set_ctas_per_sm(epsr_box *box, int32_t ctas_per_sm)
{
    if (!box || ctas_per_sm < 0 || ctas_per_sm > 4)
        return set_error(EPSR_EINVAL, "gr: CTAs per SM %d outside [0, 4]", ctas_per_sm);
    box->gr_ctas_per_sm = ctas_per_sm == 0 ? 4 : ctas_per_sm;
    return EPSR_OK;
}

extern "C" int epsr_box_get_launch(const epsr_box *box, int32_t *mc_batch, int32_t *mc_ctas,
                                   int32_t *gr_ctas_per_sm)
{
    if (!box) return set_error(EPSR_EINVAL, "NULL argument");
    if (mc_batch) *mc_batch = box->mc_batch;
    if (mc_ctas) *mc_ctas = box->mc_ctas;
    if (gr_ctas_per_sm) *gr_ctas_per_sm = box->gr_ctas_per_sm;
    return EPSR_OK;
}

namespace epsr {
// The shape a tuning applies to: every box's atoms, types, move kind and bins, and the SM count.
std::string box_shape_key(const epsr_box *box)
{
    std::string k = "box:" + std::to_string(box->sms);
    for (int b = 0; b < box->n_boxes; ++b) {
        const epsr_box_desc &d = box->desc[b];
        k += "|" + std::to_string(d.n_atoms) + "," + std::to_string(d.n_mol) + "," + std::to_string(d.n_types) +
             "," + std::to_string(d.move_kind) + "," + std::to_string(d.n_bins);
    }
    return k;
}

int box_sms(const epsr_box *box) { return box->sms; }

int box_summary(const epsr_box *box, int b, BoxSummary *out)
{
    if (!box || !out || b < 0 || b >= box->n_boxes) return set_error(EPSR_EINVAL, "bad box index");
    const BoxDev &bx = box->hb[b];
    out->n_boxes = box->n_boxes;
    out->n_pairs = bx.n_pairs;
    out->n_bins = bx.n_bins;
    out->kT = bx.kT;
    out->rho = (double)bx.n_atoms / bx.volume;
    out->dr = bx.dr_A;
    return EPSR_OK;
}

std::string sq_plan_key(const epsr_sq_plan *p, int n_cols, int cols_per_set, bool totals);
}  // namespace epsr

extern "C" int epsr_mc_set_cells(epsr_box *box, int32_t margin_fx, int32_t escapee_cap)
{
    if (!box) return set_error(EPSR_EINVAL, "NULL argument");
    if (margin_fx < 0 || escapee_cap < -1 || escapee_cap > mc_escapee_max())
        return set_error(EPSR_EINVAL, "mc cells: margin %d must be >= 0 and escapee_cap %d in [-1, %d]",
                         margin_fx, escapee_cap, mc_escapee_max());
    for (const auto &b : box->hb)
        if (margin_fx >= b.L / 4)
            return set_error(EPSR_EINVAL, "mc cells: margin %d not below a quarter of box side %d", margin_fx, b.L);
    box->cell_margin = margin_fx;
    box->esc_cap = escapee_cap;
    return EPSR_OK;
}

extern "C" int epsr_mc_set_ctas(epsr_box *box, int32_t ctas)
{
    if (!box || ctas < 0 || ctas > 65536) return set_error(EPSR_EINVAL, "ctas out of range");
    box->mc_ctas = ctas;
    plan_mc_groups(box);
    return upload_mc_groups(box);
}

extern "C" int epsr_debug_barrier_fault(epsr_box *box, int32_t cta, double timeout_ms)
{
    if (!box || !(timeout_ms > 0)) return set_error(EPSR_EINVAL, "bad argument");
    box->fault_cta = cta;
    box->timeout_ms = cta < 0 ? 2000.0 : timeout_ms;
    return EPSR_OK;
}

extern "C" int epsr_mc_stats_get(epsr_box *box, epsr_mc_stats *stats, epsr_stream_t stream)
{
    if (!box || !stats) return set_error(EPSR_EINVAL, "NULL argument");
    CK(cudaMemcpyAsync(stats, box->stats, box->n_boxes * sizeof(epsr_mc_stats), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return EPSR_OK;
}

// Enqueues a sweep without synchronising (graph-capturable: it allocates nothing; the global
// slices a layout needs are allocated with the layout, at creation or by epsr_mc_set_ctas).
static int mc_sweep_enqueue(epsr_box *box, int64_t n_moves, uint64_t seed, uint64_t move0,
                            epsr_move_log *log, cudaStream_t s)
{
    if (!box || n_moves < 0) return set_error(EPSR_EINVAL, "bad argument");
    CK(cudaMemsetAsync(box->status, 0, sizeof(int), s));
    if (n_moves == 0) return EPSR_OK;
    McLayout lay;
    int rcl = mc_layout(box, &lay);
    if (rcl) return rcl;
    const int slice_cap = lay.slice_cap, types_cap = lay.types_cap;
    const size_t smem = lay.smem;
    const bool gslice = lay.gslice;
    if (gslice && box->slice_g_cap < (size_t)box->cta_box_len * slice_cap)
        return set_error(EPSR_EINVAL, "mc sweep: global slices not allocated for this layout");
    // moves per launch: the table (allocated at creation) holds at most 2^22 moves over all boxes
    const long long chunk = std::min<long long>(n_moves, box->moves_cap / box->n_boxes);
    // type-major spatial partition of the partners for this sweep
    int rc0 = launch_scale_coords(box->boxes, box->atom_box, box->coords, box->scaled, box->n_atoms, s);
    if (!rc0)
        rc0 = launch_spatial_sort(box->boxes, box->atom_box, box->scaled, box->coords, box->n_atoms,
                                  box->total_mc_cells + 1, 1, box->mc_sort, nullptr, nullptr,
                                  box->pos_of, s);
    if (rc0) return rc0;
    McArgs a;
    memset(&a, 0, sizeof(a));
    a.sorted_index = box->mc_sort.index;
    a.pos_of = box->pos_of;
    a.mc_offset = box->mc_sort.offset;
    a.boxes = box->boxes;
    a.coords = box->coords;
    a.mol_start = box->mol_start;
    a.thresholds = box->thresholds;
    a.ep = box->ep;
    a.cta_box = box->cta_box;
    a.slots = box->slots;
    a.flags = box->flags;
    a.stats = box->stats;
    a.log = log;
    a.status = box->status;
    a.seed = seed;
    a.log_stride = n_moves;
    a.max_spin = 1LL << 40;
    a.timeout_ns = (unsigned long long)(box->timeout_ms * 1e6);
    a.grid = box->cta_box_len;
    a.lj_cut = 0;
    for (const auto &b : box->hb) a.lj_cut |= b.lj_cut;
    a.batch_k = box->mc_batch;
    a.slice_cap = slice_cap;
    a.tbl_cap = box->tbl_cap;
    a.ep_cap = box->ep_cap;
    a.types_cap = types_cap;
    a.slice_g = gslice ? box->slice_g : nullptr;
    a.home_g = gslice ? box->home_g : nullptr;
    a.cell_margin = box->cell_margin;
    a.esc_cap = box->esc_cap < 0 ? mc_escapee_max() : box->esc_cap;
    a.skip_arrival_cta = box->fault_cta;
    a.moves = box->moves;
    a.chunk = chunk;
    for (long long c0 = 0; c0 < n_moves; c0 += chunk) {
        const long long n = std::min(chunk, n_moves - c0);
        int rc = launch_mc_moves(box->boxes, box->mol_start, box->n_boxes, chunk, n, seed,
                                 move0 + (uint64_t)c0, box->moves, s);
        if (rc) return rc;
        a.n_moves = n;
        a.move0 = move0 + (uint64_t)c0;
        a.log_off = c0;
        CK(cudaMemsetAsync(box->flags, 0, box->cta_box_len * sizeof(unsigned), s));
        rc = launch_mc_sweep(a, box->cta_box_len, smem, s);
        if (rc) return rc;
    }
    return EPSR_OK;
}

extern "C" int epsr_mc_sweep(epsr_box *box, int64_t n_moves, uint64_t seed, uint64_t move0,
                             epsr_mc_stats *stats, epsr_move_log *log, epsr_stream_t stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    int rc = mc_sweep_enqueue(box, n_moves, seed, move0, log, s);
    if (rc) return rc;
    int st = 0;
    CK(cudaMemcpyAsync(&st, box->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (stats) CK(cudaMemcpyAsync(stats, box->stats, box->n_boxes * sizeof(epsr_mc_stats), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (st & kStatusTimeout) return set_error(EPSR_ETIMEOUT, "mc sweep: a grid barrier wait exceeded %.0f ms", box->timeout_ms);
    return EPSR_OK;
}

extern "C" int epsr_mc_sweep_async(epsr_box *box, int64_t n_moves, uint64_t seed, uint64_t move0,
                                   epsr_move_log *log, epsr_stream_t stream)
{
    return mc_sweep_enqueue(box, n_moves, seed, move0, log, (cudaStream_t)stream);
}

extern "C" int epsr_mc_status(epsr_box *box, int32_t *status, epsr_stream_t stream)
{
    if (!box || !status) return set_error(EPSR_EINVAL, "NULL argument");
    int st = 0;
    CK(cudaMemcpyAsync(&st, box->status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    *status = (st & kStatusTimeout) ? EPSR_ETIMEOUT : EPSR_OK;
    return EPSR_OK;
}

// ---- pair histograms --------------------------------------------------------------------------
extern "C" int epsr_partial_gr_tiles(const epsr_box *box, int64_t *n_tiles)
{
    if (!box || !n_tiles) return set_error(EPSR_EINVAL, "NULL argument");
    *n_tiles = (int64_t)box->tiles_h.size();
    return EPSR_OK;
}

static int gr_range(epsr_box *box, long long t0, long long t1, uint64_t *hist, cudaStream_t s)
{
    if (!box || !hist) return set_error(EPSR_EINVAL, "NULL argument");
    const long long nt = (long long)box->tiles_h.size();
    if (t0 < 0 || t1 > nt || t0 > t1) return set_error(EPSR_EINVAL, "tile range [%lld, %lld) outside [0, %lld)", t0, t1, nt);
    int rc = launch_scale_coords(box->boxes, box->atom_box, box->coords, box->scaled, box->n_atoms, s);
    if (rc) return rc;
    rc = launch_spatial_sort(box->boxes, box->atom_box, box->scaled, box->coords, box->n_atoms,
                             box->total_cells, 0, box->sort, box->sorted_scaled, box->sorted_coords,
                             nullptr, s);
    if (rc) return rc;
    GrArgs a;
    a.boxes = box->boxes;
    a.coords = box->sorted_coords;
    a.scaled = box->sorted_scaled;
    a.thresholds = box->thresholds;
    a.tiles = box->tiles;
    a.tile_begin = t0;
    a.tile_end = t1;
    a.hist = (unsigned long long *)hist;
    a.max_pairs_bins = box->ep_cap;
    a.max_bins1 = box->tbl_cap;
    const int grid = (int)std::min<long long>(t1 - t0, (long long)box->sms * box->gr_ctas_per_sm);
    return launch_partial_gr(a, std::max(grid, 1), s);
}

extern "C" int epsr_partial_gr_range(epsr_box *box, int64_t tile_begin, int64_t tile_end,
                                     uint64_t *hist, epsr_stream_t stream)
{
    return gr_range(box, tile_begin, tile_end, hist, (cudaStream_t)stream);
}

extern "C" int epsr_partial_gr_cells(epsr_box *box, uint64_t *hist, float *g, int64_t n_configs,
                                     epsr_stream_t stream)
{
    if (!box || !hist) return set_error(EPSR_EINVAL, "NULL argument");
    if (g && n_configs < 1) return set_error(EPSR_EINVAL, "n_configs must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = EPSR_OK;
    if (!box->gc_items_h.empty()) {
        rc = launch_scale_coords(box->boxes, box->atom_box, box->coords, box->scaled, box->n_atoms, s);
        if (rc) return rc;
        SortScratch sc = box->sort;          // per-atom scratch shared with the all-pairs order
        sc.count = box->gc_count;
        sc.offset = box->gc_offset;
        sc.block = box->gc_block;
        rc = launch_spatial_sort(box->boxes, box->atom_box, box->scaled, box->coords, box->n_atoms,
                                 box->total_gcells + 1, 2, sc, box->gc_scaled, box->gc_coords, nullptr, s);
        if (rc) return rc;
        GcArgs a;
        a.boxes = box->boxes;
        a.coords = box->gc_coords;
        a.scaled = box->gc_scaled;
        a.cell_start = box->gc_offset;
        a.cell_count = box->gc_count;
        a.thresholds = box->thresholds;
        a.items = box->gc_items;
        a.n_items = (long long)box->gc_items_h.size();
        a.hist = (unsigned long long *)hist;
        a.max_pairs_bins = box->ep_cap;
        a.max_bins1 = box->tbl_cap;
        const int grid = (int)std::min<long long>(a.n_items, (long long)box->sms * 8);
        rc = launch_partial_gr_cells(a, std::max(grid, 1), s);
        if (rc) return rc;
    }
    // boxes too small for three cells per side: the all-pairs tiles of those boxes
    for (int b = 0; b < box->n_boxes; ++b)
        if (box->hb[b].gc_n == 0 && (rc = gr_range(box, box->tile_lo[b], box->tile_hi[b], hist, s)))
            return rc;
    if (g) return epsr_normalize_g(box, hist, g, n_configs, stream);
    return EPSR_OK;
}

extern "C" int epsr_normalize_g(epsr_box *box, const uint64_t *hist, float *g, int64_t n_configs,
                                epsr_stream_t stream)
{
    if (!box || !hist || !g || n_configs < 1) return set_error(EPSR_EINVAL, "bad argument");
    return launch_normalize_g(box->boxes, box->n_boxes, (const unsigned long long *)hist, g, n_configs,
                              box->hist_len, box->hist_box, (cudaStream_t)stream);
}

extern "C" int epsr_partial_gr(epsr_box *box, uint64_t *hist, float *g, int64_t n_configs,
                               epsr_stream_t stream)
{
    if (!box || !hist) return set_error(EPSR_EINVAL, "NULL argument");
    if (g && n_configs < 1) return set_error(EPSR_EINVAL, "n_configs must be >= 1");
    int rc = gr_range(box, 0, (long long)box->tiles_h.size(), hist, (cudaStream_t)stream);
    if (rc) return rc;
    if (g) return epsr_normalize_g(box, hist, g, n_configs, stream);
    return EPSR_OK;
}

extern "C" int epsr_sq_weights(const epsr_box *box, int32_t b, double *w, double *flat)
{
    if (!box || b < 0 || b >= box->n_boxes || !w || !flat) return set_error(EPSR_EINVAL, "bad argument");
    const epsr_box_desc &d = box->desc[b];
    const BoxDev &bx = box->hb[b];
    const double N = (double)d.n_atoms;
    const double rho = N / bx.volume;
    const double pi = 3.14159265358979323846;
    double fl = 0.0;
    for (int a = 0; a < d.n_types; ++a) {
        const double ca = (double)bx.count[a] / N, ba = d.b[a] * 0.1;
        fl += ca * ba * ba;
        for (int c = a; c < d.n_types; ++c) {
            const double cc = (double)bx.count[c] / N, bc = d.b[c] * 0.1;
            w[pair_index(a, c, d.n_types)] = 4.0 * pi * rho * (a == c ? 1.0 : 2.0) * ca * cc * ba * bc;
        }
    }
    *flat = fl;
    return EPSR_OK;
}

// ---- S(Q) -----------------------------------------------------------------------------------
struct epsr_sq_plan {
    int nQ = 0, n_bins = 0, mode = 0, max_cols = 0;
    double dr = 0;
    float *Q = nullptr;
    float *Kt = nullptr;
    float *Sp_scratch = nullptr;
    double *res = nullptr;      // chi^2 residuals [nQ]
    double *chiF = nullptr;     // chi^2 basis values [max basis][nQ] (allocated on first use)
    // tensor-core modes
    unsigned char *a_packed = nullptr;
    int *tc_status = nullptr;
    int fmt_bf16 = 1, np = 2, kt = 64, stages = 0, m_tiles = 0, n_products = 0;
    int tc_n_chunk = 0, tc_k_split = 0;   // tensor-core tiling set by epsr_sq_plan_set_tiles (0 = rule)
    int sms = 0;
    ~epsr_sq_plan()
    {
        void *ptrs[] = {Q, Kt, Sp_scratch, res, chiF, a_packed, tc_status};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
};

static int gcd_i(int a, int b) { return b ? gcd_i(b, a % b) : a; }

// Tiling of the tensor-core contraction: columns per CTA (a multiple of 16, and of the set size
// when the set totals are fused into the epilogue) and the number of CTAs sharing one output
// tile along K (one cluster). The rule aims at about two CTAs per SM with power-of-two clusters;
// a tiling set on the plan (epsr_sq_plan_set_tiles, e.g. by the autotuner) takes precedence.
static int tc_choose_tiles(const epsr_sq_plan *p, int n_cols, int cps, bool want_sets, int *n_chunk,
                           int *k_split, bool *fused)
{
    const int L = 16 / gcd_i(16, cps) * cps;          // lcm(16, cols_per_set)
    const bool user = p->tc_n_chunk > 0 || p->tc_k_split > 0;
    int nc, unit;
    if (p->tc_n_chunk > 0) {
        nc = std::min(p->tc_n_chunk, std::max(16, (n_cols + 15) / 16 * 16));
        *fused = want_sets && nc % cps == 0;
        unit = 16;
    } else {
        *fused = want_sets && L <= 256;
        unit = *fused ? L : 16;
        nc = unit * std::max(1, 64 / unit);
        nc = std::min(nc, (n_cols + unit - 1) / unit * unit);
    }
    const int tiles = p->m_tiles * ((n_cols + nc - 1) / nc);
    int ks = p->tc_k_split;
    if (ks <= 0) {
        // about two CTAs per SM, in clusters of a power of two (they pack onto the GPCs better)
        const int want = std::min((2 * std::max(1, p->sms) + tiles - 1) / tiles, std::min(kTcMaxKSplit, p->stages));
        ks = 1;
        while (ks * 2 <= want) ks *= 2;
    }
    ks = std::max(1, std::min(ks, std::min(kTcMaxKSplit, p->stages)));
    const int grp = *fused ? cps : 1;
    while (tc_smem_bytes(nc, p->np, ks, grp) == 0) {
        if (user) return set_error(EPSR_EINVAL, "sq exec: tiling (%d, %d) does not fit in shared memory", nc, ks);
        if (nc > unit) nc -= unit;
        else if (ks > 1) --ks;
        else return set_error(EPSR_EINVAL, "sq exec: no tiling fits in shared memory");
    }
    *n_chunk = nc;
    *k_split = ks;
    return EPSR_OK;
}

namespace epsr {
std::string sq_plan_key(const epsr_sq_plan *p, int n_cols, int cols_per_set, bool totals)
{
    return "sq:" + std::to_string(p->sms) + "|" + std::to_string(p->nQ) + "," + std::to_string(p->n_bins) + "," +
           std::to_string(p->mode) + "," + std::to_string(n_cols) + "," + std::to_string(cols_per_set) + "," +
           std::to_string((int)totals);
}
int sq_plan_mode(const epsr_sq_plan *p) { return p->mode; }
void sq_plan_dims(const epsr_sq_plan *p, int *nQ, int *n_bins, int *max_cols)
{
    *nQ = p->nQ;
    *n_bins = p->n_bins;
    *max_cols = p->max_cols;
}
int sq_plan_stages(const epsr_sq_plan *p) { return p->stages; }
}  // namespace epsr

extern "C" int epsr_sq_plan_set_tiles(epsr_sq_plan *plan, int32_t n_chunk, int32_t k_split)
{
    if (!plan) return set_error(EPSR_EINVAL, "plan is NULL");
    if (plan->mode == EPSR_SQ_FP32) return n_chunk == 0 && k_split == 0 ? EPSR_OK
        : set_error(EPSR_EINVAL, "sq plan: the FP32 mode has no tensor-core tiling");
    if (n_chunk < 0 || n_chunk > 256 || n_chunk % 16 || k_split < 0 || k_split > kTcMaxKSplit ||
        k_split > plan->stages)
        return set_error(EPSR_EINVAL, "sq plan: tiling (%d, %d) out of range", n_chunk, k_split);
    if (n_chunk > 0 && tc_smem_bytes(n_chunk, plan->np, std::max(1, k_split), 1) == 0)
        return set_error(EPSR_EINVAL, "sq plan: %d columns per CTA do not fit in shared memory", n_chunk);
    plan->tc_n_chunk = n_chunk;
    plan->tc_k_split = k_split;
    return EPSR_OK;
}

extern "C" int epsr_sq_plan_get_tiles(const epsr_sq_plan *plan, int32_t n_cols, int32_t cols_per_set,
                                      int32_t with_totals, int32_t *n_chunk, int32_t *k_split)
{
    if (!plan || !n_chunk || !k_split || n_cols < 1 || n_cols > plan->max_cols || cols_per_set < 1)
        return set_error(EPSR_EINVAL, "sq plan: bad argument");
    *n_chunk = *k_split = 0;
    if (plan->mode == EPSR_SQ_FP32) return EPSR_OK;
    int nc = 0, ks = 0;
    bool fused = false;
    int rc = tc_choose_tiles(plan, n_cols, cols_per_set, with_totals != 0, &nc, &ks, &fused);
    if (rc) return rc;
    *n_chunk = nc;
    *k_split = ks;
    return EPSR_OK;
}

extern "C" int epsr_sq_plan_create(const float *Q, int32_t nQ, int32_t n_bins, double dr, int32_t mode,
                                   int32_t max_cols, epsr_stream_t stream, epsr_sq_plan **out)
{
    if (!out) return set_error(EPSR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!Q || nQ < 1 || nQ > (1 << 20) || n_bins < 1 || n_bins > EPSR_MAX_BINS || !(dr > 0) ||
        max_cols < 1 || max_cols > EPSR_SQ_MAX_COLS)
        return set_error(EPSR_EINVAL, "sq plan: argument out of range");
    if (mode < EPSR_SQ_FP32 || mode > EPSR_SQ_BF16X6) return set_error(EPSR_EINVAL, "sq plan: mode %d unknown", mode);
    for (int i = 0; i < nQ; ++i)
        if (!(Q[i] > 0) || !std::isfinite(Q[i])) return set_error(EPSR_EINVAL, "sq plan: Q[%d] must be > 0", i);
    epsr_sq_plan *p = new (std::nothrow) epsr_sq_plan();
    if (!p) return set_error(EPSR_ENOMEM, "host allocation failed");
    p->nQ = nQ; p->n_bins = n_bins; p->mode = mode; p->max_cols = max_cols; p->dr = dr;
    int rc;
    if ((rc = dalloc(&p->Q, nQ)) || (rc = dalloc(&p->Kt, (size_t)nQ * n_bins)) ||
        (rc = dalloc(&p->Sp_scratch, (size_t)max_cols * nQ)) || (rc = dalloc(&p->res, (size_t)nQ))) {
        delete p;
        return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(p->Q, Q, nQ * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) { delete p; return set_cuda_error(e, "sq plan upload"); }
    if ((rc = sq_build_kt(p->Q, nQ, n_bins, dr, p->Kt, s))) { delete p; return rc; }
    if (mode != EPSR_SQ_FP32) {
        p->fmt_bf16 = mode == EPSR_SQ_TF32X3 ? 0 : 1;
        p->np = mode == EPSR_SQ_BF16X6 ? 3 : 2;
        const int esize = p->fmt_bf16 ? 2 : 4;
        p->kt = 128 / esize;                       // 128-byte rows per stage
        p->stages = (n_bins + p->kt - 1) / p->kt;
        p->m_tiles = (nQ + 127) / 128;
        p->n_products = p->np * (p->np + 1) / 2;      // split products with i + j < np
        const size_t a_bytes = (size_t)p->m_tiles * p->stages * p->np * 128 * p->kt * esize;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev);
        if ((rc = dalloc(&p->a_packed, a_bytes)) || (rc = dalloc(&p->tc_status, 1))) {
            delete p;
            return rc;
        }
        cudaMemsetAsync(p->tc_status, 0, sizeof(int), s);
        if ((rc = tc_pack_a(p->Kt, nQ, n_bins, p->m_tiles, p->stages, p->kt, p->np, p->fmt_bf16,
                            p->a_packed, s))) {
            delete p;
            return rc;
        }
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { delete p; return set_cuda_error(e, "sq plan sync"); }
    *out = p;
    return EPSR_OK;
}

extern "C" int epsr_sq_plan_destroy(epsr_sq_plan *plan)
{
    if (!plan) return EPSR_OK;
    cudaDeviceSynchronize();
    delete plan;
    return EPSR_OK;
}

extern "C" int epsr_sq_exec(epsr_sq_plan *plan, const float *g, int32_t n_cols, const double *w,
                            int32_t cols_per_set, const double *flat, float *S_partial, float *S_total,
                            epsr_stream_t stream)
{
    if (!plan || !g || !w || n_cols < 1 || n_cols > plan->max_cols || cols_per_set < 1 ||
        n_cols % cols_per_set != 0)
        return set_error(EPSR_EINVAL, "sq exec: bad argument");
    if (S_total && !flat) return set_error(EPSR_EINVAL, "sq exec: flat is NULL");
    if (!S_partial && !S_total) return EPSR_OK;
    SqArgs *a = new (std::nothrow) SqArgs();
    if (!a) return set_error(EPSR_ENOMEM, "host allocation failed");
    a->g = g;
    a->Kt = plan->Kt;
    a->S_partial = S_partial ? S_partial : plan->Sp_scratch;
    a->nQ = plan->nQ;
    a->n_bins = plan->n_bins;
    a->n_cols = n_cols;
    for (int c = 0; c < n_cols; ++c) a->w[c] = w[c];
    int rc = EPSR_OK;
    bool totals_done = false;
    if (plan->mode == EPSR_SQ_FP32) {
        rc = sq_exec_fp32(*a, (cudaStream_t)stream);
    } else {
        // tensor cores: one clustered launch over (M tiles, column chunks, K split)
        TcArgs *t = new (std::nothrow) TcArgs();
        if (!t) { delete a; return set_error(EPSR_ENOMEM, "host allocation failed"); }
        int n_chunk = 0, k_split = 0;
        bool fused = false;
        rc = tc_choose_tiles(plan, n_cols, cols_per_set, S_total != nullptr, &n_chunk, &k_split, &fused);
        if (!rc) {
            t->a_packed = plan->a_packed;
            t->g = g;
            t->S_partial = (S_partial || !fused) ? a->S_partial : nullptr;
            t->S_total = fused ? S_total : nullptr;
            t->status = plan->tc_status;
            t->nQ = plan->nQ;
            t->n_bins = plan->n_bins;
            t->n_cols = n_cols;
            t->m_tiles = plan->m_tiles;
            t->units = plan->stages;
            t->ku = plan->kt;
            t->np_a = t->np_b = plan->np;
            t->fmt_bf16 = plan->fmt_bf16;
            t->n_products = plan->n_products;
            t->n_chunk = n_chunk;
            t->k_split = k_split;
            int tc = 32;
            while (tc < n_chunk) tc <<= 1;
            t->tmem_cols = tc;
            t->cols_per_set = cols_per_set;
            const int grp = fused ? cols_per_set : 1;
            const long long ctas = (long long)plan->m_tiles * ((n_cols + n_chunk - 1) / n_chunk) * k_split;
            t->slots = tc_slots_for(n_chunk, plan->np, (plan->stages + k_split - 1) / k_split, k_split, grp,
                                    ctas <= plan->sms);
            t->recv_cols = tc_recv_cols(n_chunk, grp, k_split);
            for (int c = 0; c < n_cols; ++c) t->w[c] = (float)w[c];
            if (fused)
                for (int s_ = 0; s_ < n_cols / cols_per_set; ++s_) t->flat[s_] = (float)flat[s_];
            rc = tc_exec(*t, (cudaStream_t)stream);
            totals_done = fused;
        }
        delete t;
    }
    if (!rc && S_total && !totals_done) {
        SqWeights *W = new (std::nothrow) SqWeights();
        if (!W) { delete a; return set_error(EPSR_ENOMEM, "host allocation failed"); }
        for (int s = 0; s < n_cols / cols_per_set; ++s) W->flat[s] = flat[s];
        rc = sq_totals(a->S_partial, n_cols / cols_per_set, cols_per_set, plan->nQ, *W, S_total,
                       (cudaStream_t)stream);
        delete W;
    }
    delete a;
    return rc;
}

extern "C" int epsr_sq(const float *g, int32_t n_cols, int32_t n_bins, double dr, const float *Q,
                       int32_t nQ, const double *w, int32_t cols_per_set, const double *flat,
                       float *S_partial, float *S_total, int32_t mode, epsr_stream_t stream)
{
    epsr_sq_plan *p = nullptr;
    int rc = epsr_sq_plan_create(Q, nQ, n_bins, dr, mode, n_cols, stream, &p);
    if (rc) return rc;
    rc = epsr_sq_exec(p, g, n_cols, w, cols_per_set, flat, S_partial, S_total, stream);
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) rc = set_cuda_error(e, "sq sync");
    }
    if (!rc && p->tc_status) {
        int st = 0;
        cudaMemcpy(&st, p->tc_status, sizeof(int), cudaMemcpyDeviceToHost);
        if (st) rc = set_error(EPSR_ETIMEOUT, "sq: a tensor-core completion wait gave up");
    }
    epsr_sq_plan_destroy(p);
    return rc;
}

extern "C" int epsr_sq_plan_status(epsr_sq_plan *p, int32_t *status, epsr_stream_t stream)
{
    if (!p || !status) return set_error(EPSR_EINVAL, "NULL argument");
    *status = EPSR_OK;
    if (!p->tc_status) return EPSR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    CK(cudaMemcpyAsync(&st, p->tc_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(p->tc_status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    *status = st ? EPSR_ETIMEOUT : EPSR_OK;
    return EPSR_OK;
}

// ---- empirical-potential update -------------------------------------------------------------
extern "C" int epsr_ep_update(epsr_box *box, int32_t b, const float *dS, int32_t n_data,
                              const double *w, const float *Q, int32_t nQ, int32_t n_basis,
                              double s_basis, double gamma, double alpha, double *C_out,
                              epsr_stream_t stream)
{
    if (!box || b < 0 || b >= box->n_boxes || !dS || !w || !Q)
        return set_error(EPSR_EINVAL, "ep update: bad argument");
    BoxDev &bx = box->hb[b];
    const int P = bx.n_pairs;
    if (n_data < 1 || n_data > kEpMaxData || n_basis < 1 || n_basis > kEpMaxBasis || nQ < n_basis ||
        nQ > (1 << 20) || !(s_basis > 0) || !(gamma >= 0) || !std::isfinite(alpha))
        return set_error(EPSR_EINVAL, "ep update: sizes or parameters out of range");
    if (n_data < P && !(gamma > 0))
        return set_error(EPSR_EINVAL, "ep update: %d datasets for %d pairs need gamma > 0", n_data, P);
    for (int i = 0; i < nQ; ++i)
        if (!(Q[i] > 0) || !std::isfinite(Q[i])) return set_error(EPSR_EINVAL, "ep update: Q[%d] must be > 0", i);
    cudaStream_t s = (cudaStream_t)stream;
    if (box->ep_cap_Q < nQ) {
        void *ptrs[] = {box->ep_F, box->ep_Y, box->ep_C, box->ep_Q};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        box->ep_F = box->ep_Y = box->ep_C = nullptr;
        box->ep_Q = nullptr;
        box->ep_cap_Q = 0;
        int rc;
        if ((rc = dalloc(&box->ep_F, (size_t)kEpMaxBasis * nQ)) || (rc = dalloc(&box->ep_Y, (size_t)kEpMaxPairs * nQ)) ||
            (rc = dalloc(&box->ep_C, (size_t)kEpMaxPairs * kEpMaxBasis)) || (rc = dalloc(&box->ep_Q, (size_t)nQ)))
            return rc;
        box->ep_cap_Q = nQ;
    }
    EpArgs *a = new (std::nothrow) EpArgs();
    if (!a) return set_error(EPSR_ENOMEM, "host allocation failed");
    a->dS = dS;
    a->Q = box->ep_Q;
    a->nQ = nQ;
    a->n_data = n_data;
    a->n_pairs = P;
    a->n_basis = n_basis;
    a->n_bins = bx.n_bins;
    for (int i = 0; i < n_data * P; ++i) a->w[i] = w[i];
    a->s = s_basis;
    a->gamma = gamma;
    a->alpha = alpha;
    a->kT = bx.kT;
    a->rho = (double)bx.n_atoms / bx.volume;
    a->dr = bx.dr_A;
    a->F = box->ep_F;
    a->Y = box->ep_Y;
    a->C_out = box->ep_C;
    a->ep = box->ep + bx.ep_off;
    cudaError_t e = cudaMemcpyAsync(box->ep_Q, Q, nQ * sizeof(float), cudaMemcpyHostToDevice, s);
    int rc = e == cudaSuccess ? launch_ep_update(*a, s) : set_cuda_error(e, "ep update: Q upload");
    delete a;
    if (rc) return rc;
    bx.has_ep = 1;
    set_near(bx);
    CK(cudaMemcpyAsync(box->boxes + b, &bx, sizeof(BoxDev), cudaMemcpyHostToDevice, s));
    if (C_out) CK(cudaMemcpyAsync(C_out, box->ep_C, (size_t)P * n_basis * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return EPSR_OK;
}

// ---- differentiable form: smeared histogram, adjoints, chi^2 ----------------------------------
// The cell-list form serves when every box has a cell list and 5 sigma fits in the cells'
// margin; otherwise the all-pairs tiles (any sigma, any box).
static bool smear_uses_cells(const epsr_box *box, double sigma)
{
    if (box->gc_items_h.empty() || 5.0 * sigma > kCellSmearMarginA) return false;
    for (const auto &b : box->hb)
        if (b.gc_n == 0) return false;
    return true;
}

static int smear_common(epsr_box *box, double sigma, cudaStream_t s)
{
    if (!(sigma > 0) || sigma > 2.0) return set_error(EPSR_EINVAL, "smeared g: sigma must be in (0, 2] A");
    int rc = launch_scale_coords(box->boxes, box->atom_box, box->coords, box->scaled, box->n_atoms, s);
    if (rc) return rc;
    if (smear_uses_cells(box, sigma)) {
        SortScratch sc = box->sort;
        sc.count = box->gc_count;
        sc.offset = box->gc_offset;
        sc.block = box->gc_block;
        return launch_spatial_sort(box->boxes, box->atom_box, box->scaled, box->coords, box->n_atoms,
                                   box->total_gcells + 1, 2, sc, box->gc_scaled, box->gc_coords, nullptr, s);
    }
    return launch_spatial_sort(box->boxes, box->atom_box, box->scaled, box->coords, box->n_atoms,
                               box->total_cells, 0, box->sort, box->sorted_scaled, box->sorted_coords,
                               nullptr, s);
}

static SmearArgs smear_args(epsr_box *box, double sigma)
{
    SmearArgs a;
    memset(&a, 0, sizeof(a));
    a.boxes = box->boxes;
    a.index = box->sort.index;
    a.sigma = sigma;
    a.max_pairs_bins = box->ep_cap;
    if (smear_uses_cells(box, sigma)) {
        a.coords = box->gc_coords;
        a.scaled = box->gc_scaled;
        a.items = box->gc_items;
        a.n_items = (long long)box->gc_items_h.size();
        a.cell_start = box->gc_offset;
        a.cell_count = box->gc_count;
    } else {
        a.coords = box->sorted_coords;
        a.scaled = box->sorted_scaled;
        a.tiles = box->tiles;
        a.n_tiles = (long long)box->tiles_h.size();
    }
    return a;
}

static int smear_launch(epsr_box *box, const SmearArgs &a, bool backward, cudaStream_t s)
{
    if (a.items) return launch_smear_cells(a, backward, (int)std::min<long long>(a.n_items, (long long)box->sms * 8), s);
    return launch_smear(a, backward, box->sms * 2, s);
}

extern "C" int epsr_gr_smeared_fwd(epsr_box *box, double sigma, double *Ht, float *gt, epsr_stream_t stream)
{
    if (!box || !Ht) return set_error(EPSR_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = smear_common(box, sigma, s);
    if (rc) return rc;
    CK(cudaMemsetAsync(box->smear_acc, 0, (size_t)box->hist_len * sizeof(unsigned long long), s));
    SmearArgs a = smear_args(box, sigma);
    a.acc = box->smear_acc;
    rc = smear_launch(box, a, false, s);
    if (rc) return rc;
    return launch_smear_norm(box->boxes, box->n_boxes, box->smear_acc, Ht, gt, box->hist_len,
                             box->hist_box, s);
}

extern "C" int epsr_gr_smeared_bwd(epsr_box *box, double sigma, const float *dgt, float *grad,
                                   epsr_stream_t stream)
{
    if (!box || !dgt || !grad) return set_error(EPSR_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = smear_common(box, sigma, s);
    if (rc) return rc;
    rc = launch_smear_lambda(box->boxes, box->n_boxes, dgt, box->lambda, box->hist_len, box->hist_box, s);
    if (rc) return rc;
    CK(cudaMemsetAsync(grad, 0, (size_t)box->n_atoms * 3 * sizeof(float), s));
    SmearArgs a = smear_args(box, sigma);
    a.lambda = box->lambda;
    a.grad = grad;
    return smear_launch(box, a, true, s);
}

extern "C" int epsr_sq_exec_adjoint(epsr_sq_plan *plan, const float *dS_total, int32_t n_cols,
                                    const double *w, int32_t cols_per_set, float *dg, epsr_stream_t stream)
{
    if (!plan || !dS_total || !w || !dg || n_cols < 1 || n_cols > plan->max_cols || cols_per_set < 1 ||
        n_cols % cols_per_set != 0)
        return set_error(EPSR_EINVAL, "sq adjoint: bad argument");
    SqArgs *a = new (std::nothrow) SqArgs();
    if (!a) return set_error(EPSR_ENOMEM, "host allocation failed");
    a->Kt = plan->Kt;
    a->nQ = plan->nQ;
    a->n_bins = plan->n_bins;
    a->n_cols = n_cols;
    for (int c = 0; c < n_cols; ++c) a->w[c] = w[c];
    int rc = sq_exec_adjoint(*a, dS_total, cols_per_set, dg, (cudaStream_t)stream);
    delete a;
    return rc;
}

extern "C" int epsr_chi2(epsr_sq_plan *plan, const float *S, const float *target, const double *W,
                         int32_t P, const double *C, int32_t n_basis, double s_basis, double rho,
                         double *chi2, float *dS, double *dC, epsr_stream_t stream)
{
    if (!plan || !S || !target || !W || !chi2 || !dS || P < 1 || P > kEpMaxPairs ||
        (C && (n_basis < 1 || n_basis > kEpMaxBasis || !(s_basis > 0) || !(rho > 0))))
        return set_error(EPSR_EINVAL, "chi2: bad argument");
    ChiParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.P = P;
    prm.n_basis = C ? n_basis : 0;
    prm.s = s_basis;
    prm.rho = rho;
    for (int p = 0; p < P; ++p) prm.W[p] = W[p];
    prm.res_scratch = plan->res;
    if (C && !plan->chiF) {
        if (cudaMalloc(&plan->chiF, (size_t)kEpMaxBasis * plan->nQ * sizeof(double)) != cudaSuccess) {
            plan->chiF = nullptr;
            return set_error(EPSR_ENOMEM, "chi2: basis scratch");
        }
    }
    prm.F_scratch = plan->chiF;
    return launch_chi2(S, target, plan->Q, plan->nQ, prm, C, chi2, dS, C ? dC : nullptr,
                       (cudaStream_t)stream);
}

// ---- checkpoint / resume ------------------------------------------------------------------------
// Layout: magic, version, n_boxes, n_atoms, ep_len; then int32 [n_atoms][3] coordinates,
// float [ep_len] empirical-potential tables, epsr_mc_stats [n_boxes], int32 [n_boxes] has_ep.
struct CkptHeader {
    uint64_t magic;
    uint32_t version, n_boxes;
    int64_t n_atoms, ep_len;
};
static const uint64_t kCkptMagic = 0x5450434b52535045ull;   // "EPSRCKPT"

static size_t ckpt_bytes(const epsr_box *box, long long ep_len)
{
    return sizeof(CkptHeader) + (size_t)box->n_atoms * 3 * sizeof(int32_t) + (size_t)ep_len * sizeof(float) +
           (size_t)box->n_boxes * (sizeof(epsr_mc_stats) + sizeof(int32_t));
}

static long long ep_total(const epsr_box *box)
{
    long long n = 0;
    for (const auto &b : box->hb) n += (long long)b.n_pairs * b.n_bins;
    return n;
}

extern "C" int epsr_checkpoint_size(const epsr_box *box, size_t *bytes)
{
    if (!box || !bytes) return set_error(EPSR_EINVAL, "NULL argument");
    *bytes = ckpt_bytes(box, ep_total(box));
    return EPSR_OK;
}

extern "C" int epsr_checkpoint_save(epsr_box *box, void *buf, size_t len, epsr_stream_t stream)
{
    if (!box || !buf) return set_error(EPSR_EINVAL, "NULL argument");
    const long long ep_len = ep_total(box);
    if (len < ckpt_bytes(box, ep_len)) return set_error(EPSR_EINVAL, "checkpoint buffer too small");
    unsigned char *p = static_cast<unsigned char *>(buf);
    CkptHeader h{kCkptMagic, 1u, (uint32_t)box->n_boxes, box->n_atoms, ep_len};
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    int rc = epsr_box_get_coords(box, reinterpret_cast<int32_t *>(p), stream);
    if (rc) return rc;
    p += (size_t)box->n_atoms * 3 * sizeof(int32_t);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(p, box->ep, (size_t)ep_len * sizeof(float), cudaMemcpyDeviceToHost, s));
    p += (size_t)ep_len * sizeof(float);
    CK(cudaMemcpyAsync(p, box->stats, box->n_boxes * sizeof(epsr_mc_stats), cudaMemcpyDeviceToHost, s));
    p += box->n_boxes * sizeof(epsr_mc_stats);
    for (int b = 0; b < box->n_boxes; ++b) reinterpret_cast<int32_t *>(p)[b] = box->hb[b].has_ep;
    CK(cudaStreamSynchronize(s));
    return EPSR_OK;
}

extern "C" int epsr_checkpoint_load(epsr_box *box, const void *buf, size_t len, epsr_stream_t stream)
{
    if (!box || !buf) return set_error(EPSR_EINVAL, "NULL argument");
    const long long ep_len = ep_total(box);
    if (len < sizeof(CkptHeader)) return set_error(EPSR_EINVAL, "checkpoint too short");
    CkptHeader h;
    memcpy(&h, buf, sizeof(h));
    if (h.magic != kCkptMagic || h.version != 1u || h.n_boxes != (uint32_t)box->n_boxes ||
        h.n_atoms != box->n_atoms || h.ep_len != ep_len || len < ckpt_bytes(box, ep_len))
        return set_error(EPSR_EINVAL, "checkpoint does not match this handle");
    const unsigned char *p = static_cast<const unsigned char *>(buf) + sizeof(h);
    int rc = epsr_box_set_coords(box, reinterpret_cast<const int32_t *>(p), stream);
    if (rc) return rc;
    p += (size_t)box->n_atoms * 3 * sizeof(int32_t);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(box->ep, p, (size_t)ep_len * sizeof(float), cudaMemcpyHostToDevice, s));
    p += (size_t)ep_len * sizeof(float);
    CK(cudaMemcpyAsync(box->stats, p, box->n_boxes * sizeof(epsr_mc_stats), cudaMemcpyHostToDevice, s));
    p += box->n_boxes * sizeof(epsr_mc_stats);
    for (int b = 0; b < box->n_boxes; ++b) {
        box->hb[b].has_ep = reinterpret_cast<const int32_t *>(p)[b];
        set_near(box->hb[b]);
    }
    CK(cudaMemcpyAsync(box->boxes, box->hb.data(), box->hb.size() * sizeof(BoxDev), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return EPSR_OK;
}
