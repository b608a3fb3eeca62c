// epsr_tune.cu -- the autotuner of the launch shapes.
//
// The throughput of the hot path depends on launch parameters that do not change its
// results: the moves the Monte Carlo sweep takes per grid barrier and the CTAs it runs on,
// the persistent CTAs per SM of the all-pair histogram, and the tiling of the tensor-core
// S(Q) contraction. Fixed rules pick them by default; the tuner times a small set of
// candidates on the caller's own handle (its atom counts, types, bins and the SM count of
// the device), keeps the fastest, and caches it per shape for the rest of the process, so a
// second handle of the same shape is configured without timing.
//
// The Monte Carlo candidates run real sweeps, so the tuner saves the handle's state
// (coordinates, empirical potentials, running statistics) in a host checkpoint first and
// restores it afterwards: a tuned handle continues from exactly the state it had. Every
// candidate computes the same sequential Metropolis chain (the batch size changes only the
// FP32 summation order of dU) and the same integer histograms.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "epsr.h"
#include "epsr_internal.h"

using namespace epsr;

namespace {

// Keeps the GPU busy for `ns` nanoseconds (a bounded wait on the global timer), so that the
// launches timed after it are enqueued before the GPU reaches them and the events bracket
// device time only.
__global__ void tune_delay_kernel(unsigned long long ns)
{
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    } while (t - t0 < ns);
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~EventPair() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
};

struct BoxTuning {
    int mc_batch = 0, mc_ctas = 0, gr_ctas_per_sm = 4;
    double mc_us_per_move = 0, gr_ms = 0;
};

struct SqTuning {
    int n_chunk = 0, k_split = 0;
    double us = 0;
};

std::mutex g_tune_mu;
std::map<std::string, BoxTuning> g_box_cache;
std::map<std::string, SqTuning> g_sq_cache;

// Device time of `enqueue` (run `reps` times back to back), in milliseconds per run.
template <class F>
int time_ms(cudaStream_t s, int reps, F enqueue, double *ms)
{
    EventPair ev;
    if (!ev.a || !ev.b) return set_error(EPSR_ECUDA, "tune: cudaEventCreate failed");
    tune_delay_kernel<<<1, 1, 0, s>>>(100000ull);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e, "tune: delay kernel");
    if ((e = cudaEventRecord(ev.a, s)) != cudaSuccess) return set_cuda_error(e, "tune: event");
    for (int r = 0; r < reps; ++r) {
        int rc = enqueue();
        if (rc) return rc;
    }
    if ((e = cudaEventRecord(ev.b, s)) != cudaSuccess) return set_cuda_error(e, "tune: event");
    if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) return set_cuda_error(e, "tune: event sync");
    float f = 0.f;
    if ((e = cudaEventElapsedTime(&f, ev.a, ev.b)) != cudaSuccess) return set_cuda_error(e, "tune: elapsed");
    *ms = (double)f / reps;
    return EPSR_OK;
}

int apply_box(epsr_box *box, const BoxTuning &t)
{
    int rc = epsr_mc_set_ctas(box, t.mc_ctas);
    if (!rc) rc = epsr_mc_set_batch(box, t.mc_batch);
    if (!rc) rc = epsr_gr_set_ctas_per_sm(box, t.gr_ctas_per_sm);
    return rc;
}

void fill(epsr_tuning *out, const BoxTuning &t, int from_cache)
{
    if (!out) return;
    out->mc_batch = t.mc_batch;
    out->mc_ctas = t.mc_ctas;
    out->gr_ctas_per_sm = t.gr_ctas_per_sm;
    out->from_cache = from_cache;
    out->mc_us_per_move = t.mc_us_per_move;
    out->gr_ms = t.gr_ms;
}

}  // namespace

extern "C" int epsr_autotune(epsr_box *box, uint64_t seed, int32_t probe_moves, epsr_tuning *out,
                             epsr_stream_t stream)
{
    if (!box || probe_moves < 0 || probe_moves > (1 << 20)) return set_error(EPSR_EINVAL, "autotune: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = box_shape_key(box);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_box_cache.find(key);
        if (it != g_box_cache.end()) {
            int rc = apply_box(box, it->second);
            if (!rc) fill(out, it->second, 1);
            return rc;
        }
    }
    const int n_probe = probe_moves > 0 ? probe_moves : 2048;
    int32_t n_boxes = 0;
    int64_t n_atoms = 0, hist_len = 0;
    int rc = epsr_box_info(box, &n_boxes, &n_atoms, &hist_len);
    if (rc) return rc;
    // the state the candidates disturb, restored at the end
    size_t ck_bytes = 0;
    if ((rc = epsr_checkpoint_size(box, &ck_bytes))) return rc;
    std::vector<unsigned char> ck(ck_bytes);
    if ((rc = epsr_checkpoint_save(box, ck.data(), ck.size(), stream))) return rc;
    int32_t batch0 = 0, ctas0 = 0, gr0 = 4;
    epsr_box_get_launch(box, &batch0, &ctas0, &gr0);
    const int sms = std::max(1, box_sms(box));

    // Monte Carlo: CTA budget x moves per barrier
    std::vector<int> budgets = {sms, sms * 3 / 4, sms / 2};
    budgets.erase(std::remove_if(budgets.begin(), budgets.end(), [&](int b) { return b < n_boxes; }), budgets.end());
    std::sort(budgets.begin(), budgets.end());
    budgets.erase(std::unique(budgets.begin(), budgets.end()), budgets.end());
    if (budgets.empty()) budgets.push_back(0);
    BoxTuning best;
    best.mc_us_per_move = 1e30;
    uint64_t move0 = 0;
    for (int budget : budgets) {
        if ((rc = epsr_mc_set_ctas(box, budget))) break;
        for (int batch : {16, 32, 64}) {
            if ((rc = epsr_mc_set_batch(box, batch))) break;
            double ms = 0, best_ms = 1e30;
            for (int rep = 0; rep < 3 && !rc; ++rep) {     // the first run warms up
                rc = time_ms(s, 1, [&]() { return epsr_mc_sweep_async(box, n_probe, seed, move0, nullptr, stream); }, &ms);
                move0 += (uint64_t)n_probe;
                int32_t st = EPSR_OK;
                if (!rc) rc = epsr_mc_status(box, &st, stream);
                if (!rc && st != EPSR_OK) rc = set_error(st, "autotune: a probe sweep reported status %d", st);
                if (rep > 0) best_ms = std::min(best_ms, ms);
            }
            if (rc) break;
            const double us = 1e3 * best_ms / n_probe;
            if (us < best.mc_us_per_move) {
                best.mc_us_per_move = us;
                best.mc_batch = batch;
                best.mc_ctas = budget;
            }
        }
        if (rc) break;
    }
    // all-pair histogram: persistent CTAs per SM
    uint64_t *hist = nullptr;
    if (!rc) {
        cudaError_t e = cudaMalloc(&hist, (size_t)std::max<int64_t>(1, hist_len) * sizeof(uint64_t));
        if (e != cudaSuccess) { cudaGetLastError(); rc = set_error(EPSR_ENOMEM, "autotune: scratch histogram"); }
    }
    best.gr_ms = 1e30;
    for (int per_sm = 2; per_sm <= 4 && !rc; ++per_sm) {
        if ((rc = epsr_gr_set_ctas_per_sm(box, per_sm))) break;
        double ms = 0, best_ms = 1e30;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            rc = time_ms(s, 1, [&]() { return epsr_partial_gr(box, hist, nullptr, 1, stream); }, &ms);
            if (rep > 0) best_ms = std::min(best_ms, ms);
        }
        if (!rc && best_ms < best.gr_ms) {
            best.gr_ms = best_ms;
            best.gr_ctas_per_sm = per_sm;
        }
    }
    if (hist) cudaFree(hist);
    // restore the state; keep the winner (or, after a failure, the settings the handle had)
    int rc2 = epsr_checkpoint_load(box, ck.data(), ck.size(), stream);
    if (rc) {
        BoxTuning prev;
        prev.mc_batch = batch0;
        prev.mc_ctas = ctas0;
        prev.gr_ctas_per_sm = gr0;
        apply_box(box, prev);
        return rc;
    }
    if (rc2) return rc2;
    if ((rc = apply_box(box, best))) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_box_cache[key] = best;
    }
    fill(out, best, 0);
    return EPSR_OK;
}

extern "C" int epsr_sq_plan_autotune(epsr_sq_plan *plan, const float *g, int32_t n_cols, const double *w,
                                     int32_t cols_per_set, const double *flat, float *S_partial, float *S_total,
                                     int32_t *n_chunk, int32_t *k_split, double *us, epsr_stream_t stream)
{
    if (!plan || !g || !w || n_cols < 1 || cols_per_set < 1 || n_cols % cols_per_set || (!S_partial && !S_total))
        return set_error(EPSR_EINVAL, "sq autotune: bad argument");
    if (n_chunk) *n_chunk = 0;
    if (k_split) *k_split = 0;
    if (us) *us = 0;
    if (sq_plan_mode(plan) == EPSR_SQ_FP32) return EPSR_OK;       // nothing to tune
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = sq_plan_key(plan, n_cols, cols_per_set, S_total != nullptr);
    SqTuning best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_sq_cache.find(key);
        if (it != g_sq_cache.end()) { best = it->second; cached = true; }
    }
    if (!cached) {
        const int gcd16 = [](int a, int b) { while (b) { int t = a % b; a = b; b = t; } return a; }(16, cols_per_set);
        const int L = 16 / gcd16 * cols_per_set;
        const int n_pad = (n_cols + 15) / 16 * 16;
        std::vector<int> chunks = {16, 32, 64};
        if (S_total && L <= 256) { chunks.push_back(L); if (2 * L <= 128) chunks.push_back(2 * L); }
        std::sort(chunks.begin(), chunks.end());
        chunks.erase(std::unique(chunks.begin(), chunks.end()), chunks.end());
        const int stages = sq_plan_stages(plan);
        best.us = 1e30;
        for (int nc : chunks) {
            if (nc > std::max(16, n_pad)) continue;
            for (int ks : {1, 2, 4, 8}) {
                if (ks > stages) continue;
                if (epsr_sq_plan_set_tiles(plan, nc, ks) != EPSR_OK) continue;    // does not fit
                double ms = 0;
                int rc = epsr_sq_exec(plan, g, n_cols, w, cols_per_set, flat, S_partial, S_total, stream);   // warm
                if (!rc) rc = time_ms(s, 3, [&]() {
                    return epsr_sq_exec(plan, g, n_cols, w, cols_per_set, flat, S_partial, S_total, stream);
                }, &ms);
                if (rc) { epsr_sq_plan_set_tiles(plan, 0, 0); return rc; }
                if (1e3 * ms < best.us) {
                    best.us = 1e3 * ms;
                    best.n_chunk = nc;
                    best.k_split = ks;
                }
            }
        }
        if (best.n_chunk == 0) { epsr_sq_plan_set_tiles(plan, 0, 0); return set_error(EPSR_EINVAL, "sq autotune: no tiling fits"); }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_sq_cache[key] = best;
    }
    int rc = epsr_sq_plan_set_tiles(plan, best.n_chunk, best.k_split);
    if (rc) return rc;
    int32_t st = EPSR_OK;
    if ((rc = epsr_sq_plan_status(plan, &st, stream))) return rc;
    if (st != EPSR_OK) return set_error(st, "sq autotune: a tensor-core wait gave up");
    if (n_chunk) *n_chunk = best.n_chunk;
    if (k_split) *k_split = best.k_split;
    if (us) *us = best.us;
    return EPSR_OK;
}
