// epsr_refine.cu -- the EPSR refinement loop around the hot path.
//
// Sec. 2.2 of the paper runs the method as a loop: Monte Carlo moves with the reference
// potential plus the current empirical potential (item III), the structure factor of the
// simulated box by Eq. (1) compared with the measured one (IV), the difference
// Delta S(Q) = S_measured - S_simulated fitted with Poisson functions in Q space and turned
// into an addition to the empirical potential through the pair weights of Eq. (2) (V), and
// the loop repeated with statistics accumulated (VI) until the empirical potential stops
// changing (Sec. 2.1). One epsr_refine_step is one pass: a sweep, the pair histograms
// (accumulated or fresh), S(Q) of every dataset as one contraction (the histogram's g
// columns repeated once per dataset with that dataset's weights), Delta S and chi^2 on the
// device, then epsr_ep_update. Every step of the pass is a library kernel; this file only
// orders them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "epsr.h"
#include "epsr_internal.h"

using namespace epsr;

struct epsr_refiner {
    epsr_box *box = nullptr;
    epsr_sq_plan *plan = nullptr;
    int n_data = 0, P = 0, n_bins = 0, nQ = 0;
    double kT = 0, rho = 0, dr = 0;
    epsr_refine_params prm{};
    std::vector<double> w, w_cols, flat;
    std::vector<float> Q;
    const float *target = nullptr;       // caller's device [n_data][nQ]
    uint64_t *hist = nullptr;            // [P][n_bins], accumulated over the passes
    float *g = nullptr;                  // [P][n_bins]
    float *g_rep = nullptr;              // [n_data][P][n_bins]
    float *S = nullptr;                  // [n_data][nQ]
    float *dS = nullptr;                 // [n_data][nQ]
    double *chi2 = nullptr;              // [1]
    long long n_cfg = 0, iteration = 0;
    uint64_t move0 = 0;
    std::vector<double> C;               // the last fit [P][n_basis]
    ~epsr_refiner()
    {
        void *ptrs[] = {hist, g, g_rep, S, dS, chi2};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
};

namespace {

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return set_cuda_error(e_, #call);   \
    } while (0)

constexpr int kDeltaThreads = 256;

// dS = target - S and chi^2 = sum dS^2 (FP64; per-thread sums in index order, then a fixed
// tree), one CTA.
__global__ void __launch_bounds__(kDeltaThreads) refine_delta_kernel(const float *target, const float *S, float *dS,
                                                                     int n, double *chi2)
{
    __shared__ double part[kDeltaThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kDeltaThreads) {
        const float d = target[i] - S[i];
        dS[i] = d;
        acc += (double)d * (double)d;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kDeltaThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *chi2 = part[0];
}

template <class T>
int dalloc_n(T **p, size_t n)
{
    if (cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(1, n) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(EPSR_ENOMEM, "refiner: cudaMalloc of %zu bytes failed", n * sizeof(T));
    }
    return EPSR_OK;
}

// p_n(r) = (r / (n s))^n exp(n - r / s): the Poisson function with its peak, 1, at r = n s.
double poisson_p(int n, double s, double r)
{
    return r > 0 ? std::exp(n * std::log(r / (n * s)) + n - r / s) : 0.0;
}

}  // namespace

extern "C" int epsr_refiner_create(epsr_box *box, epsr_sq_plan *plan, const float *target, int32_t n_data,
                                   const double *w, const double *flat, const float *Q, int32_t nQ,
                                   const epsr_refine_params *params, epsr_stream_t stream, epsr_refiner **out)
{
    if (!out) return set_error(EPSR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!box || !plan || !target || !w || !flat || !Q || !params || n_data < 1 || n_data > 16 || nQ < 1)
        return set_error(EPSR_EINVAL, "refiner: bad argument");
    BoxSummary bs;
    int rc = box_summary(box, 0, &bs);
    if (rc) return rc;
    if (bs.n_boxes != 1) return set_error(EPSR_EINVAL, "refiner: the handle must hold one box (it has %d)", bs.n_boxes);
    int pQ = 0, pbins = 0, pcols = 0;
    sq_plan_dims(plan, &pQ, &pbins, &pcols);
    if (pQ != nQ || pbins != bs.n_bins || pcols < n_data * bs.n_pairs)
        return set_error(EPSR_EINVAL, "refiner: the plan has %d Q, %d bins, %d columns; %d, %d, %d needed", pQ, pbins,
                         pcols, nQ, bs.n_bins, n_data * bs.n_pairs);
    if (params->moves_per_pass < 0 || params->n_basis < 1 || params->n_basis > 40 || !(params->s_basis > 0) ||
        !(params->gamma >= 0) || !std::isfinite(params->alpha) || (n_data < bs.n_pairs && !(params->gamma > 0)))
        return set_error(EPSR_EINVAL, "refiner: parameters out of range");
    epsr_refiner *r = new (std::nothrow) epsr_refiner();
    if (!r) return set_error(EPSR_ENOMEM, "host allocation failed");
    r->box = box;
    r->plan = plan;
    r->n_data = n_data;
    r->P = bs.n_pairs;
    r->n_bins = bs.n_bins;
    r->nQ = nQ;
    r->kT = bs.kT;
    r->rho = bs.rho;
    r->dr = bs.dr;
    r->prm = *params;
    r->w.assign(w, w + (size_t)n_data * r->P);
    r->flat.assign(flat, flat + n_data);
    r->Q.assign(Q, Q + nQ);
    r->w_cols.resize((size_t)n_data * r->P);
    for (size_t i = 0; i < r->w_cols.size(); ++i) r->w_cols[i] = 4.0 * M_PI * r->rho * r->w[i];
    r->target = target;
    r->move0 = params->move0;
    const size_t hp = (size_t)r->P * r->n_bins;
    if ((rc = dalloc_n(&r->hist, hp)) || (rc = dalloc_n(&r->g, hp)) || (rc = dalloc_n(&r->g_rep, hp * n_data)) ||
        (rc = dalloc_n(&r->S, (size_t)n_data * nQ)) || (rc = dalloc_n(&r->dS, (size_t)n_data * nQ)) ||
        (rc = dalloc_n(&r->chi2, 1))) {
        delete r;
        return rc;
    }
    cudaError_t e = cudaMemsetAsync(r->hist, 0, hp * sizeof(uint64_t), (cudaStream_t)stream);
    if (e != cudaSuccess) { delete r; return set_cuda_error(e, "refiner: memset"); }
    *out = r;
    return EPSR_OK;
}

extern "C" int epsr_refiner_destroy(epsr_refiner *r)
{
    if (!r) return EPSR_OK;
    cudaDeviceSynchronize();
    delete r;
    return EPSR_OK;
}

extern "C" int epsr_refine_step(epsr_refiner *r, epsr_move_log *log, epsr_refine_result *res, epsr_stream_t stream)
{
    if (!r) return set_error(EPSR_EINVAL, "refiner is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t hp = (size_t)r->P * r->n_bins;
    epsr_mc_stats st{};
    int rc = EPSR_OK;
    // III: Monte Carlo with the reference plus the current empirical potential
    if (r->prm.moves_per_pass > 0) {
        if ((rc = epsr_mc_sweep(r->box, r->prm.moves_per_pass, r->prm.seed, r->move0, &st, log, stream))) return rc;
        r->move0 += (uint64_t)r->prm.moves_per_pass;
    } else if ((rc = epsr_mc_stats_get(r->box, &st, stream))) {
        return rc;
    }
    // VI / IV: pair histograms (accumulated over the passes, or of this configuration only) and g
    if (!r->prm.accumulate) {
        CK(cudaMemsetAsync(r->hist, 0, hp * sizeof(uint64_t), s));
        r->n_cfg = 0;
    }
    ++r->n_cfg;
    if ((rc = epsr_partial_gr(r->box, r->hist, r->g, r->n_cfg, stream))) return rc;
    // IV: S(Q) of every dataset by Eq. (1), one contraction over n_data x P columns
    for (int d = 0; d < r->n_data; ++d)
        CK(cudaMemcpyAsync(r->g_rep + (size_t)d * hp, r->g, hp * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if ((rc = epsr_sq_exec(r->plan, r->g_rep, r->n_data * r->P, r->w_cols.data(), r->P, r->flat.data(), nullptr,
                           r->S, stream)))
        return rc;
    // Delta S = S_measured - S_simulated, chi^2
    const int n = r->n_data * r->nQ;
    refine_delta_kernel<<<1, kDeltaThreads, 0, s>>>(r->target, r->S, r->dS, n, r->chi2);
    note_launch();
    CK(cudaGetLastError());
    // V: fit the Poisson series to Delta S (pair-resolved through the weights) and add it (Eq. 2)
    r->C.assign((size_t)r->P * r->prm.n_basis, 0.0);
    if ((rc = epsr_ep_update(r->box, 0, r->dS, r->n_data, r->w.data(), r->Q.data(), r->nQ, r->prm.n_basis,
                             r->prm.s_basis, r->prm.gamma, r->prm.alpha, r->C.data(), stream)))
        return rc;
    double chi2 = 0.0;
    CK(cudaMemcpyAsync(&chi2, r->chi2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ++r->iteration;
    if (res) {
        // the largest change this pass made to the table: alpha kT |sum_n C_pn p_n(r_k)|
        double dmax = 0.0;
        for (int p = 0; p < r->P; ++p)
            for (int k = 0; k < r->n_bins; ++k) {
                const double rk = (k + 0.5) * r->dr;
                double v = 0.0;
                for (int nb = 1; nb <= r->prm.n_basis; ++nb) v += r->C[(size_t)p * r->prm.n_basis + nb - 1] * poisson_p(nb, r->prm.s_basis, rk);
                dmax = std::max(dmax, std::fabs(r->prm.alpha * r->kT * v));
            }
        res->iteration = r->iteration;
        res->chi2 = chi2;
        res->ep_change_max = dmax;
        res->attempted = st.attempted;
        res->accepted = st.accepted;
        res->n_configs = r->n_cfg;
        res->next_move = r->move0;
    }
    return EPSR_OK;
}

extern "C" int epsr_refiner_get(const epsr_refiner *r, uint64_t *hist, float *g, float *S, float *dS, double *C,
                                epsr_stream_t stream)
{
    if (!r) return set_error(EPSR_EINVAL, "refiner is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t hp = (size_t)r->P * r->n_bins, sq = (size_t)r->n_data * r->nQ;
    if (hist) CK(cudaMemcpyAsync(hist, r->hist, hp * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (g) CK(cudaMemcpyAsync(g, r->g, hp * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (S) CK(cudaMemcpyAsync(S, r->S, sq * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (dS) CK(cudaMemcpyAsync(dS, r->dS, sq * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (C)
        for (size_t i = 0; i < r->C.size(); ++i) C[i] = r->C[i];
    CK(cudaStreamSynchronize(s));
    return EPSR_OK;
}
