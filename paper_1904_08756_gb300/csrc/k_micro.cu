// k_micro.cu -- two measurements that bound the Monte Carlo sweep on this GPU, run by the
// library's own kernels so that they see the same code generation as the sweep:
//  - the grid-barrier floor: a cooperative persistent grid that does nothing but the sweep's
//    per-batch exchange (64 partials and the pair corrections to the slot buffer, release add
//    on a counter, acquire poll, fixed-order gather), i.e. the least time per batch;
//  - the integer and FP32 issue rates: independent dependency chains of 32-bit adds or FP32
//    fused multiply-adds in every lane, counted as lane-operations per second.
#include "epsr_device.cuh"
#include "epsr_internal.h"
#include "epsr_probe.h"

namespace epsr {

constexpr int kMicroThreads = 512;
constexpr int kMicroPartials = kMcBatchMax;    // partials per CTA (moves per batch)
constexpr int kMicroCorr = kMcCorrPerCta;      // batch-pair corrections per group
static_assert(kMicroThreads == 8 * kMicroPartials, "8 threads per partial");

// Slot buffer per parity: partials [kMicroPartials][G], then kMicroCorr corrections, pair pq
// written by CTA pq mod G; the layout and the order of operations are the sweep's.
__global__ void __launch_bounds__(kMicroThreads, 1)
barrier_floor_kernel(unsigned *counter, float *slots, int iters, unsigned long long timeout_ns, int *status,
                     float *sink)
{
    __shared__ float part[kMicroPartials];
    __shared__ float base[kMicroPartials];
    __shared__ float corr[kMicroCorr];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, cta = blockIdx.x;
    if (tid == 0) abort_flag = 0;
    if (tid < kMicroPartials) part[tid] = (float)(cta + tid);
    __syncthreads();
    const int n_local = kMicroCorr > cta ? (kMicroCorr - cta + G - 1) / G : 0;
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        float *ps = slots + (size_t)(it & 1) * ((size_t)kMicroPartials * G + kMicroCorr);
        float *cs = ps + (size_t)kMicroPartials * G;
        if (warp == 0) {
            for (int k = lane; k < kMicroPartials; k += 32) ps[(size_t)k * G + cta] = part[k];
            for (int u = lane; u < n_local; u += 32) cs[cta + u * G] = (float)u;
            __syncwarp();
            if (lane == 0) {
                red_add_release_gpu(counter, 1u);
                const unsigned target = (unsigned)(it + 1) * (unsigned)G;
                const uint64_t t0 = globaltimer_ns();
                long long spins = 0;
                bool timed_out = false;
                while (ld_acquire_gpu(counter) < target) {
                    if ((++spins & 255) == 0 && (globaltimer_ns() - t0 > timeout_ns || ld_relaxed_gpu(status) != 0)) {
                        timed_out = true;
                        break;
                    }
                }
                if (timed_out) {
                    atomicOr(status, kStatusTimeout);
                    abort_flag = 1;
                }
            }
        }
        __syncthreads();
        if (abort_flag) return;
        {
            const int k = tid >> 3, sub = tid & 7;
            float v = 0.f, pv[20];
#pragma unroll
            for (int i = 0; i < 20; ++i) pv[i] = sub + 8 * i < G ? __ldcg(&ps[(size_t)k * G + sub + 8 * i]) : 0.f;
#pragma unroll
            for (int i = 0; i < 20; ++i) v += pv[i];
            for (int r = sub + 160; r < G; r += 8) v += __ldcg(&ps[(size_t)k * G + r]);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (sub == 0) base[k] = v;
        }
        {
            constexpr int kLoads = (kMicroCorr + kMicroThreads - 1) / kMicroThreads;
            float cv[kLoads];
#pragma unroll
            for (int i = 0; i < kLoads; ++i) cv[i] = tid + i * kMicroThreads < kMicroCorr ? __ldcg(&cs[tid + i * kMicroThreads]) : 0.f;
#pragma unroll
            for (int i = 0; i < kLoads; ++i)
                if (tid + i * kMicroThreads < kMicroCorr) corr[tid + i * kMicroThreads] = cv[i];
        }
        __syncthreads();
        if (tid < kMicroPartials) acc += base[tid] + corr[tid];
    }
    if (tid < kMicroPartials && acc == -1.f) sink[cta] = acc;   // keeps the gather live
}

// 8 independent chains per lane; kind 0: 32-bit exclusive-or and add (two lane-operations
// per step), kind 1: FP32 fused multiply-add (one per step).
__global__ void alu_rate_kernel(int kind, int iters, unsigned *sink)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (kind == 0) {
        unsigned a0 = t, a1 = t ^ 1u, a2 = t ^ 2u, a3 = t ^ 3u, a4 = t ^ 4u, a5 = t ^ 5u, a6 = t ^ 6u, a7 = t ^ 7u;
        unsigned s = t | 1u, r = t * 2654435761u;
        for (int i = 0; i < iters; ++i) {
            // (a ^ s) + r: an exclusive-or then an add, two integer operations that no single
            // instruction performs together and that do not reassociate across steps
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                a0 = (a0 ^ s) + r; a1 = (a1 ^ s) + r; a2 = (a2 ^ s) + r; a3 = (a3 ^ s) + r;
                a4 = (a4 ^ s) + r; a5 = (a5 ^ s) + r; a6 = (a6 ^ s) + r; a7 = (a7 ^ s) + r;
            }
            s += 0x9e3779b9u;
            r ^= s;
        }
        if ((a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7) == 0x12345678u) sink[t] = a0;
    } else {
        float a0 = (float)t, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f, a4 = a0 + 4.f, a5 = a0 + 5.f,
              a6 = a0 + 6.f, a7 = a0 + 7.f;
        const float m = 0.9999999f, c = 1e-7f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
                a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
            }
        }
        if (a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7 == -1.f) sink[t] = 1u;
    }
}

int micro_barrier_floor(int ctas, int iters, double timeout_ms, double *ns_per_barrier, cudaStream_t stream)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_floor_kernel, kMicroThreads, 0);
    if (e != cudaSuccess) return set_cuda_error(e, "occupancy(barrier floor)");
    if (ctas < 1 || ctas > per_sm * sms) return set_error(EPSR_EINVAL, "barrier floor: %d CTAs (1..%d)", ctas, per_sm * sms);
    unsigned *counter = nullptr;
    float *slots = nullptr, *sink = nullptr;
    int *status = nullptr;
    int rc = EPSR_OK;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaMalloc(&counter, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&slots, (size_t)2 * ((size_t)kMicroPartials * ctas + kMicroCorr) * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&sink, (size_t)ctas * sizeof(float)) != cudaSuccess) {
        rc = set_error(EPSR_ENOMEM, "barrier floor scratch");
    }
    if (!rc && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
        rc = set_error(EPSR_ECUDA, "barrier floor events");
    unsigned long long tns = (unsigned long long)(timeout_ms * 1e6);
    float ms = 0.f;
    int st = 0;
    for (int pass = 0; !rc && pass < 2; ++pass) {       // pass 0 warms up
        cudaMemsetAsync(counter, 0, sizeof(unsigned), stream);
        cudaMemsetAsync(status, 0, sizeof(int), stream);
        void *params[] = {&counter, &slots, &iters, &tns, &status, &sink};
        cudaEventRecord(a, stream);
        e = cudaLaunchCooperativeKernel((const void *)barrier_floor_kernel, dim3(ctas), dim3(kMicroThreads), params, 0, stream);
        if (e != cudaSuccess) { rc = set_cuda_error(e, "barrier floor launch"); break; }
        note_launch();
        cudaEventRecord(b, stream);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) { rc = set_cuda_error(e, "barrier floor sync"); break; }
        cudaEventElapsedTime(&ms, a, b);
        cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
        if (st) { rc = set_error(EPSR_ETIMEOUT, "barrier floor: a wait exceeded %.0f ms", timeout_ms); break; }
    }
    if (!rc) *ns_per_barrier = (double)ms * 1e6 / iters;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(counter); cudaFree(status); cudaFree(slots); cudaFree(sink);
    return rc;
}

int micro_alu_rate(int kind, double *lane_ops_per_s, cudaStream_t stream)
{
    if (kind != 0 && kind != 1) return set_error(EPSR_EINVAL, "alu rate: kind 0 (int32 add) or 1 (fp32 fma)");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = sms * 8, iters = 4096;
    unsigned *sink = nullptr;
    if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(unsigned)) != cudaSuccess)
        return set_error(EPSR_ENOMEM, "alu rate scratch");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    int rc = EPSR_OK;
    for (int pass = 0; pass < 2; ++pass) {
        cudaEventRecord(a, stream);
        alu_rate_kernel<<<blocks, threads, 0, stream>>>(kind, iters, sink);
        note_launch();
        cudaEventRecord(b, stream);
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) { rc = set_cuda_error(e, "alu rate"); break; }
        cudaEventElapsedTime(&ms, a, b);
    }
    if (!rc) *lane_ops_per_s = (double)blocks * threads * iters * 16.0 * 8.0 * (kind == 0 ? 2.0 : 1.0) /
                               ((double)ms * 1e-3);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return rc;
}

}  // namespace epsr

extern "C" int epsr_bench_barrier_floor(int32_t ctas, int32_t iters, double *ns_per_barrier, epsr_stream_t stream)
{
    if (!ns_per_barrier || iters < 1) return epsr::set_error(EPSR_EINVAL, "bad argument");
    return epsr::micro_barrier_floor(ctas, iters, 2000.0, ns_per_barrier, (cudaStream_t)stream);
}

extern "C" int epsr_bench_alu_rate(int32_t kind, double *lane_ops_per_s, epsr_stream_t stream)
{
    if (!lane_ops_per_s) return epsr::set_error(EPSR_EINVAL, "NULL argument");
    return epsr::micro_alu_rate(kind, lane_ops_per_s, (cudaStream_t)stream);
}

