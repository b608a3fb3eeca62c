/*
 * epsr_probe.h -- measurements of this GPU for the benchmark (libepsr_probe.so). They have no
 * counterpart in the paper and are not part of the method: they measure the bounds the Monte
 * Carlo sweep runs against (the least cost of its grid exchange and the lane-operation rates of
 * the integer and FP32 pipes), which the benchmark reports beside its roofline figures. The
 * library links against libepsr.so and shares its status codes and error messages
 * (epsr_strerror, epsr_last_error_detail).
 */
#ifndef EPSR_PROBE_H
#define EPSR_PROBE_H

#include "epsr.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * epsr_bench_barrier_floor: the least time of one batch exchange of the Monte Carlo sweep:
 * `ctas` co-resident CTAs of 512 threads repeat, `iters` times, nothing but the sweep's grid
 * barrier (64 partials and the batch-pair corrections to the exchange buffer, release add,
 * acquire poll, fixed-order gather). Returns ns per barrier; EPSR_EINVAL if the CTAs cannot be co-resident,
 * EPSR_ETIMEOUT if a wait exceeded 2 s. Synchronises.
 * epsr_bench_alu_rate: lane-operations per second of independent chains in every lane on
 * every SM; kind 0 = 32-bit integer exclusive-or/add pairs, 1 = FP32 fused multiply-adds.
 * Synchronises. */
int epsr_bench_barrier_floor(int32_t ctas, int32_t iters, double *ns_per_barrier, epsr_stream_t stream);
int epsr_bench_alu_rate(int32_t kind, double *lane_ops_per_s, epsr_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* EPSR_PROBE_H */
