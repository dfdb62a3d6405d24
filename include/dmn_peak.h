/*
 * dmn_peak.h - measured arithmetic peaks of the current GPU, the denominators
 * of this library's compute rooflines.
 *
 * The DMN update is bound by the FP64 pipe (the mixed forms by FP64 + FP32),
 * not by memory.  The paper reports CPU timings only, so these entry points
 * have no counterpart there: they measure, on the GPU they run on, how many
 * fused multiply-adds per second the FP64 and FP32 pipes sustain, so that a
 * kernel's achieved flop rate can be stated as a fraction of a measured peak
 * rather than of a datasheet figure.
 */
#ifndef DMN_PEAK_H
#define DMN_PEAK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { DMN_PEAK_FP64_FMA = 0, DMN_PEAK_FP32_FMA = 1 };

/* Sustained FMA throughput of the current device: every SM runs 64 warps (16
 * CTAs of 128 threads), each thread 8 independent chains x = fma(x, a, b) (2
 * flops per FMA), repeated in launches of about 20 ms until `seconds` have
 * elapsed (CUDA events on `stream`, a cudaStream_t as void*, NULL = legacy
 * default stream).  Writes the achieved GFLOP/s over all launches to *gflops
 * and the measured time to *ms.  Allocates a scratch buffer of 2048 x 8 bytes
 * per SM (freed before return) and synchronises the stream.  Errors:
 * DMN_ERR_ARG (-1) for an unknown kind, seconds <= 0 or NULL outputs;
 * DMN_ERR_CUDA (-2) if a CUDA call fails (the message is returned by
 * dmn_last_error(NULL)). */
int dmn_peak_gflops(int32_t kind, double seconds, double* gflops, double* ms, void* stream);

/* The same measurement for a chosen occupancy and instruction-level
 * parallelism: warps_per_sm resident warps per SM (1..4, or a multiple of 4 up
 * to 64), `chains` independent FMA chains per thread (1, 2, 4 or 8), and only
 * the first active_lanes (1..32) lanes of every warp running the chains.
 * *gflops counts the flops of the active lanes only, so a pipe that spends
 * the same time on a warp instruction whatever its active lanes shows a rate
 * proportional to active_lanes.  dmn_peak_gflops is (64, 8, 32).  Errors as
 * above, and DMN_ERR_ARG for parameters outside these ranges. */
int dmn_fma_throughput(int32_t kind, int32_t warps_per_sm, int32_t chains, int32_t active_lanes, double seconds,
                       double* gflops, double* ms, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DMN_PEAK_H */
