/*
 * fpe_bench.h -- measurement support for libfpe (no counterpart in the paper).
 *
 * The FP64 window kernels of fpe.h are bound by the FP64 FMA pipe and the
 * tensor-core window sums by the bf16 mma.sync rate; neither is a published
 * constant for this GPU, so these calls measure them on the current device
 * and roofline fractions use denominators taken on the same GPU at the same
 * time.
 */
#ifndef FPE_BENCH_H_
#define FPE_BENCH_H_

#include "fpe.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * fpe_measure_fma_peak -- FMA throughput of the current device.
 *   precision   64 for FP64 (double) FMA, 32 for FP32 (float) FMA.
 *   fma_per_s   receives the best of `reps` timed launches, in fused
 *               multiply-adds per second (flop/s is twice that).
 *   reps        >= 1 timed launches after one warm-up launch.
 * Each launch runs 8 independent FMA chains per thread on 4 blocks of 256
 * threads per SM.  Synchronous (uses its own CUDA events on the legacy
 * default stream).  Errors: FPE_ERR_INVALID_ARG, FPE_ERR_CUDA.
 */
fpe_status fpe_measure_fma_peak(int precision, int reps, double *fma_per_s);

/*
 * fpe_measure_mma_peak -- bf16 tensor-core throughput of the instruction the
 *   tensor-core window sums issue (mma.sync m16n8k16, fp32 accumulation):
 *   eight independent accumulators per warp, operands in registers, 8 warps
 *   per block and 2 blocks per SM.  flop_per_s receives the best of `reps`
 *   timed launches (2 flop per multiply-add).  Synchronous, as above.
 *   Errors: FPE_ERR_INVALID_ARG, FPE_ERR_CUDA.
 */
fpe_status fpe_measure_mma_peak(int reps, double *flop_per_s);

#ifdef __cplusplus
}
#endif
#endif /* FPE_BENCH_H_ */
