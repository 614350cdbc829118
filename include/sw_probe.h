/*
 * sw_probe.h -- measurement helper of libswgb: the issue rate of the integer
 * instruction forms the alignment kernels use, measured on the running GPU.
 * It gives the integer-ALU roofline a measured denominator; the paper has
 * no counterpart (it reports profiler counters of its own kernels only,
 * Section 4.2, Table 4).
 */
#ifndef SWGB_SW_PROBE_H
#define SWGB_SW_PROBE_H

#include "sw.h"

#ifdef __cplusplus
extern "C" {
#endif

/* instruction forms */
#define SW_PROBE_IADD               0   /* 32-bit integer add */
#define SW_PROBE_IMAX               1   /* 32-bit signed max */
#define SW_PROBE_VIADDMAX_S32       2   /* __viaddmax_s32: max(a + b, c) */
#define SW_PROBE_VIMAX3_S32_RELU    3   /* __vimax3_s32_relu: max(a, b, c, 0) */
#define SW_PROBE_VIADDMAX_S16X2     4   /* __viaddmax_s16x2, two 16-bit lanes */
#define SW_PROBE_VIMAX3_S16X2_RELU  5   /* __vimax3_s16x2_relu, two 16-bit lanes */
#define SW_PROBE_PRMT               6   /* byte permute */
#define SW_PROBE_SHFL               7   /* warp shuffle (plus one xor) */
#define SW_PROBE_VADDUS4            8   /* __vaddus4: four saturating unsigned 8-bit adds */
#define SW_PROBE_VSUBUS4            9   /* __vsubus4: four saturating unsigned 8-bit subtracts */
#define SW_PROBE_VMAXU4            10   /* __vmaxu4: four unsigned 8-bit maxima */

/*
 * Run `op` on every SM (8 blocks of 256 threads per SM, eight independent
 * dependency chains per thread, iters x 16 steps per chain).  Writes the
 * measured thread-level results per SM per SM clock (e.g. 128 means four
 * warp instructions per clock) and the SM clock in MHz observed during the
 * run.  Synchronous on the context's stream.  iters >= 1.
 */
int sw_probe_int_rate(sw_ctx *ctx, int op, int iters, double *per_sm_per_clk, double *sm_mhz);

/*
 * Latency of `op`: one warp runs one chain of iters x 32 instructions, each
 * needing the previous one's result; writes SM clocks per instruction
 * (the shuffle probe adds one integer add per step).  Synchronous on the
 * context's stream.  iters >= 1.
 */
int sw_probe_latency(sw_ctx *ctx, int op, int iters, double *cycles_per_op);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_SW_PROBE_H */
