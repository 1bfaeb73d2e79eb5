/*
 * sm_debug.h -- test hooks of the library (not needed by normal callers).
 *
 * They let a test drive the bounded-wait path of the wavefront sweep without
 * any GPU fault: with skip_publish enabled, the first strip of every chain
 * never releases its row counters, so every downstream wait runs into its
 * time limit, records SM_ERR_TIMEOUT in the device status word and returns;
 * sm_synchronize() then reports SM_ERR_TIMEOUT and the problem stays usable.
 * The paper has no counterpart (its sweeps run on CPUs without such waits).
 */
#ifndef SM_TRT_DEBUG_H
#define SM_TRT_DEBUG_H

#include "sm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Time limit of every wavefront wait of this problem, in nanoseconds
 * (default 2e9).  INVALID_ARG for ns <= 0. */
sm_status sm_debug_set_wait_limit_ns(sm_problem *p, long long ns);

/* Non-zero: strip 0 of each chain withholds its row counters (see above). */
sm_status sm_debug_skip_publish(sm_problem *p, int enable);

/* Non-zero: the last block of the cooperative low-order kernel leaves before
 * its first grid barrier, so every other block's barrier wait runs into the
 * time limit; the solve returns SM_ERR_TIMEOUT and the problem stays usable. */
sm_status sm_debug_withhold_lo_block(sm_problem *p, int enable);

/* Form of the conjugate gradients in the low-order solves of this problem:
 * SM_DEBUG_PCG_AUTO (the library's choice: the single-reduction form below
 * 4096 cells, else the textbook form),
 * SM_DEBUG_PCG_TEXTBOOK (FP64, two grid reductions per iteration),
 * SM_DEBUG_PCG_SINGLE (FP64, Chronopoulos-Gear, one reduction per iteration)
 * or SM_DEBUG_PCG_MIXED (iterative refinement: FP32 conjugate gradients on
 * FP32 copies of the operator, FP64 residual updates; the same FP64 stopping
 * test, and the FP64 textbook form from the current iterate if a refinement
 * cycle stops halving the residual).  The FP64 forms compute the same iterates
 * up to rounding; every form stops at the same FP64 relative residual.  The
 * batched time step (sm_batch_step) runs the FP64 forms (mixed: textbook).
 * INVALID_ARG for other values. */
enum {
    SM_DEBUG_PCG_AUTO = 0,
    SM_DEBUG_PCG_TEXTBOOK = 1,
    SM_DEBUG_PCG_SINGLE = 2,
    SM_DEBUG_PCG_MIXED = 3
};
sm_status sm_debug_set_pcg_form(sm_problem *p, int form);

/* The form (SM_DEBUG_PCG_TEXTBOOK, _SINGLE or _MIXED) that the problem's
 * last low-order solve used, or SM_DEBUG_PCG_AUTO if it has run none. */
sm_status sm_debug_get_pcg_form(const sm_problem *p, int *form);

/* Emission of an FP32-sweep problem's sweeps: 0 (the default) evaluates the
 * Planck group integrals in double-FP32 arithmetic (pairs of FP32 numbers,
 * about 48 significant bits, on the FP32 pipes); non-zero takes the FP64
 * evaluation that FP64 problems and sm_emission use, so that a test can
 * compare the two.  INVALID_ARG for a NULL problem. */
sm_status sm_debug_set_emission_fp64(sm_problem *p, int fp64);

/* Low-order solves of sm_batch_step: non-zero (the default) runs every
 * member's Newton iteration in one cooperative launch, each member on its own
 * share of the blocks; 0 runs one cooperative launch per member, one after
 * another, as sm_step does.  Both solve the same systems (the block counts,
 * and so the order of the grid sums, differ).  INVALID_ARG for a NULL batch. */
sm_status sm_debug_set_batch_lo(sm_batch *b, int batched);

/* out_dev[i] = e^{-x_dev[i]} for i < n, evaluated by the emission kernels'
 * table-driven routine (Tang's method) for 0 <= x < 708, so that a test can
 * compare it with CUDA's exp directly; elsewhere out_dev[i] = exp(-x) of the
 * CUDA math library.  FP64 device arrays; asynchronous on stream (a
 * cudaStream_t, NULL = legacy default stream).  INVALID_ARG for n < 0 or a
 * NULL array with n > 0. */
sm_status sm_debug_exp_neg(const double *x_dev, double *out_dev, int n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SM_TRT_DEBUG_H */
