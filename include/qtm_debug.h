/*
 * qtm_debug.h -- host-side inspection of a plan's schedule.
 *
 * These calls never touch the GPU and are never used by qtm_forward /
 * qtm_adjoint.  They exist so the planner (the schedule of passes, phases and
 * ops that the CUDA kernels execute) can be validated on a machine without a
 * GPU: qtm_debug_emulate interprets exactly that schedule in FP64 on the host.
 */
#ifndef QTM_DEBUG_H
#define QTM_DEBUG_H

#include "qtm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Human-readable dump of the plan's passes (tile qubit sets, sources/sinks,
 * register-group phases and ops).  The string is owned by the plan and stays
 * valid until the next call on it or qtm_destroy. */
const char *qtm_debug_describe(const qtm_plan *plan);

/* Interpret the fused schedule in FP64 on the host (n <= 24).  HOST pointers:
 * x [B][n_inputs], w [n_weights], gE [B][n_obs] (NULL: forward only);
 * outputs E [B][n_obs], gx [B][n_inputs], gw [B][n_weights] (per sample), each
 * may be NULL.  Returns QTM_EUNSUPPORTED for naive-path plans or n > 24 and
 * QTM_EINVAL if the schedule breaks a locality rule (see qtm_last_error). */
qtm_status qtm_debug_emulate(const qtm_plan *plan, int B, const double *x, const double *w,
                             const double *gE, double *E, double *gx, double *gw);

/* Source of the specialised kernel qtm_compile(plan, flags) would build for
 * forward (which = 0) or reverse (which = 1) pass `index` ("" if not
 * eligible).  The string is owned by the plan until the next call. */
const char *qtm_debug_jit_source(const qtm_plan *plan, int which, int index, int flags);

/* Generate and compile every pass with NVRTC as qtm_compile(plan, flags)
 * would, without loading anything (host only).  QTM_EINVAL with the compiler
 * log in qtm_last_error on failure. */
qtm_status qtm_debug_jit_compile(qtm_plan *plan, int flags);

/* Measured FMA throughput of this GPU in the real type of `dtype` (QTM_C64:
 * FP32, QTM_C128: FP64), flop/s with an FMA counted as 2: a register-only
 * loop of independent FMA chains over 16 CTAs of 256 threads per SM, best of
 * three launches timed with CUDA events on the current device.  Synchronises
 * the device.  A roofline denominator for the pass kernels, which are FMA
 * bound at 12 qubits; not used by any compute call. */
qtm_status qtm_debug_fma_rate(int dtype, double *flops_per_s);

/* Measured throughput of the complex-pair kernels' own reverse arithmetic on
 * this GPU, flop/s counted as the plans count it (a gradient op with its two
 * gates: 40 flop per amplitude): a register-only loop over the kernels'
 * gradient sums and gates (f32x2 FMAs), 256 threads with the register budget
 * of two CTAs per SM, four waves, best of three launches timed with CUDA
 * events on the current device.  It shows how much of the derived FP32 peak
 * this arithmetic can reach at all (the f32x2 FMAs' operands, not the FMA
 * units, limit it); a context figure for the 12-qubit reverse pass's
 * roofline, not used by any compute call.  Synchronises the device. */
qtm_status qtm_debug_gate_rate(double *flops_per_s);

/* The uneven batch's task list (host only), in the order the persistent
 * kernel hands tasks out: tasks[3i .. 3i+2] = (item, step, tile); step = -1
 * is a whole item, step >= 0 one pass (forward passes, then reverse passes)
 * of an item whose state spans several tiles, and tile its tile.
 * items[2i .. 2i+1] = (circuit, sample) of item i.  At most `capacity` tasks
 * and `item_capacity` items are written; *n_tasks and *n_items (each may be
 * NULL) receive the full counts. */
qtm_status qtm_debug_multi_tasks(const qtm_multi *multi, int32_t *tasks, int capacity, int *n_tasks,
                                 int32_t *items, int item_capacity, int *n_items);

/* The task list of one launch kind (host only): which = 0 qtm_multi_run
 * (the list qtm_debug_multi_tasks returns), 1 qtm_multi_forward (forward
 * passes only), 2 qtm_multi_adjoint (reverse passes only; a tile task's step
 * still counts the forward passes first).  Triples as above. */
qtm_status qtm_debug_multi_mode_tasks(const qtm_multi *multi, int which, int32_t *tasks, int capacity,
                                      int *n_tasks);

/* Failure injection for the persistent kernel's bounded waits: replace the
 * task list by n (item, step, tile) triples and set the limit of one task's
 * wait to wait_ns (> 0; 10 s by default).  Every index is range-checked, but
 * not the order or completeness: a tile task whose item's previous pass is
 * never listed waits out the limit, the run drains, and qtm_multi_sync
 * reports QTM_ETIMEOUT.  Waits for the device when tables were uploaded.  The
 * next qtm_multi_set_config (or qtm_multi_tune) restores the normal list and
 * limit. */
qtm_status qtm_debug_multi_inject(qtm_multi *multi, const int32_t *tasks, int n, long long wait_ns);

#ifdef __cplusplus
}
#endif

#endif /* QTM_DEBUG_H */
