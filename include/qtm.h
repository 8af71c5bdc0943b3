/*
 * qtm.h -- C ABI of the GB300 (sm_103a) batched statevector QNN library.
 *
 * What it computes (arXiv 2404.06314, Sec. II):
 *   For every sample b of a batch, the state |psi_b> = U(Theta, s_b)|0> of an
 *   n-qubit parameterised circuit is evolved ONCE and all M observables are
 *   read from it (Eq. (qnn), Sec. II-A "evolve once"):
 *       E[b][m] = <psi_b| O_m |psi_b>,   O_m = sum_{t: obs_t = m} c_t Z^{mask_t}.
 *   The vector-Jacobian product with a cotangent gE[b][m] is computed by the
 *   adjoint ("reverse") method (Sec. II-A, Jones & Gacon Alg. 1, extended to M
 *   observables by weighting them into a single costate), then mapped through
 *   the angle bindings to gradients w.r.t. weights and inputs (Eq. (qnn_grad),
 *   Eq. (qnn_batched)).
 *
 * Conventions:
 *   - qubit q is bit q of the amplitude index (little endian, Qiskit order);
 *   - R_P(t) = exp(-i t P / 2) for P in {X, Y, Z};
 *   - angle of a rotation for sample b:
 *       t = coef * (w_idx >= 0 ? w[w_idx] : 1) * (x_idx >= 0 ? x[b][x_idx] : 1),
 *     which covers variational weights, angle encoding and trainable input
 *     scaling (Sec. II-C; Eq. (concrete_ansatz));
 *   - weights keep their construction order (Sec. II-C), never alphabetical.
 *
 * Memory and ownership:
 *   - x, w, expvals, grad_expvals, grad_x, grad_w are DEVICE pointers owned by
 *     the caller, row-major and contiguous, of the plan's real type:
 *     float for QTM_C64 plans, double for QTM_C128 plans;
 *   - gates/terms passed to qtm_build are HOST arrays, copied by the plan;
 *   - the plan owns its device tables and a state workspace (phi and, for
 *     n > 12, lambda: B x 2^n complex each), allocated lazily on the first
 *     call on a device and grown when a larger batch arrives;
 *   - every call enqueues work on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) and returns without synchronising.
 *
 * Errors: every entry point returns a qtm_status.  Arguments are validated on
 * the host before any launch (QTM_EINVAL).  CUDA errors map to QTM_ECUDA.
 * Kernels never trap: a device-side wait that gives up records a status word
 * that qtm_sync() reports as QTM_ETIMEOUT.  Nothing calls abort() or exit().
 */
#ifndef QTM_H
#define QTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QTM_OK = 0,
    QTM_EINVAL = 1,        /* bad argument (detected on the host, nothing launched) */
    QTM_ENOMEM = 2,        /* device or host allocation failed */
    QTM_ECUDA = 3,         /* a CUDA runtime/driver call failed */
    QTM_EUNSUPPORTED = 4,  /* valid request outside what the library supports */
    QTM_ETIMEOUT = 5,      /* a bounded device-side wait gave up (see qtm_sync) */
    QTM_ESTATE = 6         /* call order violated (e.g. adjoint without forward) */
} qtm_status;

typedef enum { QTM_RX = 0, QTM_RY = 1, QTM_RZ = 2, QTM_CZ = 3, QTM_CNOT = 4, QTM_HADAMARD = 5, QTM_RZZ = 6 } qtm_gate_kind;

typedef enum { QTM_C64 = 0, QTM_C128 = 1 } qtm_dtype;

/* Execution path.  FUSED: whole-circuit shared-memory kernel for n <= 12 and
 * fused HBM sweeps above; NAIVE: one kernel launch per gate over the batch
 * (the plain baseline the fused path is measured against). */
typedef enum { QTM_PATH_AUTO = 0, QTM_PATH_FUSED = 1, QTM_PATH_NAIVE = 2 } qtm_path;

/* One gate (32 bytes).
 *   rotations (QTM_RX/RY/RZ): q0 = target, q1 = -1;
 *   QTM_CZ:   q0, q1 = the two qubits (symmetric);
 *   QTM_CNOT: q0 = control, q1 = target;
 *   QTM_HADAMARD: Hadamard on q0, q1 = -1, no parameters (coef unused);
 *   QTM_RZZ:  exp(-i theta Z_q0 Z_q1 / 2) on q0 != q1, theta as for rotations.
 * The planner lowers H to RX(pi) RY(pi/2) (equal up to a global phase) and
 * RZZ to CNOT(q0, q1) RZ_q1(theta) CNOT(q0, q1) (equal); gradients and
 * Jacobian columns refer to the gates as given.
 * w_idx / x_idx = -1 means "factor 1" (Sec. II-C bindings, see above). */
typedef struct {
    int32_t kind;
    int32_t q0;
    int32_t q1;
    int32_t w_idx;
    int32_t x_idx;
    int32_t reserved;   /* must be 0 */
    double coef;
} qtm_gate;

/* One Z-string term of an observable (24 bytes): O_obs += coef * Z^{zmask}. */
typedef struct {
    uint64_t zmask;
    double coef;
    int32_t obs;
    int32_t reserved;   /* must be 0 */
} qtm_zterm;

/* One Pauli-string term (32 bytes): O_obs += coef * P with P = prod_q sigma_q,
 * sigma_q = X where only xmask has bit q, Y where xmask and zmask both have
 * it, Z where only zmask has it (identity elsewhere). */
typedef struct {
    uint64_t xmask;
    uint64_t zmask;
    double coef;
    int32_t obs;
    int32_t reserved;   /* must be 0 */
} qtm_pauli_term;

typedef struct qtm_plan qtm_plan;

/* Static description of a plan's schedule (host-side; no GPU needed). */
typedef struct {
    int32_t n_qubits;
    int32_t dtype;
    int32_t path;            /* resolved path (FUSED or NAIVE) */
    int32_t tile_qubits;     /* K: qubits per shared-memory tile */
    int32_t fwd_passes;      /* kernel passes over the state in qtm_forward */
    int32_t adj_passes;      /* passes in qtm_adjoint (without recompute) */
    int32_t fwd_launches;    /* kernel launches per qtm_forward (one-sample kernels; with plans of
                              * one tile per sample, one per-call kernel for the sines and
                              * cosines of rotations without an input) */
    int32_t adj_launches;    /* kernel launches per qtm_adjoint (per-sample grad_w; one more
                              * for the batch-summed grad_w) */
    int32_t n_runs;          /* fused single-qubit rotation runs */
    int32_t n_prefix_runs;   /* runs folded into the analytic product-state init */
    int32_t n_prefix_ents;   /* CZ/CNOT folded into the init */
    int32_t reserved0;
    double fwd_state_bytes;  /* HBM bytes moved over the state per sample, forward */
    double adj_state_bytes;  /* same, adjoint */
    /* Arithmetic per sample, counted per operation of the schedule over the
     * N = 2^n amplitudes with a complex multiply as 6 flop and a complex add
     * as 2: a fused 2x2 rotation 14 N, an adjoint gradient step 12 N (the
     * three inner products) plus 28 N (the rotation undone on phi and lam),
     * expectation values (3 + terms) N, costate (terms + 2) N, the analytic
     * product-state init 6 (ceil(n/4) - 1) N, 4 N per string with X/Y factors
     * (expectation value, and again for its costate part); sign flips and
     * permutations 0. */
    double fwd_flops;        /* forward */
    double adj_flops;        /* adjoint */
} qtm_plan_info;

/* Flags of qtm_adjoint. */
#define QTM_ADJ_GW_PER_SAMPLE 1  /* grad_w is [B][P] per sample instead of the batch sum [P] */
#define QTM_ADJ_RECOMPUTE 2      /* re-run the forward instead of using the stored state */

/*
 * qtm_build: plan a circuit (Sec. II-A problem statement: circuit, observables).
 *   n_qubits  1 .. 30;  gates/terms: host arrays (copied);  n_obs >= 1;
 *   n_weights, n_inputs >= 0;  dtype: qtm_dtype;  path: qtm_path.
 * Validates every index (qubits < n, CZ/CNOT with distinct qubits, w_idx <
 * n_weights, x_idx < n_inputs, zmask < 2^n, obs < n_obs).  Host-only: does no
 * CUDA call, so it works without a GPU.  On success *out owns the plan.
 */
qtm_status qtm_build(int n_qubits, const qtm_gate *gates, int n_gates,
                     const qtm_zterm *terms, int n_terms, int n_obs,
                     int n_weights, int n_inputs, int dtype, int path, qtm_plan **out);

/*
 * qtm_build_pauli: as qtm_build, with observables that are real combinations
 * of Pauli strings (X, Y and Z terms; Sec. II-A's expectation values of
 * general observables, all from one evolved state).  Fused (and AUTO) plans
 * evolve each sample once: Z strings are measured inside the pass kernels,
 * strings with X/Y factors on the final state the last forward pass leaves
 * in memory, and their part of the adjoint's costate is formed there before
 * the reverse passes.  Naive-path plans instead group the terms by their X
 * and Y qubits and measure each group on its own plan of the circuit followed
 * by the basis change V = RY(-pi/2) on X qubits and RX(pi/2) on Y qubits
 * (V sigma V^dagger = Z), summing the groups' outputs in group order
 * (qtm_plan_parts counts them).  Every entry point below applies, except that
 * qtm_forward_noalloc returns QTM_EUNSUPPORTED for plans with X/Y terms.
 * With Z strings only this is qtm_build.
 */
qtm_status qtm_build_pauli(int n_qubits, const qtm_gate *gates, int n_gates,
                           const qtm_pauli_term *terms, int n_terms, int n_obs,
                           int n_weights, int n_inputs, int dtype, int path, qtm_plan **out);

/* Number of measurement groups of a plan (1 unless built from X/Y terms). */
int qtm_plan_parts(const qtm_plan *plan);

/*
 * qtm_forward: expectation values, Eq. (qnn) for every sample of the batch
 * (Eq. (qnn_batched)).  x: [B][n_inputs], w: [n_weights], expvals: [B][n_obs]
 * (device, plan real type).  B >= 0; B = 0 is an empty batch: nothing is
 * computed and no pointer is read (QTM_ECUDA still without a CUDA device).
 * Keeps the final states in the plan's workspace for a following qtm_adjoint
 * on the same stream.
 */
qtm_status qtm_forward(qtm_plan *plan, int B, const void *x, const void *w,
                       void *expvals, void *stream);

/*
 * qtm_adjoint: vector-Jacobian product by the adjoint method (Sec. II-A).
 *   grad_expvals [B][n_obs] is the cotangent of expvals;  outputs
 *   grad_x [B][n_inputs] (or NULL) and grad_w ([n_weights], or [B][n_weights]
 *   with QTM_ADJ_GW_PER_SAMPLE; or NULL).  Outputs are overwritten.
 * Uses the states stored by the last qtm_forward on this plan, which must have
 * had the same B, x and w, on the same stream; pass QTM_ADJ_RECOMPUTE to
 * evolve them again (required if anything else ran on the plan since).  Returns
 * QTM_ESTATE when no stored forward matches (B, x, w pointers).  The stored
 * states are consumed.  B = 0 (empty batch): no stored forward is needed,
 * nothing is computed, and a batch-summed grad_w is set to zero on the stream.
 */
qtm_status qtm_adjoint(qtm_plan *plan, int B, const void *grad_expvals, const void *x,
                       const void *w, void *grad_x, void *grad_w, int flags, void *stream);

/*
 * qtm_jacobian: full Jacobian J[b][m][g] = d<O_m>/d theta_g with respect to
 * every gate angle (device, plan real type, [B][n_obs][n_gates], zero for
 * CZ/CNOT): the (B, M, |Theta|) output of Sec. II-B, one costate per
 * observable (the reverse passes run once per observable with cotangent
 * e_m).  Runs the forward itself; fused plans only (QTM_EUNSUPPORTED on the
 * naive path).  Leaves no stored forward state behind.  B = 0: nothing.
 */
qtm_status qtm_jacobian(qtm_plan *plan, int B, const void *x, const void *w, void *jac,
                        void *stream);

/* Size of the device array behind qtm_forward_noalloc (bytes, per GPU). */
#define QTM_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * qtm_forward_noalloc: the expectation values of qtm_forward, without any
 * device allocation.  The paper has no counterpart; this exists for callers
 * that cannot call cudaMalloc: host programs whose GPU memory is owned by
 * another allocator with a fixed budget (a framework that reserves the
 * device's memory up front, an application that forbids its plugins to
 * allocate), and loops that must not stall on an allocation, which can
 * synchronise the device.
 *
 * Instead of plan-owned buffers it uses one file-scope device array of
 * QTM_NOALLOC_SCRATCH_BYTES (8 MiB) that the library keeps on every GPU it is
 * loaded on until the process exits.  Arguments are those of qtm_forward
 * (device pointers, plan real type), with B >= 1.  Supported for fused plans
 * whose state fits one shared-memory tile (n <= 12): otherwise
 * QTM_EUNSUPPORTED.  A batch whose tables and scratch exceed the array returns
 * QTM_EINVAL before any work is enqueued (about 2.8 MB for 12 qubits, 6
 * layers, B = 1024).  The call copies the plan's tables (a few KB) from host
 * memory each time; those copies return once the bytes are staged.
 *
 * Set-up: the first call on each device (and the first after that device's
 * context was reset) loads the library's device code there and resolves the
 * array's device address (cudaGetSymbolAddress, with that device current), so
 * make that first call before any stream capture.  Every call shares the
 * array and no call clears what an earlier one left in it: calls that overlap
 * on the GPU (different streams, or different plans at the same time) race
 * and must be serialised by the caller.  It stores no state for qtm_adjoint.
 */
qtm_status qtm_forward_noalloc(qtm_plan *plan, int B, const void *x, const void *w,
                               void *expvals, void *stream);

/* Per-launch timing (profiling aid).  enable = 1: every later qtm_forward /
 * qtm_adjoint records a pair of CUDA events around each of its kernel
 * launches, on the call's stream; enable = 2: only around the pass kernels
 * of qtm_adjoint (each event between two kernels delays the second by a
 * microsecond or two, so timing the dominant kernel alone perturbs the rest
 * least); enable = 0 stops recording.  Other values: QTM_EINVAL. */
qtm_status qtm_set_profiling(qtm_plan *plan, int enable);

/* After the stream has been synchronised: the device durations (ms) of the
 * kernel launches of the last profiled qtm_forward (which = 0) or qtm_adjoint
 * (which = 1), in launch order.  kinds[i] (optional) receives 0 for a pass
 * kernel over the state and 1 for a finalize/reduce kernel.  *count receives
 * the number of launches (at most cap are written). */
qtm_status qtm_get_launch_times(qtm_plan *plan, int which, float *ms, int *kinds, int cap,
                                int *count);

/* ------------------------------------------------------------------------
 * Uneven batches: many circuits of different qubit counts and depths, each
 * with `batch` samples, evaluated (forward + adjoint) in ONE persistent kernel
 * launch, optionally replayed from a captured CUDA graph.  Sec. II-B's batch
 * parallelism extended across circuits.
 * ------------------------------------------------------------------------ */

/* One circuit of an uneven batch (host arrays, copied by qtm_build_multi). */
typedef struct {
    int32_t n_qubits;
    int32_t n_gates;
    const qtm_gate *gates;
    int32_t n_terms;
    int32_t n_obs;
    const qtm_zterm *terms;
    int32_t n_weights;
    int32_t n_inputs;
} qtm_circuit;

typedef struct qtm_multi qtm_multi;

/* Packed buffers of qtm_multi_run: circuit c's block starts at element
 * offsets[c] (from qtm_multi_offsets) of the buffer named by `which`:
 *   QTM_MULTI_X  x       [batch][n_inputs_c]    QTM_MULTI_W  w    [n_weights_c]
 *   QTM_MULTI_GE cotangents [batch][n_obs_c]    QTM_MULTI_E  E    [batch][n_obs_c]
 *   QTM_MULTI_GX grad_x  [batch][n_inputs_c]    QTM_MULTI_GW grad_w [n_weights_c] (batch sum) */
#define QTM_MULTI_X 0
#define QTM_MULTI_W 1
#define QTM_MULTI_GE 2
#define QTM_MULTI_E 3
#define QTM_MULTI_GX 4
#define QTM_MULTI_GW 5

/* Launch configuration chosen by qtm_multi_tune (or set by hand). */
typedef struct {
    int32_t ctas_per_sm;   /* persistent grid = ctas_per_sm x SM count (capped by the work) */
    int32_t order;         /* 0: costliest (circuit, sample) items first; 1: as given */
    int32_t fuse_width;    /* most rotations fused into one run (1 .. 32) */
    int32_t split;         /* 0: one CTA runs a whole item; 1 (default): items of n > 12
                            * qubits are split into one task per (pass, tile), spread over
                            * CTAs; a task waits (bounded) for its item's previous pass */
} qtm_multi_config;

/* Build plans for n_circuits circuits (validated as in qtm_build), batch >= 1
 * samples each.  Host-only until the first run. */
qtm_status qtm_build_multi(const qtm_circuit *circuits, int n_circuits, int batch, int dtype,
                           qtm_multi **out);

/* Element offsets of every circuit's block in a packed buffer: offsets[0..n_circuits],
 * offsets[n_circuits] = total elements. */
qtm_status qtm_multi_offsets(const qtm_multi *multi, int which, int64_t *offsets);

/* Forward + adjoint of every (circuit, sample) in one persistent launch (the
 * fused fast path; qtm_multi_forward and qtm_multi_adjoint below split it): a
 * device work counter hands tasks to CTAs in a fixed list order; circuits with
 * n <= 12 run both directions in shared memory as one task, larger ones sweep
 * tiles of their own states, either inside one CTA (split = 0) or as one task
 * per (pass, tile) that waits, bounded, for the tiles of the item's previous
 * pass (split = 1; every wait is on a task listed earlier, so waits end).
 * Device pointers, plan real type.
 * flags: QTM_MULTI_GRAPH replays a CUDA graph captured on first use for
 * these buffers (re-captured when a pointer changes). */
#define QTM_MULTI_GRAPH 1
qtm_status qtm_multi_run(qtm_multi *multi, const void *x, const void *w, const void *grad_expvals,
                         void *expvals, void *grad_x, void *grad_w, int flags, void *stream);

/*
 * qtm_multi_forward: the expectation values alone (Eq. (qnn) for every
 * circuit's samples, Sec. II-B's batched forward) in one persistent launch:
 * prep, the forward passes of every (circuit, sample), the fixed-order sums
 * into E.  x, w, E: packed device buffers as for qtm_multi_run.  Every item's
 * final state stays in the batch's workspace for one following
 * qtm_multi_adjoint with the same x and w on the same stream (an inference-
 * only caller just never calls it).  flags: QTM_MULTI_GRAPH (a graph of its
 * own, captured on first use for these buffers).
 */
qtm_status qtm_multi_forward(qtm_multi *multi, const void *x, const void *w, void *expvals, int flags,
                             void *stream);

/*
 * qtm_multi_adjoint: the vector-Jacobian product (Sec. II-A adjoint method,
 * per circuit and sample as in Sec. II-B) from the states the last
 * qtm_multi_forward stored: the reverse passes of every (circuit, sample) in
 * one persistent launch, then grad_x [batch][n_inputs_c] and the batch-summed
 * grad_w [n_weights_c] of every circuit (packed, overwritten).  The stored
 * states are consumed.  Returns QTM_ESTATE, before any CUDA call, when no
 * stored forward matches (x, w), or when qtm_multi_run, qtm_multi_tune or a
 * configuration change ran since; with QTM_MULTI_RECOMPUTE the forward is
 * evolved again inside the same launch instead (E is not written) and no
 * stored forward is needed.  flags: QTM_MULTI_GRAPH | QTM_MULTI_RECOMPUTE.
 */
#define QTM_MULTI_RECOMPUTE 2
qtm_status qtm_multi_adjoint(qtm_multi *multi, const void *x, const void *w, const void *grad_expvals,
                             void *grad_x, void *grad_w, int flags, void *stream);

/* Message of the last error recorded on this uneven batch ("" if none);
 * owned by the batch, valid until the next call on it. */
const char *qtm_multi_last_error(const qtm_multi *multi);

/* Autotune the launch configuration on these buffers: time each candidate
 * (CTAs per SM x item order x fusion width x split) with CUDA events and keep the
 * fastest.  cache_path (or NULL): a JSON file of earlier choices keyed by the
 * batch's signature and the device name; a hit skips the timing. */
qtm_status qtm_multi_tune(qtm_multi *multi, const void *x, const void *w, const void *grad_expvals,
                          void *expvals, void *grad_x, void *grad_w, void *stream,
                          const char *cache_path);

/* Synchronise `stream`, then report the persistent kernel's self-checks:
 * QTM_ETIMEOUT if a CTA ran past its 20 s deadline or a task's wait for its
 * item's previous pass gave up after 10 s (the run stops taking work),
 * QTM_EINVAL if an index check failed; the status is cleared after reading. */
qtm_status qtm_multi_sync(qtm_multi *multi, void *stream);

qtm_status qtm_multi_get_config(const qtm_multi *multi, qtm_multi_config *cfg);
qtm_status qtm_multi_set_config(qtm_multi *multi, const qtm_multi_config *cfg);
qtm_status qtm_multi_destroy(qtm_multi *multi);

/* qtm_compile: specialise the plan's pass kernels.  The schedule is fixed
 * once a plan is built, so every register position, table slot, CZ sign
 * pattern, CNOT form and observable sign pattern of each pass is written out
 * as CUDA source, compiled with NVRTC for sm_103a (compiled images are cached
 * on disk under $QTM_JIT_CACHE, default /tmp/qtm_jit_cache) and loaded on the
 * current device; later qtm_forward / qtm_adjoint / qtm_jacobian calls on that
 * device launch them in place of the general pass kernel.  The kernels run one
 * sample per CTA with each complex amplitude one of Blackwell's f32x2
 * register pairs (re, im; paired fma / mul / add); a stretch of phases that
 * repeats one phase program with shifted run slots (a layered circuit's
 * layers) is emitted once, as a loop.  flags: 0 (reserved; other values
 * QTM_EINVAL).  Applies to complex64 fused plans with tiles of >= 9 qubits
 * (QTM_EUNSUPPORTED otherwise, or when NVRTC is unavailable; the plan keeps
 * the general kernels).  Synchronises the device and drops the workspace and
 * any stored forward state. */
qtm_status qtm_compile(qtm_plan *plan, int flags);

/* The schedule of a plan: the planner's and the kernels' choices, which do
 * not change the results beyond rounding (Sec. II-A's computation either way);
 * the knobs of qtm_tune. */
typedef struct {
    int32_t phase_mode;   /* register phases: 0 greedy (the most ready gates per phase), 1 round
                           * robin (the register groups in turn, one run per qubit per phase),
                           * 2 automatic (qtm_set_schedule only: round robin where most of the
                           * work then repeats phase after phase, else greedy) */
    int32_t tile_qubits;  /* qubits per shared-memory tile of a state that spans several tiles
                           * (9 .. 12 complex64, 9 .. 11 complex128; 0 = the largest); a state
                           * that fits one tile is always one tile (qtm_get_schedule reports its
                           * width, and qtm_set_schedule ignores the field for it) */
    int32_t low_min;      /* narrowest low block of a tile (4 .. tile_qubits): rows of 2^low_min
                           * contiguous amplitudes in memory */
    int32_t kernels;      /* 0 the general pass kernel, 1 the specialised kernels (qtm_compile) */
    int32_t minb_fwd;     /* CTAs per SM the specialised forward / reverse kernels' registers are */
    int32_t minb_rev;     /*   budgeted for (1 .. 4) */
} qtm_schedule;

/* Current schedule of a fused plan (host only). */
qtm_status qtm_get_schedule(const qtm_plan *plan, qtm_schedule *sched);

/* Re-plan a fused plan with `sched` and load its kernels (NVRTC compile for
 * kernels = 1).  Where the specialised kernels do not apply (complex128, a
 * tile below 9 qubits, no NVRTC) it returns QTM_EUNSUPPORTED and the plan
 * keeps its old schedule, on the general kernel.  Synchronises the device
 * and drops the workspace and any stored forward state.  Composite (grouped
 * Pauli) and naive-path plans: QTM_EUNSUPPORTED. */
qtm_status qtm_set_schedule(qtm_plan *plan, const qtm_schedule *sched);

/* qtm_tune: choose the schedule of a fused plan for batches of B samples by
 * timing forward + adjoint (CUDA events on `stream`, median of 5 after 2
 * warm-up steps) over candidate schedules, one knob at a time from the
 * current one (phase grouping; tile width and low-block width of multi-tile
 * states; specialised or general kernels and the specialised kernels'
 * register budgets), keeping a change only when it is at least 1 % faster;
 * the fastest is applied.  x [B][n_inputs], w, grad_expvals [B][n_obs]: device
 * inputs of the plan's real type (read only); the outputs go to scratch the
 * call allocates and frees.  cache_path (or NULL): a JSON-lines file of
 * earlier choices keyed by the circuit, observables, dtype, B and the device
 * name; a hit applies the stored schedule without timing, a miss appends the
 * choice.  Synchronises the device. */
qtm_status qtm_tune(qtm_plan *plan, int B, const void *x, const void *w, const void *grad_expvals, void *stream,
                    const char *cache_path);

/* Number of specialised pass kernels loaded for the current device (0 before
 * qtm_compile, or on another device). */
int qtm_compiled_passes(const qtm_plan *plan);

/* Synchronise `stream`, then report (and clear) any status a kernel of this
 * plan recorded on the device: QTM_ETIMEOUT if a bounded wait gave up. */
qtm_status qtm_sync(qtm_plan *plan, void *stream);

/* Schedule summary of a plan (host-side). */
qtm_status qtm_get_plan_info(const qtm_plan *plan, qtm_plan_info *info);

/* Release the plan and its device memory (synchronises the device first). */
qtm_status qtm_destroy(qtm_plan *plan);

/* Message of the last error recorded on this plan ("" if none).  Owned by
 * the plan; valid until the next call on it. */
const char *qtm_last_error(const qtm_plan *plan);

/* Static string for a status code. */
const char *qtm_status_str(int status);

/* Library version, e.g. "qtm 0.1 sm_103a". */
const char *qtm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QTM_H */
