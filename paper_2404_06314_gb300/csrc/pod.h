// Plain-data types shared by the host planner, the kernels and the kernels
// generated at run time (NVRTC): no host headers when compiled by NVRTC.
#pragma once

#ifdef __CUDACC_RTC__
typedef int int32_t;
typedef unsigned int uint32_t;
typedef short int16_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
enum { QTM_RX = 0, QTM_RY = 1, QTM_RZ = 2, QTM_CZ = 3, QTM_CNOT = 4 };
#else
#include <stdint.h>
#include "../../include/qtm.h"
#endif

namespace qtm {

// Tile geometry ------------------------------------------------------------
// A pass streams the state through shared memory in tiles of 2^K amplitudes.
// The tile's qubits are S = {0 .. l-1} U {h .. h+m-1} (K = l + m, l >= 4): the
// low block keeps global memory access contiguous, the high block reaches the
// qubits above.  Tile-local bit i < l is global qubit i; tile-local bit l + j
// is global qubit h + j.  Each thread holds 16 amplitudes in registers: the 4
// tile-local bits [lo, lo + 4) of its current "register group".

constexpr int kRegBits = 4;
constexpr int kRegs = 16;
constexpr int kMaxTileQubits = 12;   // complex64 tiles (32 KiB)
constexpr int kMaxTileQubits128 = 11;
constexpr int kMaxQubits = 30;
constexpr int kMaxRunLen = 32;       // rotations fused into one 2x2
constexpr int kMaxMaskTerms = 8;     // closed-form analytic state: max mask terms

enum OpType : int32_t {
    OP_U2 = 1,       // apply fused run matrix (forward)                 a = local bit, slot
    OP_GRAD = 2,     // v += Im<lam|sigma phi>, then apply U^dagger      a = local bit, slot, flags
    OP_CZ = 3,       // a, b operands
    OP_CNOT = 4,     // a = control operand, b = target (local bit)
    OP_EXPVAL = 5,   // accumulate <O_m> partials
    OP_COSTATE = 6,  // lam = (sum_m gE_m O_m) phi
    OP_DIAG = 7,     // product of CZ gates (diag_pairs[a .. a+b)): one sign mask
};
constexpr int32_t OPF_SKIP_APPLY = 1;   // GRAD: no later op touches this qubit
constexpr int32_t OPF_ACCUMULATE = 2;   // COSTATE: add to the lam already in memory (its X/Y part)

// Operand encoding: 0..31 = tile-local bit; kFixed + Q = global qubit Q that is
// constant within the tile (outside S).
constexpr int32_t kFixed = 32;

struct DevOp {
    int16_t type;
    int16_t flags;
    int16_t a;
    int16_t b;
    int32_t slot;   // pass-local run slot (U2 / GRAD)
    int32_t pad;
};
static_assert(sizeof(DevOp) == 16, "DevOp layout");

struct DiagPair {   // one CZ of a DIAG op (operand encoding as DevOp::a/b)
    int16_t a, b;
};

// Analytic prefix state in closed form: with x = A^{-1} y evaluated as
// XOR over linear terms (d, m) of shift(y, d) & m (shift right by d >= 0, left
// by -d), the folded CZ/CNOT prefix contributes the sign
// (-1)^{popcount(x & dlin) + sum over quadratic terms (d, m) of popcount(x & (x >> d) & m)}.
struct MaskTerm {
    int32_t d;
    uint32_t mask;
};

struct DevPhase {
    int32_t lo;        // register group: tile-local bits [lo, lo + 4)
    int32_t op_begin;  // into the plan's op array
    int32_t op_end;
    int32_t flags;     // PHF_*
};
// The phase's ops leave phi and lam as they are (gradients of runs' last
// reverse ops, whose undo is skipped, and expectation values): it need not
// store them back to shared memory.
constexpr int32_t PHF_KEEPS_STATE = 1;

enum Src : int32_t { SRC_NONE = 0, SRC_LOAD = 1, SRC_ANALYTIC = 2, SRC_COSTATE = 3 };

struct PassDesc {
    int32_t K, l, h, m;         // tile geometry
    int32_t phi_src;            // SRC_LOAD / SRC_ANALYTIC
    int32_t lam_src;            // reverse only: SRC_COSTATE (first pass) / SRC_LOAD
    int32_t analytic_ents;      // prefix entanglers still applied to the analytic phi
    int32_t ents_begin;         // ... listed (circuit order) at plan.pass_ents[ents_begin ..)
    int32_t store_phi, store_lam;
    int32_t phase_begin, phase_end;
    int32_t slot_begin, slot_end;   // pass-local run slots -> run ids (plan.slot_runs)
    int32_t has_expval, has_grad;
    int32_t reverse;
    // closed form of the analytic phi (used when amap_lin >= 0)
    int32_t amap_begin, amap_lin, amap_quad;   // terms [begin, begin+lin) linear, then quad
    uint32_t amap_dlin;
};

// A run: consecutive rotations on one qubit (forward order).
struct Run {
    int32_t q;
    int32_t rot_begin, rot_end;   // into the rotation arrays
    int32_t prefix;               // 1 if folded into the analytic init
};

// A rotation (one gate of the circuit).
struct Rot {
    int32_t kind;    // QTM_RX / RY / RZ
    int32_t gate;    // index in the circuit's gate list
    int32_t w_idx, x_idx;
    double coef;
};

struct Ent {        // CZ / CNOT
    int32_t kind, a, b, gate;
};

struct Term {
    uint64_t zmask;
    double coef;
    int32_t obs;
    int32_t pad;
};

// Pauli string with X or Y factors, evaluated on the final state outside the
// pass kernels: P|x> = i^ny (-1)^popcount(x & zmask) |x ^ xmask>, with Y where
// both masks have the qubit (ny of them), X where only xmask has it.
struct PauliTerm {
    uint64_t xmask, zmask;
    double coef;
    int32_t obs, ny;
};

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define QTM_POD_HD __host__ __device__ inline
#else
#define QTM_POD_HD inline
#endif

// status word bits recorded by kernels
constexpr unsigned kStatusTimeout = 1u;

// Kernel parameters of one pass over the state (k_pass and the generated kernels).
struct PassArgs {
    // geometry
    int K, l, h, m;
    int state_qubits, n;
    int tiles, log_tiles;
    int B;
    int rank;                     // tensor-map rank of this pass
    int low_dims, gap_dim, high_dims;   // dims per segment (for coordinates)
    // program
    const DevOp *ops;
    const DiagPair *diag;
    const DevPhase *phases;
    int phase_begin, phase_end;
    const int32_t *slot_runs;
    int slot_begin, nslots;
    int n_runs;
    const void *mats;             // [B][n_runs][4] fused run matrices U (plan complex type)
    const void *tabs;             // [B][ntab][16] product-state tables (plan complex type)
    // analytic init
    const Ent *prefix_ents;
    int analytic_ents;
    const MaskTerm *amap;         // closed form of the analytic state (amap_lin >= 0)
    int amap_lin, amap_quad;
    uint32_t amap_dlin;
    // sources / sinks
    int phi_src, lam_src, store_phi, store_lam, has_expval;
    // observables
    const Term *terms;
    int n_terms, M;
    // data (plan real type)
    const void *x, *w, *gE;
    int n_in;
    double *Epart;                // [B][tiles][M]
    double *Gpart;                // [B][n_runs][tiles][3]
    unsigned *status;
    int smem_bytes;
    // Per-sample steps fused into the pass (plans of one tile per sample,
    // where a CTA holds a whole sample): prep_fused, the first forward pass
    // also computes its sample's run matrices, product-state tables and half
    // angles (mats, tabs, cs; as k_prep); finalize_fused, the last reverse
    // pass also turns its sample's run sums into angle gradients and applies
    // the chain rule (abar, gx, gw_out / gw_ws; as k_grad_finalize).
    int prep_fused, finalize_fused;
    const Run *runs;
    const Rot *rots;
    const int32_t *prq;           // prefix run of each qubit (-1: none)
    void *cs;                     // [B][n_rots] (cos, sin) of half angles, FP64 pairs (may be null)
    int n_rots, n_weights;
    const int32_t *w_ptr, *w_rots, *x_ptr, *x_rots;
    double *abar;                 // [B][n_rots]
    void *gx, *gw_out;            // [B][n_in], [B][n_weights] plan real type (may be null)
    double *gw_ws;                // [B][n_weights] (may be null)
    // Plans of one tile per sample: the forward pass that measures also writes
    // the expectation values [B][M] (plan real type) here, so no separate
    // finalize runs; null otherwise.
    void *E_out;
    // Fused prep of complex64 plans (may be null): rot_rep[i] is the first
    // rotation with rotation i's coefficient, weight and input (the same angle
    // for every sample), and cs_shared[rot_rep[i]] the FP64 (cos, sin) of the
    // half angle of a rotation without an input, computed once per call.
    const int32_t *rot_rep;
    const void *cs_shared;
};

}  // namespace qtm
