// Internal plan representation shared by the host planner, the host-side
// schedule interpreter and the CUDA launch code.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qtm.h"

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
    int32_t pad;
};

enum Src : int32_t { SRC_NONE = 0, SRC_LOAD = 1, SRC_ANALYTIC = 2, SRC_COSTATE = 3 };

struct PassDesc {
    int32_t K, l, h, m;         // tile geometry
    int32_t phi_src;            // SRC_LOAD / SRC_ANALYTIC
    int32_t lam_src;            // reverse only: SRC_COSTATE (first pass) / SRC_LOAD
    int32_t analytic_ents;      // prefix entanglers still applied to the analytic phi
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

struct Plan {
    // circuit
    int n = 0, dtype = QTM_C64, path = QTM_PATH_FUSED;
    int n_obs = 0, n_weights = 0, n_inputs = 0;
    std::vector<qtm_gate> gates;
    std::vector<Term> terms;            // sorted by obs

    // runs and rotations
    std::vector<Run> runs;
    std::vector<Rot> rots;
    std::vector<int32_t> prefix_run_of_q;   // [n] run id or -1
    std::vector<Ent> prefix_ents;           // folded CZ/CNOT, in circuit order
    std::vector<int32_t> rot_of_gate;       // [G] rotation id or -1

    // chain rule: CSR over weights and inputs -> rotation ids
    std::vector<int32_t> w_ptr, w_rots, x_ptr, x_rots;

    // schedule
    int K = 0;                 // tile qubits
    int state_qubits = 0;      // max(n, 4): per-sample stride is 2^state_qubits
    int tiles_per_sample = 1;
    std::vector<PassDesc> fwd, rev;
    std::vector<DevPhase> phases;
    std::vector<DevOp> ops;
    std::vector<DiagPair> diag_pairs;
    std::vector<MaskTerm> amap_terms;
    std::vector<int32_t> slot_runs;

    int max_slots = 0;         // max run slots of any pass
    int max_phases = 0;

    std::string describe() const;
};

// Build the plan (host only).  Returns QTM_OK or an error with `err` set.
// max_run: most rotations fused into one run (the fusion width).
qtm_status make_plan(int n, const qtm_gate *gates, int n_gates, const qtm_zterm *terms,
                     int n_terms, int n_obs, int n_weights, int n_inputs, int dtype, int path,
                     Plan &out, std::string &err, int max_run = kMaxRunLen);

// Per-sample cost model of a plan (bytes over the state, arithmetic).
void plan_costs(const Plan &p, double &fwd_bytes, double &adj_bytes, double &fwd_flops,
                double &adj_flops);

inline int elem_bytes(int dtype) { return dtype == QTM_C128 ? 16 : 8; }

}  // namespace qtm
