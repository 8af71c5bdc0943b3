// Internal plan representation shared by the host planner, the host-side
// schedule interpreter and the CUDA launch code.  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qtm.h"
#include "pod.h"

namespace qtm {

// How a pass's ops are grouped into register phases (see plan.cpp);
// PHASES_AUTO plans round robin and keeps it when at least half of the ops
// lie in periodic stretches of phases (periodic_fraction), else greedy;
// complex128 plans (interpreter kernels only) always get greedy.
enum { PHASES_GREEDY = 0, PHASES_ROUND_ROBIN = 1, PHASES_AUTO = 2 };

// Schedule choices of the planner (the autotuner's knobs).
struct PlanOptions {
    int max_run = kMaxRunLen;          // most rotations fused into one run (fusion width)
    int phase_mode = PHASES_GREEDY;    // PHASES_GREEDY, PHASES_ROUND_ROBIN or PHASES_AUTO
    int tile_qubits = 0;               // K of plans whose state spans several tiles (0: the largest)
    int low_min = kRegBits;            // narrowest low block l of a tile (contiguous 2^l-amplitude rows)
};

struct Plan {
    // circuit
    int n = 0, dtype = QTM_C64, path = QTM_PATH_FUSED;
    int phase_mode = PHASES_GREEDY;    // resolved (never PHASES_AUTO)
    int low_min = kRegBits;
    int n_obs = 0, n_weights = 0, n_inputs = 0;
    std::vector<qtm_gate> gates;        // lowered to RX/RY/RZ/CZ/CNOT (H and RZZ expanded)
    int n_user_gates = 0;               // gates as given to qtm_build (Jacobian columns)
    std::vector<Term> terms;            // sorted by obs
    std::vector<PauliTerm> pterms;      // terms with X/Y factors (fused plans of qtm_build_pauli)

    // runs and rotations
    std::vector<Run> runs;
    std::vector<Rot> rots;
    std::vector<int32_t> prefix_run_of_q;   // [n] run id or -1
    std::vector<Ent> prefix_ents;           // folded CZ/CNOT, in circuit order
    // per analytic pass, the folded entanglers still applied (circuit order):
    // [0, |prefix_ents|) is the forward's full list; reverse prefix passes append
    // the subset not yet undone (undone ones may leave out of list order when
    // they commute, so a pass's subset is not a list prefix in general)
    std::vector<Ent> pass_ents;
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
qtm_status make_plan(int n, const qtm_gate *gates, int n_gates, const qtm_zterm *terms,
                     int n_terms, int n_obs, int n_weights, int n_inputs, int dtype, int path,
                     Plan &out, std::string &err, const PlanOptions &opt = PlanOptions());

// Fraction of a plan's phase ops that lie in periodic stretches of its
// passes' phases (the same phase program repeated with shifted run slots),
// which the specialised kernels emit as loops.
double periodic_fraction(const Plan &P);

// Give a fused plan observables with X/Y factors: the last forward pass keeps
// the final state in memory, where the X/Y terms' expectation values and
// their part of the costate are evaluated, and the first reverse pass loads
// that costate part and adds the Z part to it.
void attach_pauli_terms(Plan &P, const std::vector<PauliTerm> &terms);

// Per-sample cost model of a plan (bytes over the state, arithmetic).
void plan_costs(const Plan &p, double &fwd_bytes, double &adj_bytes, double &fwd_flops,
                double &adj_flops);

inline int elem_bytes(int dtype) { return dtype == QTM_C128 ? 16 : 8; }

}  // namespace qtm
