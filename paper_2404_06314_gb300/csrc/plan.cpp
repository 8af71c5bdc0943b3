// Host-side circuit planner.
//
// Turns a gate list into the schedule the CUDA kernels execute:
//   1. Prefix folding.  Every qubit starts in |0>; the leading single-qubit
//      rotations of each qubit make a product state, and CZ/CNOT gates that
//      act only on such untouched product qubits permute/sign its amplitudes.
//      That prefix is evaluated analytically (psi[y] = sign * prod_q u_q[x_q]
//      with x = y pushed back through the folded entanglers), so the first
//      layer costs no pass over the state.
//   2. Runs.  Consecutive rotations on one qubit fuse into one 2x2 matrix
//      forward, and into one 3-component inner product Im<lam|sigma phi>
//      backward (the gradients of the run's rotations follow from it by SO(3)
//      rotations, see the finalize kernel).
//   3. Passes.  n <= K: one pass holds the whole state in shared memory.
//      n > K: greedy sweeps, each over a tile qubit set S = {0..l-1} U
//      {h..h+m-1} chosen to execute the most ready gates; CZ gates and the
//      control of a CNOT may lie outside S (they are constant per tile).
//   4. Phases.  Inside a pass each thread keeps 16 amplitudes in registers
//      (4 tile bits); a phase is a greedy maximal set of ready gates local to
//      one 4-bit register group.  Two rules pick the group: the group whose
//      set holds the most gates (PHASES_GREEDY), or the groups in turn with
//      at most one run per qubit in a phase (PHASES_ROUND_ROBIN), which gives
//      a layered circuit the same few phase programs layer after layer.
// The reverse (adjoint) schedule runs the same greedy on the reversed gate
// DAG, then on the folded prefix, whose state is again analytic.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <queue>
#include <sstream>

namespace qtm {

namespace {

bool is_rot(int k) { return k == QTM_RX || k == QTM_RY || k == QTM_RZ; }
constexpr double kPi = 3.14159265358979323846264338327950288;

struct Node {
    int type;      // 0 = run, 1 = entangler
    int run;       // run id (type 0)
    Ent ent;       // (type 1)
    bool prefix;
    std::vector<int> preds;
    int q0() const { return type == 0 ? -1 : ent.a; }
};

struct Seq {
    std::vector<Node> nodes;
};

// qubits touched by a node
inline void touched(const Node &nd, const std::vector<Run> &runs, int &a, int &b)
{
    if (nd.type == 0) { a = runs[nd.run].q; b = -1; }
    else { a = nd.ent.a; b = nd.ent.b; }
}

// Dependencies in circuit order.  CZ gates are diagonal and commute with one
// another, so a CZ waits only for the last run or CNOT on each of its qubits,
// and a run or CNOT waits for every CZ on its qubits since then; a CZ ring
// therefore does not chain around the qubits, and a register group can apply
// its part of a ring as soon as its neighbours' runs are done.
void build_deps(std::vector<Node> &nodes, const std::vector<Run> &runs, int n)
{
    std::vector<int> last(n, -1);                  // last run / CNOT on the qubit
    std::vector<std::vector<int>> diag(n);         // CZs on the qubit since then
    auto add = [](std::vector<int> &v, int x) {
        if (x >= 0 && std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
    };
    for (int i = 0; i < (int)nodes.size(); ++i) {
        int a, b;
        touched(nodes[i], runs, a, b);
        std::vector<int> &pr = nodes[i].preds;
        pr.clear();
        const bool cz = nodes[i].type == 1 && nodes[i].ent.kind == QTM_CZ;
        for (int q : {a, b}) {
            if (q < 0) continue;
            add(pr, last[q]);
            if (!cz)
                for (int d : diag[q]) add(pr, d);
        }
        for (int q : {a, b}) {
            if (q < 0) continue;
            if (cz) {
                diag[q].push_back(i);
            } else {
                last[q] = i;
                diag[q].clear();
            }
        }
    }
}

struct TileSet {
    int l, h, m;   // S = [0, l) U [h, h + m)
    bool has(int q) const { return q < l || (m > 0 && q >= h && q < h + m); }
    int local(int q) const { return q < l ? q : l + (q - h); }
};

// Can node run in tile S, register group [lo, lo+4) (lo < 0: any group)?
bool executable(const Node &nd, const std::vector<Run> &runs, const TileSet &S, int lo)
{
    if (nd.type == 0) {
        int q = runs[nd.run].q;
        if (!S.has(q)) return false;
        if (lo < 0) return true;
        int p = S.local(q);
        return p >= lo && p < lo + kRegBits;
    }
    if (nd.ent.kind == QTM_CZ) return true;   // diagonal: any layout
    int t = nd.ent.b;                          // CNOT target must be in registers
    if (!S.has(t)) return false;
    if (lo < 0) return true;
    int p = S.local(t);
    return p >= lo && p < lo + kRegBits;
}

double node_weight(const Node &nd)
{
    if (nd.type == 0) return 1.0;
    return nd.ent.kind == QTM_CNOT ? 1.0 : 0.01;
}

// Closure of ready nodes executable under (S, lo) among the nodes with
// member[i] true and done[i] false.  Returns them in execution order.
// one_run_per_qubit: a qubit's second run waits for the next phase.
std::vector<int> closure(const std::vector<Node> &nodes, const std::vector<Run> &runs,
                         const std::vector<char> &member, const std::vector<char> &done,
                         const TileSet &S, int lo, double *weight, bool one_run_per_qubit = false)
{
    const int N = (int)nodes.size();
    std::vector<char> d(done);
    std::vector<char> ran(one_run_per_qubit ? kMaxQubits : 0, 0);
    std::vector<int> order;
    double w = 0.0;
    // simple fixed-point sweep in index order (nodes are topologically sorted)
    bool progress = true;
    while (progress) {
        progress = false;
        for (int i = 0; i < N; ++i) {
            if (!member[i] || d[i]) continue;
            bool ready = true;
            for (int p : nodes[i].preds)
                if (!d[p]) { ready = false; break; }
            if (!ready) continue;
            if (!executable(nodes[i], runs, S, lo)) continue;
            if (one_run_per_qubit && nodes[i].type == 0) {
                const int q = runs[nodes[i].run].q;
                if (ran[q]) continue;
                ran[q] = 1;
            }
            d[i] = 1;
            order.push_back(i);
            w += node_weight(nodes[i]);
            progress = true;
        }
    }
    if (weight) *weight = w;
    return order;
}

struct Builder {
    Plan &P;
    explicit Builder(Plan &p) : P(p) {}

    int operand(const TileSet &S, int q) const { return S.has(q) ? S.local(q) : kFixed + q; }

    // Emit the phases and ops of one pass over `pass_nodes` (execution order
    // from the sweep closure).  Returns the PassDesc with phases/slots filled.
    PassDesc emit_pass(const std::vector<Node> &nodes, const std::vector<int> &pass_nodes,
                       const TileSet &S, int K, bool reverse, const std::vector<int> &last_touch)
    {
        PassDesc pd{};
        pd.K = K; pd.l = S.l; pd.h = S.h; pd.m = S.m;
        pd.reverse = reverse ? 1 : 0;
        pd.phase_begin = (int)P.phases.size();
        pd.slot_begin = (int)P.slot_runs.size();

        const int N = (int)nodes.size();
        std::vector<char> member(N, 0), done(N, 0);
        for (int i : pass_nodes) member[i] = 1;
        // nodes not in this pass: treat as done if they precede it (they were
        // scheduled earlier); nodes after it are never preds of pass members.
        for (int i = 0; i < N; ++i)
            if (!member[i]) done[i] = 1;

        std::vector<int> slot_of_run;
        auto slot = [&](int run) {
            if ((int)slot_of_run.size() <= run) slot_of_run.resize(run + 1, -1);
            if (slot_of_run[run] < 0) {
                slot_of_run[run] = (int)P.slot_runs.size() - pd.slot_begin;
                P.slot_runs.push_back(run);
            }
            return slot_of_run[run];
        };

        const int ngroups = (K + kRegBits - 1) / kRegBits;
        const bool rr = P.phase_mode == PHASES_ROUND_ROBIN;
        int remaining = (int)pass_nodes.size();
        int last_lo = -1, last_g = -1;
        while (remaining > 0) {
            int best_lo = -1, best_g = -1;
            double best_w = -1.0;
            std::vector<int> best;
            if (rr) {
                // the groups in turn, skipping a group with nothing ready
                for (int k = 1; k <= ngroups && best.empty(); ++k) {
                    const int g = (last_g + k) % ngroups;
                    const int lo = std::min(g * kRegBits, K - kRegBits);
                    std::vector<int> c = closure(nodes, P.runs, member, done, S, lo, nullptr, true);
                    if (!c.empty()) { best_g = g; best_lo = lo; best = std::move(c); }
                }
            } else {
                for (int g = 0; g < ngroups; ++g) {
                    int lo = std::min(g * kRegBits, K - kRegBits);
                    double w;
                    std::vector<int> c = closure(nodes, P.runs, member, done, S, lo, &w);
                    // prefer staying in the current group on ties (no smem round trip saved,
                    // but keeps phases fewer)
                    if (w > best_w + 1e-9 || (std::fabs(w - best_w) <= 1e-9 && lo == last_lo)) {
                        best_w = w; best_lo = lo; best_g = g; best = std::move(c);
                    }
                }
            }
            if (best.empty()) break;   // cannot happen for a valid DAG
            DevPhase ph{};
            ph.lo = best_lo;
            ph.op_begin = (int)P.ops.size();
            for (int i : best) {
                const Node &nd = nodes[i];
                DevOp op{};
                if (nd.type == 0) {
                    const Run &r = P.runs[nd.run];
                    op.type = reverse ? OP_GRAD : OP_U2;
                    op.a = S.local(r.q);
                    op.b = -1;
                    op.slot = slot(nd.run);
                    if (reverse && last_touch[r.q] == i) op.flags |= OPF_SKIP_APPLY;
                } else if (nd.ent.kind == QTM_CZ) {
                    op.type = OP_CZ;
                    op.a = operand(S, nd.ent.a);
                    op.b = operand(S, nd.ent.b);
                    op.slot = -1;
                } else {
                    op.type = OP_CNOT;
                    op.a = operand(S, nd.ent.a);
                    op.b = S.local(nd.ent.b);
                    op.slot = -1;
                }
                P.ops.push_back(op);
                done[i] = 1;
                --remaining;
            }
            ph.op_end = (int)P.ops.size();
            P.phases.push_back(ph);
            last_lo = best_lo;
            last_g = best_g;
        }
        if (P.phases.size() == (size_t)pd.phase_begin) {   // empty pass: one empty phase
            DevPhase ph{};
            ph.lo = 0;
            ph.op_begin = ph.op_end = (int)P.ops.size();
            P.phases.push_back(ph);
        }
        pd.phase_end = (int)P.phases.size();
        pd.slot_end = (int)P.slot_runs.size();
        return pd;
    }

    // Greedy sweep selection over the nodes [begin, end) of `nodes` not done.
    // pass_nodes (optional) receives each emitted pass's node list.
    void schedule_stage(const std::vector<Node> &nodes, int begin, int end, int K, bool reverse,
                        const std::vector<int> &last_touch, std::vector<PassDesc> &out,
                        std::vector<std::vector<int>> *pass_nodes = nullptr)
    {
        const int N = (int)nodes.size();
        const int n = P.n;
        std::vector<char> member(N, 0), done(N, 1);
        for (int i = begin; i < end; ++i) { member[i] = 1; done[i] = 0; }
        int remaining = end - begin;
        if (n <= K) {
            // whole state in one tile
            TileSet S{K, K, 0};
            std::vector<int> all;
            for (int i = begin; i < end; ++i) all.push_back(i);
            if (!all.empty() || out.empty()) {
                // emit in a topological order that the phase greedy will refine
                out.push_back(emit_pass(nodes, all, S, K, reverse, last_touch));
                if (pass_nodes) pass_nodes->push_back(all);
            }
            return;
        }
        // candidate tile sets
        std::vector<TileSet> cands;
        for (int l = std::max(kRegBits, P.low_min); l <= K; ++l) {
            int m = K - l;
            if (m == 0) { cands.push_back({l, l, 0}); continue; }
            for (int h = l; h + m <= n; ++h) cands.push_back({l, h, m});
        }
        while (remaining > 0) {
            double best_w = -1.0;
            TileSet bestS{K, K, 0};
            std::vector<int> best;
            for (const TileSet &S : cands) {
                double w;
                std::vector<int> c = closure(nodes, P.runs, member, done, S, -1, &w);
                if (w > best_w + 1e-9) { best_w = w; bestS = S; best = std::move(c); }
            }
            if (best.empty()) break;
            out.push_back(emit_pass(nodes, best, bestS, K, reverse, last_touch));
            if (pass_nodes) pass_nodes->push_back(best);
            for (int i : best) done[i] = 1;
            remaining -= (int)best.size();
        }
    }
};

// Closed form of the first `e` folded entanglers acting on basis states:
// y = A x, phase (-1)^{x^T Q x + D.x}.  Returns false if the mask form would
// cost more bit operations per amplitude than undoing the gates one by one.
bool closed_form(const std::vector<Ent> &ents, int e, int n, std::vector<MaskTerm> &terms,
                 int &n_lin, int &n_quad, uint32_t &dlin)
{
    std::vector<uint32_t> row(n);
    for (int i = 0; i < n; ++i) row[i] = 1u << i;
    std::vector<uint32_t> Q(n, 0u);   // Q[i] bit j (j > i): x_i x_j term
    uint32_t D = 0;
    for (int k = 0; k < e; ++k) {
        const Ent &g = ents[k];
        if (g.kind == QTM_CNOT) {
            row[g.b] ^= row[g.a];
        } else {
            const uint32_t ra = row[g.a], rb = row[g.b];
            D ^= ra & rb;
            for (int i = 0; i < n; ++i)
                for (int j = i + 1; j < n; ++j) {
                    const uint32_t t = (((ra >> i) & (rb >> j)) ^ ((ra >> j) & (rb >> i))) & 1u;
                    Q[i] ^= t << j;
                }
        }
    }
    // invert A (rows) over GF(2): augmented 64-bit rows [A | I]
    std::vector<uint64_t> aug(n);
    for (int i = 0; i < n; ++i) aug[i] = (uint64_t)row[i] | ((uint64_t)1 << (32 + i));
    for (int col = 0; col < n; ++col) {
        int piv = -1;
        for (int r = col; r < n; ++r)
            if ((aug[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) return false;   // cannot happen: CNOT products are invertible
        std::swap(aug[col], aug[piv]);
        for (int r = 0; r < n; ++r)
            if (r != col && ((aug[r] >> col) & 1)) aug[r] ^= aug[col];
    }
    // A^{-1}[i][j] = bit (32 + j) of aug[i]
    terms.clear();
    n_lin = 0;
    for (int d = -(n - 1); d <= n - 1; ++d) {
        uint32_t m = 0;
        for (int i = 0; i < n; ++i) {
            const int j = i + d;
            if (j < 0 || j >= n) continue;
            if ((aug[i] >> (32 + j)) & 1) m |= 1u << i;
        }
        if (m) { terms.push_back({d, m}); ++n_lin; }
    }
    n_quad = 0;
    for (int d = 1; d <= n - 1; ++d) {
        uint32_t m = 0;
        for (int i = 0; i + d < n; ++i)
            if ((Q[i] >> (i + d)) & 1) m |= 1u << i;
        if (m) { terms.push_back({d, m}); ++n_quad; }
    }
    dlin = D;
    return n_lin + n_quad <= kMaxMaskTerms && 3 * (n_lin + n_quad) + 2 <= 4 * e;
}

}  // namespace

namespace {

qtm_status make_plan_mode(int n, const qtm_gate *gates, int n_gates, const qtm_zterm *terms,
                          int n_terms, int n_obs, int n_weights, int n_inputs, int dtype, int path,
                          Plan &P, std::string &err, const PlanOptions &opt, int phase_mode)
{
    const int max_run = std::min(std::max(opt.max_run, 1), kMaxRunLen);
    auto bad = [&](const std::string &m) { err = m; return QTM_EINVAL; };
    if (n < 1 || n > kMaxQubits) return bad("n_qubits out of range 1..30");
    if (n_gates < 0 || (n_gates > 0 && !gates)) return bad("bad gate array");
    if (n_terms < 0 || (n_terms > 0 && !terms)) return bad("bad term array");
    if (n_obs < 1) return bad("n_obs must be >= 1");
    if (n_weights < 0 || n_inputs < 0) return bad("negative n_weights / n_inputs");
    if (dtype != QTM_C64 && dtype != QTM_C128) return bad("unknown dtype");
    if (path != QTM_PATH_AUTO && path != QTM_PATH_FUSED && path != QTM_PATH_NAIVE)
        return bad("unknown path");
    for (int g = 0; g < n_gates; ++g) {
        const qtm_gate &G = gates[g];
        std::ostringstream s;
        s << "gate " << g << ": ";
        if (G.reserved != 0) return bad(s.str() + "reserved field must be 0");
        if (!std::isfinite(G.coef)) return bad(s.str() + "coef not finite");
        if (is_rot(G.kind)) {
            if (G.q0 < 0 || G.q0 >= n) return bad(s.str() + "qubit out of range");
            if (G.q1 != -1) return bad(s.str() + "rotation must have q1 = -1");
            if (G.w_idx < -1 || G.w_idx >= n_weights) return bad(s.str() + "w_idx out of range");
            if (G.x_idx < -1 || G.x_idx >= n_inputs) return bad(s.str() + "x_idx out of range");
        } else if (G.kind == QTM_CZ || G.kind == QTM_CNOT) {
            if (G.q0 < 0 || G.q0 >= n || G.q1 < 0 || G.q1 >= n) return bad(s.str() + "qubit out of range");
            if (G.q0 == G.q1) return bad(s.str() + "two-qubit gate on one qubit");
            if (G.w_idx != -1 || G.x_idx != -1) return bad(s.str() + "CZ/CNOT take no parameters");
        } else if (G.kind == QTM_HADAMARD) {
            if (G.q0 < 0 || G.q0 >= n) return bad(s.str() + "qubit out of range");
            if (G.q1 != -1) return bad(s.str() + "H must have q1 = -1");
            if (G.w_idx != -1 || G.x_idx != -1) return bad(s.str() + "H takes no parameters");
        } else if (G.kind == QTM_RZZ) {
            if (G.q0 < 0 || G.q0 >= n || G.q1 < 0 || G.q1 >= n) return bad(s.str() + "qubit out of range");
            if (G.q0 == G.q1) return bad(s.str() + "two-qubit gate on one qubit");
            if (G.w_idx < -1 || G.w_idx >= n_weights) return bad(s.str() + "w_idx out of range");
            if (G.x_idx < -1 || G.x_idx >= n_inputs) return bad(s.str() + "x_idx out of range");
        } else {
            return bad(s.str() + "unknown gate kind");
        }
    }
    for (int t = 0; t < n_terms; ++t) {
        const qtm_zterm &T = terms[t];
        std::ostringstream s;
        s << "term " << t << ": ";
        if (T.reserved != 0) return bad(s.str() + "reserved field must be 0");
        if (n < 64 && (T.zmask >> n) != 0) return bad(s.str() + "zmask has bits >= n");
        if (T.obs < 0 || T.obs >= n_obs) return bad(s.str() + "obs out of range");
        if (!std::isfinite(T.coef)) return bad(s.str() + "coef not finite");
    }

    P = Plan();
    P.phase_mode = phase_mode == PHASES_ROUND_ROBIN ? PHASES_ROUND_ROBIN : PHASES_GREEDY;
    P.low_min = std::min(std::max(opt.low_min, kRegBits), kMaxTileQubits);
    P.n = n; P.dtype = dtype; P.n_obs = n_obs; P.n_weights = n_weights; P.n_inputs = n_inputs;
    P.path = (path == QTM_PATH_NAIVE) ? QTM_PATH_NAIVE : QTM_PATH_FUSED;
    P.n_user_gates = n_gates;

    // ---- 0. lower H and RZZ to the native gate set -------------------------
    // H = RX(pi) RY(pi/2) up to the global phase -i (no expectation value or
    // gradient sees a global phase); RZZ(t) = CNOT(q0 -> q1) RZ_q1(t) CNOT,
    // exactly (CNOT Z_q1 CNOT = Z_q0 Z_q1), so RZ's angle gradient is RZZ's.
    // origin[g]: the user gate whose angle lowered gate g carries (-1: none).
    std::vector<qtm_gate> lowered;
    std::vector<int> origin;
    for (int g = 0; g < n_gates; ++g) {
        const qtm_gate &G = gates[g];
        if (G.kind == QTM_HADAMARD) {
            lowered.push_back({QTM_RY, G.q0, -1, -1, -1, 0, 0.5 * kPi});
            origin.push_back(-1);
            lowered.push_back({QTM_RX, G.q0, -1, -1, -1, 0, kPi});
            origin.push_back(-1);
        } else if (G.kind == QTM_RZZ) {
            lowered.push_back({QTM_CNOT, G.q0, G.q1, -1, -1, 0, 1.0});
            origin.push_back(-1);
            lowered.push_back({QTM_RZ, G.q1, -1, G.w_idx, G.x_idx, 0, G.coef});
            origin.push_back(g);
            lowered.push_back({QTM_CNOT, G.q0, G.q1, -1, -1, 0, 1.0});
            origin.push_back(-1);
        } else {
            lowered.push_back(G);
            origin.push_back(is_rot(G.kind) ? g : -1);
        }
    }
    gates = lowered.data();
    n_gates = (int)lowered.size();
    P.gates = lowered;
    for (int t = 0; t < n_terms; ++t)
        P.terms.push_back({terms[t].zmask, terms[t].coef, terms[t].obs, 0});
    std::stable_sort(P.terms.begin(), P.terms.end(),
                     [](const Term &a, const Term &b) { return a.obs < b.obs; });

    // ---- 1. prefix folding ------------------------------------------------
    std::vector<char> blocked(n, 0), ent_touched(n, 0), in_prefix(n_gates, 0);
    std::vector<std::vector<int>> prefix_rots(n);
    for (int g = 0; g < n_gates; ++g) {
        const qtm_gate &G = gates[g];
        if (is_rot(G.kind)) {
            int q = G.q0;
            if (!blocked[q] && !ent_touched[q]) { in_prefix[g] = 1; prefix_rots[q].push_back(g); }
            else blocked[q] = 1;
        } else {
            if (!blocked[G.q0] && !blocked[G.q1]) {
                in_prefix[g] = 1;
                ent_touched[G.q0] = ent_touched[G.q1] = 1;
                P.prefix_ents.push_back({G.kind, G.q0, G.q1, g});
            } else {
                blocked[G.q0] = blocked[G.q1] = 1;
            }
        }
    }
    if (P.path == QTM_PATH_NAIVE) {
        // the naive path applies every gate; no folding
        std::fill(in_prefix.begin(), in_prefix.end(), 0);
        P.prefix_ents.clear();
        for (auto &v : prefix_rots) v.clear();
    }

    // ---- 2. runs --------------------------------------------------------
    P.rot_of_gate.assign(n_gates, -1);
    P.prefix_run_of_q.assign(n, -1);
    auto add_rot = [&](int g) {
        const qtm_gate &G = gates[g];
        P.rot_of_gate[g] = (int)P.rots.size();
        P.rots.push_back({G.kind, origin[g], G.w_idx, G.x_idx, G.coef});   // gate = user gate (or -1)
    };
    for (int q = 0; q < n; ++q) {
        if (prefix_rots[q].empty()) continue;
        Run r{};
        r.q = q; r.prefix = 1; r.rot_begin = (int)P.rots.size();
        for (int g : prefix_rots[q]) add_rot(g);
        r.rot_end = (int)P.rots.size();
        P.prefix_run_of_q[q] = (int)P.runs.size();
        P.runs.push_back(r);
    }
    // non-prefix nodes, in circuit order
    std::vector<Node> fwd_nodes;
    {
        std::vector<int> open(n, -1);   // open run id per qubit
        std::vector<std::vector<int>> run_gates;
        for (int g = 0; g < n_gates; ++g) {
            if (in_prefix[g]) continue;
            const qtm_gate &G = gates[g];
            if (is_rot(G.kind)) {
                int q = G.q0;
                int rid = open[q];
                if (rid >= 0 && (int)run_gates[rid].size() < max_run) {
                    run_gates[rid].push_back(g);
                } else {
                    rid = (int)run_gates.size();
                    run_gates.push_back({g});
                    open[q] = rid;
                    Node nd{};
                    nd.type = 0; nd.run = rid; nd.prefix = false;
                    fwd_nodes.push_back(nd);
                }
            } else {
                open[G.q0] = open[G.q1] = -1;
                Node nd{};
                nd.type = 1; nd.ent = {G.kind, G.q0, G.q1, g}; nd.prefix = false;
                fwd_nodes.push_back(nd);
            }
        }
        // materialise runs (ids after the prefix runs)
        int base = (int)P.runs.size();
        for (auto &rg : run_gates) {
            Run r{};
            r.q = gates[rg[0]].q0; r.prefix = 0; r.rot_begin = (int)P.rots.size();
            for (int g : rg) add_rot(g);
            r.rot_end = (int)P.rots.size();
            P.runs.push_back(r);
        }
        for (auto &nd : fwd_nodes)
            if (nd.type == 0) nd.run += base;
    }

    // chain-rule CSR
    P.w_ptr.assign(n_weights + 1, 0);
    P.x_ptr.assign(n_inputs + 1, 0);
    for (const Rot &r : P.rots) {
        if (r.w_idx >= 0) P.w_ptr[r.w_idx + 1]++;
        if (r.x_idx >= 0) P.x_ptr[r.x_idx + 1]++;
    }
    for (int j = 0; j < n_weights; ++j) P.w_ptr[j + 1] += P.w_ptr[j];
    for (int k = 0; k < n_inputs; ++k) P.x_ptr[k + 1] += P.x_ptr[k];
    P.w_rots.assign(P.w_ptr[n_weights], 0);
    P.x_rots.assign(P.x_ptr[n_inputs], 0);
    {
        std::vector<int> wf(P.w_ptr.begin(), P.w_ptr.end() - 1), xf(P.x_ptr.begin(), P.x_ptr.end() - 1);
        for (int i = 0; i < (int)P.rots.size(); ++i) {
            if (P.rots[i].w_idx >= 0) P.w_rots[wf[P.rots[i].w_idx]++] = i;
            if (P.rots[i].x_idx >= 0) P.x_rots[xf[P.rots[i].x_idx]++] = i;
        }
    }

    if (P.path == QTM_PATH_NAIVE) {
        P.K = 0;
        P.state_qubits = n;
        return QTM_OK;
    }

    // ---- 3/4. schedule ---------------------------------------------------
    const int Kmax = dtype == QTM_C128 ? kMaxTileQubits128 : kMaxTileQubits;
    const int smem_limit = kMaxTileQubits;   // whole-state tile for either dtype
    P.state_qubits = std::max(n, kRegBits);
    // a state that spans several tiles: tiles of Kmax qubits unless the
    // options ask for a narrower one (at least 9: full warps of 16 registers)
    const int Kmulti = (opt.tile_qubits >= 9 && opt.tile_qubits <= Kmax) ? opt.tile_qubits : Kmax;
    P.K = (P.state_qubits <= smem_limit) ? P.state_qubits : Kmulti;
    if (P.low_min > P.K) P.low_min = P.K;
    P.tiles_per_sample = 1 << (P.state_qubits - P.K);

    P.pass_ents = P.prefix_ents;   // [0, |prefix_ents|): the forward's analytic state
    Builder bld(P);
    // forward
    build_deps(fwd_nodes, P.runs, n);
    {
        std::vector<int> last_touch(n, -1);
        bld.schedule_stage(fwd_nodes, 0, (int)fwd_nodes.size(), P.K, false, last_touch, P.fwd);
        if (P.fwd.empty())
            P.fwd.push_back(bld.emit_pass(fwd_nodes, {}, TileSet{P.K, P.K, 0}, P.K, false, last_touch));
    }
    // reverse sequence: reversed non-prefix nodes, then the reversed prefix
    // (folded entanglers in reverse order, then the prefix runs)
    std::vector<Node> rev_nodes;
    for (int i = (int)fwd_nodes.size() - 1; i >= 0; --i) {
        Node nd = fwd_nodes[i];
        nd.preds.clear();
        rev_nodes.push_back(nd);
    }
    const int n_main = (int)rev_nodes.size();
    for (int i = (int)P.prefix_ents.size() - 1; i >= 0; --i) {
        Node nd{};
        nd.type = 1; nd.ent = P.prefix_ents[i]; nd.prefix = true;
        rev_nodes.push_back(nd);
    }
    for (int q = 0; q < n; ++q)
        if (P.prefix_run_of_q[q] >= 0) {
            Node nd{};
            nd.type = 0; nd.run = P.prefix_run_of_q[q]; nd.prefix = true;
            rev_nodes.push_back(nd);
        }
    build_deps(rev_nodes, P.runs, n);
    std::vector<int> last_touch(n, -1);
    for (int i = 0; i < (int)rev_nodes.size(); ++i) {
        int a, b;
        touched(rev_nodes[i], P.runs, a, b);
        last_touch[a] = i;
        if (b >= 0) last_touch[b] = i;
    }
    if (n <= P.K) {
        // one pass: everything in shared memory
        std::vector<int> all;
        for (int i = 0; i < (int)rev_nodes.size(); ++i) all.push_back(i);
        P.rev.push_back(bld.emit_pass(rev_nodes, all, TileSet{P.K, P.K, 0}, P.K, true, last_touch));
    } else {
        bld.schedule_stage(rev_nodes, 0, n_main, P.K, true, last_touch, P.rev);
        size_t first_prefix_pass = P.rev.size();
        std::vector<std::vector<int>> prefix_pass_nodes;
        bld.schedule_stage(rev_nodes, n_main, (int)rev_nodes.size(), P.K, true, last_touch, P.rev,
                           &prefix_pass_nodes);
        // analytic phi for prefix-only passes: the folded entanglers not undone
        // by an earlier pass, in circuit order.  rev node n_main + k undoes
        // prefix entangler |prefix_ents| - 1 - k.
        const int ne = (int)P.prefix_ents.size();
        std::vector<char> undone(ne, 0);
        for (size_t i = first_prefix_pass; i < P.rev.size(); ++i) {
            PassDesc &pd = P.rev[i];
            pd.phi_src = SRC_ANALYTIC;
            pd.ents_begin = (int)P.pass_ents.size();
            for (int k = 0; k < ne; ++k)
                if (!undone[k]) P.pass_ents.push_back(P.prefix_ents[k]);
            pd.analytic_ents = (int)P.pass_ents.size() - pd.ents_begin;
            for (int node : prefix_pass_nodes[i - first_prefix_pass])
                if (rev_nodes[node].type == 1) undone[ne - 1 - (node - n_main)] = 1;
        }
        if (P.rev.empty()) {
            P.rev.push_back(bld.emit_pass(rev_nodes, {}, TileSet{P.K, P.K, 0}, P.K, true, last_touch));
        }
    }

    // ---- sources, sinks, expval / costate ops ---------------------------------
    const int nf = (int)P.fwd.size();
    for (int i = 0; i < nf; ++i) {
        PassDesc &pd = P.fwd[i];
        pd.phi_src = (i == 0) ? SRC_ANALYTIC : SRC_LOAD;
        pd.analytic_ents = (int)P.prefix_ents.size();
        pd.ents_begin = 0;
        pd.lam_src = SRC_NONE;
        pd.store_phi = 1;
        pd.store_lam = 0;
    }
    {
        // EXPVAL goes at the end of the last phase of the last forward pass
        PassDesc &pd = P.fwd.back();
        DevPhase &ph = P.phases[pd.phase_end - 1];
        // the op arrays are laid out pass after pass; the last pass's last
        // phase is the last one emitted in forward order only if no reverse
        // phases follow it: insert and shift later indices.
        DevOp op{};
        op.type = OP_EXPVAL; op.a = op.b = -1; op.slot = -1;
        int at = ph.op_end;
        P.ops.insert(P.ops.begin() + at, op);
        for (auto &p2 : P.phases) {
            if (&p2 == &ph) { p2.op_end++; continue; }
            if (p2.op_begin >= at) { p2.op_begin++; p2.op_end++; }
        }
        pd.has_expval = 1;
    }
    const int nr = (int)P.rev.size();
    for (int i = 0; i < nr; ++i) {
        PassDesc &pd = P.rev[i];
        if (pd.phi_src != SRC_ANALYTIC) {
            pd.phi_src = SRC_LOAD;
            pd.analytic_ents = 0;
        }
        pd.lam_src = (i == 0) ? SRC_COSTATE : SRC_LOAD;
        pd.store_lam = (i < nr - 1) ? 1 : 0;
        pd.store_phi = (i < nr - 1 && P.rev[i + 1].phi_src != SRC_ANALYTIC) ? 1 : 0;
        pd.has_grad = 0;
        for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph)
            for (int o = P.phases[ph].op_begin; o < P.phases[ph].op_end; ++o)
                if (P.ops[o].type == OP_GRAD) pd.has_grad = 1;
    }
    {
        // COSTATE first in the first phase of the first reverse pass
        PassDesc &pd = P.rev.front();
        DevPhase &ph = P.phases[pd.phase_begin];
        DevOp op{};
        op.type = OP_COSTATE; op.a = op.b = -1; op.slot = -1;
        int at = ph.op_begin;
        P.ops.insert(P.ops.begin() + at, op);
        for (auto &p2 : P.phases) {
            if (&p2 == &ph) { p2.op_end++; continue; }
            if (p2.op_begin >= at) { p2.op_begin++; p2.op_end++; }
        }
    }
    // ---- closed forms of the analytic states ---------------------------------
    for (auto *v : {&P.fwd, &P.rev})
        for (auto &pd : *v) {
            pd.amap_lin = -1;
            pd.amap_quad = 0;
            pd.amap_begin = 0;
            pd.amap_dlin = 0;
            if (pd.phi_src != SRC_ANALYTIC || pd.analytic_ents == 0) continue;
            std::vector<MaskTerm> t;
            int nl, nq;
            uint32_t dl;
            // over all state qubits: those above n (padding when n < 4) keep identity rows
            const std::vector<Ent> sub(P.pass_ents.begin() + pd.ents_begin,
                                       P.pass_ents.begin() + pd.ents_begin + pd.analytic_ents);
            if (!closed_form(sub, pd.analytic_ents, P.state_qubits, t, nl, nq, dl)) continue;
            pd.amap_begin = (int)P.amap_terms.size();
            pd.amap_lin = nl;
            pd.amap_quad = nq;
            pd.amap_dlin = dl;
            P.amap_terms.insert(P.amap_terms.end(), t.begin(), t.end());
        }

    // ---- place the CZ gates of each pass so that they merge into few DIAG ops --
    // A CZ may sit anywhere between the nearest ops of its pass, before and
    // after it, that do not commute with it: a run or gradient on one of its
    // qubits, a CNOT whose target is one of them, an expectation value or the
    // costate.  The fewest positions that cover every CZ's range are chosen
    // greedily (latest range start first, each new position at that start, so
    // no CZ moves later than the merge needs) and the CZs of one position
    // become consecutive ops.  In a reverse pass that stores nothing, a CZ
    // whose range reaches the pass's end is left out: it would multiply phi
    // and lam by the same signs, which no later op of the pass tells apart
    // (each commutes with it, and <D lam|sigma_c|D phi> = <lam|sigma_c|phi>
    // for a qubit c outside it).
    {
        std::vector<std::vector<DevOp>> placed(P.phases.size());
        std::vector<char> in_pass(P.phases.size(), 0);
        auto commutes = [](const DevOp &op, int a, int b) {
            switch (op.type) {
            case OP_CZ: return true;
            case OP_U2: case OP_GRAD: return op.a != a && op.a != b;
            case OP_CNOT: return op.b != a && op.b != b;
            default: return false;
            }
        };
        struct Range { int s, e, i; };   // gaps s..e (gap g lies before position g); the CZ's position i
        for (auto *v : {&P.fwd, &P.rev})
            for (const PassDesc &pd : *v) {
                std::vector<int> seq, phase_of;   // the pass's ops, phase after phase
                for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph) {
                    in_pass[ph] = 1;
                    for (int o = P.phases[ph].op_begin; o < P.phases[ph].op_end; ++o) {
                        seq.push_back(o);
                        phase_of.push_back(ph);
                    }
                }
                const int len = (int)seq.size();
                std::vector<Range> rs;
                for (int i = 0; i < len; ++i) {
                    const DevOp &cz = P.ops[seq[i]];
                    if (cz.type != OP_CZ) continue;
                    int s = i, e = i + 1;
                    while (s > 0 && commutes(P.ops[seq[s - 1]], cz.a, cz.b)) --s;
                    while (e < len && commutes(P.ops[seq[e]], cz.a, cz.b)) ++e;
                    rs.push_back({s, e, i});
                }
                const bool drop_tail = pd.reverse && !pd.store_phi && !pd.store_lam;
                std::vector<int> gap_of(len, -1);   // per CZ position its gap, -1 left out
                std::sort(rs.begin(), rs.end(), [](const Range &x, const Range &y) {
                    return x.s != y.s ? x.s > y.s : x.i < y.i;
                });
                int point = -1;
                for (const Range &r : rs) {
                    if (drop_tail && r.e == len) continue;
                    if (point < 0 || r.e < point) point = r.s;
                    gap_of[r.i] = point;
                }
                auto emit_gap = [&](int g, int ph) {
                    for (int i = 0; i < len; ++i)
                        if (gap_of[i] == g) placed[ph].push_back(P.ops[seq[i]]);
                };
                for (int i = 0; i < len; ++i) {
                    // a gap between two phases goes to the end of the earlier one
                    emit_gap(i, (i > 0 && phase_of[i - 1] != phase_of[i]) ? phase_of[i - 1] : phase_of[i]);
                    if (P.ops[seq[i]].type != OP_CZ) placed[phase_of[i]].push_back(P.ops[seq[i]]);
                }
                if (len > 0) emit_gap(len, phase_of[len - 1]);
            }
        std::vector<DevOp> ops;
        ops.reserve(P.ops.size());
        for (size_t ph = 0; ph < P.phases.size(); ++ph) {
            DevPhase &d = P.phases[ph];
            const int nb = (int)ops.size();
            if (in_pass[ph]) ops.insert(ops.end(), placed[ph].begin(), placed[ph].end());
            else ops.insert(ops.end(), P.ops.begin() + d.op_begin, P.ops.begin() + d.op_end);
            d.op_begin = nb;
            d.op_end = (int)ops.size();
        }
        P.ops.swap(ops);
    }

    // ---- merge runs of consecutive CZ ops inside a phase into one DIAG op -----
    {
        std::vector<DevOp> ops;
        ops.reserve(P.ops.size());
        for (auto &ph : P.phases) {
            const int nb = (int)ops.size();
            for (int o = ph.op_begin; o < ph.op_end;) {
                if (P.ops[o].type != OP_CZ) { ops.push_back(P.ops[o]); ++o; continue; }
                DevOp d{};
                d.type = OP_DIAG;
                d.a = (int16_t)P.diag_pairs.size();
                d.slot = -1;
                while (o < ph.op_end && P.ops[o].type == OP_CZ) {
                    P.diag_pairs.push_back({P.ops[o].a, P.ops[o].b});
                    ++o;
                }
                d.b = (int16_t)(P.diag_pairs.size() - d.a);
                ops.push_back(d);
            }
            ph.op_begin = nb;
            ph.op_end = (int)ops.size();
        }
        P.ops.swap(ops);
        if (P.diag_pairs.size() > 32000) { err = "too many CZ gates"; return QTM_EUNSUPPORTED; }
    }
    for (auto *v : {&P.fwd, &P.rev})
        for (auto &pd : *v) {
            P.max_slots = std::max(P.max_slots, pd.slot_end - pd.slot_begin);
            P.max_phases = std::max(P.max_phases, pd.phase_end - pd.phase_begin);
        }
    for (DevPhase &ph : P.phases) {
        bool keeps = true;
        for (int o = ph.op_begin; o < ph.op_end && keeps; ++o) {
            const DevOp &op = P.ops[o];
            keeps = op.type == OP_EXPVAL || (op.type == OP_GRAD && (op.flags & OPF_SKIP_APPLY));
        }
        ph.flags = keeps ? PHF_KEEPS_STATE : 0;
    }
    return QTM_OK;
}

}  // namespace

void attach_pauli_terms(Plan &P, const std::vector<PauliTerm> &terms)
{
    P.pterms = terms;
    if (terms.empty() || P.path != QTM_PATH_FUSED || P.fwd.empty() || P.rev.empty()) return;
    P.fwd.back().store_phi = 1;
    PassDesc &pd = P.rev.front();
    pd.lam_src = SRC_LOAD;
    for (int o = P.phases[pd.phase_begin].op_begin; o < P.phases[pd.phase_begin].op_end; ++o)
        if (P.ops[o].type == OP_COSTATE) P.ops[o].flags |= OPF_ACCUMULATE;
}

namespace {

// Ops of a pass's phase as a comparable key: register group, then per op its
// type, operands, flags, run slot relative to the phase's first slot and,
// for DIAG ops, the CZ pairs.
std::vector<int64_t> phase_key(const Plan &P, const DevPhase &ph)
{
    int sb = -1;
    for (int o = ph.op_begin; o < ph.op_end; ++o)
        if (P.ops[o].slot >= 0 && (sb < 0 || P.ops[o].slot < sb)) sb = P.ops[o].slot;
    std::vector<int64_t> k{ph.lo};
    for (int o = ph.op_begin; o < ph.op_end; ++o) {
        const DevOp &op = P.ops[o];
        if (op.type == OP_DIAG) {   // a and b locate the pairs in the shared list: key the pairs
            k.insert(k.end(), {op.type, op.b, op.flags});
            for (int d = op.a; d < op.a + op.b; ++d) k.insert(k.end(), {P.diag_pairs[d].a, P.diag_pairs[d].b});
        } else {
            k.insert(k.end(), {op.type, op.a, op.b, op.flags, op.slot >= 0 ? op.slot - sb : -1});
        }
    }
    return k;
}

}  // namespace

double periodic_fraction(const Plan &P)
{
    double in_loops = 0.0, total = 0.0;
    for (const auto *v : {&P.fwd, &P.rev})
        for (const PassDesc &pd : *v) {
            const int nph = pd.phase_end - pd.phase_begin;
            std::vector<std::vector<int64_t>> key(nph);
            std::vector<int> sb(nph, 0), ops(nph, 0);
            for (int i = 0; i < nph; ++i) {
                const DevPhase &ph = P.phases[pd.phase_begin + i];
                key[i] = phase_key(P, ph);
                ops[i] = ph.op_end - ph.op_begin;
                int m = -1;
                for (int o = ph.op_begin; o < ph.op_end; ++o)
                    if (P.ops[o].slot >= 0 && (m < 0 || P.ops[o].slot < m)) m = P.ops[o].slot;
                sb[i] = m < 0 ? 0 : m;
                total += ops[i];
            }
            // the longest stretch [st, st + p * r) of phases repeating with a fixed slot stride
            int best = 0, best_st = 0;
            for (int p = 1; p <= 8 && 2 * p <= nph; ++p)
                for (int st = 0; st + 2 * p <= nph; ++st) {
                    const int stride = sb[st + p] - sb[st];
                    int r = 1;
                    while (st + (r + 1) * p <= nph) {
                        bool ok = true;
                        for (int i = 0; i < p && ok; ++i) {
                            const int a = st + i, b = st + r * p + i;
                            ok = key[b] == key[a] && sb[b] - sb[a] == r * stride;
                        }
                        if (!ok) break;
                        ++r;
                    }
                    if (r >= 2 && p * r > best) { best = p * r; best_st = st; }
                }
            for (int i = best_st; i < best_st + best; ++i) in_loops += ops[i];
        }
    return total > 0.0 ? in_loops / total : 0.0;
}

qtm_status make_plan(int n, const qtm_gate *gates, int n_gates, const qtm_zterm *terms,
                     int n_terms, int n_obs, int n_weights, int n_inputs, int dtype, int path,
                     Plan &P, std::string &err, const PlanOptions &opt)
{
    if (opt.phase_mode != PHASES_AUTO)
        return make_plan_mode(n, gates, n_gates, terms, n_terms, n_obs, n_weights, n_inputs, dtype, path, P, err,
                              opt, opt.phase_mode);
    // round robin where it makes most of the work periodic, else greedy; the
    // interpreter kernels (complex128 plans) run a few percent slower on the
    // extra phases, so those keep greedy
    if (dtype == QTM_C128)
        return make_plan_mode(n, gates, n_gates, terms, n_terms, n_obs, n_weights, n_inputs, dtype, path, P, err,
                              opt, PHASES_GREEDY);
    qtm_status st = make_plan_mode(n, gates, n_gates, terms, n_terms, n_obs, n_weights, n_inputs, dtype, path, P,
                                   err, opt, PHASES_ROUND_ROBIN);
    if (st != QTM_OK || P.path != QTM_PATH_FUSED || periodic_fraction(P) >= 0.5) return st;
    return make_plan_mode(n, gates, n_gates, terms, n_terms, n_obs, n_weights, n_inputs, dtype, path, P, err,
                          opt, PHASES_GREEDY);
}

void plan_costs(const Plan &p, double &fwd_bytes, double &adj_bytes, double &fwd_flops,
                double &adj_flops)
{
    const double N = std::ldexp(1.0, p.n);
    const double sb = N * elem_bytes(p.dtype);
    const double T = (double)p.terms.size();
    fwd_bytes = adj_bytes = fwd_flops = adj_flops = 0.0;
    if (p.path == QTM_PATH_NAIVE) {
        // every gate reads and writes the state once; reverse: rotations read
        // phi and lam twice (inner product, then update), entanglers once.
        int nrot = 0, nent = 0;
        for (const auto &g : p.gates) (is_rot(g.kind) ? nrot : nent)++;
        fwd_bytes = sb * (1 + 2.0 * (nrot + nent) + 1);
        adj_bytes = sb * (2.0 + 2 * 2.0 * nrot + 4.0 * nrot + 4.0 * nent);
        fwd_flops = N * (7.0 * nrot + 3.0 + T);
        adj_flops = N * (10.5 * nrot + 14.0 * nrot + T + 2.0);
        return;
    }
    auto pass_flops = [&](const PassDesc &pd) {
        double f = 0.0;
        for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph)
            for (int o = p.phases[ph].op_begin; o < p.phases[ph].op_end; ++o) {
                const DevOp &op = p.ops[o];
                switch (op.type) {
                case OP_U2: f += 14.0 * N; break;                       // 2x2 complex on N/2 pairs
                case OP_GRAD: f += 12.0 * N + ((op.flags & OPF_SKIP_APPLY) ? 0.0 : 28.0 * N); break;
                case OP_EXPVAL: f += (3.0 + T) * N; break;
                case OP_DIAG: break;
                case OP_COSTATE: f += (T + 2.0) * N; break;
                default: break;
                }
            }
        if (pd.phi_src == SRC_ANALYTIC) f += 6.0 * ((p.n + 3) / 4 - 1) * N;
        return f;
    };
    for (const auto &pd : p.fwd) {
        fwd_bytes += sb * ((pd.phi_src == SRC_LOAD) + pd.store_phi);
        fwd_flops += pass_flops(pd);
    }
    for (const auto &pd : p.rev) {
        adj_bytes += sb * ((pd.phi_src == SRC_LOAD) + (pd.lam_src == SRC_LOAD) + pd.store_phi +
                           pd.store_lam);
        adj_flops += pass_flops(pd);
    }
    // strings with X/Y factors on the final state: one read of it per string
    // (its partner amplitudes come from the same cache lines or L2), 4 flop per
    // amplitude and string (Re conj(a) b, or the cotangent-weighted add); the
    // costate part is written once
    const double TP = (double)p.pterms.size();
    if (TP > 0) {
        fwd_bytes += sb * TP;
        fwd_flops += 4.0 * TP * N;
        adj_bytes += sb * (TP + 1.0);
        adj_flops += 4.0 * TP * N;
    }
}

std::string Plan::describe() const
{
    std::ostringstream s;
    s << "plan n=" << n << " K=" << K << " tiles/sample=" << tiles_per_sample
      << " runs=" << runs.size() << " rots=" << rots.size()
      << " prefix_ents=" << prefix_ents.size() << "\n";
    auto dump = [&](const char *name, const std::vector<PassDesc> &v) {
        for (size_t i = 0; i < v.size(); ++i) {
            const PassDesc &pd = v[i];
            s << name << "[" << i << "] S=[0," << pd.l << ")";
            if (pd.m) s << "+[" << pd.h << "," << pd.h + pd.m << ")";
            s << " phi=" << pd.phi_src << " lam=" << pd.lam_src << " ents=" << pd.analytic_ents;
            if (pd.phi_src == SRC_ANALYTIC) s << " closed=" << pd.amap_lin << "/" << pd.amap_quad;
            s
              << " store=" << pd.store_phi << pd.store_lam << " phases=";
            for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph) {
                s << "{lo" << phases[ph].lo << ":";
                for (int o = phases[ph].op_begin; o < phases[ph].op_end; ++o) {
                    const DevOp &op = ops[o];
                    const char *nm[] = {"?", "U", "G", "CZ", "CX", "E", "C", "D"};
                    s << " " << nm[op.type];
                    if (op.type <= OP_CNOT) s << op.a;
                    if (op.type == OP_CZ || op.type == OP_CNOT) s << "," << op.b;
                    if (op.type == OP_DIAG) {
                        s << "[";
                        for (int k = op.a; k < op.a + op.b; ++k)
                            s << (k > op.a ? " " : "") << diag_pairs[k].a << "," << diag_pairs[k].b;
                        s << "]";
                    }
                    if (op.type == OP_GRAD && (op.flags & OPF_SKIP_APPLY)) s << "s";
                }
                s << "}";
            }
            s << "\n";
        }
    };
    dump("fwd", fwd);
    dump("rev", rev);
    return s.str();
}

}  // namespace qtm
