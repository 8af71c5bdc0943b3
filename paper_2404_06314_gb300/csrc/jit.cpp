// Run-time specialised pass kernels.
//
// The interpreter kernel (k_pass) reads every op's type, register bit, slot
// and operands at run time.  For a fixed plan all of them are known, so this
// file writes the pass's phase program out as CUDA source in which every
// register bit, slot offset, CZ sign pattern and CNOT form is a compile-time
// constant, compiles it with NVRTC for sm_103a, and loads it through the
// driver API.  The generated kernel reuses the library's tile program
// (pass_body in tile.cuh: TMA staging, analytic state, partial sums) and
// replaces only the phase interpreter.  NVRTC is loaded with dlopen; when it
// is missing, plans keep the interpreter kernels.
#include "jit.h"

#include "device.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

namespace qtm {

extern const char *const kJitPrelude;   // pod.h + finalize_math.h + tile.cuh (generated at build time)

namespace {

// ---- source generation ---------------------------------------------------------

const char *kRegMask[4] = {"0xAAAAu", "0xCCCCu", "0xF0F0u", "0xFF00u"};
const uint32_t kRegMaskV[4] = {0xAAAAu, 0xCCCCu, 0xF0F0u, 0xFF00u};

std::string operand_bit(int o)
{
    std::ostringstream s;
    if (o >= kFixed) s << "(base >> " << (o - kFixed) << ")";
    else s << "(xt >> " << o << ")";
    return s.str();
}

}  // namespace

bool jit_eligible(const Plan &P, const PassDesc &pd)
{
    return P.path == QTM_PATH_FUSED && pd.K >= 9 && P.dtype == QTM_C64;
}

namespace {

// tile-local Z mask of a term for the pass geometry (l, h, m)
uint32_t local_mask(const PassDesc &pd, uint64_t zm)
{
    return (uint32_t)(zm & ((1ull << pd.l) - 1ull)) | (uint32_t)(((zm >> pd.h) & ((1ull << pd.m) - 1ull)) << pd.l);
}

bool has_reg_bit(int x, int lo) { return x < kFixed && x >= lo && x < lo + kRegBits; }

// byte offset of the complex-pair matrix table from the tile program's
// aligned shared base (it follows the tile program's shared memory)
size_t cpx_table_offset(const Plan &P, const PassDesc &pd)
{
    return pass_smem_bytes(pd.K, P.dtype, pd.reverse != 0, pd.slot_end - pd.slot_begin, (int)P.terms.size(), P.n_obs,
                           P.state_qubits, pd.phi_src == SRC_ANALYTIC ? pd.analytic_ents : 0) - 1024;
}

// The DIAG op as sign flips of single registers: a register's sign is its
// constant part (CZ pairs of two register bits) XOR the thread's sign words,
// one per register bit paired with thread bits and one for the pairs of two
// thread bits, each computed once per op.
std::string diag_flip_cpx(const Plan &P, const DevOp &op, int lo, bool rev)
{
    uint32_t C = 0;
    std::vector<std::vector<int>> per_reg(kRegBits);
    std::vector<std::pair<int, int>> other;
    for (int k = op.a; k < op.a + op.b; ++k) {
        const DiagPair dp = P.diag_pairs[k];
        const bool ra = has_reg_bit(dp.a, lo), rb = has_reg_bit(dp.b, lo);
        if (ra && rb) C ^= kRegMaskV[dp.a - lo] & kRegMaskV[dp.b - lo];
        else if (ra) per_reg[dp.a - lo].push_back(dp.b);
        else if (rb) per_reg[dp.b - lo].push_back(dp.a);
        else other.push_back({dp.a, dp.b});
    }
    std::ostringstream o;
    o << "{";
    for (int r = 0; r < kRegBits; ++r) {
        if (per_reg[r].empty()) continue;
        o << " const uint32_t t" << r << " = (0u - ((";
        for (size_t i = 0; i < per_reg[r].size(); ++i) o << (i ? " ^ " : "") << operand_bit(per_reg[r][i]);
        o << ") & 1u)) & 0x80000000u;";
    }
    if (!other.empty()) {
        o << " const uint32_t to = (0u - ((";
        for (size_t i = 0; i < other.size(); ++i)
            o << (i ? " ^ " : "") << "(" << operand_bit(other[i].first) << " & " << operand_bit(other[i].second) << ")";
        o << ") & 1u)) & 0x80000000u;";
    }
    for (int j = 0; j < (1 << kRegBits); ++j) {
        std::string s;
        for (int r = 0; r < kRegBits; ++r)
            if (((j >> r) & 1) && !per_reg[r].empty()) s += (s.empty() ? "t" : " ^ t") + std::to_string(r);
        if (!other.empty()) s += s.empty() ? "to" : " ^ to";
        const bool c = (C >> j) & 1u;
        if (s.empty() && !c) continue;
        if (s.empty()) s = "0x80000000u";
        else if (c) s += " ^ 0x80000000u";
        o << " flip_reg<" << (rev ? "true" : "false") << ", " << j << ">(p, q, " << s << ");";
    }
    o << " }";
    return o.str();
}

// Phases emitted straight-line (default; measured 5 % faster at 12 and 20
// qubits) or as a loop over a phase table with one copy of each distinct phase
// program (QTM_JIT_PHASE_LOOP=1, a tuning switch).
bool straight_phases(size_t, size_t)
{
    const char *v = std::getenv("QTM_JIT_PHASE_LOOP");
    return !(v && *v == '1');
}

// Repeated phase programs emitted once as a loop (default) or every phase
// straight-line (QTM_JIT_REPEAT_LOOPS=0, a tuning switch).
bool repeat_loops()
{
    const char *v = std::getenv("QTM_JIT_REPEAT_LOOPS");
    return !(v && *v == '0');
}

// The longest periodic stretch of a pass's phase table (pairs of program
// index, first run slot): phases [start, start + period * reps) where phase
// start + r * period + i runs the program of phase start + i with its slots
// shifted by r * stride.  A layered circuit scheduled with one run per qubit
// per phase (PHASES_ROUND_ROBIN) repeats a few phase programs layer after
// layer; emitted as a loop they are fetched once per CTA instead of once per
// layer.  reps < 2: no such stretch.
struct Repeat {
    int start = 0, period = 0, reps = 0, stride = 0;
};

Repeat find_repeat(const std::vector<int> &table, int nph)
{
    Repeat best;
    for (int p = 1; p <= 8 && 2 * p <= nph; ++p)
        for (int st = 0; st + 2 * p <= nph; ++st) {
            const int stride = table[2 * (st + p) + 1] - table[2 * st + 1];
            int r = 1;
            while (st + (r + 1) * p <= nph) {
                bool ok = true;
                for (int i = 0; i < p && ok; ++i) {
                    const int a = st + i, b = st + r * p + i;
                    ok = table[2 * b] == table[2 * a] && table[2 * b + 1] - table[2 * a + 1] == r * stride;
                }
                if (!ok) break;
                ++r;
            }
            if (r >= 2 && p * r > best.period * best.reps) best = {st, p, r, stride};
        }
    return best;
}

// Phase transitions inside one warp.  A thread of a phase with register
// group [lo, lo + 4) holds the tile amplitudes whose other K - 4 bits are its
// index bits in order (thread bit k is tile bit k below lo, k + 4 above), so
// warp w of 2^(K-4) threads holds the amplitudes whose bits at the positions
// of thread bits 5 .. K-5 spell w.  When two consecutive phases put those
// warp bits on the same tile bits, every amplitude a warp stores is loaded
// back by the same warp, and a warp barrier orders the shared-memory store
// and load; other state shared across warps (tables, per-warp partial sums)
// is not written between phases.
bool warp_local_transition(int K, int lo_a, int lo_b)
{
    if (K - 4 <= 5) return true;   // one warp per CTA
    for (int k = 5; k < K - 4; ++k) {
        const int ba = k < lo_a ? k : k + 4, bb = k < lo_b ? k : k + 4;
        if (ba != bb) return false;
    }
    return true;
}

// warp barriers between phases that stay within a warp (default) or CTA
// barriers everywhere (QTM_JIT_WARP_BARRIERS=0, a tuning switch)
bool warp_local_barriers()
{
    const char *v = std::getenv("QTM_JIT_WARP_BARRIERS");
    return !(v && *v == '0');
}

// Body of one phase with its run slots written relative to the phase's first
// slot `sb` (a runtime value): layers of a layered circuit repeat the same
// body with other slots and then share one copy of the code.
// ---- complex-pair one-sample kernels (tile_cpx.cuh) ----------------------------------

constexpr int kCpxSlotPairsHost = 8;   // f32x2 pairs per run slot in the complex-pair table

void gen_expval_cpx(std::ostringstream &o, const Plan &P, const PassDesc &pd, int lo)
{
    // per register sign pattern rm: sum of |p_jj|^2 with sign (-1)^popc(jj & rm),
    // as two FMA chains (plus / minus) straight from the amplitudes
    o << "        {\n";
    std::vector<int> seen(16, 0);
    for (const Term &t : P.terms) {
        const int rm = (int)((local_mask(pd, t.zmask) >> lo) & 15u);
        if (seen[rm]) continue;
        seen[rm] = 1;
        std::string pos = "", neg = "";
        for (int jj = 0; jj < 16; ++jj) {
            std::string &acc = (__builtin_popcount(jj & rm) & 1) ? neg : pos;
            const std::string pj = "p[" + std::to_string(jj) + "]";
            acc = acc.empty() ? "mul2(" + pj + ", " + pj + ")" : "fma2(" + pj + ", " + pj + ", " + acc + ")";
        }
        o << "            const f2 a" << rm << " = " << (neg.empty() ? pos : "sub2(" + pos + ", " + neg + ")") << ";\n";
        o << "            const float s" << rm << " = lane0(a" << rm << ") + lane1(a" << rm << ");\n";
    }
    for (int m = 0; m < P.n_obs; ++m) {
        bool any = false;
        for (size_t t = 0; t < P.terms.size(); ++t) {
            if (P.terms[t].obs != m) continue;
            if (!any) o << "            { float e = 0.f;\n";
            any = true;
            const uint32_t lm = local_mask(pd, P.terms[t].zmask);
            const int rm = (int)((lm >> lo) & 15u);
            o << "              e = fmaf((__popc(xt & 0x" << std::hex << lm << std::dec << "u) & 1u) ? -S.tcoef[" << t
              << "] : S.tcoef[" << t << "], s" << rm << ", e);\n";
        }
        if (any)
            o << "              e = warp_sum(e, 32, 0xffffffffu); if (lane == 0) S.redE[warp * " << P.n_obs << " + "
              << m << "] = e; }\n";
    }
    o << "        }\n";
}

// acc: q holds the costate's X/Y part (loaded from memory); add the Z part.
void gen_costate_cpx(std::ostringstream &o, const Plan &P, const PassDesc &pd, int lo, bool acc)
{
    o << "        {\n";
    std::vector<std::vector<size_t>> by_rm(16);
    for (size_t t = 0; t < P.terms.size(); ++t) by_rm[(local_mask(pd, P.terms[t].zmask) >> lo) & 15u].push_back(t);
    std::vector<int> rms;
    for (int rm = 0; rm < 16; ++rm) {
        if (by_rm[rm].empty()) continue;
        rms.push_back(rm);
        o << "            const float c" << rm << " = 0.f";
        for (size_t t : by_rm[rm])
            o << " + ((__popc(xt & 0x" << std::hex << local_mask(pd, P.terms[t].zmask) << std::dec
              << "u) & 1u) ? -S.tcoef[" << t << "] : S.tcoef[" << t << "])";
        o << ";\n";
    }
    for (int jj = 0; jj < 16; ++jj) {
        std::string e = "0.f";
        for (int rm : rms) e += std::string(__builtin_popcount(jj & rm) & 1 ? " - c" : " + c") + std::to_string(rm);
        o << "            { const float d = " << e << "; q[" << jj << "] = "
          << (acc ? "fma2(pack2(d, d), p[" + std::to_string(jj) + "], q[" + std::to_string(jj) + "]); }\n"
                  : "mul2(pack2(d, d), p[" + std::to_string(jj) + "]); }\n");
    }
    o << "        }\n";
}

// An analytic pass whose closed form is known (or that has no folded
// entangler): the complex-pair kernel computes phi straight into its first
// phase's registers instead of the tile program filling shared memory.
bool cpx_fill(const PassDesc &pd)
{
    return pd.phi_src == SRC_ANALYTIC && (pd.amap_lin >= 0 || pd.analytic_ents == 0);
}

// Closed form of the analytic phi (the tile program's fill_analytic, with
// every constant of the pass written out).  Amplitude index y (global bits)
// of register jj of a thread: y = y_t | Y_jj with Y_jj the tile bits of jj,
// so the linear part x = X(y_t) ^ X(Y_jj) and the linear sign parity split
// into a per-thread value and a per-register constant; the quadratic parity
// terms are evaluated per register.  phi_y = sign * prod_q T_q[nibble q of x]:
// tables whose nibble no register changes are multiplied once per thread.
void gen_fill_cpx(std::ostringstream &o, const Plan &P, const PassDesc &pd, int lo)
{
    const int L = pd.l, H = pd.h;
    const uint32_t LM = (1u << L) - 1u;
    auto yloc = [&](uint32_t v) { return (v & LM) | ((v >> L) << H); };
    std::vector<MaskTerm> lin, quad;
    uint32_t dlin = 0;
    const bool identity = pd.amap_lin < 0;   // no folded entangler: x = y
    if (!identity) {
        for (int k = 0; k < pd.amap_lin; ++k) lin.push_back(P.amap_terms[pd.amap_begin + k]);
        for (int k = 0; k < pd.amap_quad; ++k) quad.push_back(P.amap_terms[pd.amap_begin + pd.amap_lin + k]);
        dlin = pd.amap_dlin;
    }
    auto X = [&](uint32_t y) {
        if (identity) return y;
        uint32_t x = 0;
        for (const MaskTerm &t : lin) x ^= (t.d >= 0 ? (y >> t.d) : (y << -t.d)) & t.mask;
        return x;
    };
    const int ntab = (P.state_qubits + 3) >> 2;
    std::vector<uint32_t> C(16);
    std::vector<int> PC(16);
    for (int jj = 0; jj < 16; ++jj) {
        C[jj] = X(yloc((uint32_t)jj << lo));
        PC[jj] = __builtin_popcount(C[jj] & dlin) & 1;
    }
    std::vector<int> vary, fixed;
    for (int q = 0; q < ntab; ++q) {
        bool v = false;
        for (int jj = 0; jj < 16; ++jj) v |= ((C[jj] >> (4 * q)) & 15u) != 0;
        (v ? vary : fixed).push_back(q);
    }
    o << "        {   // analytic phi, closed form, straight into the registers\n";
    o << "            const uint32_t yt = base | (xt & 0x" << std::hex << LM << "u) | ((xt >> " << std::dec << L
      << ") << " << H << ");\n";
    if (identity) {
        o << "            const uint32_t x0 = yt;\n";
    } else {
        o << "            uint32_t x0 = 0u;\n";
        for (const MaskTerm &t : lin)
            o << "            x0 ^= (yt " << (t.d >= 0 ? ">> " : "<< ") << std::abs(t.d) << ") & 0x" << std::hex << t.mask
              << std::dec << "u;\n";
    }
    o << "            const uint32_t s0 = " << (dlin ? "__popc(x0 & 0x" : "0u") ;
    if (dlin) o << std::hex << dlin << std::dec << "u) & 1u";
    o << ";\n";
    o << "            const uint32_t tb = smem_u32(S.tabs), tt = smem_u32(TT);\n";
    for (int q = 0; q < ntab; ++q)
        o << "            const uint32_t n" << q << " = (x0 >> " << 4 * q << ") & 15u;\n";
    // thread-constant product of the tables no register changes
    if (!fixed.empty()) {
        o << "            f2 pt = lds_f2(tb + 8u * (" << 16 * fixed[0] << "u + n" << fixed[0] << "));\n";
        for (size_t i = 1; i < fixed.size(); ++i)
            o << "            pt = cmul_tab(tt + 16u * (" << 16 * fixed[i] << "u + n" << fixed[i] << "), pt);\n";
    }
    for (int jj = 0; jj < 16; ++jj) {
        o << "            { ";
        size_t first = 0;
        if (!fixed.empty()) {
            o << "f2 a = pt;";
        } else {
            const int q = vary[0];
            o << "f2 a = lds_f2(tb + 8u * (" << 16 * q << "u + (n" << q << " ^ " << ((C[jj] >> (4 * q)) & 15u) << "u)));";
            first = 1;
        }
        for (size_t i = first; i < vary.size(); ++i) {
            const int q = vary[i];
            o << " a = cmul_tab(tt + 16u * (" << 16 * q << "u + (n" << q << " ^ " << ((C[jj] >> (4 * q)) & 15u)
              << "u)), a);";
        }
        o << " uint32_t s = s0 ^ " << PC[jj] << "u;";
        if (!quad.empty()) {
            o << " const uint32_t xx = x0 ^ 0x" << std::hex << C[jj] << std::dec << "u;";
            for (const MaskTerm &t : quad)
                o << " s ^= __popc(xx & (xx >> " << t.d << ") & 0x" << std::hex << t.mask << std::dec << "u) & 1u;";
        }
        o << " p[" << jj << "] = a ^ (((f2)s << 63) | ((f2)s << 31)); }\n";
    }
    o << "        }\n";
}

// One op of a complex-pair phase (register group lo); `slot` is the C
// expression of its run slot.  deferred (reverse phases): GRAD ops keep their
// reduced sums in registers vr[i] and the phase stores them at its end (slot
// expressions collected here), so no shared store waits on a reduction
// between one run's gradient and the next run's table loads (12 qubits:
// reverse pass 287 -> 280 us).
void cpx_op(std::ostringstream &o, const Plan &P, const PassDesc &pd, int k, int lo, const std::string &slot,
            std::vector<std::string> *deferred = nullptr)
{
    const bool rev = pd.reverse != 0;
    const int nslots = pd.slot_end - pd.slot_begin;
    const DevOp &op = P.ops[k];
    const bool reg_a = has_reg_bit(op.a, lo);
    const bool reg_b = has_reg_bit(op.b, lo);
    if (((op.type == OP_U2 || op.type == OP_GRAD) && !reg_a) || (op.type == OP_CNOT && !reg_b) ||
        ((op.type == OP_U2 || op.type == OP_GRAD) && (op.slot < 0 || op.slot >= nslots)) ||
        (op.type == OP_DIAG && (op.a < 0 || op.a + op.b > (int)P.diag_pairs.size()))) {
        o << "#error \"op " << k << " has an operand outside its phase\"\n";
        return;
    }
    const int rb = op.a - lo;
    const std::string tab = "CT + " + std::to_string(kCpxSlotPairsHost) + " * " + slot;
    switch (op.type) {
    case OP_U2:
        o << "        u2_cpx<" << rb << ">(p, " << tab << ");\n";
        break;
    case OP_GRAD:
        o << "        { float vx, vy, vz; grad_cpx<" << rb << ">(p, q, vx, vy, vz);";
        if (deferred) {
            o << " vr[" << deferred->size() << "] = warp_sum3(vx, vy, vz, lane);";
            deferred->push_back(slot);
        } else {
            o << " const float v = warp_sum3(vx, vy, vz, lane);"
              << " if ((lane & 7) == 0 && lane < 24) S.redG[warp * " << 3 * nslots << " + 3 * " << slot
              << " + (lane >> 3)] = v;";
        }
        if (!(op.flags & OPF_SKIP_APPLY))
            o << " u2_cpx<" << rb << ">(p, " << tab << "); u2_cpx<" << rb << ">(q, " << tab << ");";
        o << " }\n";
        break;
    case OP_DIAG:
        o << "        " << diag_flip_cpx(P, op, lo, rev) << "\n";
        break;
    case OP_CNOT: {
        const int rt = op.b - lo;
        if (has_reg_bit(op.a, lo)) {
            o << "        cnot_static_cpx<" << (op.a - lo) << ", " << rt << ">(p);";
            if (rev) o << " cnot_static_cpx<" << (op.a - lo) << ", " << rt << ">(q);";
            o << "\n";
        } else {
            o << "        { const int c = (int)(" << operand_bit(op.a) << " & 1u); cnot_cpx<" << rt << ">(p, c);";
            if (rev) o << " cnot_cpx<" << rt << ">(q, c);";
            o << " }\n";
        }
        break;
    }
    case OP_EXPVAL: gen_expval_cpx(o, P, pd, lo); break;
    case OP_COSTATE: gen_costate_cpx(o, P, pd, lo, (op.flags & OPF_ACCUMULATE) != 0); break;
    default: break;
    }
}

std::string phase_body(const Plan &P, const PassDesc &pd, const DevPhase &phs, bool lam_valid, int sb,
                       bool fill = false, bool store = true)
{
    const bool rev = pd.reverse != 0;
    const int lo = phs.lo;
    std::ostringstream o;
    auto slot = [&](int s) { return "(sb + " + std::to_string(s - sb) + ")"; };
    o << "        constexpr int LO = " << lo << ";\n";
    o << "        const uint32_t xt = ((uint32_t)tid & ((1u << LO) - 1u)) | (((uint32_t)tid >> LO) << (LO + 4));\n";
    if (fill) {   // phi from the closed form, lam (if any) from shared memory
        if (lam_valid) o << "        regs_load_cpx_lam<LO>(q, S, xt);\n";
        gen_fill_cpx(o, P, pd, lo);
    } else {
        o << "        regs_load_cpx<LO, " << (lam_valid ? "true" : "false") << ">(p, q, S, xt);\n";
    }
    std::vector<std::string> deferred;
    const bool defer = rev;
    int ngrad = 0;
    for (int k = phs.op_begin; k < phs.op_end; ++k) ngrad += P.ops[k].type == OP_GRAD;
    if (defer && ngrad) o << "        float vr[" << ngrad << "];\n";
    for (int k = phs.op_begin; k < phs.op_end; ++k)
        cpx_op(o, P, pd, k, lo, slot(P.ops[k].slot), defer && ngrad ? &deferred : nullptr);
    if (!deferred.empty()) {
        const int nslots = pd.slot_end - pd.slot_begin;
        o << "        if ((lane & 7) == 0 && lane < 24) {";
        for (size_t i = 0; i < deferred.size(); ++i)
            o << " S.redG[warp * " << 3 * nslots << " + 3 * " << deferred[i] << " + (lane >> 3)] = vr[" << i << "];";
        o << " }\n";
    }
    if (store) o << "        regs_store_cpx<LO, " << (rev ? "true" : "false") << ">(p, q, S, xt);\n";
    return o.str();
}

}  // namespace

std::string jit_source(const Plan &P, const PassDesc &pd, int min_blocks)
{
    const bool rev = pd.reverse != 0;
    // distinct phase bodies (templates) and, per phase, (template, first slot)
    std::vector<std::string> tpl;
    std::vector<int> table;
    std::vector<int> stores;   // per phase: it writes phi / lam back to shared memory
    bool lam_valid = rev && pd.lam_src == SRC_LOAD;
    for (int ph = pd.phase_begin; ph < pd.phase_end; ++ph) {
        const DevPhase &phs = P.phases[ph];
        int sb = -1;
        for (int k = phs.op_begin; k < phs.op_end; ++k)
            if ((P.ops[k].type == OP_U2 || P.ops[k].type == OP_GRAD) && (sb < 0 || P.ops[k].slot < sb))
                sb = P.ops[k].slot;
        if (sb < 0) sb = 0;
        const bool fill = cpx_fill(pd) && ph == pd.phase_begin;
        // a phase that leaves phi and lam as they are (the planner's flag) need
        // not store them back, unless it computed phi in registers itself
        const bool store = fill || !(phs.flags & PHF_KEEPS_STATE);
        stores.push_back(store ? 1 : 0);
        const std::string body = phase_body(P, pd, phs, lam_valid, sb, fill, store);
        size_t t = 0;
        while (t < tpl.size() && tpl[t] != body) ++t;
        if (t == tpl.size()) tpl.push_back(body);
        table.push_back((int)t);
        table.push_back(sb);
        if (rev) lam_valid = true;
    }
    const int nph = pd.phase_end - pd.phase_begin;
    std::ostringstream o;
    o << "namespace qtm {\nnamespace {\n";
    o << "// " << nph << " phases, " << tpl.size() << " distinct phase programs\n";
    o << "__constant__ int kPhaseTable[" << (table.empty() ? 2 : table.size()) << "] = {";
    for (size_t i = 0; i < table.size(); ++i) o << (i ? ", " : "") << table[i];
    if (table.empty()) o << "0, 0";
    o << "};\n";
    const int nslots = pd.slot_end - pd.slot_begin;
    o << "template <typename R>\n__device__ __forceinline__ void gen_phases(const TileJob &j, const TileSmem<R> &S, "
         "bool)\n{\n    f2 p[kRegs];\n    f2 q[kRegs];\n"
      << "    // complex-pair matrix table after the tile program's shared memory\n"
      << "    f2 *CT = reinterpret_cast<f2 *>(reinterpret_cast<unsigned char *>(S.phi) + " << cpx_table_offset(P, pd)
      << ");\n    stage_cpx_table(S.mats, CT, " << nslots << ");\n"
      << (cpx_fill(pd) ? "    f2 *TT = CT + " + std::to_string(kCpxSlotPairsHost * std::max(1, nslots)) +
                             ";   // product-state tables, broadcast form\n    stage_cpx_tabs(S.tabs, TT, " +
                             std::to_string(16 * ((P.state_qubits + 3) >> 2)) + ");\n"
                       : std::string())
      << "    __syncthreads();\n";
    o << "    const int tid = threadIdx.x;\n    const int warp = tid >> 5, lane = tid & 31;\n";
    o << "    const uint32_t base = j.base;\n    (void)base; (void)lane; (void)warp; (void)j;\n";
    if (straight_phases(tpl.size(), (size_t)nph)) {
        // every phase its own block, in order (slots as constants through sb),
        // except a periodic stretch, which becomes a loop over its first
        // period with the slots shifted by the stride each time round;
        // complex-pair kernels end a phase with a warp barrier where the next
        // phase's warps hold the same amplitudes (see warp_local_transition)
        auto lo_of = [&](int ph) { return P.phases[pd.phase_begin + ph].lo; };
        auto local = [&](int a, int b) {
            return b < nph && warp_local_barriers() && warp_local_transition(pd.K, lo_of(a), lo_of(b));
        };
        auto barrier = [&](bool warp_only) {
            return warp_only ? "        __syncwarp();\n" : "        __syncthreads();\n";
        };
        // The shared tile changes only in phases that store: two neighbouring
        // phases that both leave it alone need no barrier between them, if
        // every store so far has been published by a CTA barrier (a warp
        // barrier after a store only publishes it within the warp, and the
        // next phase may read another warp's part).  Once a barrier has been
        // left out, warps may be phases apart, so the next barrier is a CTA
        // barrier (a warp barrier before a storing phase would let a warp
        // overwrite what a lagging warp still reads).  The last phase always
        // ends with one: the partial sums are read next.
        bool published = true;   // every store so far seen by every warp
        bool drift = false;      // a barrier left out since the last CTA barrier
        auto after = [&](int a, int b, bool warp_only) -> std::string {
            if (b < nph && !stores[a] && !stores[b] && published) {
                drift = true;
                return "";
            }
            if (drift || !warp_only) {
                drift = false;
                published = true;
                return barrier(false);
            }
            if (stores[a]) published = false;
            return barrier(true);
        };
        const Repeat rp = repeat_loops() ? find_repeat(table, nph) : Repeat{};
        const int loop_end = rp.reps >= 2 ? rp.start + rp.period * rp.reps : 0;
        for (int ph = 0; ph < nph; ++ph) {
            if (rp.reps >= 2 && ph == rp.start) {
                o << "    // phases " << rp.start << " .. " << loop_end - 1 << ": " << rp.reps << " x the next "
                  << rp.period << " phase programs, slots + " << rp.stride << " each time\n";
                o << "#pragma unroll 1\n    for (int it = 0; it < " << rp.reps << "; ++it) {\n";
                for (int i = 0; i < rp.period; ++i) {
                    const int a = rp.start + i;
                    // the last program of the period hands over to the period's first
                    // (next time round) or to the phase after the loop
                    const bool wl = i + 1 < rp.period ? local(a, a + 1)
                                                      : local(a, rp.start) && loop_end < nph && local(a, loop_end);
                    o << "    {\n        const int sb = " << table[2 * a + 1] << " + it * " << rp.stride
                      << ";\n        (void)sb;\n" << tpl[table[2 * a]] << barrier(wl) << "    }\n";
                    if (i + 1 == rp.period) {   // the loop's last barrier hands over to the phase after it
                        published = !wl;   // only a CTA barrier publishes the loop's stores
                        drift = false;
                    }
                }
                o << "    }\n";
                ph = loop_end - 1;
                continue;
            }
            o << "    {\n        const int sb = " << table[2 * ph + 1] << ";\n        (void)sb;\n"
              << tpl[table[2 * ph]] << after(ph, ph + 1, local(ph, ph + 1)) << "    }\n";
        }
    } else {
        o << "#pragma unroll 1\n    for (int ph = 0; ph < " << nph << "; ++ph) {\n";
        o << "        const int sb = kPhaseTable[2 * ph + 1];\n        (void)sb;\n";
        o << "        switch (kPhaseTable[2 * ph]) {\n";
        for (size_t t = 0; t < tpl.size(); ++t) {
            o << "        " << (t + 1 < tpl.size() ? "case " + std::to_string(t) + ":" : "default:") << " {\n";
            o << tpl[t] << "        } break;\n";
        }
        o << "        }\n        __syncthreads();\n    }\n";
    }
    o << "}\n}  // namespace\n}  // namespace qtm\n\n";
    o << "extern \"C\" __global__ void __launch_bounds__(256, " << min_blocks << ") qtm_gen_pass("
      << "const __grid_constant__ qtm::PassArgs a, const __grid_constant__ CUtensorMap tm_phi, "
      << "const __grid_constant__ CUtensorMap tm_lam)\n{\n";
    o << "    qtm::pass_body<float, " << (rev ? "true" : "false") << (cpx_fill(pd) ? ", false" : "")
      << ">(a, &tm_phi, &tm_lam, "
      << "[](const qtm::TileJob &j, const qtm::TileSmem<float> &S, bool lv) { qtm::gen_phases<float>(j, S, lv); "
         "});\n}\n";
    return o.str();
}

size_t jit_smem_bytes_cpx(const Plan &P, const PassDesc &pd)
{
    return cpx_table_offset(P, pd) + 1024 + (size_t)8 * kCpxSlotPairsHost * std::max(1, pd.slot_end - pd.slot_begin) +
           (cpx_fill(pd) ? (size_t)256 * ((P.state_qubits + 3) >> 2) : 0);
}


// ---- NVRTC and the driver API ---------------------------------------------------

namespace {

struct Nvrtc {
    bool ok = false;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

const Nvrtc &nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
        n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
        n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
        n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    });
    return n;
}

struct Drv {
    bool ok = false;
    PFN_cuModuleLoadData_v2000 load = nullptr;
    PFN_cuModuleGetFunction_v2000 get = nullptr;
    PFN_cuModuleUnload_v2000 unload = nullptr;
    PFN_cuFuncSetAttribute_v9000 set_attr = nullptr;
    PFN_cuLaunchKernel_v4000 launch = nullptr;
    PFN_cuLaunchKernelEx_v11060 launch_ex = nullptr;   // optional: programmatic dependent launches
};

const Drv &drv()
{
    static Drv d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto get = [](const char *name, void **fn) {
            cudaDriverEntryPointQueryResult q;
            return cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
                   q == cudaDriverEntryPointSuccess;
        };
        d.ok = get("cuModuleLoadData", reinterpret_cast<void **>(&d.load)) &&
               get("cuModuleGetFunction", reinterpret_cast<void **>(&d.get)) &&
               get("cuModuleUnload", reinterpret_cast<void **>(&d.unload)) &&
               get("cuFuncSetAttribute", reinterpret_cast<void **>(&d.set_attr)) &&
               get("cuLaunchKernel", reinterpret_cast<void **>(&d.launch));
        if (!get("cuLaunchKernelEx", reinterpret_cast<void **>(&d.launch_ex))) d.launch_ex = nullptr;
    });
    return d;
}

uint64_t fnv1a(const std::string &s)
{
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : s) { h ^= c; h *= 1099511628211ull; }
    return h;
}

std::string cache_dir()
{
    const char *e = std::getenv("QTM_JIT_CACHE");
    if (e && *e) return e;
    return "/tmp/qtm_jit_cache";
}

bool read_file(const std::string &path, std::vector<char> &out)
{
    std::ifstream f(path, std::ios::binary);
    if (!f) return false;
    out.assign(std::istreambuf_iterator<char>(f), std::istreambuf_iterator<char>());
    return !out.empty();
}

}  // namespace

bool jit_available() { return nvrtc().ok && drv().ok; }
bool jit_nvrtc_available() { return nvrtc().ok; }

bool jit_compile(const std::string &body, std::vector<char> &cubin, std::string &log)
{
    const Nvrtc &N = nvrtc();
    if (!N.ok) { log = "NVRTC not found"; return false; }
    const std::string src = std::string(kJitPrelude) + "\n" + body;
    // QTM_JIT_VERBOSE=1: bypass the cache and print ptxas resource usage
    const char *vb = std::getenv("QTM_JIT_VERBOSE");
    const bool verbose = vb && *vb == '1';
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
    const int nopts = verbose ? 4 : 3;
    char key[32];
    std::snprintf(key, sizeof(key), "%016llx", (unsigned long long)fnv1a(src));
    const std::string dir = cache_dir(), path = dir + "/" + key + ".cubin";
    if (!verbose && read_file(path, cubin)) return true;
    nvrtcProgram prog;
    if (N.create(&prog, src.c_str(), "qtm_gen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return false;
    }
    const nvrtcResult r = N.compile(prog, nopts, opts);
    size_t ls = 0;
    N.log_size(prog, &ls);
    if (ls > 1) {
        log.resize(ls);
        N.log(prog, &log[0]);
    }
    bool ok = r == NVRTC_SUCCESS;
    if (ok) {
        size_t cs = 0;
        ok = N.cubin_size(prog, &cs) == NVRTC_SUCCESS && cs > 0;
        if (ok) {
            cubin.resize(cs);
            ok = N.cubin(prog, cubin.data()) == NVRTC_SUCCESS;
        }
    }
    N.destroy(&prog);
    if (verbose) std::fprintf(stderr, "%s\n", log.c_str());
    if (ok) {   // best-effort disk cache keyed by the source hash
        ::mkdir(dir.c_str(), 0755);
        const std::string tmp = path + ".tmp" + std::to_string((unsigned long long)::getpid());
        std::ofstream f(tmp, std::ios::binary);
        if (f) {
            f.write(cubin.data(), (std::streamsize)cubin.size());
            f.close();
            std::rename(tmp.c_str(), path.c_str());
        }
    }
    return ok;
}

bool jit_load(const std::vector<char> &cubin, int smem, JitKernel &k, std::string &err)
{
    const Drv &D = drv();
    if (!D.ok) { err = "driver entry points unavailable"; return false; }
    CUmodule mod = nullptr;
    CUfunction fn = nullptr;
    if (D.load(&mod, cubin.data()) != CUDA_SUCCESS) { err = "cuModuleLoadData failed"; return false; }
    if (D.get(&fn, mod, "qtm_gen_pass") != CUDA_SUCCESS ||
        D.set_attr(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, smem) != CUDA_SUCCESS) {
        D.unload(mod);
        err = "kernel lookup / attribute failed";
        return false;
    }
    k.mod = mod;
    k.fn = fn;
    k.smem = smem;
    return true;
}

void jit_unload(JitKernel &k)
{
    if (k.mod && drv().ok) drv().unload(static_cast<CUmodule>(k.mod));
    k.mod = nullptr;
    k.fn = nullptr;
}

cudaError_t jit_launch(const JitKernel &k, const PassArgs &a, const CUtensorMap &tm_phi, const CUtensorMap &tm_lam,
                       cudaStream_t s, bool pdl)
{
    PassArgs args = a;
    CUtensorMap t0 = tm_phi, t1 = tm_lam;
    void *params[] = {&args, &t0, &t1};
    const unsigned grid = (unsigned)a.B * (unsigned)a.tiles, block = 1u << (a.K - 4);
    CUresult r;
    if (pdl && drv().launch_ex) {
        CUlaunchAttribute at[1];
        at[0].id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
        at[0].value.programmaticStreamSerializationAllowed = 1;
        CUlaunchConfig cfg{};
        cfg.gridDimX = grid; cfg.gridDimY = 1; cfg.gridDimZ = 1;
        cfg.blockDimX = block; cfg.blockDimY = 1; cfg.blockDimZ = 1;
        cfg.sharedMemBytes = (unsigned)a.smem_bytes;
        cfg.hStream = reinterpret_cast<CUstream>(s);
        cfg.attrs = at;
        cfg.numAttrs = 1;
        r = drv().launch_ex(&cfg, static_cast<CUfunction>(k.fn), params, nullptr);
    } else {
        r = drv().launch(static_cast<CUfunction>(k.fn), grid, 1, 1, block, 1, 1, (unsigned)a.smem_bytes,
                         reinterpret_cast<CUstream>(s), params, nullptr);
    }
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorLaunchFailure;
}

}  // namespace qtm
