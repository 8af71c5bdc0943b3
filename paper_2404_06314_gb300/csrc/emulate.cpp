// Host-side interpreter of a plan's device schedule (FP64).
//
// Executes exactly the passes, tiles, phases and ops the CUDA kernels execute
// -- tile gathers over S = [0,l) U [h,h+m), per-tile constant operands, the
// analytic product-state init, register-group locality, skip-apply, partial
// sums per tile, the SO(3) finalize and the chain rule -- in plain scalar
// loops.  It exists to validate the planner without a GPU and is never called
// by qtm_forward / qtm_adjoint.
#include <cmath>
#include <complex>
#include <stdexcept>
#include <vector>

#include "finalize_math.h"
#include "plan.h"

namespace qtm {

namespace {

using cd = std::complex<double>;

struct Mat2 { cd a[2][2]; };

Mat2 mul(const Mat2 &A, const Mat2 &B)
{
    Mat2 C;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) C.a[r][c] = A.a[r][0] * B.a[0][c] + A.a[r][1] * B.a[1][c];
    return C;
}

Mat2 rot_matrix(int kind, double t)
{
    double c = std::cos(0.5 * t), s = std::sin(0.5 * t);
    Mat2 m;
    if (kind == QTM_RX) { m.a[0][0] = c; m.a[0][1] = cd(0, -s); m.a[1][0] = cd(0, -s); m.a[1][1] = c; }
    else if (kind == QTM_RY) { m.a[0][0] = c; m.a[0][1] = -s; m.a[1][0] = s; m.a[1][1] = c; }
    else { m.a[0][0] = cd(c, -s); m.a[0][1] = 0; m.a[1][0] = 0; m.a[1][1] = cd(c, s); }
    return m;
}

Mat2 dag(const Mat2 &m)
{
    Mat2 d;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) d.a[r][c] = std::conj(m.a[c][r]);
    return d;
}

double rot_angle(const Rot &r, const double *xb, const double *w)
{
    double t = r.coef;
    if (r.w_idx >= 0) t *= w[r.w_idx];
    if (r.x_idx >= 0) t *= xb[r.x_idx];
    return t;
}

Mat2 run_matrix(const Plan &P, int run, const double *xb, const double *w)
{
    Mat2 U;
    U.a[0][0] = 1; U.a[0][1] = 0; U.a[1][0] = 0; U.a[1][1] = 1;
    const Run &R = P.runs[run];
    for (int i = R.rot_begin; i < R.rot_end; ++i)
        U = mul(rot_matrix(P.rots[i].kind, rot_angle(P.rots[i], xb, w)), U);
    return U;
}

uint64_t deposit_bits(uint64_t v, uint64_t mask)
{
    uint64_t r = 0;
    for (int b = 0; mask; ++b) {
        uint64_t low = mask & (~mask + 1);
        if ((v >> b) & 1) r |= low;
        mask &= mask - 1;
    }
    return r;
}

struct Emu {
    const Plan &P;
    int B;
    const double *x, *w, *gE;
    int NS;                    // per-sample stride (2^state_qubits)
    std::vector<cd> phi, lam;  // [B][NS]
    std::vector<double> Epart;    // [B][tiles][M]
    std::vector<double> Gpart;    // [B][runs][tiles][3]

    Emu(const Plan &p, int b, const double *x_, const double *w_, const double *gE_)
        : P(p), B(b), x(x_), w(w_), gE(gE_)
    {
        NS = 1 << P.state_qubits;
        phi.assign((size_t)B * NS, 0.0);
        lam.assign((size_t)B * NS, 0.0);
        Epart.assign((size_t)B * P.tiles_per_sample * P.n_obs, 0.0);
        Gpart.assign((size_t)B * P.runs.size() * P.tiles_per_sample * 3, 0.0);
    }

    const double *xb(int b) const { return x + (size_t)b * P.n_inputs; }

    // analytic prefix state at global index y, with the first `ents` folded
    // entanglers applied
    cd analytic(const PassDesc &pd, uint64_t y, const std::vector<cd> &u) const
    {
        uint64_t xx = y;
        int sign = 0;
        if (pd.amap_lin >= 0) {   // closed form, exactly as the kernel evaluates it
            uint32_t yy = (uint32_t)y, x32 = 0;
            for (int k = 0; k < pd.amap_lin; ++k) {
                const MaskTerm t = P.amap_terms[pd.amap_begin + k];
                x32 ^= (t.d >= 0 ? (yy >> t.d) : (yy << -t.d)) & t.mask;
            }
            int par = __builtin_popcount(x32 & pd.amap_dlin);
            for (int k = 0; k < pd.amap_quad; ++k) {
                const MaskTerm t = P.amap_terms[pd.amap_begin + pd.amap_lin + k];
                par += __builtin_popcount(x32 & (x32 >> t.d) & t.mask);
            }
            xx = x32;
            sign = par & 1;
        } else {
            for (int k = pd.analytic_ents - 1; k >= 0; --k) {
                const Ent &e = P.pass_ents[pd.ents_begin + k];
                if (e.kind == QTM_CNOT) xx ^= ((xx >> e.a) & 1ull) << e.b;
                else sign ^= (int)((xx >> e.a) & (xx >> e.b) & 1ull);
            }
        }
        cd a = 1.0;
        for (int q = 0; q < P.state_qubits; ++q) a *= u[2 * q + ((xx >> q) & 1)];
        return sign ? -a : a;
    }

    // (P psi)_y of a string with X/Y factors: i^ny (-1)^popcount(x & zmask) psi_x, x = y ^ xmask
    cd pauli_apply(const PauliTerm &t, const cd *psi, uint64_t y) const
    {
        const uint64_t xx = y ^ t.xmask;
        cd v = psi[xx];
        if (__builtin_popcountll(xx & t.zmask) & 1) v = -v;
        static const cd ipow[4] = {cd(1, 0), cd(0, 1), cd(-1, 0), cd(0, -1)};
        return ipow[t.ny & 3] * v;
    }

    // X/Y strings on the final state: expectation values added to E, and the
    // costate part written to lam (what the device does between the passes)
    void pauli_expvals(double *E) const
    {
        for (int b = 0; b < B; ++b) {
            const cd *psi = &phi[(size_t)b * NS];
            for (const PauliTerm &t : P.pterms) {
                double s = 0.0;
                for (uint64_t y = 0; y < (uint64_t)NS; ++y) s += std::real(std::conj(psi[y]) * pauli_apply(t, psi, y));
                E[(size_t)b * P.n_obs + t.obs] += t.coef * s;
            }
        }
    }

    void pauli_costate()
    {
        for (int b = 0; b < B; ++b) {
            const cd *psi = &phi[(size_t)b * NS];
            cd *la = &lam[(size_t)b * NS];
            for (uint64_t y = 0; y < (uint64_t)NS; ++y) {
                cd v = 0.0;
                for (const PauliTerm &t : P.pterms) v += gE[(size_t)b * P.n_obs + t.obs] * t.coef * pauli_apply(t, psi, y);
                la[y] = v;
            }
        }
    }

    std::vector<cd> prefix_factors(int b) const
    {
        std::vector<cd> u(2 * P.state_qubits);
        for (int q = 0; q < P.state_qubits; ++q) {
            u[2 * q] = 1.0; u[2 * q + 1] = 0.0;
            if (q < P.n && P.prefix_run_of_q[q] >= 0) {
                Mat2 U = run_matrix(P, P.prefix_run_of_q[q], xb(b), w);
                u[2 * q] = U.a[0][0]; u[2 * q + 1] = U.a[1][0];
            }
        }
        return u;
    }

    void run_pass(const PassDesc &pd)
    {
        const int K = pd.K, T = 1 << K;
        const int tiles = P.tiles_per_sample;
        uint64_t Smask = ((1ull << pd.l) - 1) | (pd.m ? (((1ull << pd.m) - 1) << pd.h) : 0);
        uint64_t outmask = ((1ull << P.state_qubits) - 1) & ~Smask;
        std::vector<cd> tp(T), tl(T);
        for (int b = 0; b < B; ++b) {
            std::vector<cd> u = prefix_factors(b);
            // matrices of this pass's runs
            std::vector<Mat2> mats;
            for (int s = pd.slot_begin; s < pd.slot_end; ++s) {
                Mat2 U = run_matrix(P, P.slot_runs[s], xb(b), w);
                mats.push_back(pd.reverse ? dag(U) : U);
            }
            for (int t = 0; t < tiles; ++t) {
                uint64_t base = deposit_bits((uint64_t)t, outmask);
                auto gidx = [&](int e) { return base | deposit_bits((uint64_t)e, Smask); };
                cd *ph = &phi[(size_t)b * NS], *la = &lam[(size_t)b * NS];
                for (int e = 0; e < T; ++e) {
                    uint64_t y = gidx(e);
                    tp[e] = pd.phi_src == SRC_ANALYTIC ? analytic(pd, y, u) : ph[y];
                    if (pd.lam_src == SRC_LOAD) tl[e] = la[y];
                }
                auto bitval = [&](int operand, int e) -> int {
                    if (operand >= kFixed) return (int)((base >> (operand - kFixed)) & 1ull);
                    return (e >> operand) & 1;
                };
                for (int phz = pd.phase_begin; phz < pd.phase_end; ++phz) {
                    const DevPhase &phs = P.phases[phz];
                    auto in_group = [&](int p) { return p >= phs.lo && p < phs.lo + kRegBits; };
                    for (int o = phs.op_begin; o < phs.op_end; ++o) {
                        const DevOp &op = P.ops[o];
                        switch (op.type) {
                        case OP_U2: {
                            if (!in_group(op.a)) throw std::runtime_error("U2 outside register group");
                            const Mat2 &m = mats[op.slot];
                            int bit = 1 << op.a;
                            for (int e = 0; e < T; ++e)
                                if (!(e & bit)) {
                                    cd a0 = tp[e], a1 = tp[e | bit];
                                    tp[e] = m.a[0][0] * a0 + m.a[0][1] * a1;
                                    tp[e | bit] = m.a[1][0] * a0 + m.a[1][1] * a1;
                                }
                            break;
                        }
                        case OP_GRAD: {
                            if (!in_group(op.a)) throw std::runtime_error("GRAD outside register group");
                            int bit = 1 << op.a;
                            double vx = 0, vy = 0, vz = 0;
                            for (int e = 0; e < T; ++e)
                                if (!(e & bit)) {
                                    cd a0 = tp[e], a1 = tp[e | bit], b0 = tl[e], b1 = tl[e | bit];
                                    vz += std::imag(std::conj(b0) * a0) - std::imag(std::conj(b1) * a1);
                                    vx += std::imag(std::conj(b0) * a1) + std::imag(std::conj(b1) * a0);
                                    vy += -std::real(std::conj(b0) * a1) + std::real(std::conj(b1) * a0);
                                }
                            int run = P.slot_runs[pd.slot_begin + op.slot];
                            double *g = &Gpart[(((size_t)b * P.runs.size() + run) * tiles + t) * 3];
                            g[0] += vx; g[1] += vy; g[2] += vz;
                            if (!(op.flags & OPF_SKIP_APPLY)) {
                                const Mat2 &m = mats[op.slot];
                                for (int e = 0; e < T; ++e)
                                    if (!(e & bit)) {
                                        cd a0 = tp[e], a1 = tp[e | bit];
                                        tp[e] = m.a[0][0] * a0 + m.a[0][1] * a1;
                                        tp[e | bit] = m.a[1][0] * a0 + m.a[1][1] * a1;
                                        a0 = tl[e]; a1 = tl[e | bit];
                                        tl[e] = m.a[0][0] * a0 + m.a[0][1] * a1;
                                        tl[e | bit] = m.a[1][0] * a0 + m.a[1][1] * a1;
                                    }
                            }
                            break;
                        }
                        case OP_CZ:
                            for (int e = 0; e < T; ++e)
                                if (bitval(op.a, e) & bitval(op.b, e)) {
                                    tp[e] = -tp[e];
                                    if (pd.reverse) tl[e] = -tl[e];
                                }
                            break;
                        case OP_DIAG:
                            for (int k = op.a; k < op.a + op.b; ++k) {
                                const DiagPair dp = P.diag_pairs[k];
                                for (int e = 0; e < T; ++e)
                                    if (bitval(dp.a, e) & bitval(dp.b, e)) {
                                        tp[e] = -tp[e];
                                        if (pd.reverse) tl[e] = -tl[e];
                                    }
                            }
                            break;
                        case OP_CNOT: {
                            if (!in_group(op.b)) throw std::runtime_error("CNOT target outside group");
                            int bit = 1 << op.b;
                            for (int e = 0; e < T; ++e)
                                if (!(e & bit) && bitval(op.a, e)) {
                                    std::swap(tp[e], tp[e | bit]);
                                    if (pd.reverse) std::swap(tl[e], tl[e | bit]);
                                }
                            break;
                        }
                        case OP_EXPVAL:
                            for (int e = 0; e < T; ++e) {
                                uint64_t y = gidx(e);
                                double p = std::norm(tp[e]);
                                for (const Term &tm : P.terms) {
                                    int par = __builtin_popcountll(y & tm.zmask) & 1;
                                    Epart[((size_t)b * tiles + t) * P.n_obs + tm.obs] +=
                                        (par ? -tm.coef : tm.coef) * p;
                                }
                            }
                            break;
                        case OP_COSTATE:
                            for (int e = 0; e < T; ++e) {
                                uint64_t y = gidx(e);
                                double d = 0.0;
                                for (const Term &tm : P.terms) {
                                    int par = __builtin_popcountll(y & tm.zmask) & 1;
                                    double k = gE[(size_t)b * P.n_obs + tm.obs] * tm.coef;
                                    d += par ? -k : k;
                                }
                                tl[e] = (op.flags & OPF_ACCUMULATE) ? tl[e] + d * tp[e] : d * tp[e];
                            }
                            break;
                        default:
                            throw std::runtime_error("bad op");
                        }
                    }
                }
                for (int e = 0; e < T; ++e) {
                    uint64_t y = gidx(e);
                    if (pd.store_phi) ph[y] = tp[e];
                    if (pd.store_lam) la[y] = tl[e];
                }
            }
        }
    }
};

}  // namespace

// FP64 interpretation of the fused schedule.  E [B][M], gx [B][n_in],
// gw [B][P] per sample (any may be NULL; gE may be NULL for forward only).
qtm_status emulate_plan(const Plan &P, int B, const double *x, const double *w, const double *gE,
                        double *E, double *gx, double *gw, std::string &err)
{
    if (P.path != QTM_PATH_FUSED) { err = "emulation covers the fused path"; return QTM_EUNSUPPORTED; }
    if (P.state_qubits > 24) { err = "emulation limited to n <= 24"; return QTM_EUNSUPPORTED; }
    try {
        Emu em(P, B, x, w, gE);
        for (const auto &pd : P.fwd) em.run_pass(pd);
        const int tiles = P.tiles_per_sample;
        if (E)
            for (int b = 0; b < B; ++b)
                for (int m = 0; m < P.n_obs; ++m) {
                    double s = 0.0;
                    for (int t = 0; t < tiles; ++t) s += em.Epart[((size_t)b * tiles + t) * P.n_obs + m];
                    E[(size_t)b * P.n_obs + m] = s;
                }
        if (E && !P.pterms.empty()) em.pauli_expvals(E);
        if (!gE) return QTM_OK;
        if (!P.pterms.empty()) em.pauli_costate();
        for (const auto &pd : P.rev) em.run_pass(pd);
        std::vector<double> abar(P.rots.size());
        for (int b = 0; b < B; ++b) {
            const double *xb = x + (size_t)b * P.n_inputs;
            for (size_t r = 0; r < P.runs.size(); ++r) {
                double v[3] = {0, 0, 0};
                for (int t = 0; t < tiles; ++t)
                    for (int c = 0; c < 3; ++c)
                        v[c] += em.Gpart[(((size_t)b * P.runs.size() + r) * tiles + t) * 3 + c];
                const Run &R = P.runs[r];
                int m = R.rot_end - R.rot_begin;
                std::vector<int> kv(m);
                std::vector<double> tv(m), out(m);
                for (int i = 0; i < m; ++i) {
                    kv[i] = P.rots[R.rot_begin + i].kind;
                    tv[i] = rot_angle(P.rots[R.rot_begin + i], xb, w);
                }
                run_angle_grads(m, kv.data(), tv.data(), v, out.data());
                for (int i = 0; i < m; ++i) abar[R.rot_begin + i] = out[i];
            }
            if (gw)
                for (int j = 0; j < P.n_weights; ++j) {
                    double s = 0.0;
                    for (int k = P.w_ptr[j]; k < P.w_ptr[j + 1]; ++k) {
                        const Rot &r = P.rots[P.w_rots[k]];
                        s += abar[P.w_rots[k]] * r.coef * (r.x_idx >= 0 ? xb[r.x_idx] : 1.0);
                    }
                    gw[(size_t)b * P.n_weights + j] = s;
                }
            if (gx)
                for (int i = 0; i < P.n_inputs; ++i) {
                    double s = 0.0;
                    for (int k = P.x_ptr[i]; k < P.x_ptr[i + 1]; ++k) {
                        const Rot &r = P.rots[P.x_rots[k]];
                        s += abar[P.x_rots[k]] * r.coef * (r.w_idx >= 0 ? w[r.w_idx] : 1.0);
                    }
                    gx[(size_t)b * P.n_inputs + i] = s;
                }
        }
    } catch (const std::exception &ex) {
        err = ex.what();
        return QTM_EINVAL;
    }
    return QTM_OK;
}

}  // namespace qtm
