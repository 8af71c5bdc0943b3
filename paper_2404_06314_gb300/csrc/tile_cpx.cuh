// Complex-pair registers for the one-sample specialised pass kernels.
//
// A thread's 16 amplitudes (register bits [lo, lo+4) of a phase) are held as
// 16 f32x2 register pairs, each one complex amplitude (re, im): the layout of
// the amplitude in shared memory, so loads and stores move whole pairs.  A
// complex product is two f32x2 instructions on the pair and its lane swap:
//     u x = (u.re, u.re) * (x.re, x.im) + (-u.im, u.im) * (x.im, x.re),
// and Blackwell's f32x2 FMA takes the swapped operand without a register move.
// Every register bit is alike: a gate on register bit RB pairs whole
// registers, a CNOT permutes them, a CZ sign flips both lanes of a register.
// The sample, the shared-memory layout and the tile program (tile.cuh) are
// those of the one-sample kernel.
#pragma once

#include "f32x2.cuh"

namespace qtm {

namespace {

// Every run matrix is special unitary, U = [[a, -conj(b)], [b, conj(a)]]
// (a product of rotations; U^dagger has the same form with a -> conj(a),
// b -> -b), so its four entries in broadcast form, (e.re, e.re) and
// (-e.im, e.im), hold six distinct pairs: A_r = (a.re, a.re),
// A_n = (-a.im, a.im), B_r = (b.re, b.re), B_n = (-b.im, b.im) and the
// negations -B_r, -A_n.  A slot keeps those six (of eight places).
constexpr int kCpxSlotPairs = 8;

// Complex-pair table of every run slot from the staged matrices (U or U^dagger).
__device__ __forceinline__ void stage_cpx_table(const Cx<float> *mats, f2 *tab, int nslots)
{
    for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
        f2 *t = tab + kCpxSlotPairs * s;
        const Cx<float> a = mats[4 * s], b = mats[4 * s + 2];
        t[0] = pack2(a.x, a.x);     // A_r
        t[1] = pack2(-a.y, a.y);    // A_n
        t[2] = pack2(b.x, b.x);     // B_r
        t[3] = pack2(-b.y, b.y);    // B_n
        t[4] = pack2(-b.x, -b.x);   // -B_r
        t[5] = pack2(a.y, -a.y);    // -A_n
    }
}

// Shared-space accesses of one amplitude (8 bytes) or two neighbouring ones (16 bytes).
__device__ __forceinline__ f2 lds_f2(uint32_t addr)
{
    f2 v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void lds_f2x2(uint32_t addr, f2 &a, f2 &b)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}
__device__ __forceinline__ void sts_f2(uint32_t addr, f2 v)
{
    asm volatile("st.shared.b64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
__device__ __forceinline__ void sts_f2x2(uint32_t addr, f2 a, f2 b)
{
    asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

// Registers <-> shared tile for register group LO (compile time).  Group 0:
// two neighbouring amplitudes per 16-byte access (the swizzle keeps 16-byte
// chunks whole); other groups: one 8-byte access per amplitude.
template <int LO, bool LAM>
__device__ __forceinline__ void regs_load_cpx(f2 (&p)[kRegs], f2 (&q)[kRegs], const TileSmem<float> &T, uint32_t xt)
{
    const uint32_t ph = smem_u32(T.phi), lm = smem_u32(T.lam);
    if constexpr (LO == 0) {
#pragma unroll
        for (int k = 0; k < kRegs / 2; ++k) {
            const uint32_t o = 8u * (uint32_t)swz<float>((int)xt + 2 * k);
            lds_f2x2(ph + o, p[2 * k], p[2 * k + 1]);
            if (LAM) lds_f2x2(lm + o, q[2 * k], q[2 * k + 1]);
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) {
            const uint32_t o = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)jj << LO)));
            p[jj] = lds_f2(ph + o);
            if (LAM) q[jj] = lds_f2(lm + o);
        }
    }
}

template <int LO, bool LAM>
__device__ __forceinline__ void regs_store_cpx(const f2 (&p)[kRegs], const f2 (&q)[kRegs], const TileSmem<float> &T,
                                               uint32_t xt)
{
    const uint32_t ph = smem_u32(T.phi), lm = smem_u32(T.lam);
    if constexpr (LO == 0) {
#pragma unroll
        for (int k = 0; k < kRegs / 2; ++k) {
            const uint32_t o = 8u * (uint32_t)swz<float>((int)xt + 2 * k);
            sts_f2x2(ph + o, p[2 * k], p[2 * k + 1]);
            if (LAM) sts_f2x2(lm + o, q[2 * k], q[2 * k + 1]);
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) {
            const uint32_t o = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)jj << LO)));
            sts_f2(ph + o, p[jj]);
            if (LAM) sts_f2(lm + o, q[jj]);
        }
    }
}

// lam only (the generated first phase of an analytic pass computes phi itself).
template <int LO>
__device__ __forceinline__ void regs_load_cpx_lam(f2 (&q)[kRegs], const TileSmem<float> &T, uint32_t xt)
{
    const uint32_t lm = smem_u32(T.lam);
    if constexpr (LO == 0) {
#pragma unroll
        for (int k = 0; k < kRegs / 2; ++k)
            lds_f2x2(lm + 8u * (uint32_t)swz<float>((int)xt + 2 * k), q[2 * k], q[2 * k + 1]);
    } else {
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) q[jj] = lds_f2(lm + 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)jj << LO))));
    }
}

// Product-state tables in broadcast form for complex products: entry e as
// (e.re, e.re), (-e.im, e.im), so that amp <- e * amp is
// fma2((e.re, e.re), amp, (-e.im, e.im) * swap(amp)).
__device__ __forceinline__ void stage_cpx_tabs(const Cx<float> *tabs, f2 *tt, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Cx<float> e = tabs[i];
        tt[2 * i] = pack2(e.x, e.x);
        tt[2 * i + 1] = pack2(-e.y, e.y);
    }
}

// amp <- e * amp with e read in broadcast form at shared address addr.
__device__ __forceinline__ f2 cmul_tab(uint32_t addr, f2 amp)
{
    f2 er, en;
    lds_f2x2(addr, er, en);
    return fma2(er, amp, mul2(en, swap2(amp)));
}

// The special-unitary product on one register pair (x0, x1):
// y0 = a x0 - conj(b) x1 = A_r x0 + A_n s0 - B_r x1 + B_n s1,
// y1 = b x0 + conj(a) x1 = B_r x0 + B_n s0 + A_r x1 - A_n s1 (s = lane swap).
template <int RB>
__device__ __forceinline__ void su2_apply(f2 (&a)[kRegs], f2 A_r, f2 A_n, f2 B_r, f2 B_n, f2 NB_r, f2 NA_n)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RB)) continue;
        const f2 x0 = a[j], x1 = a[j | (1 << RB)];
        const f2 s0 = swap2(x0), s1 = swap2(x1);
        a[j] = fma2(A_r, x0, fma2(A_n, s0, fma2(NB_r, x1, mul2(B_n, s1))));
        a[j | (1 << RB)] = fma2(B_r, x0, fma2(B_n, s0, fma2(A_r, x1, mul2(NA_n, s1))));
    }
}

// a <- U a on register bit RB with U's six pairs from the slot table t.
template <int RB>
__device__ __forceinline__ void u2_cpx(f2 (&a)[kRegs], const f2 *t)
{
    f2 A_r, A_n, B_r, B_n, NB_r, NA_n;
    lds_table2<true>(t, A_r, A_n); lds_table2<true>(t + 2, B_r, B_n); lds_table2<true>(t + 4, NB_r, NA_n);
    su2_apply<RB>(a, A_r, A_n, B_r, B_n, NB_r, NA_n);
}

// (vx, vy, vz) on register bit RB, the same sums as grad_acc in tile.cuh:
// with b = lam and a = phi, Im(conj(b) a) = lane0 - lane1 of b * swap(a) and
// Re(conj(b) a) = lane0 + lane1 of b * a.  Z's second term enters with a
// plus sign as swap(b1) * a1 (whose lane0 - lane1 is minus that of
// b1 * swap(a1)), and X's two terms add, so Z and X each take one
// accumulator: four instead of six.
template <int RB>
__device__ __forceinline__ void grad_cpx(const f2 (&a)[kRegs], const f2 (&b)[kRegs], float &vx, float &vy, float &vz)
{
    f2 zs, xs, yp, yn;
#pragma unroll
    for (int j = 0, first = 1; j < kRegs; ++j) {
        if (j & (1 << RB)) continue;
        const f2 a0 = a[j], a1 = a[j | (1 << RB)], b0 = b[j], b1 = b[j | (1 << RB)];
        const f2 s0 = swap2(a0), s1 = swap2(a1);
        if (first) {   // the first pair starts the accumulators (no zero fill)
            zs = fma2(swap2(b1), a1, mul2(b0, s0));
            xs = fma2(b1, s0, mul2(b0, s1));
            yp = mul2(b1, a0); yn = mul2(b0, a1);
            first = 0;
        } else {
            zs = fma2(b0, s0, zs); zs = fma2(swap2(b1), a1, zs);
            xs = fma2(b0, s1, xs); xs = fma2(b1, s0, xs);
            yp = fma2(b1, a0, yp); yn = fma2(b0, a1, yn);
        }
    }
    const f2 Y = sub2(yp, yn);
    vz = lane0(zs) - lane1(zs);
    vx = lane0(xs) - lane1(xs);
    vy = lane0(Y) + lane1(Y);
}

// CNOT with control and target both register bits: a fixed register permutation.
template <int RC, int RT>
__device__ __forceinline__ void cnot_static_cpx(f2 (&a)[kRegs])
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        if ((jj & (1 << RT)) || !(jj & (1 << RC))) continue;
        const f2 t = a[jj];
        a[jj] = a[jj | (1 << RT)];
        a[jj | (1 << RT)] = t;
    }
}

// CNOT on target register bit RT with a control bit c known per thread.
template <int RT>
__device__ __forceinline__ void cnot_cpx(f2 (&a)[kRegs], int c)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RT)) continue;
        const f2 t0 = a[j], t1 = a[j | (1 << RT)];
        a[j] = c ? t1 : t0;
        a[j | (1 << RT)] = c ? t0 : t1;
    }
}

// Negate amplitude jj where bit jj of m is set (phi, and lam in reverse).
template <bool REV>
__device__ __forceinline__ void flip_cpx(f2 (&p)[kRegs], f2 (&q)[kRegs], uint32_t m)
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        const uint32_t sb = (m << (31 - jj)) & 0x80000000u;   // bit jj of m as a sign bit
        const f2 s = ((f2)sb << 32) | sb;                     // in both lanes
        p[jj] ^= s;
        if (REV) q[jj] ^= s;
    }
}

// Negate register J (phi, and lam in reverse) by the sign word s (0 or 0x80000000).
template <bool REV, int J>
__device__ __forceinline__ void flip_reg(f2 (&p)[kRegs], f2 (&q)[kRegs], uint32_t s)
{
    const f2 v = ((f2)s << 32) | s;
    p[J] ^= v;
    if (REV) q[J] ^= v;
}

// ---- the phase interpreter on complex pairs (complex64 general kernels) ----

// a <- U a on register bit RB with U read as four complex entries (the
// general kernels' staged matrices) and put in broadcast form here.
template <int RB>
__device__ __forceinline__ void u2_cpx_m(f2 (&a)[kRegs], const Cx<float> *m)
{
    const Cx<float> u00 = m[0], u10 = m[2];   // special unitary: u01 = -conj(u10), u11 = conj(u00)
    su2_apply<RB>(a, pack2(u00.x, u00.x), pack2(-u00.y, u00.y), pack2(u10.x, u10.x), pack2(-u10.y, u10.y),
                  pack2(-u10.x, -u10.x), pack2(u00.y, -u00.y));
}

__device__ __forceinline__ void u2_cpx_dispatch(int rb, f2 (&a)[kRegs], const Cx<float> *m)
{
    switch (rb) {
    case 0: u2_cpx_m<0>(a, m); break;
    case 1: u2_cpx_m<1>(a, m); break;
    case 2: u2_cpx_m<2>(a, m); break;
    default: u2_cpx_m<3>(a, m); break;
    }
}

__device__ __forceinline__ void grad_cpx_dispatch(int rb, const f2 (&a)[kRegs], const f2 (&b)[kRegs], float &vx,
                                                  float &vy, float &vz)
{
    switch (rb) {
    case 0: grad_cpx<0>(a, b, vx, vy, vz); break;
    case 1: grad_cpx<1>(a, b, vx, vy, vz); break;
    case 2: grad_cpx<2>(a, b, vx, vy, vz); break;
    default: grad_cpx<3>(a, b, vx, vy, vz); break;
    }
}

// CNOT on target register bit RT; control a register bit rc (>= 0) or the
// thread-known bit vc.
template <int RT>
__device__ __forceinline__ void cnot_regs_cpx(f2 (&a)[kRegs], int rc, int vc)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RT)) continue;
        const int c = rc >= 0 ? ((j >> rc) & 1) : vc;
        const f2 t0 = a[j], t1 = a[j | (1 << RT)];
        a[j] = c ? t1 : t0;
        a[j | (1 << RT)] = c ? t0 : t1;
    }
}

__device__ __forceinline__ void cnot_cpx_dispatch(int rt, f2 (&a)[kRegs], int rc, int vc)
{
    switch (rt) {
    case 0: cnot_regs_cpx<0>(a, rc, vc); break;
    case 1: cnot_regs_cpx<1>(a, rc, vc); break;
    case 2: cnot_regs_cpx<2>(a, rc, vc); break;
    default: cnot_regs_cpx<3>(a, rc, vc); break;
    }
}

// The pass's phases over the tile in shared memory (after a barrier), the op
// records read at run time as in run_phases (tile.cuh), with each amplitude an
// f32x2 pair; ends with a barrier.  lam_valid: the costate tile holds lam.
template <bool REV>
__device__ __forceinline__ void run_phases_cpx(const TileJob &j, const TileSmem<float> &S, bool lam_valid)
{
    const int tid = threadIdx.x, T = j.T;
    const bool active = tid < T;
    const int warp = tid >> 5, lane = tid & 31;
    const int wwidth = T < 32 ? T : 32;
    const unsigned wmask = T < 32 ? ((1u << T) - 1u) : 0xffffffffu;
    const uint32_t base = j.base;
    const uint32_t ph_s = smem_u32(S.phi), lm_s = smem_u32(S.lam);
    f2 p[kRegs];
    f2 q[kRegs];
    for (int phz = j.phase_begin; phz < j.phase_end; ++phz) {
        // threads beyond the tile's 2^(K-4) skip the work but reach the same
        // barrier instruction at the end of the phase
        if (active) {
        const DevPhase ph = j.phases[phz];
        const int lo = ph.lo;
        const uint32_t xt = ((uint32_t)tid & ((1u << lo) - 1u)) | (((uint32_t)tid >> lo) << (lo + 4));
        if (lo == 0) {
#pragma unroll
            for (int k = 0; k < kRegs / 2; ++k) {
                const uint32_t o = 8u * (uint32_t)swz<float>((int)xt + 2 * k);
                lds_f2x2(ph_s + o, p[2 * k], p[2 * k + 1]);
                if (REV && lam_valid) lds_f2x2(lm_s + o, q[2 * k], q[2 * k + 1]);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < kRegs; ++jj) {
                const uint32_t o = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)jj << lo)));
                p[jj] = lds_f2(ph_s + o);
                if (REV && lam_valid) q[jj] = lds_f2(lm_s + o);
            }
        }
        DevOp nxt = j.ops[ph.op_begin < ph.op_end ? ph.op_begin : 0];
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
            const DevOp op = nxt;
            if (o + 1 < ph.op_end) nxt = j.ops[o + 1];
            switch (op.type) {
            case OP_DIAG: {
                uint32_t msk = 0;
#pragma unroll 4
                for (int k = op.a; k < op.a + op.b; ++k) {
                    const DiagPair dp = j.diag[k];
                    msk ^= operand_pattern(dp.a, lo, xt, base) & operand_pattern(dp.b, lo, xt, base);
                }
                flip_cpx<REV>(p, q, msk);
                break;
            }
            case OP_U2:
                u2_cpx_dispatch(op.a - lo, p, S.mats + 4 * op.slot);
                break;
            case OP_GRAD:
                if constexpr (REV) {
                    float vx, vy, vz;
                    grad_cpx_dispatch(op.a - lo, p, q, vx, vy, vz);
                    float *g = S.redG + (size_t)warp * 3 * j.nslots + 3 * op.slot;
                    if (T >= 32) {
                        const float v = warp_sum3(vx, vy, vz, lane);
                        if ((lane & 7) == 0 && lane < 24) g[lane >> 3] = v;
                    } else {
                        vx = warp_sum(vx, wwidth, wmask);
                        vy = warp_sum(vy, wwidth, wmask);
                        vz = warp_sum(vz, wwidth, wmask);
                        if (lane == 0) { g[0] = vx; g[1] = vy; g[2] = vz; }
                    }
                    if (!(op.flags & OPF_SKIP_APPLY)) {
                        u2_cpx_dispatch(op.a - lo, p, S.mats + 4 * op.slot);
                        u2_cpx_dispatch(op.a - lo, q, S.mats + 4 * op.slot);
                    }
                }
                break;
            case OP_CNOT: {
                int rc = -1, vc = 0;
                if (op.a >= kFixed) vc = (int)((base >> (op.a - kFixed)) & 1u);
                else if (op.a >= lo && op.a < lo + kRegBits) rc = op.a - lo;
                else vc = (int)((xt >> op.a) & 1u);
                cnot_cpx_dispatch(op.b - lo, p, rc, vc);
                if (REV) cnot_cpx_dispatch(op.b - lo, q, rc, vc);
                break;
            }
            case OP_EXPVAL: {
                float pr[kRegs];
#pragma unroll
                for (int jj = 0; jj < kRegs; ++jj) {
                    const f2 t = mul2(p[jj], p[jj]);
                    pr[jj] = lane0(t) + lane1(t);
                }
                op_expval_pr<float>(pr, S, j, xt, lo, warp, lane, wwidth, wmask);
                break;
            }
            case OP_COSTATE:
                if constexpr (REV) {
                    float d[kRegs];
                    costate_diag<float>(d, S, j, xt, lo);
                    if (op.flags & OPF_ACCUMULATE) {   // q holds the costate's X/Y part
#pragma unroll
                        for (int jj = 0; jj < kRegs; ++jj) q[jj] = fma2(pack2(d[jj], d[jj]), p[jj], q[jj]);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < kRegs; ++jj) q[jj] = mul2(pack2(d[jj], d[jj]), p[jj]);
                    }
                    lam_valid = true;
                }
                break;
            default:
                break;
            }
        }
        if (lo == 0) {
#pragma unroll
            for (int k = 0; k < kRegs / 2; ++k) {
                const uint32_t o = 8u * (uint32_t)swz<float>((int)xt + 2 * k);
                sts_f2x2(ph_s + o, p[2 * k], p[2 * k + 1]);
                if (REV) sts_f2x2(lm_s + o, q[2 * k], q[2 * k + 1]);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < kRegs; ++jj) {
                const uint32_t o = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)jj << lo)));
                sts_f2(ph_s + o, p[jj]);
                if (REV) sts_f2(lm_s + o, q[jj]);
            }
        }
        if (REV) lam_valid = true;
        }
        __syncthreads();
    }
}

// The interpreter for a plan's real type: complex pairs for complex64.
template <typename R, bool REV>
__device__ __forceinline__ void run_phases_any(const TileJob &j, const TileSmem<R> &S, bool lam_valid)
{
    if constexpr (sizeof(R) == 4) run_phases_cpx<REV>(j, S, lam_valid);
    else run_phases<R, REV>(j, S, lam_valid);
}

}  // namespace

}  // namespace qtm
