// Paired-sample tile program: the general paired pass kernel (k_pass_x2, op
// tables read at run time) and the run-time specialised paired kernels.
//
// Blackwell's FP32 datapath executes fma / mul / add / sub on .f32x2 register
// pairs: one instruction issues two lanes of work.  A paired pass CTA takes two
// samples of the batch, b0 = 2 * pair and b1 = b0 + 1 (b1 = b0 again, results
// discarded, when the batch is odd), and keeps the amplitude of one basis state
// of both samples in one register pair.  The samples share the circuit, so
// every sign pattern, register permutation and closed-form index is common to
// both and only the numbers differ: each gate op is a two-lane SIMD op with
// the same schedule as the one-sample tile program in tile.cuh.
//
// Memory layout (shared and global): an element is 16 bytes,
// (re_b0, re_b1, im_b0, im_b1), so the state of a sample pair is laid out like
// a complex128 state with half as many samples and uses the same TMA geometry
// and 128-byte swizzle (16-byte chunk index XOR row mod 8).  Run matrices and
// product-state tables are staged as pairs (re, im, -im) per entry.
#pragma once

#include "tile.cuh"

namespace qtm {

namespace {

typedef unsigned long long f2;   // lanes (sample b0, sample b1) of one f32x2 register pair
constexpr f2 kSign2 = 0x8000000080000000ull;

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// register-pair moves (no arithmetic)
__device__ __forceinline__ f2 pack2(float a, float b)
{
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float lane0(f2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float lane1(f2 v)
{
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}

struct A2 { f2 r, i; };   // amplitude of one basis state in both samples

__device__ __forceinline__ int swz16(int e) { return e ^ ((e >> 3) & 7); }

__device__ __forceinline__ A2 lds_a2(const A2 *base, int s)
{
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(base + s);
    return {v.x, v.y};
}
__device__ __forceinline__ void sts_a2(A2 *base, int s, A2 a)
{
    *reinterpret_cast<ulonglong2 *>(base + s) = make_ulonglong2(a.r, a.i);
}

// ---- register-group kernels ---------------------------------------------------

// a <- U a on register bit RB; m: the slot's 12 pairs (u00, u01, u10, u11) x (re, im, -im)
template <int RB>
__device__ __forceinline__ void u2x2(A2 (&a)[kRegs], const f2 *m)
{
    const ulonglong2 *mv = reinterpret_cast<const ulonglong2 *>(m);
    const ulonglong2 w0 = mv[0], w1 = mv[1], w2 = mv[2], w3 = mv[3], w4 = mv[4], w5 = mv[5];
    const f2 a_r = w0.x, a_i = w0.y, a_n = w1.x;   // u00
    const f2 b_r = w1.y, b_i = w2.x, b_n = w2.y;   // u01
    const f2 c_r = w3.x, c_i = w3.y, c_n = w4.x;   // u10
    const f2 d_r = w4.y, d_i = w5.x, d_n = w5.y;   // u11
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RB)) continue;
        const A2 x0 = a[j], x1 = a[j | (1 << RB)];
        a[j].r = fma2(a_r, x0.r, fma2(a_n, x0.i, fma2(b_r, x1.r, mul2(b_n, x1.i))));
        a[j].i = fma2(a_r, x0.i, fma2(a_i, x0.r, fma2(b_r, x1.i, mul2(b_i, x1.r))));
        a[j | (1 << RB)].r = fma2(c_r, x0.r, fma2(c_n, x0.i, fma2(d_r, x1.r, mul2(d_n, x1.i))));
        a[j | (1 << RB)].i = fma2(c_r, x0.i, fma2(c_i, x0.r, fma2(d_r, x1.i, mul2(d_i, x1.r))));
    }
}

// (vx, vy, vz) = sum over the pairs on register bit RB of Im<lam|sigma phi>,
// sigma = X, Y, Z; a = phi, b = lam.  Positive and negative terms accumulate
// separately (no negated operands needed) and are subtracted once.
template <int RB>
__device__ __forceinline__ void grad_x2(const A2 (&a)[kRegs], const A2 (&b)[kRegs], f2 &vx, f2 &vy, f2 &vz)
{
    f2 xp = 0, xn = 0, yp = 0, yn = 0, zp = 0, zn = 0;
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RB)) continue;
        const A2 a0 = a[j], a1 = a[j | (1 << RB)], b0 = b[j], b1 = b[j | (1 << RB)];
        // Z: Im(conj(b0) a0) - Im(conj(b1) a1)
        zp = fma2(b0.r, a0.i, zp); zn = fma2(b0.i, a0.r, zn);
        zn = fma2(b1.r, a1.i, zn); zp = fma2(b1.i, a1.r, zp);
        // X: Im(conj(b0) a1) + Im(conj(b1) a0)
        xp = fma2(b0.r, a1.i, xp); xn = fma2(b0.i, a1.r, xn);
        xp = fma2(b1.r, a0.i, xp); xn = fma2(b1.i, a0.r, xn);
        // Y: Re(conj(b1) a0) - Re(conj(b0) a1)
        yp = fma2(b1.r, a0.r, yp); yp = fma2(b1.i, a0.i, yp);
        yn = fma2(b0.r, a1.r, yn); yn = fma2(b0.i, a1.i, yn);
    }
    vx = sub2(xp, xn);
    vy = sub2(yp, yn);
    vz = sub2(zp, zn);
}

__device__ __forceinline__ f2 warp_sum2(f2 v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = add2(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// CNOT on target register bit RT with a control bit c known per thread.
template <int RT>
__device__ __forceinline__ void cnot_x2(A2 (&a)[kRegs], int c)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RT)) continue;
        const A2 t0 = a[j], t1 = a[j | (1 << RT)];
        a[j] = c ? t1 : t0;
        a[j | (1 << RT)] = c ? t0 : t1;
    }
}

// CNOT with control and target both register bits: a fixed register permutation.
template <int RC, int RT>
__device__ __forceinline__ void cnot_static_x2(A2 (&a)[kRegs])
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if ((j & (1 << RT)) || !(j & (1 << RC))) continue;
        const A2 t = a[j];
        a[j] = a[j | (1 << RT)];
        a[j | (1 << RT)] = t;
    }
}

// Negate register j (both samples, phi and in reverse lam) where bit j of m is set.
template <bool REV>
__device__ __forceinline__ void flip_x2(A2 (&p)[kRegs], A2 (&q)[kRegs], uint32_t m)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        const f2 s = ((m >> j) & 1u) ? kSign2 : 0ull;
        p[j].r ^= s; p[j].i ^= s;
        if (REV) { q[j].r ^= s; q[j].i ^= s; }
    }
}

// ---- tile program -------------------------------------------------------------

struct TileJobX2 : TileJob {
    const void *mats1, *tabs1, *gE1;   // second sample's tables (== the first's on an odd tail)
    int has_b1;
};

struct TileSmemX2 {
    A2 *phi, *lam;
    f2 *mats, *tabs, *tcoef;
    uint32_t *tmask;
    int32_t *tobs;
    Ent *ents;
    f2 *redE, *redG;
    uint64_t *bar;
};

__device__ __forceinline__ TileSmemX2 carve_x2(unsigned char *smem, const LayoutX2 &L)
{
    TileSmemX2 t;
    t.phi = reinterpret_cast<A2 *>(smem + L.phi);
    t.lam = reinterpret_cast<A2 *>(smem + L.lam);
    t.mats = reinterpret_cast<f2 *>(smem + L.mats);
    t.tabs = reinterpret_cast<f2 *>(smem + L.tabs);
    t.tcoef = reinterpret_cast<f2 *>(smem + L.tcoef);
    t.tmask = reinterpret_cast<uint32_t *>(smem + L.tmask);
    t.tobs = reinterpret_cast<int32_t *>(smem + L.tobs);
    t.ents = reinterpret_cast<Ent *>(smem + L.ents);
    t.redE = reinterpret_cast<f2 *>(smem + L.redE);
    t.redG = reinterpret_cast<f2 *>(smem + L.redG);
    t.bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    return t;
}

__device__ __forceinline__ void put3(f2 *d, Cx<float> u0, Cx<float> u1)
{
    d[0] = pack2(u0.x, u1.x);
    d[1] = pack2(u0.y, u1.y);
    d[2] = pack2(-u0.y, -u1.y);
}

// Stage both samples' run matrices (U, or U^dagger in reverse), the observable
// coefficients as seen from this tile (times each sample's cotangent in
// reverse) and (analytic phi) the product-state tables.  Ends without a barrier.
template <bool REV>
__device__ __forceinline__ void stage_tables_x2(const TileJobX2 &j, const TileSmemX2 &S, int nwarps)
{
    const int tid = threadIdx.x, T = blockDim.x;
    for (int i = tid; i < nwarps * (j.M > 0 ? j.M : 1); i += T) S.redE[i] = 0ull;
    for (int i = tid; i < nwarps * 3 * (j.nslots > 0 ? j.nslots : 1); i += T) S.redG[i] = 0ull;
    const Cx<float> *g0 = static_cast<const Cx<float> *>(j.mats);
    const Cx<float> *g1 = static_cast<const Cx<float> *>(j.mats1);
    for (int i = tid; i < 4 * j.nslots; i += T) {
        const int s = i >> 2, k = i & 3;
        const int run = j.slot_runs[s];
        if (REV) {   // U^dagger: entry (r, c) <- conj(U[c][r])
            const int src = 4 * run + ((k & 1) << 1 | (k >> 1));
            const Cx<float> u0 = g0[src], u1 = g1[src];
            put3(S.mats + 3 * i, {u0.x, -u0.y}, {u1.x, -u1.y});
        } else {
            put3(S.mats + 3 * i, g0[4 * run + k], g1[4 * run + k]);
        }
    }
    const uint64_t Smask = ((1ull << j.l) - 1ull) | (j.m ? (((1ull << j.m) - 1ull) << j.h) : 0ull);
    for (int t = tid; t < j.n_terms; t += T) {
        const Term tm = j.terms[t];
        const uint64_t zm = tm.zmask;
        const int fixed = __popcll(zm & ~Smask & (uint64_t)j.base) & 1;
        float c0 = (float)tm.coef, c1 = c0;
        if (REV) {
            c0 *= static_cast<const float *>(j.gE)[tm.obs];
            c1 *= static_cast<const float *>(j.gE1)[tm.obs];
        }
        S.tcoef[t] = fixed ? pack2(-c0, -c1) : pack2(c0, c1);
        S.tmask[t] = (uint32_t)(zm & ((1ull << j.l) - 1ull)) | (uint32_t)(((zm >> j.h) & ((1ull << j.m) - 1ull)) << j.l);
        S.tobs[t] = tm.obs;
    }
    if (j.phi_src == SRC_ANALYTIC) {
        for (int k = tid; k < j.analytic_ents; k += T) S.ents[k] = j.prefix_ents[k];
        const int ntab = (j.sq + 3) >> 2;
        const Cx<float> *t0 = static_cast<const Cx<float> *>(j.tabs);
        const Cx<float> *t1 = static_cast<const Cx<float> *>(j.tabs1);
        for (int i = tid; i < ntab * 16; i += T) put3(S.tabs + 3 * i, t0[i], t1[i]);
    }
}

// phi tile of both samples from the folded product-state prefix (after
// stage_tables_x2 + barrier); same index arithmetic as fill_analytic.
__device__ __forceinline__ void fill_analytic_x2(const TileJobX2 &j, const TileSmemX2 &S)
{
    const int tid = threadIdx.x, T = blockDim.x;
    const int ntab = (j.sq + 3) >> 2;
    const int E = 1 << j.K;
    int td[kMaxMaskTerms];
    uint32_t tmk[kMaxMaskTerms];
    const int nl = j.amap_lin, nt = j.amap_lin + j.amap_quad;
#pragma unroll
    for (int k = 0; k < kMaxMaskTerms; ++k) {
        const MaskTerm t = k < nt ? j.amap[k] : MaskTerm{0, 0u};
        td[k] = t.d;
        tmk[k] = t.mask;
    }
    for (int e = tid; e < E; e += T) {
        const uint32_t y = j.base | ((uint32_t)e & ((1u << j.l) - 1u)) | (((uint32_t)e >> j.l) << j.h);
        uint32_t xx = y;
        int sign = 0;
        if (nl >= 0) {   // closed form: x = A^{-1} y, sign from the quadratic form
            xx = 0;
#pragma unroll
            for (int k = 0; k < kMaxMaskTerms; ++k)
                if (k < nl) xx ^= (td[k] >= 0 ? (y >> td[k]) : (y << -td[k])) & tmk[k];
            int par = __popc(xx & j.amap_dlin);
#pragma unroll
            for (int k = 0; k < kMaxMaskTerms; ++k)
                if (k >= nl && k < nt) par += __popc(xx & (xx >> td[k]) & tmk[k]);
            sign = par & 1;
        } else {
            for (int k = j.analytic_ents - 1; k >= 0; --k) {
                const Ent en = S.ents[k];
                if (en.kind == QTM_CNOT) xx ^= ((xx >> en.a) & 1u) << en.b;
                else sign ^= (int)((xx >> en.a) & (xx >> en.b) & 1u);
            }
        }
        const f2 *t = S.tabs + 3 * (xx & 15u);
        A2 amp{t[0], t[1]};
        for (int q = 1; q < ntab; ++q) {
            const f2 *u = S.tabs + 3 * (16 * q + ((xx >> (4 * q)) & 15u));
            const A2 o = amp;
            amp.r = fma2(o.r, u[0], mul2(o.i, u[2]));
            amp.i = fma2(o.r, u[1], mul2(o.i, u[0]));
        }
        if (sign) { amp.r ^= kSign2; amp.i ^= kSign2; }
        sts_a2(S.phi, swz16(e), amp);
    }
}

// Registers <-> shared tile for register group [LO, LO+4) (compile-time LO).
template <int LO, bool LAM>
__device__ __forceinline__ void regs_load_x2(A2 (&p)[kRegs], A2 (&q)[kRegs], const TileSmemX2 &S, uint32_t xt)
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        const int s = swz16((int)(xt | ((uint32_t)jj << LO)));
        p[jj] = lds_a2(S.phi, s);
        if (LAM) q[jj] = lds_a2(S.lam, s);
    }
}

template <int LO, bool LAM>
__device__ __forceinline__ void regs_store_x2(const A2 (&p)[kRegs], const A2 (&q)[kRegs], const TileSmemX2 &S,
                                              uint32_t xt)
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        const int s = swz16((int)(xt | ((uint32_t)jj << LO)));
        sts_a2(S.phi, s, p[jj]);
        if (LAM) sts_a2(S.lam, s, q[jj]);
    }
}

// One GRAD op's warp-reduced (vx, vy, vz) for both samples into the slot's partials.
__device__ __forceinline__ void grad_store_x2(const TileSmemX2 &S, int nslots, int slot, int warp, int lane, f2 vx,
                                              f2 vy, f2 vz)
{
    vx = warp_sum2(vx);
    vy = warp_sum2(vy);
    vz = warp_sum2(vz);
    if (lane == 0) {
        f2 *g = S.redG + (size_t)warp * 3 * nslots + 3 * slot;
        g[0] = vx; g[1] = vy; g[2] = vz;
    }
}

// Per-tile partial sums of both samples (fixed order over warps, FP64).
template <bool REV>
__device__ __forceinline__ void write_partials_x2(const TileJobX2 &j, const TileSmemX2 &S, int nwarps,
                                                  bool has_expval, double *Ep0, double *Ep1, double *Gp0,
                                                  double *Gp1, int tiles, int tile)
{
    const int tid = threadIdx.x, T = blockDim.x;
    if (!REV) {
        if (!has_expval) return;
        for (int i = tid; i < j.M; i += T) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                const f2 v = S.redE[w * j.M + i];
                s0 += (double)lane0(v);
                s1 += (double)lane1(v);
            }
            Ep0[i] = s0;
            if (j.has_b1) Ep1[i] = s1;
        }
    } else {
        const int nv = 3 * j.nslots;
        for (int i = tid; i < nv; i += T) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                const f2 v = S.redG[w * nv + i];
                s0 += (double)lane0(v);
                s1 += (double)lane1(v);
            }
            const int run = j.slot_runs[i / 3];
            const size_t o = ((size_t)run * tiles + tile) * 3 + (i % 3);
            Gp0[o] = s0;
            if (j.has_b1) Gp1[o] = s1;
        }
    }
}

// ---- phase interpreter (general paired kernel) ------------------------------------

template <int RT>
__device__ __forceinline__ void cnot_x2_dyn(A2 (&a)[kRegs], int rc, int vc)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RT)) continue;
        const int c = rc >= 0 ? ((j >> rc) & 1) : vc;
        const A2 t0 = a[j], t1 = a[j | (1 << RT)];
        a[j] = c ? t1 : t0;
        a[j | (1 << RT)] = c ? t0 : t1;
    }
}

// <O_m> partials of both samples over the thread's 16 registers (terms sorted
// by observable), warp-reduced into S.redE.
__device__ __forceinline__ void expval_x2(const A2 (&p)[kRegs], const TileSmemX2 &S, const TileJobX2 &j, uint32_t xt,
                                          int lo, int warp, int lane)
{
    f2 pr[kRegs];
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) pr[jj] = fma2(p[jj].r, p[jj].r, mul2(p[jj].i, p[jj].i));
    int cur = -1;
    f2 acc = 0ull;
    for (int t = 0; t < j.n_terms; ++t) {
        const int ob = S.tobs[t];
        if (ob != cur) {
            if (cur >= 0) {
                acc = warp_sum2(acc);
                if (lane == 0) S.redE[warp * j.M + cur] = acc;
            }
            cur = ob;
            acc = 0ull;
        }
        const uint32_t lm = S.tmask[t];
        const uint32_t tpar = (uint32_t)__popc(xt & lm);
        const uint32_t rm = (lm >> lo) & 15u;
        f2 sacc = 0ull;
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj)
            sacc = add2(sacc, pr[jj] ^ (((tpar + __popc((uint32_t)jj & rm)) & 1u) ? kSign2 : 0ull));
        acc = fma2(S.tcoef[t], sacc, acc);
    }
    if (cur >= 0) {
        acc = warp_sum2(acc);
        if (lane == 0) S.redE[warp * j.M + cur] = acc;
    }
}

// lam = (sum_m gE_m O_m) phi for both samples (Sec. II-A costate).
__device__ __forceinline__ void costate_x2(const A2 (&p)[kRegs], A2 (&q)[kRegs], const TileSmemX2 &S,
                                           const TileJobX2 &j, uint32_t xt, int lo)
{
    f2 d[kRegs];
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) d[jj] = 0ull;
    for (int t = 0; t < j.n_terms; ++t) {
        const uint32_t lm = S.tmask[t];
        const uint32_t tpar = (uint32_t)__popc(xt & lm);
        const uint32_t rm = (lm >> lo) & 15u;
        const f2 k = S.tcoef[t];
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj)
            d[jj] = add2(d[jj], k ^ (((tpar + __popc((uint32_t)jj & rm)) & 1u) ? kSign2 : 0ull));
    }
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        q[jj].r = mul2(d[jj], p[jj].r);
        q[jj].i = mul2(d[jj], p[jj].i);
    }
}

// The pass's phases read from the op tables: same op semantics as run_phases,
// each op applied to both samples.  All threads of the CTA (2^(K-4) >= 32)
// run every phase.
template <bool REV>
__device__ __forceinline__ void run_phases_x2(const TileJobX2 &j, const TileSmemX2 &S, bool lam_valid)
{
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t base = j.base;
    A2 p[kRegs];
    A2 q[kRegs];
    for (int phz = j.phase_begin; phz < j.phase_end; ++phz) {
        const DevPhase ph = j.phases[phz];
        const int lo = ph.lo;
        const uint32_t xt = ((uint32_t)tid & ((1u << lo) - 1u)) | (((uint32_t)tid >> lo) << (lo + 4));
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) {
            const int s = swz16((int)(xt | ((uint32_t)jj << lo)));
            p[jj] = lds_a2(S.phi, s);
            if (REV && lam_valid) q[jj] = lds_a2(S.lam, s);
        }
        DevOp nxt = j.ops[ph.op_begin < ph.op_end ? ph.op_begin : 0];
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
            const DevOp op = nxt;
            if (o + 1 < ph.op_end) nxt = j.ops[o + 1];
            // one flat dispatch key: op type x register bit
            const int sub = (op.type == OP_CNOT ? op.b : op.a) - lo;
            const int key = op.type * 4 + ((op.type == OP_U2 || op.type == OP_GRAD || op.type == OP_CNOT) ? (sub & 3) : 0);
            const f2 *m = S.mats + 12 * op.slot;
            switch (key) {
            case OP_U2 * 4 + 0: u2x2<0>(p, m); break;
            case OP_U2 * 4 + 1: u2x2<1>(p, m); break;
            case OP_U2 * 4 + 2: u2x2<2>(p, m); break;
            case OP_U2 * 4 + 3: u2x2<3>(p, m); break;
#define QTM_GRAD_CASE(RB)                                                             \
            case OP_GRAD * 4 + RB:                                                    \
                if constexpr (REV) {                                                  \
                    f2 vx, vy, vz;                                                    \
                    grad_x2<RB>(p, q, vx, vy, vz);                                    \
                    grad_store_x2(S, j.nslots, op.slot, warp, lane, vx, vy, vz);      \
                    if (!(op.flags & OPF_SKIP_APPLY)) { u2x2<RB>(p, m); u2x2<RB>(q, m); } \
                }                                                                     \
                break;
            QTM_GRAD_CASE(0)
            QTM_GRAD_CASE(1)
            QTM_GRAD_CASE(2)
            QTM_GRAD_CASE(3)
#undef QTM_GRAD_CASE
            case OP_DIAG * 4: {
                uint32_t msk = 0;
                for (int k = op.a; k < op.a + op.b; ++k) {
                    const DiagPair dp = j.diag[k];
                    msk ^= operand_pattern(dp.a, lo, xt, base) & operand_pattern(dp.b, lo, xt, base);
                }
                flip_x2<REV>(p, q, msk);
                break;
            }
#define QTM_CNOT_CASE(RT)                                                              \
            case OP_CNOT * 4 + RT: {                                                   \
                int rc = -1, vc = 0;                                                   \
                if (op.a >= kFixed) vc = (int)((base >> (op.a - kFixed)) & 1u);        \
                else if (op.a >= lo && op.a < lo + kRegBits) rc = op.a - lo;           \
                else vc = (int)((xt >> op.a) & 1u);                                    \
                cnot_x2_dyn<RT>(p, rc, vc);                                            \
                if (REV) cnot_x2_dyn<RT>(q, rc, vc);                                   \
                break;                                                                 \
            }
            QTM_CNOT_CASE(0)
            QTM_CNOT_CASE(1)
            QTM_CNOT_CASE(2)
            QTM_CNOT_CASE(3)
#undef QTM_CNOT_CASE
            case OP_EXPVAL * 4: expval_x2(p, S, j, xt, lo, warp, lane); break;
            case OP_COSTATE * 4:
                if constexpr (REV) costate_x2(p, q, S, j, xt, lo);
                break;
            default: break;
            }
        }
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) {
            const int s = swz16((int)(xt | ((uint32_t)jj << lo)));
            sts_a2(S.phi, s, p[jj]);
            if (REV) sts_a2(S.lam, s, q[jj]);
        }
        if (REV) lam_valid = true;
        __syncthreads();
    }
}

// The body of a paired pass kernel: one CTA per (sample pair, tile); grid =
// ceil(B / 2) * tiles, block = 2^(K-4) threads (K >= 9).  Same stages as
// pass_body; `phases` is the generated phase program.
template <bool REV, typename PhaseFn>
__device__ __forceinline__ void pass_body_x2(const PassArgs &a, const CUtensorMap *tm_phi, const CUtensorMap *tm_lam,
                                             PhaseFn phases)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int nwarps = blockDim.x >> 5;
    const int pair = blockIdx.x >> a.log_tiles;
    const int tile = blockIdx.x & (a.tiles - 1);
    const int b0 = 2 * pair;
    const int has_b1 = b0 + 1 < a.B;
    const int b1 = has_b1 ? b0 + 1 : b0;
    const int gapbits = a.h - a.l;
    const uint32_t gap = tile & ((1u << gapbits) - 1u);
    const uint32_t rest = tile >> gapbits;

    TileJobX2 j;
    j.T = blockDim.x;
    j.K = a.K; j.l = a.l; j.h = a.h; j.m = a.m; j.sq = a.state_qubits;
    j.base = (gap << a.l) | (rest << (a.h + a.m));
    j.ops = a.ops; j.diag = a.diag; j.phases = a.phases;
    j.phase_begin = a.phase_begin; j.phase_end = a.phase_end;
    j.slot_runs = a.slot_runs + a.slot_begin; j.nslots = a.nslots;
    const int ntab16 = ((a.state_qubits + 3) >> 2) * 16;
    j.mats = static_cast<const Cx<float> *>(a.mats) + (size_t)b0 * a.n_runs * 4;
    j.mats1 = static_cast<const Cx<float> *>(a.mats) + (size_t)b1 * a.n_runs * 4;
    j.tabs = static_cast<const Cx<float> *>(a.tabs) + (size_t)b0 * ntab16;
    j.tabs1 = static_cast<const Cx<float> *>(a.tabs) + (size_t)b1 * ntab16;
    j.prefix_ents = a.prefix_ents; j.analytic_ents = a.analytic_ents;
    j.amap = a.amap; j.amap_lin = a.amap_lin; j.amap_quad = a.amap_quad; j.amap_dlin = a.amap_dlin;
    j.terms = a.terms; j.n_terms = a.n_terms; j.M = a.M;
    j.gE = REV ? static_cast<const float *>(a.gE) + (size_t)b0 * a.M : nullptr;
    j.gE1 = REV ? static_cast<const float *>(a.gE) + (size_t)b1 * a.M : nullptr;
    j.phi_src = a.phi_src; j.lam_src = a.lam_src;
    j.has_b1 = has_b1;

    const LayoutX2 L = make_layout_x2(a.K, REV, a.nslots, a.n_terms, a.M, a.state_qubits, a.analytic_ents, nwarps,
                                      (int)sizeof(Ent));
    const TileSmemX2 S = carve_x2(smem, L);

    int coord[5] = {0, 0, 0, 0, 0};
    {
        int d = a.low_dims;
        if (gapbits > 0) coord[d++] = (int)gap;
        d += a.high_dims;
        coord[d] = (int)(rest + ((uint32_t)pair << (a.state_qubits - a.h - a.m)));
    }
    const bool load_phi = a.phi_src == SRC_LOAD;
    const bool load_lam = REV && a.lam_src == SRC_LOAD;
    const uint32_t tile_bytes = 16u << a.K;
    if (tid == 0 && (load_phi || load_lam)) {
        mbar_init(S.bar, 1);
        mbar_expect_tx(S.bar, tile_bytes * ((load_phi ? 1u : 0u) + (load_lam ? 1u : 0u)));
        if (load_phi) tma_load(S.phi, tm_phi, coord, a.rank, S.bar);
        if (load_lam) tma_load(S.lam, tm_lam, coord, a.rank, S.bar);
    }
    stage_tables_x2<REV>(j, S, nwarps);
    __syncthreads();
    if (a.phi_src == SRC_ANALYTIC) fill_analytic_x2(j, S);
    if (load_phi || load_lam) {
        if (!wait_tile_loads(S.bar, a.status)) return;
    } else {
        __syncthreads();
    }

    phases(j, S, load_lam);

    write_partials_x2<REV>(j, S, nwarps, a.has_expval != 0, a.Epart + ((size_t)b0 * a.tiles + tile) * a.M,
                           a.Epart + ((size_t)b1 * a.tiles + tile) * a.M,
                           REV ? a.Gpart + (size_t)b0 * a.n_runs * a.tiles * 3 : nullptr,
                           REV ? a.Gpart + (size_t)b1 * a.n_runs * a.tiles * 3 : nullptr, a.tiles, tile);

    if (a.store_phi || (REV && a.store_lam)) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (a.store_phi) tma_store(tm_phi, coord, a.rank, S.phi);
            if (REV && a.store_lam) tma_store(tm_lam, coord, a.rank, S.lam);
            tma_store_commit_and_drain();
        }
    }
}

}  // namespace

}  // namespace qtm
