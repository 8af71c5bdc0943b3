// Device-side building blocks shared by the pass kernel (fused.cu) and the
// persistent multi-circuit kernel (multi.cu): complex arithmetic, the shared-
// memory swizzle, TMA/mbarrier helpers, the register-group gate kernels, the
// FP64 run-matrix builder, and the tile program (table staging, analytic
// product state, register-phase interpreter, per-tile partial sums).
#pragma once

#ifdef __CUDACC_RTC__
struct alignas(64) CUtensorMap_st { unsigned long long opaque[16]; };
typedef CUtensorMap_st CUtensorMap;
#else
#include <cstdint>
#include <cuda.h>
#endif

#include "finalize_math.h"
#include "pod.h"

namespace qtm {

namespace {

constexpr unsigned long long kWaitLimitNs = 1000000000ull;   // bounded mbarrier wait: 1 s

template <typename R>
struct Cx { R x, y; };

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// a*b + c
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> c)
{
    return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}

// element index -> swizzled shared-memory slot, matching the TMA 128-byte
// swizzle (16-byte chunk index within a 128-byte row XOR row mod 8)
template <typename R>
__device__ __forceinline__ int swz(int e);
template <>
__device__ __forceinline__ int swz<float>(int e) { return e ^ (((e >> 4) & 7) << 1); }
template <>
__device__ __forceinline__ int swz<double>(int e) { return e ^ ((e >> 3) & 7); }

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- TMA / mbarrier -------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait, bounded, for this CTA's tile loads (phase 0 of `bar`); every thread
// calls it.  After kWaitLimitNs the CTA records kStatusTimeout (qtm_sync
// reports QTM_ETIMEOUT) and waits once more, again at most kWaitLimitNs, for
// the copies still in flight, so that none is left writing this CTA's shared
// memory when it exits.  Returns false when the caller must return.
__device__ __forceinline__ bool wait_tile_loads(uint64_t *bar, unsigned *status)
{
    bool ok = false;
    unsigned long long t0 = global_ns();
    while (!(ok = mbar_try_wait(bar, 0)))
        if (global_ns() - t0 > kWaitLimitNs) break;
    if (!__syncthreads_or(!ok)) return true;
    if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
    t0 = global_ns();
    while (!mbar_try_wait(bar, 0))
        if (global_ns() - t0 > kWaitLimitNs) break;
    __syncthreads();
    return false;
}

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *tm, const int *c, int rank,
                                         uint64_t *bar)
{
    uint32_t d = smem_u32(dst), b = smem_u32(bar);
    uint64_t t = reinterpret_cast<uint64_t>(tm);
    switch (rank) {
    case 1:
        asm volatile("cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2}], [%3];" ::"r"(d), "l"(t), "r"(c[0]), "r"(b) : "memory");
        break;
    case 2:
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3}], [%4];" ::"r"(d), "l"(t), "r"(c[0]), "r"(c[1]), "r"(b)
                     : "memory");
        break;
    case 3:
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(d), "l"(t), "r"(c[0]), "r"(c[1]),
                     "r"(c[2]), "r"(b)
                     : "memory");
        break;
    case 4:
        asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(d), "l"(t), "r"(c[0]), "r"(c[1]),
                     "r"(c[2]), "r"(c[3]), "r"(b)
                     : "memory");
        break;
    default:
        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(d), "l"(t), "r"(c[0]), "r"(c[1]),
                     "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(b)
                     : "memory");
        break;
    }
}

__device__ __forceinline__ void tma_store(const CUtensorMap *tm, const int *c, int rank, const void *src)
{
    uint32_t s = smem_u32(src);
    uint64_t t = reinterpret_cast<uint64_t>(tm);
    switch (rank) {
    case 1:
        asm volatile("cp.async.bulk.tensor.1d.global.shared::cta.tile.bulk_group [%0, {%1}], [%2];"
                     ::"l"(t), "r"(c[0]), "r"(s) : "memory");
        break;
    case 2:
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
                     ::"l"(t), "r"(c[0]), "r"(c[1]), "r"(s) : "memory");
        break;
    case 3:
        asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
                     ::"l"(t), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(s) : "memory");
        break;
    case 4:
        asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
                     ::"l"(t), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(s) : "memory");
        break;
    default:
        asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];"
                     ::"l"(t), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(s) : "memory");
        break;
    }
}

__device__ __forceinline__ void tma_store_commit_and_drain()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// ---- register-group kernels -------------------------------------------------

template <int RB, typename R>
__device__ __forceinline__ void u2(Cx<R> (&a)[kRegs], const Cx<R> *m)
{
    const Cx<R> m00 = m[0], m01 = m[1], m10 = m[2], m11 = m[3];
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RB)) continue;
        const Cx<R> a0 = a[j], a1 = a[j | (1 << RB)];
        a[j] = cfma(m00, a0, cmul(m01, a1));
        a[j | (1 << RB)] = cfma(m10, a0, cmul(m11, a1));
    }
}

template <typename R>
__device__ __forceinline__ void u2_dispatch(int rb, Cx<R> (&a)[kRegs], const Cx<R> *m)
{
    switch (rb) {
    case 0: u2<0>(a, m); break;
    case 1: u2<1>(a, m); break;
    case 2: u2<2>(a, m); break;
    default: u2<3>(a, m); break;
    }
}

// v = sum over pairs of Im<lam|sigma phi> for sigma = X, Y, Z on register bit RB
template <int RB, typename R>
__device__ __forceinline__ void grad_acc(const Cx<R> (&a)[kRegs], const Cx<R> (&b)[kRegs], R &vx,
                                         R &vy, R &vz)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RB)) continue;
        const Cx<R> a0 = a[j], a1 = a[j | (1 << RB)], b0 = b[j], b1 = b[j | (1 << RB)];
        // Im(conj(b) a) = b.x a.y - b.y a.x ;  Re(conj(b) a) = b.x a.x + b.y a.y
        vz += (b0.x * a0.y - b0.y * a0.x) - (b1.x * a1.y - b1.y * a1.x);
        vx += (b0.x * a1.y - b0.y * a1.x) + (b1.x * a0.y - b1.y * a0.x);
        vy += (b1.x * a0.x + b1.y * a0.y) - (b0.x * a1.x + b0.y * a1.y);
    }
}

template <typename R>
__device__ __forceinline__ void grad_dispatch(int rb, const Cx<R> (&a)[kRegs], const Cx<R> (&b)[kRegs],
                                              R &vx, R &vy, R &vz)
{
    switch (rb) {
    case 0: grad_acc<0>(a, b, vx, vy, vz); break;
    case 1: grad_acc<1>(a, b, vx, vy, vz); break;
    case 2: grad_acc<2>(a, b, vx, vy, vz); break;
    default: grad_acc<3>(a, b, vx, vy, vz); break;
    }
}

template <int RT, typename R>
__device__ __forceinline__ void cnot_regs(Cx<R> (&a)[kRegs], int rc, int vc)
{
#pragma unroll
    for (int j = 0; j < kRegs; ++j) {
        if (j & (1 << RT)) continue;
        const int c = rc >= 0 ? ((j >> rc) & 1) : vc;
        const Cx<R> t0 = a[j], t1 = a[j | (1 << RT)];
        a[j] = c ? t1 : t0;
        a[j | (1 << RT)] = c ? t0 : t1;
    }
}

template <typename R>
__device__ __forceinline__ void cnot_dispatch(int rt, Cx<R> (&a)[kRegs], int rc, int vc)
{
    switch (rt) {
    case 0: cnot_regs<0>(a, rc, vc); break;
    case 1: cnot_regs<1>(a, rc, vc); break;
    case 2: cnot_regs<2>(a, rc, vc); break;
    default: cnot_regs<3>(a, rc, vc); break;
    }
}

// 16-bit pattern of the registers j (tile bits [lo, lo+4)) on which an
// operand's bit is 1: register bits give fixed patterns, thread bits and
// tile-constant bits give all-or-nothing.
__device__ __forceinline__ uint32_t operand_pattern(int o, int lo, uint32_t xt, uint32_t base)
{
    if (o >= kFixed) return ((base >> (o - kFixed)) & 1u) ? 0xFFFFu : 0u;
    if (o >= lo && o < lo + kRegBits)
        return (uint32_t)(0xFF00F0F0CCCCAAAAull >> (16 * (o - lo))) & 0xFFFFu;
    return ((xt >> o) & 1u) ? 0xFFFFu : 0u;
}

__device__ __forceinline__ void flip_sign(Cx<float> &v, uint32_t bit)
{
    const uint32_t s = bit << 31;
    v.x = __uint_as_float(__float_as_uint(v.x) ^ s);
    v.y = __uint_as_float(__float_as_uint(v.y) ^ s);
}

__device__ __forceinline__ void flip_sign(Cx<double> &v, uint32_t bit)
{
    const unsigned long long s = (unsigned long long)bit << 63;
    v.x = __longlong_as_double(__double_as_longlong(v.x) ^ (long long)s);
    v.y = __longlong_as_double(__double_as_longlong(v.y) ^ (long long)s);
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v, int width, unsigned mask)
{
    for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// Full-warp sums of three values in one butterfly of 6 shuffles instead of 15:
// the first level trades half the values (lanes 0-15 keep a and b, lanes
// 16-31 keep c and a zero pad), the second level half of what is left, and
// three more levels sum the single value.  Lanes 0, 8 and 16 end with the
// sums of a, b and c.
template <typename R>
__device__ __forceinline__ R warp_sum3(R a, R b, R c, int lane)
{
    const bool hi = (lane & 16) != 0;
    const R x0 = (hi ? c : a) + __shfl_xor_sync(0xffffffffu, hi ? a : c, 16);
    const R x1 = (hi ? (R)0 : b) + __shfl_xor_sync(0xffffffffu, hi ? b : (R)0, 16);
    const bool h8 = (lane & 8) != 0;
    R y = (h8 ? x1 : x0) + __shfl_xor_sync(0xffffffffu, h8 ? x0 : x1, 8);
    y += __shfl_xor_sync(0xffffffffu, y, 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    return y;
}

// Shared-memory layout of a pass CTA (offsets from a 1024-byte aligned base).
struct Layout {
    int phi, lam, mats, tabs, tmask, tcoef, tobs, ents, redE, redG, bar, total;
};

__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline Layout make_layout(int K, int csize, bool rev, int nslots, int n_terms,
                                              int M, int sq, int n_ents, int nwarps, int rsize)
{
    Layout L{};
    int tile = csize << K;
    int o = 0;
    L.phi = o; o += tile;
    L.lam = align_up(o, 1024); o = L.lam + (rev ? tile : 0);   // swizzle pattern needs 1 KiB alignment
    o = align_up(o, 16);
    L.mats = o; o = align_up(o + 4 * csize * (nslots > 0 ? nslots : 1), 16);
    L.tabs = o; o = align_up(o + csize * 16 * ((sq + 3) / 4), 16);
    L.tmask = o; o = align_up(o + 4 * (n_terms > 0 ? n_terms : 1), 16);
    L.tcoef = o; o = align_up(o + rsize * (n_terms > 0 ? n_terms : 1), 16);
    L.tobs = o; o = align_up(o + 4 * (n_terms > 0 ? n_terms : 1), 16);
    L.ents = o; o = align_up(o + (int)sizeof(Ent) * (n_ents > 0 ? n_ents : 1), 16);
    L.redE = o; o = align_up(o + rsize * nwarps * (M > 0 ? M : 1), 16);
    L.redG = o; o = align_up(o + rsize * nwarps * 3 * (nslots > 0 ? nslots : 1), 16);
    L.bar = o; o += 16;
    L.total = o;
    return L;
}

// Fused matrix U = R_m ... R_1 of a run for sample b, in FP64 (row-major
// u00, u01, u10, u11 as (re, im) pairs).  Rotation R_P(t) = cos(t/2) I - i sin(t/2) P.
// Every R_P(t) is in SU(2), R = [[alpha, -conj(beta)], [beta, conj(alpha)]]
// (RX: alpha = c, beta = -i s; RY: alpha = c, beta = s; RZ: alpha = c - i s,
// beta = 0), so the product is carried as U = [[a, -conj(b)], [b, conj(a)]]
// and R U costs two complex products: a <- alpha a - conj(beta) b,
// b <- beta a + conj(alpha) b.  cs (may be null): each rotation's
// (cos(t/2), sin(t/2)), indexed like rots.
// (a, b) <- R (a, b) for R = R_kind(t), c = cos(t/2), s = sin(t/2).
__device__ __forceinline__ void su2_rotate(int kind, double c, double s, double2 &a, double2 &b)
{
    double2 na, nb;
    if (kind == QTM_RX) {          // a' = c a - i s b, b' = -i s a + c b
        na = {c * a.x + s * b.y, c * a.y - s * b.x};
        nb = {s * a.y + c * b.x, c * b.y - s * a.x};
    } else if (kind == QTM_RY) {   // a' = c a - s b, b' = s a + c b
        na = {c * a.x - s * b.x, c * a.y - s * b.y};
        nb = {s * a.x + c * b.x, s * a.y + c * b.y};
    } else {                       // a' = (c - i s) a, b' = (c + i s) b
        na = {c * a.x + s * a.y, c * a.y - s * a.x};
        nb = {c * b.x - s * b.y, c * b.y + s * b.x};
    }
    a = na;
    b = nb;
}

template <typename R>
__device__ void run_matrix_f64(const Run rr, const Rot *rots, const R *xb, const R *w, double2 *U, double2 *cs)
{
    double2 a{1, 0}, b{0, 0};
    for (int i = rr.rot_begin; i < rr.rot_end; ++i) {
        const Rot ro = rots[i];
        double t = ro.coef;
        if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
        if (ro.x_idx >= 0) t *= (double)xb[ro.x_idx];
        double s, c;
        sincos(0.5 * t, &s, &c);
        if (cs) cs[i] = double2{c, s};
        su2_rotate(ro.kind, c, s, a, b);
    }
    U[0] = a; U[1] = double2{-b.x, b.y}; U[2] = b; U[3] = double2{a.x, -a.y};
}

// One CTA: every run's fused matrix for one sample (FP64, rounded once), and
// the product-state tables T_j[v] = prod_{k<4} u_{4j+k}[bit k of v], u_q = U_prefix(q)|0>.
// cs_b (may be null): this sample's per-rotation (cos(t/2), sin(t/2)).
template <typename R>
__device__ __forceinline__ void prep_sample(const Run *runs, const Rot *rots, const int32_t *prefix_run_of_q,
                                            int n_runs, int n, int sq, const R *xb, const R *w,
                                            Cx<R> *mats, Cx<R> *tabs, double2 *ufac, double2 *cs_b)
{
    for (int r = threadIdx.x; r < n_runs; r += blockDim.x) {
        double2 U[4];
        const Run rr = runs[r];
        run_matrix_f64<R>(rr, rots, xb, w, U, cs_b);
        for (int k = 0; k < 4; ++k) mats[4 * r + k] = {(R)U[k].x, (R)U[k].y};
        if (rr.prefix) { ufac[2 * rr.q] = U[0]; ufac[2 * rr.q + 1] = U[2]; }
    }
    for (int q = threadIdx.x; q < sq; q += blockDim.x)
        if (q >= n || prefix_run_of_q[q] < 0) { ufac[2 * q] = {1, 0}; ufac[2 * q + 1] = {0, 0}; }
    __syncthreads();
    const int ntab = (sq + 3) >> 2;
    for (int i = threadIdx.x; i < ntab * 16; i += blockDim.x) {
        const int j = i >> 4, v = i & 15;
        double2 p{1, 0};
        for (int k = 0; k < 4; ++k) {
            const int q = 4 * j + k;
            if (q < sq) {
                const double2 u = ufac[2 * q + ((v >> k) & 1)];
                p = double2{p.x * u.x - p.y * u.y, p.x * u.y + p.y * u.x};
            }
        }
        tabs[i] = {(R)p.x, (R)p.y};
    }
}

// prep_sample with the angles shared: sines and cosines of the rotations
// without an input come from cs_shared (computed once per call), those of the
// others once per distinct angle (rep[i] == i) into scratch (shared memory,
// n_rots pairs); then every run's product as in run_matrix_f64.  Same
// outputs as prep_sample, with FP64 sines and cosines per sample only for
// distinct input-dependent angles (the FP64 pipe runs at 1/64 of the FP32
// rate on this GPU).
template <typename R>
__device__ __forceinline__ void prep_sample_shared(const Run *runs, const Rot *rots, const int32_t *rep,
                                                   const double2 *cs_shared, const int32_t *prefix_run_of_q,
                                                   int n_runs, int n_rots, int n, int sq, const R *xb, const R *w,
                                                   Cx<R> *mats, Cx<R> *tabs, double2 *ufac, double2 *cs_b,
                                                   double2 *scratch)
{
    for (int i = threadIdx.x; i < n_rots; i += blockDim.x) {
        const Rot ro = rots[i];
        if (ro.x_idx < 0 || rep[i] != i) continue;
        double t = ro.coef;   // the factor order of run_matrix_f64 (the same pair, bit for bit)
        if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
        t *= (double)xb[ro.x_idx];
        double s, c;
        sincos(0.5 * t, &s, &c);
        scratch[i] = double2{c, s};
    }
    __syncthreads();
    // cs_shared comes from the kernel launched just before this one, which
    // this one may overlap (programmatic dependent launch): wait for it here
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int r = threadIdx.x; r < n_runs; r += blockDim.x) {
        const Run rr = runs[r];
        double2 a{1, 0}, b{0, 0};
        for (int i = rr.rot_begin; i < rr.rot_end; ++i) {
            const Rot ro = rots[i];
            const double2 cs = ro.x_idx < 0 ? cs_shared[rep[i]] : scratch[rep[i]];
            if (cs_b) cs_b[i] = cs;
            su2_rotate(ro.kind, cs.x, cs.y, a, b);
        }
        const double2 U[4] = {a, double2{-b.x, b.y}, b, double2{a.x, -a.y}};
        for (int k = 0; k < 4; ++k) mats[4 * r + k] = {(R)U[k].x, (R)U[k].y};
        if (rr.prefix) { ufac[2 * rr.q] = U[0]; ufac[2 * rr.q + 1] = U[2]; }
    }
    for (int q = threadIdx.x; q < sq; q += blockDim.x)
        if (q >= n || prefix_run_of_q[q] < 0) { ufac[2 * q] = {1, 0}; ufac[2 * q + 1] = {0, 0}; }
    __syncthreads();
    const int ntab = (sq + 3) >> 2;
    for (int i = threadIdx.x; i < ntab * 16; i += blockDim.x) {
        const int j = i >> 4, v = i & 15;
        double2 p{1, 0};
        for (int k = 0; k < 4; ++k) {
            const int q = 4 * j + k;
            if (q < sq) {
                const double2 u = ufac[2 * q + ((v >> k) & 1)];
                p = double2{p.x * u.x - p.y * u.y, p.x * u.y + p.y * u.x};
            }
        }
        tabs[i] = {(R)p.x, (R)p.y};
    }
}

// Everything one CTA needs to run a pass over one tile of one sample.
struct TileJob {
    int T;                          // threads running the phases: 2^(K-4) (the rest only join barriers)
    int K, l, h, m, sq;
    uint32_t base;                  // global index bits of the tile outside S
    const DevOp *ops;
    const DiagPair *diag;
    const DevPhase *phases;
    int phase_begin, phase_end;
    const int32_t *slot_runs;       // already offset to the pass's first slot
    int nslots;
    const void *mats;               // this sample's run matrices [n_runs][4]
    const void *tabs;               // this sample's product-state tables
    const Ent *prefix_ents;
    int analytic_ents;
    const MaskTerm *amap;
    int amap_lin, amap_quad;
    uint32_t amap_dlin;
    const Term *terms;
    int n_terms, M;
    const void *gE;                 // this sample's cotangents [M] (reverse)
    int phi_src, lam_src;
};

template <typename R>
struct TileSmem {
    Cx<R> *phi, *lam, *mats, *tabs;
    uint32_t *tmask;
    R *tcoef;
    int32_t *tobs;
    Ent *ents;
    R *redE, *redG;
    uint64_t *bar;
};

template <typename R>
__device__ __forceinline__ TileSmem<R> carve(unsigned char *smem, const Layout &L)
{
    TileSmem<R> t;
    t.phi = reinterpret_cast<Cx<R> *>(smem + L.phi);
    t.lam = reinterpret_cast<Cx<R> *>(smem + L.lam);
    t.mats = reinterpret_cast<Cx<R> *>(smem + L.mats);
    t.tabs = reinterpret_cast<Cx<R> *>(smem + L.tabs);
    t.tmask = reinterpret_cast<uint32_t *>(smem + L.tmask);
    t.tcoef = reinterpret_cast<R *>(smem + L.tcoef);
    t.tobs = reinterpret_cast<int32_t *>(smem + L.tobs);
    t.ents = reinterpret_cast<Ent *>(smem + L.ents);
    t.redE = reinterpret_cast<R *>(smem + L.redE);
    t.redG = reinterpret_cast<R *>(smem + L.redG);
    t.bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    return t;
}

// Stage the pass's run matrices (U, or U^dagger in reverse), the observable
// terms as seen from this tile, and (analytic phi) the product-state tables.
// Ends without a barrier.
template <typename R, bool REV>
__device__ __forceinline__ void stage_tables(const TileJob &j, const TileSmem<R> &S, int nwarps)
{
    const int tid = threadIdx.x, T = blockDim.x;
    for (int i = tid; i < nwarps * (j.M > 0 ? j.M : 1); i += T) S.redE[i] = (R)0;
    for (int i = tid; i < nwarps * 3 * (j.nslots > 0 ? j.nslots : 1); i += T) S.redG[i] = (R)0;
    const Cx<R> *gm = static_cast<const Cx<R> *>(j.mats);
    for (int i = tid; i < 4 * j.nslots; i += T) {
        const int s = i >> 2, k = i & 3;
        const int run = j.slot_runs[s];
        if (REV) {   // U^dagger: (k = 2r + c) <- conj(U[c][r])
            const Cx<R> u = gm[4 * run + ((k & 1) << 1 | (k >> 1))];
            S.mats[i] = {u.x, -u.y};
        } else {
            S.mats[i] = gm[4 * run + k];
        }
    }
    const uint64_t Smask = ((1ull << j.l) - 1ull) | (j.m ? (((1ull << j.m) - 1ull) << j.h) : 0ull);
    for (int t = tid; t < j.n_terms; t += T) {
        const Term tm = j.terms[t];
        const uint64_t zm = tm.zmask;
        const uint32_t lm = (uint32_t)(zm & ((1ull << j.l) - 1ull)) |
                            (uint32_t)(((zm >> j.h) & ((1ull << j.m) - 1ull)) << j.l);
        const int fixed = __popcll(zm & ~Smask & (uint64_t)j.base) & 1;
        R coef = (R)tm.coef;
        if (REV) coef *= static_cast<const R *>(j.gE)[tm.obs];
        S.tmask[t] = lm;
        S.tcoef[t] = fixed ? -coef : coef;
        S.tobs[t] = tm.obs;
    }
    if (j.phi_src == SRC_ANALYTIC) {
        for (int k = tid; k < j.analytic_ents; k += T) S.ents[k] = j.prefix_ents[k];
        const int ntab = (j.sq + 3) >> 2;
        const Cx<R> *gt = static_cast<const Cx<R> *>(j.tabs);
        for (int i = tid; i < ntab * 16; i += T) S.tabs[i] = gt[i];
    }
}

// phi tile from the folded product-state prefix (after stage_tables + barrier).
template <typename R>
__device__ __forceinline__ void fill_analytic(const TileJob &j, const TileSmem<R> &S)
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
        Cx<R> amp = S.tabs[xx & 15u];
        for (int q = 1; q < ntab; ++q) amp = cmul(amp, S.tabs[16 * q + ((xx >> (4 * q)) & 15u)]);
        if (sign) { amp.x = -amp.x; amp.y = -amp.y; }
        S.phi[swz<R>(e)] = amp;
    }
}

// <O_m> partials over the thread's 16 registers (terms sorted by observable),
// warp-reduced, one value per (warp, observable) in S.redE.
// pr: |amplitude|^2 of the thread's registers.
template <typename R>
__device__ __forceinline__ void op_expval_pr(const R (&pr)[kRegs], const TileSmem<R> &S, const TileJob &j,
                                             uint32_t xt, int lo, int warp, int lane, int wwidth, unsigned wmask)
{
    int cur = -1;
    R acc = 0;
    for (int t = 0; t < j.n_terms; ++t) {
        const int ob = S.tobs[t];
        if (ob != cur) {
            if (cur >= 0) {
                acc = warp_sum(acc, wwidth, wmask);
                if (lane == 0) S.redE[warp * j.M + cur] = acc;
            }
            cur = ob;
            acc = 0;
        }
        const uint32_t lm = S.tmask[t];
        const int tpar = __popc(xt & lm);
        const uint32_t rm = (lm >> lo) & 15u;
        R sacc = 0;
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj)
            sacc += ((tpar + __popc((uint32_t)jj & rm)) & 1) ? -pr[jj] : pr[jj];
        acc = fma(S.tcoef[t], sacc, acc);
    }
    if (cur >= 0) {
        acc = warp_sum(acc, wwidth, wmask);
        if (lane == 0) S.redE[warp * j.M + cur] = acc;
    }
}

template <typename R>
__device__ __forceinline__ void op_expval(const Cx<R> (&p)[kRegs], const TileSmem<R> &S, const TileJob &j,
                                          uint32_t xt, int lo, int warp, int lane, int wwidth, unsigned wmask)
{
    R pr[kRegs];
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) pr[jj] = p[jj].x * p[jj].x + p[jj].y * p[jj].y;
    op_expval_pr<R>(pr, S, j, xt, lo, warp, lane, wwidth, wmask);
}

// lam = (sum_m gE_m O_m) phi on the thread's registers (Sec. II-A costate).
// d[jj]: the diagonal of sum_m gE_m O_m on the thread's registers.
template <typename R>
__device__ __forceinline__ void costate_diag(R (&d)[kRegs], const TileSmem<R> &S, const TileJob &j, uint32_t xt,
                                             int lo)
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) d[jj] = 0;
    for (int t = 0; t < j.n_terms; ++t) {
        const uint32_t lm = S.tmask[t];
        const int tpar = __popc(xt & lm);
        const uint32_t rm = (lm >> lo) & 15u;
        const R k = S.tcoef[t];
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj)
            d[jj] += ((tpar + __popc((uint32_t)jj & rm)) & 1) ? -k : k;
    }
}

// acc: q already holds the costate's X/Y part (loaded from memory); add to it.
template <typename R>
__device__ __forceinline__ void op_costate(const Cx<R> (&p)[kRegs], Cx<R> (&q)[kRegs], const TileSmem<R> &S,
                                           const TileJob &j, uint32_t xt, int lo, bool acc = false)
{
    R d[kRegs];
    costate_diag<R>(d, S, j, xt, lo);
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj)
        q[jj] = acc ? Cx<R>{q[jj].x + d[jj] * p[jj].x, q[jj].y + d[jj] * p[jj].y}
                    : Cx<R>{d[jj] * p[jj].x, d[jj] * p[jj].y};
}

// CNOT with control and target both register bits: a fixed register permutation.
template <int RC, int RT, typename R>
__device__ __forceinline__ void cnot_static(Cx<R> (&a)[kRegs])
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        if ((jj & (1 << RT)) || !(jj & (1 << RC))) continue;
        const Cx<R> t = a[jj];
        a[jj] = a[jj | (1 << RT)];
        a[jj | (1 << RT)] = t;
    }
}

// Registers <-> shared tile for register group [LO, LO+4) (compile-time LO).
template <typename R, int LO, bool LAM>
__device__ __forceinline__ void regs_load(Cx<R> (&p)[kRegs], Cx<R> (&q)[kRegs], const TileSmem<R> &S, uint32_t xt)
{
    if (sizeof(R) == 4 && LO == 0) {
#pragma unroll
        for (int k = 0; k < kRegs / 2; ++k) {
            const int s = swz<R>((int)xt + 2 * k);
            const float4 v = *reinterpret_cast<const float4 *>(&S.phi[s]);
            p[2 * k] = {(R)v.x, (R)v.y};
            p[2 * k + 1] = {(R)v.z, (R)v.w};
            if (LAM) {
                const float4 u = *reinterpret_cast<const float4 *>(&S.lam[s]);
                q[2 * k] = {(R)u.x, (R)u.y};
                q[2 * k + 1] = {(R)u.z, (R)u.w};
            }
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) {
            const int s = swz<R>((int)(xt | ((uint32_t)jj << LO)));
            p[jj] = S.phi[s];
            if (LAM) q[jj] = S.lam[s];
        }
    }
}

template <typename R, int LO, bool LAM>
__device__ __forceinline__ void regs_store(const Cx<R> (&p)[kRegs], const Cx<R> (&q)[kRegs], const TileSmem<R> &S,
                                           uint32_t xt)
{
    if (sizeof(R) == 4 && LO == 0) {
#pragma unroll
        for (int k = 0; k < kRegs / 2; ++k) {
            const int s = swz<R>((int)xt + 2 * k);
            *reinterpret_cast<float4 *>(&S.phi[s]) =
                make_float4((float)p[2 * k].x, (float)p[2 * k].y, (float)p[2 * k + 1].x, (float)p[2 * k + 1].y);
            if (LAM)
                *reinterpret_cast<float4 *>(&S.lam[s]) =
                    make_float4((float)q[2 * k].x, (float)q[2 * k].y, (float)q[2 * k + 1].x, (float)q[2 * k + 1].y);
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < kRegs; ++jj) {
            const int s = swz<R>((int)(xt | ((uint32_t)jj << LO)));
            S.phi[s] = p[jj];
            if (LAM) S.lam[s] = q[jj];
        }
    }
}

template <typename R, bool REV>
__device__ __forceinline__ void flip_mask(Cx<R> (&p)[kRegs], Cx<R> (&q)[kRegs], uint32_t msk)
{
#pragma unroll
    for (int jj = 0; jj < kRegs; ++jj) {
        const uint32_t bit = (msk >> jj) & 1u;
        flip_sign(p[jj], bit);
        if (REV) flip_sign(q[jj], bit);
    }
}

// The pass's phases over the tile in shared memory (after a barrier); ends
// with a barrier.  lam_valid: the costate tile already holds lam.
template <typename R, bool REV>
__device__ __forceinline__ void run_phases(const TileJob &j, const TileSmem<R> &S, bool lam_valid)
{
    const int tid = threadIdx.x, T = j.T;
    const bool active = tid < T;
    const int warp = tid >> 5, lane = tid & 31;
    const int wwidth = T < 32 ? T : 32;
    const unsigned wmask = T < 32 ? ((1u << T) - 1u) : 0xffffffffu;
    const uint32_t base = j.base;
    Cx<R> p[kRegs];
    Cx<R> q[kRegs];
    for (int phz = j.phase_begin; phz < j.phase_end; ++phz) {
        // threads beyond the tile's 2^(K-4) skip the work but reach the same
        // barrier instruction at the end of the phase (never a second one)
        if (active) {
        const DevPhase ph = j.phases[phz];
        const int lo = ph.lo;
        const uint32_t xt = ((uint32_t)tid & ((1u << lo) - 1u)) | (((uint32_t)tid >> lo) << (lo + 4));
        // load registers
        if (sizeof(R) == 4 && lo == 0) {
#pragma unroll
            for (int k = 0; k < kRegs / 2; ++k) {
                const int s = swz<R>((int)xt + 2 * k);
                const float4 v = *reinterpret_cast<const float4 *>(&S.phi[s]);
                p[2 * k] = {(R)v.x, (R)v.y};
                p[2 * k + 1] = {(R)v.z, (R)v.w};
                if (REV && lam_valid) {
                    const float4 u = *reinterpret_cast<const float4 *>(&S.lam[s]);
                    q[2 * k] = {(R)u.x, (R)u.y};
                    q[2 * k + 1] = {(R)u.z, (R)u.w};
                }
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < kRegs; ++jj) {
                const int s = swz<R>((int)(xt | ((uint32_t)jj << lo)));
                p[jj] = S.phi[s];
                if (REV && lam_valid) q[jj] = S.lam[s];
            }
        }
        // ops (the next op record is fetched while this one executes)
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
#pragma unroll
                for (int jj = 0; jj < kRegs; ++jj) {
                    const uint32_t bit = (msk >> jj) & 1u;
                    flip_sign(p[jj], bit);
                    if (REV) flip_sign(q[jj], bit);
                }
                break;
            }
            case OP_U2:
                u2_dispatch<R>(op.a - lo, p, S.mats + 4 * op.slot);
                break;
            case OP_GRAD:
                if constexpr (REV) {
                    R vx = 0, vy = 0, vz = 0;
                    grad_dispatch<R>(op.a - lo, p, q, vx, vy, vz);
                    vx = warp_sum(vx, wwidth, wmask);
                    vy = warp_sum(vy, wwidth, wmask);
                    vz = warp_sum(vz, wwidth, wmask);
                    if (lane == 0) {
                        R *g = S.redG + (size_t)warp * 3 * j.nslots + 3 * op.slot;
                        g[0] = vx; g[1] = vy; g[2] = vz;
                    }
                    if (!(op.flags & OPF_SKIP_APPLY)) {
                        u2_dispatch<R>(op.a - lo, p, S.mats + 4 * op.slot);
                        u2_dispatch<R>(op.a - lo, q, S.mats + 4 * op.slot);
                    }
                }
                break;
            case OP_CNOT: {
                int rc = -1, vc = 0;
                if (op.a >= kFixed) vc = (int)((base >> (op.a - kFixed)) & 1u);
                else if (op.a >= lo && op.a < lo + kRegBits) rc = op.a - lo;
                else vc = (int)((xt >> op.a) & 1u);
                cnot_dispatch<R>(op.b - lo, p, rc, vc);
                if (REV) cnot_dispatch<R>(op.b - lo, q, rc, vc);
                break;
            }
            case OP_EXPVAL:
                op_expval<R>(p, S, j, xt, lo, warp, lane, wwidth, wmask);
                break;
            case OP_COSTATE:
                if constexpr (REV) {
                    op_costate<R>(p, q, S, j, xt, lo, (op.flags & OPF_ACCUMULATE) != 0);
                    lam_valid = true;
                }
                break;
            default:
                break;
            }
        }
        // store registers
        if (sizeof(R) == 4 && lo == 0) {
#pragma unroll
            for (int k = 0; k < kRegs / 2; ++k) {
                const int s = swz<R>((int)xt + 2 * k);
                *reinterpret_cast<float4 *>(&S.phi[s]) =
                    make_float4((float)p[2 * k].x, (float)p[2 * k].y, (float)p[2 * k + 1].x,
                                (float)p[2 * k + 1].y);
                if (REV)
                    *reinterpret_cast<float4 *>(&S.lam[s]) =
                        make_float4((float)q[2 * k].x, (float)q[2 * k].y, (float)q[2 * k + 1].x,
                                    (float)q[2 * k + 1].y);
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < kRegs; ++jj) {
                const int s = swz<R>((int)(xt | ((uint32_t)jj << lo)));
                S.phi[s] = p[jj];
                if (REV) S.lam[s] = q[jj];
            }
        }
        if (REV) lam_valid = true;
        }
        __syncthreads();
    }
}

// Sum of the per-warp partials p[0], p[stride], ... (nwarps of them) in
// FP64 precision.  Complex64 plans add them in FP32 with Knuth's TwoSum,
// carrying each addition's rounding error, and convert once: the same result
// as FP64 additions up to the FP32 rounding of the carried error, with three
// FP64 operations instead of 2 x nwarps (the FP64 pipe runs at 1/64 of the
// FP32 rate on this GPU).
template <typename R>
__device__ __forceinline__ double sum_warps(const R *p, int stride, int nwarps)
{
    if constexpr (sizeof(R) == 8) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += (double)p[w * stride];
        return s;
    } else {
        float s = 0.f, e = 0.f;
        for (int w = 0; w < nwarps; ++w) {
            const float x = p[w * stride];
            const float t = s + x;
            const float z = t - s;
            e += (s - (t - z)) + (x - z);
            s = t;
        }
        return (double)s + (double)e;
    }
}

// Per-tile partial sums: <O_m> partials (forward) or v per run (reverse).
// Epart_row: [M] for this (sample, tile); Gpart_b: this sample's [n_runs][tiles][3].
template <typename R, bool REV>
__device__ __forceinline__ void write_partials(const TileJob &j, const TileSmem<R> &S, int nwarps,
                                               bool has_expval, double *Epart_row, double *Gpart_b,
                                               int tiles, int tile, R *E_row = nullptr)
{
    const int tid = threadIdx.x, T = blockDim.x;   // nwarps: warps that ran the phases
    if (!REV) {
        if (!has_expval) return;
        for (int i = tid; i < j.M; i += T) {
            const double s = sum_warps<R>(S.redE + i, j.M, nwarps);
            Epart_row[i] = s;
            if (E_row) E_row[i] = (R)s;   // one tile per sample: the tile's sum is the value
        }
    } else {
        const int nv = 3 * j.nslots;
        for (int i = tid; i < nv; i += T) {
            const int run = j.slot_runs[i / 3];
            Gpart_b[((size_t)run * tiles + tile) * 3 + (i % 3)] = sum_warps<R>(S.redG + i, nv, nwarps);
        }
    }
}


// One sample's gradients (one CTA): v per run summed over tiles in fixed
// order, the SO(3) walk back through the run's rotations (finalize_math.h)
// giving every rotation's angle gradient, then the chain rule
// theta = coef * W * X  =>  dW += g * coef * X,  dX += g * coef * W.
template <typename R>
__device__ __forceinline__ void grad_finalize_sample(
    const Run *runs, const Rot *rots, int n_runs, const int32_t *w_ptr, const int32_t *w_rots,
    const int32_t *x_ptr, const int32_t *x_rots, int P, int n_in, const R *xb, const R *w,
    double *Gpart_b, int tiles, double *abar, R *gx_b, R *gw_b, double *gwws_b, const double2 *cs_b)
{
    const bool warp_sums = tiles >= 32 && blockDim.x >= 32;
    if (warp_sums) {
        // many tiles: sum every run's tiles first, one warp per run (lanes take
        // every 32nd tile, fixed butterfly), into the run's tile-0 slot
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r = threadIdx.x >> 5; r < n_runs; r += nw)
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
                for (int t = lane; t < tiles; t += 32) s += Gpart_b[((size_t)r * tiles + t) * 3 + c];
                s = warp_sum(s, 32, 0xffffffffu);
                if (lane == 0) Gpart_b[(size_t)r * tiles * 3 + c] = s;
            }
        __syncthreads();
    }
    const int tiles_left = warp_sums ? 1 : tiles;
    for (int r = threadIdx.x; r < n_runs; r += blockDim.x) {
        double v[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < tiles_left; ++t)
            for (int c = 0; c < 3; ++c) v[c] += Gpart_b[((size_t)r * tiles + t) * 3 + c];
        const Run rr = runs[r];
        for (int i = rr.rot_end - 1; i >= rr.rot_begin; --i) {
            const Rot ro = rots[i];
            abar[i] = v[ro.kind];
            if (cs_b) {   // cos t, sin t from the prep's half-angle pair
                const double2 h = cs_b[i];
                adjoint_transpose_apply_cs(ro.kind, h.x * h.x - h.y * h.y, 2.0 * h.x * h.y, v);
            } else {
                double t = ro.coef;
                if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
                if (ro.x_idx >= 0) t *= (double)xb[ro.x_idx];
                adjoint_transpose_apply(ro.kind, t, v);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        double s = 0.0;
        for (int k = w_ptr[j]; k < w_ptr[j + 1]; ++k) {
            const int ri = w_rots[k];
            const Rot ro = rots[ri];
            s += abar[ri] * ro.coef * (ro.x_idx >= 0 ? (double)xb[ro.x_idx] : 1.0);
        }
        if (gw_b) gw_b[j] = (R)s;
        if (gwws_b) gwws_b[j] = s;
    }
    if (gx_b)
        for (int k = threadIdx.x; k < n_in; k += blockDim.x) {
            double s = 0.0;
            for (int i = x_ptr[k]; i < x_ptr[k + 1]; ++i) {
                const int ri = x_rots[i];
                const Rot ro = rots[ri];
                s += abar[ri] * ro.coef * (ro.w_idx >= 0 ? (double)w[ro.w_idx] : 1.0);
            }
            gx_b[k] = (R)s;
        }
}

// The body of a pass kernel: tile coordinates, TMA loads (or the analytic
// state), table staging, the pass's phases (`phases`, the interpreter or a
// generated specialisation), per-tile partial sums and the TMA stores.
// FILL = false: the phases compute an analytic phi themselves (the tables
// are staged, the tile is not filled).
template <typename R, bool REV, bool FILL = true, typename PhaseFn>
__device__ __forceinline__ void pass_body(const PassArgs &a, const CUtensorMap *tm_phi,
                                          const CUtensorMap *tm_lam, PhaseFn phases)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x;
    const int nwarps = (blockDim.x + 31) >> 5;
    const int b = blockIdx.x >> a.log_tiles;
    const int tile = blockIdx.x & (a.tiles - 1);
    const int gapbits = a.h - a.l;
    const uint32_t gap = tile & ((1u << gapbits) - 1u);
    const uint32_t rest = tile >> gapbits;

    if constexpr (REV) {
        // a kernel launched after this one as a programmatic dependent launch
        // (the batch grad_w reduction) may start once every CTA is running;
        // it waits for this grid before reading its results
        asm volatile("griddepcontrol.launch_dependents;");
    }
    if constexpr (!REV) {
        __shared__ double2 ufac[2 * 32];
        if (a.prep_fused && a.rot_rep) {   // as below, sines and cosines shared; scratch: the idle tile
            prep_sample_shared<R>(a.runs, a.rots, a.rot_rep, static_cast<const double2 *>(a.cs_shared), a.prq,
                                  a.n_runs, a.n_rots, a.n, a.state_qubits,
                                  static_cast<const R *>(a.x) + (size_t)b * a.n_in, static_cast<const R *>(a.w),
                                  static_cast<Cx<R> *>(const_cast<void *>(a.mats)) + (size_t)b * a.n_runs * 4,
                                  static_cast<Cx<R> *>(const_cast<void *>(a.tabs)) +
                                      (size_t)b * ((a.state_qubits + 3) >> 2) * 16,
                                  ufac, a.cs ? static_cast<double2 *>(a.cs) + (size_t)b * a.n_rots : nullptr,
                                  reinterpret_cast<double2 *>(smem));
            __syncthreads();
        } else if (a.prep_fused) {   // this CTA's sample: run matrices and tables before anything reads them
            prep_sample<R>(a.runs, a.rots, a.prq, a.n_runs, a.n, a.state_qubits,
                           static_cast<const R *>(a.x) + (size_t)b * a.n_in, static_cast<const R *>(a.w),
                           static_cast<Cx<R> *>(const_cast<void *>(a.mats)) + (size_t)b * a.n_runs * 4,
                           static_cast<Cx<R> *>(const_cast<void *>(a.tabs)) +
                               (size_t)b * ((a.state_qubits + 3) >> 2) * 16,
                           ufac, a.cs ? static_cast<double2 *>(a.cs) + (size_t)b * a.n_rots : nullptr);
            __syncthreads();
        }
    }

    TileJob j;
    j.T = 1 << (a.K - 4);   // threads holding the tile's amplitudes (the CTA may have more)
    j.K = a.K; j.l = a.l; j.h = a.h; j.m = a.m; j.sq = a.state_qubits;
    j.base = (gap << a.l) | (rest << (a.h + a.m));
    j.ops = a.ops; j.diag = a.diag; j.phases = a.phases;
    j.phase_begin = a.phase_begin; j.phase_end = a.phase_end;
    j.slot_runs = a.slot_runs + a.slot_begin; j.nslots = a.nslots;
    j.mats = static_cast<const Cx<R> *>(a.mats) + (size_t)b * a.n_runs * 4;
    j.tabs = static_cast<const Cx<R> *>(a.tabs) + (size_t)b * ((a.state_qubits + 3) >> 2) * 16;
    j.prefix_ents = a.prefix_ents; j.analytic_ents = a.analytic_ents;
    j.amap = a.amap; j.amap_lin = a.amap_lin; j.amap_quad = a.amap_quad; j.amap_dlin = a.amap_dlin;
    j.terms = a.terms; j.n_terms = a.n_terms; j.M = a.M;
    j.gE = REV ? static_cast<const R *>(a.gE) + (size_t)b * a.M : nullptr;
    j.phi_src = a.phi_src; j.lam_src = a.lam_src;

    const Layout L = make_layout(a.K, (int)sizeof(Cx<R>), REV, a.nslots, a.n_terms, a.M,
                                 a.state_qubits, a.analytic_ents, nwarps, (int)sizeof(R));
    const TileSmem<R> S = carve<R>(smem, L);

    // coordinates of this tile in the tensor maps
    int coord[5] = {0, 0, 0, 0, 0};
    {
        int d = a.low_dims;
        if (gapbits > 0) coord[d++] = (int)gap;
        d += a.high_dims;
        coord[d] = (int)(rest + ((uint32_t)b << (a.state_qubits - a.h - a.m)));
    }
    const bool load_phi = a.phi_src == SRC_LOAD;
    const bool load_lam = REV && a.lam_src == SRC_LOAD;
    const uint32_t tile_bytes = (uint32_t)sizeof(Cx<R>) << a.K;
    if (tid == 0 && (load_phi || load_lam)) {
        mbar_init(S.bar, 1);
        mbar_expect_tx(S.bar, tile_bytes * ((load_phi ? 1u : 0u) + (load_lam ? 1u : 0u)));
        if (load_phi) tma_load(S.phi, tm_phi, coord, a.rank, S.bar);
        if (load_lam) tma_load(S.lam, tm_lam, coord, a.rank, S.bar);
    }
    stage_tables<R, REV>(j, S, nwarps);
    __syncthreads();
    if (FILL && a.phi_src == SRC_ANALYTIC) fill_analytic<R>(j, S);
    if (load_phi || load_lam) {
        if (!wait_tile_loads(S.bar, a.status)) return;
    } else {
        __syncthreads();
    }

    phases(j, S, load_lam);

    write_partials<R, REV>(j, S, nwarps, a.has_expval != 0,
                           a.Epart + ((size_t)b * a.tiles + tile) * a.M,
                           REV ? a.Gpart + (size_t)b * a.n_runs * a.tiles * 3 : nullptr, a.tiles, tile,
                           (!REV && a.E_out) ? static_cast<R *>(a.E_out) + (size_t)b * a.M : nullptr);

    // ---- write the tile back ----
    if (a.store_phi || (REV && a.store_lam)) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (a.store_phi) tma_store(tm_phi, coord, a.rank, S.phi);
            if (REV && a.store_lam) tma_store(tm_lam, coord, a.rank, S.lam);
            tma_store_commit_and_drain();
        }
    }

    if constexpr (REV) {
        if (a.finalize_fused) {   // this CTA's sample: every run's sums are written (one tile)
            __syncthreads();
            const R *xb = static_cast<const R *>(a.x) + (size_t)b * a.n_in;
            grad_finalize_sample<R>(a.runs, a.rots, a.n_runs, a.w_ptr, a.w_rots, a.x_ptr, a.x_rots, a.n_weights,
                                    a.n_in, xb, static_cast<const R *>(a.w),
                                    a.Gpart + (size_t)b * a.n_runs * a.tiles * 3, a.tiles,
                                    a.abar + (size_t)b * a.n_rots,
                                    a.gx ? static_cast<R *>(a.gx) + (size_t)b * a.n_in : nullptr,
                                    a.gw_out ? static_cast<R *>(a.gw_out) + (size_t)b * a.n_weights : nullptr,
                                    a.gw_ws ? a.gw_ws + (size_t)b * a.n_weights : nullptr,
                                    a.cs ? static_cast<const double2 *>(a.cs) + (size_t)b * a.n_rots : nullptr);
        }
    }
}

}  // namespace

}  // namespace qtm
