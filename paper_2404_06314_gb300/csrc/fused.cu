// Fused pass kernel, expectation/gradient finalize kernels (sm_103a).
//
// One CTA processes one tile of 2^K amplitudes of one sample (the whole state
// when n <= 12).  The tile is staged in shared memory by TMA (bulk tensor
// copies with the 128-byte swizzle) or generated analytically from the folded
// product-state prefix, then the pass's phases run: each thread holds 16
// amplitudes (tile bits [lo, lo+4)) in registers and applies every op of the
// phase there; between phases the tile goes through shared memory.  The
// forward applies fused run matrices U (Eq. (qnn)); the reverse applies U^dagger
// to the state phi and the costate lam and accumulates v = Im<lam|sigma phi>
// per run (Sec. II-A adjoint method).  Partial sums per tile are written to
// global memory and reduced in fixed order by the finalize kernels.
#include <cstdint>

#include "device.h"
#include "finalize_math.h"

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
template <typename R>
__device__ void run_matrix_f64(const Run rr, const Rot *rots, const R *xb, const R *w, double2 *U)
{
    double2 u00{1, 0}, u01{0, 0}, u10{0, 0}, u11{1, 0};
    auto mul = [](double2 a, double2 b) { return double2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; };
    auto add = [](double2 a, double2 b) { return double2{a.x + b.x, a.y + b.y}; };
    for (int i = rr.rot_begin; i < rr.rot_end; ++i) {
        const Rot ro = rots[i];
        double t = ro.coef;
        if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
        if (ro.x_idx >= 0) t *= (double)xb[ro.x_idx];
        double s, c;
        sincos(0.5 * t, &s, &c);
        double2 g00, g01, g10, g11;
        if (ro.kind == QTM_RX) { g00 = {c, 0}; g01 = {0, -s}; g10 = {0, -s}; g11 = {c, 0}; }
        else if (ro.kind == QTM_RY) { g00 = {c, 0}; g01 = {-s, 0}; g10 = {s, 0}; g11 = {c, 0}; }
        else { g00 = {c, -s}; g01 = {0, 0}; g10 = {0, 0}; g11 = {c, s}; }
        const double2 n00 = add(mul(g00, u00), mul(g01, u10));
        const double2 n01 = add(mul(g00, u01), mul(g01, u11));
        const double2 n10 = add(mul(g10, u00), mul(g11, u10));
        const double2 n11 = add(mul(g10, u01), mul(g11, u11));
        u00 = n00; u01 = n01; u10 = n10; u11 = n11;
    }
    U[0] = u00; U[1] = u01; U[2] = u10; U[3] = u11;
}

// One CTA per sample: every run's fused matrix, then the product-state tables
// T_j[v] = prod_{k<4} u_{4j+k}[bit k of v] with u_q = U_prefix(q) |0>.
template <typename R>
__global__ void k_prep(const PrepArgs a)
{
    __shared__ double2 ufac[2 * 32];
    const int b = blockIdx.x;
    const R *xb = static_cast<const R *>(a.x) + (size_t)b * a.n_in;
    const R *w = static_cast<const R *>(a.w);
    Cx<R> *mats = static_cast<Cx<R> *>(a.mats) + (size_t)b * a.n_runs * 4;
    for (int r = threadIdx.x; r < a.n_runs; r += blockDim.x) {
        double2 U[4];
        const Run rr = a.runs[r];
        run_matrix_f64<R>(rr, a.rots, xb, w, U);
        for (int k = 0; k < 4; ++k) mats[4 * r + k] = {(R)U[k].x, (R)U[k].y};
        if (rr.prefix) { ufac[2 * rr.q] = U[0]; ufac[2 * rr.q + 1] = U[2]; }
    }
    for (int q = threadIdx.x; q < a.state_qubits; q += blockDim.x)
        if (q >= a.n || a.prefix_run_of_q[q] < 0) { ufac[2 * q] = {1, 0}; ufac[2 * q + 1] = {0, 0}; }
    __syncthreads();
    const int ntab = (a.state_qubits + 3) >> 2;
    Cx<R> *tabs = static_cast<Cx<R> *>(a.tabs) + (size_t)b * ntab * 16;
    for (int i = threadIdx.x; i < ntab * 16; i += blockDim.x) {
        const int j = i >> 4, v = i & 15;
        double2 p{1, 0};
        for (int k = 0; k < 4; ++k) {
            const int q = 4 * j + k;
            if (q < a.state_qubits) {
                const double2 u = ufac[2 * q + ((v >> k) & 1)];
                p = double2{p.x * u.x - p.y * u.y, p.x * u.y + p.y * u.x};
            }
        }
        tabs[i] = {(R)p.x, (R)p.y};
    }
}

template <typename R, bool REV>
__global__ void __launch_bounds__(256, sizeof(R) == 8 ? 1 : (REV ? 2 : 3)) k_pass(const __grid_constant__ PassArgs a,
                                              const __grid_constant__ CUtensorMap tm_phi,
                                              const __grid_constant__ CUtensorMap tm_lam)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    const int tid = threadIdx.x;
    const int T = blockDim.x;
    const int nwarps = (T + 31) >> 5;
    const int warp = tid >> 5, lane = tid & 31;
    const int wwidth = T < 32 ? T : 32;
    const unsigned wmask = T < 32 ? ((1u << T) - 1u) : 0xffffffffu;

    const int b = blockIdx.x >> a.log_tiles;
    const int tile = blockIdx.x & (a.tiles - 1);
    const int K = a.K, l = a.l, h = a.h, m = a.m;
    const int gapbits = h - l;
    const uint32_t gap = tile & ((1u << gapbits) - 1u);
    const uint32_t rest = tile >> gapbits;
    const uint32_t base = (gap << l) | (rest << (h + m));

    const Layout L = make_layout(K, (int)sizeof(Cx<R>), REV, a.nslots, a.n_terms, a.M,
                                 a.state_qubits, a.analytic_ents, nwarps, (int)sizeof(R));
    Cx<R> *sphi = reinterpret_cast<Cx<R> *>(smem + L.phi);
    Cx<R> *slam = reinterpret_cast<Cx<R> *>(smem + L.lam);
    Cx<R> *mats = reinterpret_cast<Cx<R> *>(smem + L.mats);
    Cx<R> *tabs = reinterpret_cast<Cx<R> *>(smem + L.tabs);
    uint32_t *tmask = reinterpret_cast<uint32_t *>(smem + L.tmask);
    R *tcoef = reinterpret_cast<R *>(smem + L.tcoef);
    int32_t *tobs = reinterpret_cast<int32_t *>(smem + L.tobs);
    Ent *sents = reinterpret_cast<Ent *>(smem + L.ents);
    R *redE = reinterpret_cast<R *>(smem + L.redE);
    R *redG = reinterpret_cast<R *>(smem + L.redG);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.bar);

    // coordinates of this tile in the tensor maps
    int coord[5] = {0, 0, 0, 0, 0};
    {
        int d = a.low_dims;
        if (gapbits > 0) coord[d++] = (int)gap;
        d += a.high_dims;
        coord[d] = (int)(rest + ((uint32_t)b << (a.state_qubits - h - m)));
    }
    const bool load_phi = a.phi_src == SRC_LOAD;
    const bool load_lam = REV && a.lam_src == SRC_LOAD;
    const uint32_t tile_bytes = (uint32_t)sizeof(Cx<R>) << K;

    if (tid == 0 && (load_phi || load_lam)) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, tile_bytes * ((load_phi ? 1u : 0u) + (load_lam ? 1u : 0u)));
        if (load_phi) tma_load(sphi, &tm_phi, coord, a.rank, bar);
        if (load_lam) tma_load(slam, &tm_lam, coord, a.rank, bar);
    }

    // ---- per-CTA tables ----
    for (int i = tid; i < nwarps * (a.M > 0 ? a.M : 1); i += T) redE[i] = (R)0;
    for (int i = tid; i < nwarps * 3 * (a.nslots > 0 ? a.nslots : 1); i += T) redG[i] = (R)0;
    {
        const Cx<R> *gm = static_cast<const Cx<R> *>(a.mats) + (size_t)b * a.n_runs * 4;
        for (int i = tid; i < 4 * a.nslots; i += T) {
            const int s = i >> 2, k = i & 3;
            const int run = a.slot_runs[a.slot_begin + s];
            if (REV) {   // U^dagger: (k = 2r + c) <- conj(U[c][r])
                const Cx<R> u = gm[4 * run + ((k & 1) << 1 | (k >> 1))];
                mats[i] = {u.x, -u.y};
            } else {
                mats[i] = gm[4 * run + k];
            }
        }
    }
    const uint64_t Smask = ((1ull << l) - 1ull) | (m ? (((1ull << m) - 1ull) << h) : 0ull);
    for (int t = tid; t < a.n_terms; t += T) {
        const Term tm = a.terms[t];
        const uint64_t zm = tm.zmask;
        const uint32_t lm = (uint32_t)(zm & ((1ull << l) - 1ull)) |
                            (uint32_t)(((zm >> h) & ((1ull << m) - 1ull)) << l);
        const int fixed = __popcll(zm & ~Smask & (uint64_t)base) & 1;
        R coef = (R)tm.coef;
        if (REV) coef *= static_cast<const R *>(a.gE)[(size_t)b * a.M + tm.obs];
        tmask[t] = lm;
        tcoef[t] = fixed ? -coef : coef;
        tobs[t] = tm.obs;
    }
    const bool analytic = a.phi_src == SRC_ANALYTIC;
    if (analytic) {
        for (int k = tid; k < a.analytic_ents; k += T) sents[k] = a.prefix_ents[k];
        const int ntab = (a.state_qubits + 3) >> 2;
        const Cx<R> *gt = static_cast<const Cx<R> *>(a.tabs) + (size_t)b * ntab * 16;
        for (int i = tid; i < ntab * 16; i += T) tabs[i] = gt[i];
    }
    __syncthreads();
    if (analytic) {
        const int ntab = (a.state_qubits + 3) >> 2;
        const int E = 1 << K;
        int td[kMaxMaskTerms];
        uint32_t tmk[kMaxMaskTerms];
        const int nl = a.amap_lin, nt = a.amap_lin + a.amap_quad;
#pragma unroll
        for (int k = 0; k < kMaxMaskTerms; ++k) {
            const MaskTerm t = k < nt ? a.amap[k] : MaskTerm{0, 0u};
            td[k] = t.d;
            tmk[k] = t.mask;
        }
        for (int e = tid; e < E; e += T) {
            uint32_t y = base | ((uint32_t)e & ((1u << l) - 1u)) | (((uint32_t)e >> l) << h);
            uint32_t xx = y;
            int sign = 0;
            if (nl >= 0) {   // closed form: x = A^{-1} y, sign from the quadratic form
                xx = 0;
#pragma unroll
                for (int k = 0; k < kMaxMaskTerms; ++k)
                    if (k < nl) xx ^= (td[k] >= 0 ? (y >> td[k]) : (y << -td[k])) & tmk[k];
                int par = __popc(xx & a.amap_dlin);
#pragma unroll
                for (int k = 0; k < kMaxMaskTerms; ++k)
                    if (k >= nl && k < nt) par += __popc(xx & (xx >> td[k]) & tmk[k]);
                sign = par & 1;
            } else {
                for (int k = a.analytic_ents - 1; k >= 0; --k) {
                    const Ent en = sents[k];
                    if (en.kind == QTM_CNOT) xx ^= ((xx >> en.a) & 1u) << en.b;
                    else sign ^= (int)((xx >> en.a) & (xx >> en.b) & 1u);
                }
            }
            Cx<R> amp = tabs[xx & 15u];
            for (int j = 1; j < ntab; ++j) amp = cmul(amp, tabs[16 * j + ((xx >> (4 * j)) & 15u)]);
            if (sign) { amp.x = -amp.x; amp.y = -amp.y; }
            sphi[swz<R>(e)] = amp;
        }
    }
    if (load_phi || load_lam) {
        bool ok = false;
        const unsigned long long t0 = global_ns();
        while (!(ok = mbar_try_wait(bar, 0)))
            if (global_ns() - t0 > kWaitLimitNs) break;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(a.status, kStatusTimeout);
            return;
        }
    } else {
        __syncthreads();
    }

    // ---- phases ----
    Cx<R> p[kRegs];
    Cx<R> q[kRegs];
    bool lam_valid = load_lam;
    for (int phz = a.phase_begin; phz < a.phase_end; ++phz) {
        const DevPhase ph = a.phases[phz];
        const int lo = ph.lo;
        const uint32_t xt = ((uint32_t)tid & ((1u << lo) - 1u)) | (((uint32_t)tid >> lo) << (lo + 4));
        // load registers
        if (sizeof(R) == 4 && lo == 0) {
#pragma unroll
            for (int k = 0; k < kRegs / 2; ++k) {
                const int s = swz<R>((int)xt + 2 * k);
                const float4 v = *reinterpret_cast<const float4 *>(&sphi[s]);
                p[2 * k] = {(R)v.x, (R)v.y};
                p[2 * k + 1] = {(R)v.z, (R)v.w};
                if (REV && lam_valid) {
                    const float4 u = *reinterpret_cast<const float4 *>(&slam[s]);
                    q[2 * k] = {(R)u.x, (R)u.y};
                    q[2 * k + 1] = {(R)u.z, (R)u.w};
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < kRegs; ++j) {
                const int s = swz<R>((int)(xt | ((uint32_t)j << lo)));
                p[j] = sphi[s];
                if (REV && lam_valid) q[j] = slam[s];
            }
        }
        // ops (the next op record is fetched while this one executes)
        DevOp nxt = a.ops[ph.op_begin < ph.op_end ? ph.op_begin : 0];
        for (int o = ph.op_begin; o < ph.op_end; ++o) {
            const DevOp op = nxt;
            if (o + 1 < ph.op_end) nxt = a.ops[o + 1];
            switch (op.type) {
            case OP_DIAG: {
                uint32_t msk = 0;
#pragma unroll 4
                for (int k = op.a; k < op.a + op.b; ++k) {
                    const DiagPair dp = a.diag[k];
                    msk ^= operand_pattern(dp.a, lo, xt, base) & operand_pattern(dp.b, lo, xt, base);
                }
#pragma unroll
                for (int j = 0; j < kRegs; ++j) {
                    const uint32_t bit = (msk >> j) & 1u;
                    flip_sign(p[j], bit);
                    if (REV) flip_sign(q[j], bit);
                }
                break;
            }
            case OP_U2:
                u2_dispatch<R>(op.a - lo, p, mats + 4 * op.slot);
                break;
            case OP_GRAD:
                if constexpr (REV) {
                    R vx = 0, vy = 0, vz = 0;
                    grad_dispatch<R>(op.a - lo, p, q, vx, vy, vz);
                    vx = warp_sum(vx, wwidth, wmask);
                    vy = warp_sum(vy, wwidth, wmask);
                    vz = warp_sum(vz, wwidth, wmask);
                    if (lane == 0) {
                        R *g = redG + (size_t)warp * 3 * a.nslots + 3 * op.slot;
                        g[0] = vx; g[1] = vy; g[2] = vz;
                    }
                    if (!(op.flags & OPF_SKIP_APPLY)) {
                        u2_dispatch<R>(op.a - lo, p, mats + 4 * op.slot);
                        u2_dispatch<R>(op.a - lo, q, mats + 4 * op.slot);
                    }
                }
                break;
            case OP_CZ: {
                int ra = -1, rb = -1, va = 0, vb = 0;
                if (op.a >= kFixed) va = (int)((base >> (op.a - kFixed)) & 1u);
                else if (op.a >= lo && op.a < lo + kRegBits) ra = op.a - lo;
                else va = (int)((xt >> op.a) & 1u);
                if (op.b >= kFixed) vb = (int)((base >> (op.b - kFixed)) & 1u);
                else if (op.b >= lo && op.b < lo + kRegBits) rb = op.b - lo;
                else vb = (int)((xt >> op.b) & 1u);
#pragma unroll
                for (int j = 0; j < kRegs; ++j) {
                    const int ba = ra >= 0 ? ((j >> ra) & 1) : va;
                    const int bb = rb >= 0 ? ((j >> rb) & 1) : vb;
                    if (ba & bb) {
                        p[j].x = -p[j].x; p[j].y = -p[j].y;
                        if (REV) { q[j].x = -q[j].x; q[j].y = -q[j].y; }
                    }
                }
                break;
            }
            case OP_CNOT: {
                int rc = -1, vc = 0;
                if (op.a >= kFixed) vc = (int)((base >> (op.a - kFixed)) & 1u);
                else if (op.a >= lo && op.a < lo + kRegBits) rc = op.a - lo;
                else vc = (int)((xt >> op.a) & 1u);
                cnot_dispatch<R>(op.b - lo, p, rc, vc);
                if (REV) cnot_dispatch<R>(op.b - lo, q, rc, vc);
                break;
            }
            case OP_EXPVAL: {
                R pr[kRegs];
#pragma unroll
                for (int j = 0; j < kRegs; ++j) pr[j] = p[j].x * p[j].x + p[j].y * p[j].y;
                int cur = -1;
                R acc = 0;
                for (int t = 0; t < a.n_terms; ++t) {
                    const int ob = tobs[t];
                    if (ob != cur) {
                        if (cur >= 0) {
                            acc = warp_sum(acc, wwidth, wmask);
                            if (lane == 0) redE[warp * a.M + cur] = acc;
                        }
                        cur = ob;
                        acc = 0;
                    }
                    const uint32_t lm = tmask[t];
                    const int tpar = __popc(xt & lm);
                    const uint32_t rm = (lm >> lo) & 15u;
                    R s = 0;
#pragma unroll
                    for (int j = 0; j < kRegs; ++j)
                        s += ((tpar + __popc((uint32_t)j & rm)) & 1) ? -pr[j] : pr[j];
                    acc = fma(tcoef[t], s, acc);
                }
                if (cur >= 0) {
                    acc = warp_sum(acc, wwidth, wmask);
                    if (lane == 0) redE[warp * a.M + cur] = acc;
                }
                break;
            }
            case OP_COSTATE:
                if constexpr (REV) {
                    R d[kRegs];
#pragma unroll
                    for (int j = 0; j < kRegs; ++j) d[j] = 0;
                    for (int t = 0; t < a.n_terms; ++t) {
                        const uint32_t lm = tmask[t];
                        const int tpar = __popc(xt & lm);
                        const uint32_t rm = (lm >> lo) & 15u;
                        const R k = tcoef[t];
#pragma unroll
                        for (int j = 0; j < kRegs; ++j)
                            d[j] += ((tpar + __popc((uint32_t)j & rm)) & 1) ? -k : k;
                    }
#pragma unroll
                    for (int j = 0; j < kRegs; ++j) q[j] = {d[j] * p[j].x, d[j] * p[j].y};
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
                *reinterpret_cast<float4 *>(&sphi[s]) =
                    make_float4((float)p[2 * k].x, (float)p[2 * k].y, (float)p[2 * k + 1].x,
                                (float)p[2 * k + 1].y);
                if (REV)
                    *reinterpret_cast<float4 *>(&slam[s]) =
                        make_float4((float)q[2 * k].x, (float)q[2 * k].y, (float)q[2 * k + 1].x,
                                    (float)q[2 * k + 1].y);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kRegs; ++j) {
                const int s = swz<R>((int)(xt | ((uint32_t)j << lo)));
                sphi[s] = p[j];
                if (REV) slam[s] = q[j];
            }
        }
        if (REV) lam_valid = true;
        __syncthreads();
    }

    // ---- partial sums to global ----
    if (!REV && a.has_expval) {
        for (int i = tid; i < a.M; i += T) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += (double)redE[w * a.M + i];
            a.Epart[((size_t)b * a.tiles + tile) * a.M + i] = s;
        }
    } else {
        const int nv = 3 * a.nslots;
        for (int i = tid; i < nv; i += T) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += (double)redG[w * nv + i];
            const int run = a.slot_runs[a.slot_begin + i / 3];
            a.Gpart[(((size_t)b * a.n_runs + run) * a.tiles + tile) * 3 + (i % 3)] = s;
        }
    }

    // ---- write the tile back ----
    if (a.store_phi || (REV && a.store_lam)) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            if (a.store_phi) tma_store(&tm_phi, coord, a.rank, sphi);
            if (REV && a.store_lam) tma_store(&tm_lam, coord, a.rank, slam);
            tma_store_commit_and_drain();
        }
    }
}

template <typename R>
__global__ void k_expval_finalize(const double *Epart, int B, int tiles, int M, R *E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * M) return;
    const int b = i / M, m = i % M;
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += Epart[((size_t)b * tiles + t) * M + m];
    E[i] = (R)s;
}

template <typename R>
__global__ void k_grad_finalize(const FinalizeArgs f)
{
    const int b = blockIdx.x;
    const R *xb = static_cast<const R *>(f.x) + (size_t)b * f.n_in;
    const R *w = static_cast<const R *>(f.w);
    double *abar = f.abar + (size_t)b * f.n_rots;
    for (int r = threadIdx.x; r < f.n_runs; r += blockDim.x) {
        double v[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < f.tiles; ++t)
            for (int c = 0; c < 3; ++c) v[c] += f.Gpart[(((size_t)b * f.n_runs + r) * f.tiles + t) * 3 + c];
        const Run rr = f.runs[r];
        // u <- v; walk the run backwards (see finalize_math.h)
        for (int i = rr.rot_end - 1; i >= rr.rot_begin; --i) {
            const Rot ro = f.rots[i];
            double t = ro.coef;
            if (ro.w_idx >= 0) t *= (double)w[ro.w_idx];
            if (ro.x_idx >= 0) t *= (double)xb[ro.x_idx];
            abar[i] = v[ro.kind];
            adjoint_transpose_apply(ro.kind, t, v);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < f.P; j += blockDim.x) {
        double s = 0.0;
        for (int k = f.w_ptr[j]; k < f.w_ptr[j + 1]; ++k) {
            const int ri = f.w_rots[k];
            const Rot ro = f.rots[ri];
            s += abar[ri] * ro.coef * (ro.x_idx >= 0 ? (double)xb[ro.x_idx] : 1.0);
        }
        if (f.gw_out) static_cast<R *>(f.gw_out)[(size_t)b * f.P + j] = (R)s;
        if (f.gw_ws) f.gw_ws[(size_t)b * f.P + j] = s;
    }
    if (f.gx)
        for (int k = threadIdx.x; k < f.n_in; k += blockDim.x) {
            double s = 0.0;
            for (int i = f.x_ptr[k]; i < f.x_ptr[k + 1]; ++i) {
                const int ri = f.x_rots[i];
                const Rot ro = f.rots[ri];
                s += abar[ri] * ro.coef * (ro.w_idx >= 0 ? (double)w[ro.w_idx] : 1.0);
            }
            static_cast<R *>(f.gx)[(size_t)b * f.n_in + k] = (R)s;
        }
}

// grad_w[j] = sum_b gw_ws[b][j]: one CTA per weight, each thread a fixed
// strided subset of samples, then a fixed-shape tree: deterministic.
template <typename R>
__global__ void k_gw_reduce(const double *gw_ws, int B, int P, R *gw)
{
    __shared__ double red[256];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += gw_ws[(size_t)b * P + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gw[j] = (R)red[0];
}

}  // namespace

size_t pass_smem_bytes(int K, int dtype, bool reverse, int nslots, int n_terms, int M,
                       int state_qubits, int n_prefix_ents)
{
    const int csize = dtype == QTM_C128 ? 16 : 8;
    const int rsize = csize / 2;
    const int T = K >= 4 ? (1 << (K - 4)) : 1;
    const int nwarps = (T + 31) / 32;
    Layout L = make_layout(K, csize, reverse, nslots, n_terms, M, state_qubits, n_prefix_ents,
                           nwarps, rsize);
    return (size_t)L.total + 1024;
}

cudaError_t launch_pass(int dtype, bool reverse, const PassArgs &a, const CUtensorMap &tm_phi,
                        const CUtensorMap &tm_lam, cudaStream_t s)
{
    const int T = 1 << (a.K - 4);
    const dim3 grid((unsigned)a.B * (unsigned)a.tiles), block((unsigned)T);
    const size_t smem = (size_t)a.smem_bytes;
    cudaError_t e;
#define QTM_LAUNCH(R, REV)                                                                     \
    do {                                                                                       \
        auto fn = k_pass<R, REV>;                                                              \
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        if (e != cudaSuccess) return e;                                                        \
        fn<<<grid, block, smem, s>>>(a, tm_phi, tm_lam);                                       \
    } while (0)
    if (dtype == QTM_C128) {
        if (reverse) QTM_LAUNCH(double, true); else QTM_LAUNCH(double, false);
    } else {
        if (reverse) QTM_LAUNCH(float, true); else QTM_LAUNCH(float, false);
    }
#undef QTM_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_prep(int dtype, const PrepArgs &a, cudaStream_t s)
{
    if (dtype == QTM_C128) k_prep<double><<<a.B, 128, 0, s>>>(a);
    else k_prep<float><<<a.B, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_expval_finalize(int dtype, const FinalizeArgs &f, cudaStream_t s)
{
    const int n = f.B * f.M;
    const int blk = 256, grd = (n + blk - 1) / blk;
    if (dtype == QTM_C128)
        k_expval_finalize<double><<<grd, blk, 0, s>>>(f.Epart, f.B, f.tiles, f.M, static_cast<double *>(f.E));
    else
        k_expval_finalize<float><<<grd, blk, 0, s>>>(f.Epart, f.B, f.tiles, f.M, static_cast<float *>(f.E));
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(int dtype, const FinalizeArgs &f, cudaStream_t s)
{
    if (dtype == QTM_C128) k_grad_finalize<double><<<f.B, 256, 0, s>>>(f);
    else k_grad_finalize<float><<<f.B, 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_gw_reduce(int dtype, const double *gw_ws, int B, int P, void *gw, cudaStream_t s)
{
    if (P <= 0) return cudaSuccess;
    if (dtype == QTM_C128) k_gw_reduce<double><<<P, 256, 0, s>>>(gw_ws, B, P, static_cast<double *>(gw));
    else k_gw_reduce<float><<<P, 256, 0, s>>>(gw_ws, B, P, static_cast<float *>(gw));
    return cudaGetLastError();
}

}  // namespace qtm
