// Lane-paired registers for the one-sample specialised pass kernels.
//
// A thread's 16 amplitudes (register bits [lo, lo+4) of a phase) are held as
// 8 f32x2 register pairs: pair k holds the amplitudes j0, j1 that differ only
// in one chosen register bit s (lane 0: bit s = 0, lane 1: bit s = 1); k
// enumerates the other three bits.  A gate on a register bit other than s then
// pairs whole registers (k, k') and runs as two-lane SIMD with the matrix
// entries broadcast to both lanes; a gate on bit s mixes the two lanes of
// each register: Y = D * X + O * swap(X) with D = (u00, u11), O = (u01, u10).
// The sample, the shared-memory layout and the tile program (tile.cuh) are
// those of the one-sample kernel; the register file per thread is the same,
// so occupancy is unchanged while most FP32 instructions become f32x2.
#pragma once

#include "tile_x2.cuh"

namespace qtm {

namespace {

constexpr int kLanePairs = 8;
constexpr int kLaneSlotPairs = 18;   // per run slot: 12 broadcast pairs, then D_r D_i D_n O_r O_i O_n

// register index jj of lane h of pair k with s the lane bit
template <int S>
__host__ __device__ constexpr int lane_jj(int k, int h)
{
    return ((k >> S) << (S + 1)) | (h << S) | (k & ((1 << S) - 1));
}

// 16-byte table read.  VT: one the compiler may not merge with an earlier
// read (the table's registers are free between two applications), else a
// plain load the compiler may schedule and reuse freely.
template <bool VT>
__device__ __forceinline__ void lds_table2(const f2 *t, f2 &a, f2 &b)
{
    if constexpr (VT) {
        asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(smem_u32(t)));
    } else {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(t);
        a = v.x;
        b = v.y;
    }
}

__device__ __forceinline__ f2 swap2(f2 v)
{
    f2 d;
    asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tmov.b64 %0, {hi, lo};\n\t}" : "=l"(d) : "l"(v));
    return d;
}

// lane 0 of x with lane 1 of y
__device__ __forceinline__ f2 merge2(f2 x, f2 y) { return pack2(lane0(x), lane1(y)); }

// Lane-pair table of every run slot from the staged matrices (U or U^dagger).
__device__ __forceinline__ void stage_lane_table(const Cx<float> *mats, f2 *tab, int nslots)
{
    for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
        const Cx<float> u00 = mats[4 * s], u01 = mats[4 * s + 1], u10 = mats[4 * s + 2], u11 = mats[4 * s + 3];
        f2 *t = tab + kLaneSlotPairs * s;
        const Cx<float> e[4] = {u00, u01, u10, u11};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            t[3 * k] = pack2(e[k].x, e[k].x);
            t[3 * k + 1] = pack2(e[k].y, e[k].y);
            t[3 * k + 2] = pack2(-e[k].y, -e[k].y);
        }
        t[12] = pack2(u00.x, u11.x);
        t[13] = pack2(u00.y, u11.y);
        t[14] = pack2(-u00.y, -u11.y);
        t[15] = pack2(u01.x, u10.x);
        t[16] = pack2(u01.y, u10.y);
        t[17] = pack2(-u01.y, -u10.y);
    }
}

// Registers <-> shared tile (one-sample layout) for register group LO, lane bit
// S.  Scalar 32-bit accesses put every value straight into its lane of the
// destination pair (no repacking through temporaries).
__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts_f32(uint32_t addr, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Register group at tile bit 0 with lane bit 0: a 16-byte element pair
// (re0, im0, re1, im1) is exactly one lane pair; 16-byte accesses keep the
// swizzled rows free of bank conflicts.
template <bool LAM>
__device__ __forceinline__ void regs_load_lanes_lo0(A2 (&p)[kLanePairs], A2 (&q)[kLanePairs], const TileSmem<float> &T,
                                                    uint32_t xt)
{
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const int s = swz<float>((int)xt + 2 * k);
        const float4 v = *reinterpret_cast<const float4 *>(&T.phi[s]);
        p[k] = {pack2(v.x, v.z), pack2(v.y, v.w)};
        if (LAM) {
            const float4 u = *reinterpret_cast<const float4 *>(&T.lam[s]);
            q[k] = {pack2(u.x, u.z), pack2(u.y, u.w)};
        }
    }
}

template <bool LAM>
__device__ __forceinline__ void regs_store_lanes_lo0(const A2 (&p)[kLanePairs], const A2 (&q)[kLanePairs],
                                                     const TileSmem<float> &T, uint32_t xt)
{
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const int s = swz<float>((int)xt + 2 * k);
        *reinterpret_cast<float4 *>(&T.phi[s]) = make_float4(lane0(p[k].r), lane0(p[k].i), lane1(p[k].r), lane1(p[k].i));
        if (LAM)
            *reinterpret_cast<float4 *>(&T.lam[s]) =
                make_float4(lane0(q[k].r), lane0(q[k].i), lane1(q[k].r), lane1(q[k].i));
    }
}

// One complex amplitude (re, im) as a 64-bit shared access.
__device__ __forceinline__ void lds_c64(uint32_t addr, float &re, float &im)
{
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(re), "=f"(im) : "r"(addr));
}
__device__ __forceinline__ void sts_c64(uint32_t addr, float re, float im)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(re), "f"(im) : "memory");
}

// V64: 64-bit accesses outside group 0 (conflict-free rows, lanes assembled
// by register moves) instead of scalar 32-bit accesses.
template <int LO, int S, bool LAM, bool V64 = false>
__device__ __forceinline__ void regs_load_lanes(A2 (&p)[kLanePairs], A2 (&q)[kLanePairs], const TileSmem<float> &T,
                                                uint32_t xt)
{
    if constexpr (LO == 0 && S == 0) {
        regs_load_lanes_lo0<LAM>(p, q, T, xt);
        return;
    }
    const uint32_t ph = smem_u32(T.phi), lm = smem_u32(T.lam);
    if constexpr (V64) {
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const uint32_t o0 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 0) << LO)));
        const uint32_t o1 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 1) << LO)));
        float r0, i0, r1, i1;
        lds_c64(ph + o0, r0, i0);
        lds_c64(ph + o1, r1, i1);
        p[k] = {pack2(r0, r1), pack2(i0, i1)};
        if (LAM) {
            lds_c64(lm + o0, r0, i0);
            lds_c64(lm + o1, r1, i1);
            q[k] = {pack2(r0, r1), pack2(i0, i1)};
        }
    }
    return;
    }
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const uint32_t o0 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 0) << LO)));
        const uint32_t o1 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 1) << LO)));
        p[k] = {pack2(lds_f32(ph + o0), lds_f32(ph + o1)), pack2(lds_f32(ph + o0 + 4), lds_f32(ph + o1 + 4))};
        if (LAM) q[k] = {pack2(lds_f32(lm + o0), lds_f32(lm + o1)), pack2(lds_f32(lm + o0 + 4), lds_f32(lm + o1 + 4))};
    }
}

template <int LO, int S, bool LAM, bool V64 = false>
__device__ __forceinline__ void regs_store_lanes(const A2 (&p)[kLanePairs], const A2 (&q)[kLanePairs],
                                                 const TileSmem<float> &T, uint32_t xt)
{
    if constexpr (LO == 0 && S == 0) {
        regs_store_lanes_lo0<LAM>(p, q, T, xt);
        return;
    }
    const uint32_t ph = smem_u32(T.phi), lm = smem_u32(T.lam);
    if constexpr (V64) {
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const uint32_t o0 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 0) << LO)));
        const uint32_t o1 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 1) << LO)));
        sts_c64(ph + o0, lane0(p[k].r), lane0(p[k].i));
        sts_c64(ph + o1, lane1(p[k].r), lane1(p[k].i));
        if (LAM) {
            sts_c64(lm + o0, lane0(q[k].r), lane0(q[k].i));
            sts_c64(lm + o1, lane1(q[k].r), lane1(q[k].i));
        }
    }
    return;
    }
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const uint32_t o0 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 0) << LO)));
        const uint32_t o1 = 8u * (uint32_t)swz<float>((int)(xt | ((uint32_t)lane_jj<S>(k, 1) << LO)));
        sts_f32(ph + o0, lane0(p[k].r)); sts_f32(ph + o1, lane1(p[k].r));
        sts_f32(ph + o0 + 4, lane0(p[k].i)); sts_f32(ph + o1 + 4, lane1(p[k].i));
        if (LAM) {
            sts_f32(lm + o0, lane0(q[k].r)); sts_f32(lm + o1, lane1(q[k].r));
            sts_f32(lm + o0 + 4, lane0(q[k].i)); sts_f32(lm + o1 + 4, lane1(q[k].i));
        }
    }
}

// a <- U a on register bit RB != S (whole registers pair up)
template <int S, int RB, bool VT = true>
__device__ __forceinline__ void u2_lanes(A2 (&a)[kLanePairs], const f2 *t)
{
    constexpr int kb = RB < S ? RB : RB - 1;
    f2 a_r, a_i, a_n, b_r, b_i, b_n, c_r, c_i, c_n, d_r, d_i, d_n;
    lds_table2<VT>(t, a_r, a_i); lds_table2<VT>(t + 2, a_n, b_r); lds_table2<VT>(t + 4, b_i, b_n);
    lds_table2<VT>(t + 6, c_r, c_i); lds_table2<VT>(t + 8, c_n, d_r); lds_table2<VT>(t + 10, d_i, d_n);
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        if (k & (1 << kb)) continue;
        const A2 x0 = a[k], x1 = a[k | (1 << kb)];
        a[k].r = fma2(a_r, x0.r, fma2(a_n, x0.i, fma2(b_r, x1.r, mul2(b_n, x1.i))));
        a[k].i = fma2(a_r, x0.i, fma2(a_i, x0.r, fma2(b_r, x1.i, mul2(b_i, x1.r))));
        a[k | (1 << kb)].r = fma2(c_r, x0.r, fma2(c_n, x0.i, fma2(d_r, x1.r, mul2(d_n, x1.i))));
        a[k | (1 << kb)].i = fma2(c_r, x0.i, fma2(c_i, x0.r, fma2(d_r, x1.i, mul2(d_i, x1.r))));
    }
}

// a <- U a on the lane bit S: Y = D X + O swap(X)
template <bool VT = true>
__device__ __forceinline__ void u2_lanes_s(A2 (&a)[kLanePairs], const f2 *t)
{
    f2 D_r, D_i, D_n, O_r, O_i, O_n;
    lds_table2<VT>(t + 12, D_r, D_i); lds_table2<VT>(t + 14, D_n, O_r); lds_table2<VT>(t + 16, O_i, O_n);
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const A2 x = a[k];
        const f2 sr = swap2(x.r), si = swap2(x.i);
        a[k].r = fma2(D_r, x.r, fma2(D_n, x.i, fma2(O_r, sr, mul2(O_n, si))));
        a[k].i = fma2(D_r, x.i, fma2(D_i, x.r, fma2(O_r, si, mul2(O_i, sr))));
    }
}

// (vx, vy, vz) of one sample over the pairs on register bit RB != S: both
// lanes hold pairs of the same sample and are added at the end.
template <int S, int RB>
__device__ __forceinline__ void grad_lanes(const A2 (&a)[kLanePairs], const A2 (&b)[kLanePairs], float &vx, float &vy,
                                           float &vz)
{
    constexpr int kb = RB < S ? RB : RB - 1;
    f2 xp, xn, yp, yn, zp, zn;
#pragma unroll
    for (int k = 0, first = 1; k < kLanePairs; ++k) {
        if (k & (1 << kb)) continue;
        const A2 a0 = a[k], a1 = a[k | (1 << kb)], b0 = b[k], b1 = b[k | (1 << kb)];
        if (first) {   // the first pair starts the accumulators (no zero fill)
            zp = mul2(b0.r, a0.i); zn = mul2(b0.i, a0.r);
            xp = mul2(b0.r, a1.i); xn = mul2(b0.i, a1.r);
            yp = mul2(b1.r, a0.r); yn = mul2(b0.r, a1.r);
            first = 0;
        } else {
            zp = fma2(b0.r, a0.i, zp); zn = fma2(b0.i, a0.r, zn);
            xp = fma2(b0.r, a1.i, xp); xn = fma2(b0.i, a1.r, xn);
            yp = fma2(b1.r, a0.r, yp); yn = fma2(b0.r, a1.r, yn);
        }
        zn = fma2(b1.r, a1.i, zn); zp = fma2(b1.i, a1.r, zp);
        xp = fma2(b1.r, a0.i, xp); xn = fma2(b1.i, a0.r, xn);
        yp = fma2(b1.i, a0.i, yp); yn = fma2(b0.i, a1.i, yn);
    }
    const f2 X = sub2(xp, xn), Y = sub2(yp, yn), Z = sub2(zp, zn);
    vx = lane0(X) + lane1(X);
    vy = lane0(Y) + lane1(Y);
    vz = lane0(Z) + lane1(Z);
}

// (vx, vy, vz) over the pairs on the lane bit S (lane 0 = bit 0, lane 1 = bit 1).
__device__ __forceinline__ void grad_lanes_s(const A2 (&a)[kLanePairs], const A2 (&b)[kLanePairs], float &vx,
                                             float &vy, float &vz)
{
    f2 zp, zn, xp, xn, yy;
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const A2 x = a[k], l = b[k];
        const f2 sr = swap2(x.r), si = swap2(x.i);
        if (k == 0) {   // the first register starts the accumulators
            zp = mul2(l.r, x.i); zn = mul2(l.i, x.r);
            xp = mul2(l.r, si); xn = mul2(l.i, sr);
            yy = mul2(l.r, sr);
        } else {
            zp = fma2(l.r, x.i, zp); zn = fma2(l.i, x.r, zn);   // lane-wise Im(conj(lam) phi)
            xp = fma2(l.r, si, xp); xn = fma2(l.i, sr, xn);     // lane-wise Im(conj(lam) swap(phi))
            yy = fma2(l.r, sr, yy);                             // lane-wise Re(conj(lam) swap(phi))
        }
        yy = fma2(l.i, si, yy);
    }
    const f2 Z = sub2(zp, zn), X = sub2(xp, xn);
    vz = lane0(Z) - lane1(Z);
    vx = lane0(X) + lane1(X);
    vy = lane1(yy) - lane0(yy);
}

// CNOT, control and target register bits (RC, RT), lane bit S.
template <int S, int RC, int RT>
__device__ __forceinline__ void cnot_lanes_static(A2 (&a)[kLanePairs])
{
    if constexpr (RT == S) {   // swap the lanes of registers whose control bit is set
        constexpr int kc = RC < S ? RC : RC - 1;
#pragma unroll
        for (int k = 0; k < kLanePairs; ++k)
            if (k & (1 << kc)) a[k] = {swap2(a[k].r), swap2(a[k].i)};
    } else if constexpr (RC == S) {   // exchange lane 1 between the target pair of registers
        constexpr int kt = RT < S ? RT : RT - 1;
#pragma unroll
        for (int k = 0; k < kLanePairs; ++k) {
            if (k & (1 << kt)) continue;
            const A2 x0 = a[k], x1 = a[k | (1 << kt)];
            a[k] = {merge2(x0.r, x1.r), merge2(x0.i, x1.i)};
            a[k | (1 << kt)] = {merge2(x1.r, x0.r), merge2(x1.i, x0.i)};
        }
    } else {   // whole registers trade places
        constexpr int kc = RC < S ? RC : RC - 1, kt = RT < S ? RT : RT - 1;
#pragma unroll
        for (int k = 0; k < kLanePairs; ++k) {
            if ((k & (1 << kt)) || !(k & (1 << kc))) continue;
            const A2 t = a[k];
            a[k] = a[k | (1 << kt)];
            a[k | (1 << kt)] = t;
        }
    }
}

// CNOT on target register bit RT with a control bit c known per thread.
template <int S, int RT>
__device__ __forceinline__ void cnot_lanes(A2 (&a)[kLanePairs], int c)
{
    if constexpr (RT == S) {
#pragma unroll
        for (int k = 0; k < kLanePairs; ++k) {
            const A2 x = a[k];
            a[k] = c ? A2{swap2(x.r), swap2(x.i)} : x;
        }
    } else {
        constexpr int kt = RT < S ? RT : RT - 1;
#pragma unroll
        for (int k = 0; k < kLanePairs; ++k) {
            if (k & (1 << kt)) continue;
            const A2 t0 = a[k], t1 = a[k | (1 << kt)];
            a[k] = c ? t1 : t0;
            a[k | (1 << kt)] = c ? t0 : t1;
        }
    }
}

// Negate amplitude jj where bit jj of m is set (phi, and lam in reverse).
template <int S, bool REV>
__device__ __forceinline__ void flip_lanes(A2 (&p)[kLanePairs], A2 (&q)[kLanePairs], uint32_t m)
{
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const int j0 = lane_jj<S>(k, 0), j1 = lane_jj<S>(k, 1);
        const f2 s = pack2(__uint_as_float(((m >> j0) & 1u) << 31), __uint_as_float(((m >> j1) & 1u) << 31));
        p[k].r ^= s; p[k].i ^= s;
        if (REV) { q[k].r ^= s; q[k].i ^= s; }
    }
}

}  // namespace

}  // namespace qtm
