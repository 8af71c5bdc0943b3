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

// Registers <-> shared tile (one-sample layout) for register group LO, lane bit S.
template <int LO, int S, bool LAM>
__device__ __forceinline__ void regs_load_lanes(A2 (&p)[kLanePairs], A2 (&q)[kLanePairs], const TileSmem<float> &T,
                                                uint32_t xt)
{
    Cx<float> a[kRegs], b[kRegs];
    regs_load<float, LO, LAM>(a, b, T, xt);
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const int j0 = lane_jj<S>(k, 0), j1 = lane_jj<S>(k, 1);
        p[k] = {pack2(a[j0].x, a[j1].x), pack2(a[j0].y, a[j1].y)};
        if (LAM) q[k] = {pack2(b[j0].x, b[j1].x), pack2(b[j0].y, b[j1].y)};
    }
}

template <int LO, int S, bool LAM>
__device__ __forceinline__ void regs_store_lanes(const A2 (&p)[kLanePairs], const A2 (&q)[kLanePairs],
                                                 const TileSmem<float> &T, uint32_t xt)
{
    Cx<float> a[kRegs], b[kRegs];
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const int j0 = lane_jj<S>(k, 0), j1 = lane_jj<S>(k, 1);
        a[j0] = {lane0(p[k].r), lane0(p[k].i)};
        a[j1] = {lane1(p[k].r), lane1(p[k].i)};
        if (LAM) {
            b[j0] = {lane0(q[k].r), lane0(q[k].i)};
            b[j1] = {lane1(q[k].r), lane1(q[k].i)};
        }
    }
    regs_store<float, LO, LAM>(a, b, T, xt);
}

// a <- U a on register bit RB != S (whole registers pair up)
template <int S, int RB>
__device__ __forceinline__ void u2_lanes(A2 (&a)[kLanePairs], const f2 *t)
{
    constexpr int kb = RB < S ? RB : RB - 1;
    const ulonglong2 *mv = reinterpret_cast<const ulonglong2 *>(t);
    const ulonglong2 w0 = mv[0], w1 = mv[1], w2 = mv[2], w3 = mv[3], w4 = mv[4], w5 = mv[5];
    const f2 a_r = w0.x, a_i = w0.y, a_n = w1.x;
    const f2 b_r = w1.y, b_i = w2.x, b_n = w2.y;
    const f2 c_r = w3.x, c_i = w3.y, c_n = w4.x;
    const f2 d_r = w4.y, d_i = w5.x, d_n = w5.y;
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
__device__ __forceinline__ void u2_lanes_s(A2 (&a)[kLanePairs], const f2 *t)
{
    const ulonglong2 *mv = reinterpret_cast<const ulonglong2 *>(t + 12);
    const ulonglong2 w0 = mv[0], w1 = mv[1], w2 = mv[2];
    const f2 D_r = w0.x, D_i = w0.y, D_n = w1.x, O_r = w1.y, O_i = w2.x, O_n = w2.y;
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
    f2 xp = 0, xn = 0, yp = 0, yn = 0, zp = 0, zn = 0;
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        if (k & (1 << kb)) continue;
        const A2 a0 = a[k], a1 = a[k | (1 << kb)], b0 = b[k], b1 = b[k | (1 << kb)];
        zp = fma2(b0.r, a0.i, zp); zn = fma2(b0.i, a0.r, zn);
        zn = fma2(b1.r, a1.i, zn); zp = fma2(b1.i, a1.r, zp);
        xp = fma2(b0.r, a1.i, xp); xn = fma2(b0.i, a1.r, xn);
        xp = fma2(b1.r, a0.i, xp); xn = fma2(b1.i, a0.r, xn);
        yp = fma2(b1.r, a0.r, yp); yp = fma2(b1.i, a0.i, yp);
        yn = fma2(b0.r, a1.r, yn); yn = fma2(b0.i, a1.i, yn);
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
    f2 zp = 0, zn = 0, xp = 0, xn = 0, yy = 0;
#pragma unroll
    for (int k = 0; k < kLanePairs; ++k) {
        const A2 x = a[k], l = b[k];
        const f2 sr = swap2(x.r), si = swap2(x.i);
        zp = fma2(l.r, x.i, zp); zn = fma2(l.i, x.r, zn);   // lane-wise Im(conj(lam) phi)
        xp = fma2(l.r, si, xp); xn = fma2(l.i, sr, xn);     // lane-wise Im(conj(lam) swap(phi))
        yy = fma2(l.r, sr, yy); yy = fma2(l.i, si, yy);     // lane-wise Re(conj(lam) swap(phi))
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
