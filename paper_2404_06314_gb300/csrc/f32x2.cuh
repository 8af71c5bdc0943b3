// Blackwell's paired FP32 operations on f32x2 register pairs.
//
// The FP32 datapath of sm_103a executes fma / mul / add / sub on .f32x2
// operands: one instruction, two lanes of work.  The complex-pair pass kernels
// (tile_cpx.cuh) keep each complex64 amplitude as one such pair (re, im).
#pragma once

#include "tile.cuh"

namespace qtm {

namespace {

typedef unsigned long long f2;   // the two 32-bit lanes of one f32x2 register pair

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

}  // namespace

}  // namespace qtm
