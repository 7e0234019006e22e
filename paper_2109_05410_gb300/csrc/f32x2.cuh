// f32x2.cuh -- packed FP32 pairs for the sm_100-family packed instructions.
//
// add.rn.f32x2, mul.rn.f32x2 and fma.rn.f32x2 carry out two IEEE
// single-precision operations in one instruction on a 64-bit register pair,
// each lane rounded to nearest even exactly as the scalar add / mul / fma
// round (no flush to zero without .ftz).  A stencil that evaluates two
// neighbouring points with the same operation sequence therefore gives the
// bits of the scalar code with half the floating-point instructions.
#pragma once

namespace ooc {
namespace sten {

struct F2 {
    unsigned long long v;  // lane 0 in the low word
};

__device__ __forceinline__ F2 pk2(float lo, float hi)
{
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ F2 dup2(float a) { return pk2(a, a); }

__device__ __forceinline__ void unpk2(F2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}

__device__ __forceinline__ F2 add2(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ F2 mul2(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// a * b + c per lane, one rounding
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

}  // namespace sten
}  // namespace ooc
