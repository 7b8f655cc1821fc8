// f32x2.cuh -- packed FP32 pairs for sm_100-class GPUs.
//
// Blackwell executes FADD2 / FMUL2 / FFMA2 on a pair of FP32 values per lane and instruction.
// The structured-grid kernels evaluate the x-face and the y-face of a cell as the two halves of
// one pair, so every arithmetic step of the face term costs one instruction for both faces.
#pragma once
#include <cuda_runtime.h>

namespace zoomy {

struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float x, float y) { v = make_float2(x, y); }
    __device__ __forceinline__ explicit F2(float s) { v = make_float2(s, s); }
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
};

__device__ __forceinline__ unsigned long long as_u64(F2 a)
{
    return (unsigned long long)__float_as_uint(a.v.x) | ((unsigned long long)__float_as_uint(a.v.y) << 32);
}
__device__ __forceinline__ F2 from_u64(unsigned long long u)
{
    return F2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
}
// Every packed operation is written as PTX with an explicit rounding modifier.  The compiler can
// neither split such an instruction into scalar halves (it may do that with the equivalent
// intrinsics when one half of a result is unused) nor contract a .rn multiply into a later addition,
// so an expression rounds the same way wherever it is inlined.  The stage kernels rely on this for
// results that are bitwise independent of the row decomposition.
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)));
    return from_u64(d);
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)));
    return from_u64(d);
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)));
    return from_u64(d);
}
// a * b + c
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
    return from_u64(d);
}

}  // namespace zoomy
