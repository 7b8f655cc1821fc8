// f32x2.cuh -- packed FP32 pairs for sm_100-class GPUs.
//
// Blackwell executes FADD2 / FMUL2 / FFMA2 on a pair of FP32 values per lane and instruction.
// The structured-grid kernels evaluate the x-face and the y-face of a cell as the two halves of
// one pair, so every arithmetic step of the face term costs one instruction for both faces.
// Subtraction goes through sub.rn.f32x2 so that no operand needs a separate negation.
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

__device__ __forceinline__ F2 mk2(float2 a)
{
    F2 r;
    r.v = a;
    return r;
}
__device__ __forceinline__ unsigned long long as_u64(F2 a)
{
    return (unsigned long long)__float_as_uint(a.v.x) | ((unsigned long long)__float_as_uint(a.v.y) << 32);
}
__device__ __forceinline__ F2 from_u64(unsigned long long u)
{
    return F2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return mk2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return mk2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_u64(a)), "l"(as_u64(b)));
    return from_u64(d);
}
// a * b + c
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return mk2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 max2(F2 a, F2 b) { return F2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }

}  // namespace zoomy
