// Packed FP32 pairs for the two-cells-per-lane step kernel.
//
// sm_100-class GPUs execute FP32 add, multiply and fused multiply-add on a
// pair of values in one instruction (PTX add/sub/mul/fma .f32x2).  A lane of
// the step kernel owns two neighbouring cells of a row, so every operation of
// the collision is one such instruction for both cells.  Each component is
// rounded exactly like the scalar FP32 operation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

struct F2 {
    float x, y;  // the even and the odd cell of a lane
};

__device__ __forceinline__ uint64_t f2_bits(F2 a)
{
    return (uint64_t)__float_as_uint(a.x) | ((uint64_t)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ F2 f2_from_bits(uint64_t b)
{
    return F2{__uint_as_float((uint32_t)b), __uint_as_float((uint32_t)(b >> 32))};
}
__device__ __forceinline__ F2 f2(float s) { return F2{s, s}; }
__device__ __forceinline__ F2 f2(float a, float b) { return F2{a, b}; }

__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(d);
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(d);
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(d);
}
// a * b + c, one rounding per component
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from_bits(d);
}
// -a (a subtraction from zero: one packed instruction)
__device__ __forceinline__ F2 neg2(F2 a) { return f2(0.0f) - a; }
// c - a * b, fused
__device__ __forceinline__ F2 fnma2(F2 a, F2 b, F2 c) { return fma2(neg2(a), b, c); }
__device__ __forceinline__ F2 operator*(float s, F2 a) { return f2(s) * a; }
__device__ __forceinline__ F2 operator*(F2 a, float s) { return a * f2(s); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }

// 1/x per component: hardware approximation refined by one Newton-Raphson step
// (e = 1 - x r, r' = r + r e), correct to about 1 ulp.
__device__ __forceinline__ float rcp_nr(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}
__device__ __forceinline__ F2 recip2(F2 x, F2 one)
{
    F2 r{0.f, 0.f};
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(x.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(x.y));
    const F2 e = fnma2(x, r, one);
    return fma2(r, e, r);
}

}  // namespace lbm
