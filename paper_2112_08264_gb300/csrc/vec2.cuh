// vec2.cuh -- packed FP32 pairs.
//
// Blackwell executes two FP32 additions, multiplications or fused
// multiply-adds per lane in one instruction on a 64-bit register pair
// (add/sub/mul/fma .f32x2). The two components A and B of a lattice node
// undergo the same arithmetic (density sums, force sums, the equilibrium and
// the relaxation of each velocity), so a float2 holding (A, B) halves the
// instruction count of those steps. Every operation rounds to nearest-even,
// element by element, exactly as the scalar instruction would; none of them
// is contracted or reassociated by the compiler.
#pragma once
#include <cuda_runtime.h>

namespace lbgb {

__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
          "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&r);
}

}  // namespace lbgb
