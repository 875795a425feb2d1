// Two lanes of FP32 arithmetic per instruction.  The sm_100 family executes
// fma / add / mul on a pair of floats held in a 64-bit register pair
// (fma.rn.f32x2 and friends, reached through __ffma2_rn, __fadd2_rn,
// __fmul2_rn); each half is rounded exactly as the scalar fmaf / __fadd_rn /
// __fmul_rn of the same operands, so a formula evaluated on pairs gives the
// bits of the same formula evaluated one sample at a time.  The helpers below
// take float or float2 so that one formula serves both, with every operation
// explicit (nothing left for the compiler to contract into an fma).
// Functions without a packed form (the MUFU square roots and reciprocals,
// rounding to an integer, compares and selects) are applied lane by lane.
#pragma once
#include <cuda_runtime.h>

namespace vndf {

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }

template <typename V>
__device__ __forceinline__ V splat(float a);
template <>
__device__ __forceinline__ float splat<float>(float a) { return a; }
template <>
__device__ __forceinline__ float2 splat<float2>(float a) { return make_float2(a, a); }

// b - a as fma(a, -1, b): the product is exact, so this is the correctly rounded difference.
template <typename V>
__device__ __forceinline__ V vsub(V b, V a) { return vfma(a, splat<V>(-1.f), b); }

// A scalar function applied to each lane.
template <typename F>
__device__ __forceinline__ float vmap(F f, float x) { return f(x); }
template <typename F>
__device__ __forceinline__ float2 vmap(F f, float2 x) { return make_float2(f(x.x), f(x.y)); }
template <typename F>
__device__ __forceinline__ float vmap(F f, float x, float y) { return f(x, y); }
template <typename F>
__device__ __forceinline__ float2 vmap(F f, float2 x, float2 y) { return make_float2(f(x.x, y.x), f(x.y, y.y)); }

}  // namespace vndf
