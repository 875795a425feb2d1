// Two lanes of FP32 arithmetic per instruction.  The sm_100 family executes
// fma / add / sub / mul on a pair of floats held in a 64-bit register pair
// (the PTX .f32x2 forms of those instructions); each half is rounded exactly
// as the scalar instruction with the same rounding modifier, so a formula
// evaluated on pairs gives the bits of the same formula evaluated one sample at
// a time.  The helpers below take float or float2 so that one formula serves
// both, with every operation explicit: the packed forms are written as inline
// PTX with .rn, and the scalar ones as fmaf / __fmul_rn / __fadd_rn /
// __fsub_rn, so that neither width leaves a multiply and an add for the
// compiler to contract into an fma (the packed intrinsics __fmul2_rn and
// __fadd2_rn can be contracted, which changes the rounding of one width only).
// Functions without a packed form (the MUFU square roots and reciprocals,
// rounding to an integer, compares and selects) are applied lane by lane.
#pragma once
#include <cuda_runtime.h>

namespace vndf {

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }

__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
      "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "mul.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

// A roughness known to be 1 at compile time (the hemisphere configuration): products with it are the
// other factor, with no instruction (an inline-PTX multiply by 1 would not be folded away).
struct UnitAlpha {};
__device__ __forceinline__ float vmul(UnitAlpha, float x) { return x; }
__device__ __forceinline__ float2 vmul(UnitAlpha, float2 x) { return x; }
__device__ __forceinline__ float vmul(float x, UnitAlpha) { return x; }
__device__ __forceinline__ float2 vmul(float2 x, UnitAlpha) { return x; }

template <typename V>
__device__ __forceinline__ V splat(float a);
template <>
__device__ __forceinline__ float splat<float>(float a) { return a; }
template <>
__device__ __forceinline__ float2 splat<float2>(float a) { return make_float2(a, a); }

// A scalar function applied to each lane.
template <typename F>
__device__ __forceinline__ float vmap(F f, float x) { return f(x); }
template <typename F>
__device__ __forceinline__ float2 vmap(F f, float2 x) { return make_float2(f(x.x), f(x.y)); }

// Lane masks: bool for one sample, bool2 for a pair.
struct bool2 {
  bool x, y;
};
__device__ __forceinline__ bool2 operator&(bool2 a, bool2 b) { return {bool(a.x & b.x), bool(a.y & b.y)}; }
__device__ __forceinline__ bool2 operator|(bool2 a, bool2 b) { return {bool(a.x | b.x), bool(a.y | b.y)}; }
__device__ __forceinline__ bool2& operator&=(bool2& a, bool2 b) { return a = a & b; }

template <typename V>
struct MaskOf {
  using type = bool;
};
template <>
struct MaskOf<float2> {
  using type = bool2;
};
template <typename V>
using Mask = typename MaskOf<V>::type;

__device__ __forceinline__ float vsel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ float2 vsel(bool2 m, float2 a, float2 b) {
  return make_float2(m.x ? a.x : b.x, m.y ? a.y : b.y);
}
__device__ __forceinline__ bool vgt(float a, float b) { return a > b; }
__device__ __forceinline__ bool2 vgt(float2 a, float2 b) { return {a.x > b.x, a.y > b.y}; }
__device__ __forceinline__ bool vge(float a, float b) { return a >= b; }
__device__ __forceinline__ bool2 vge(float2 a, float2 b) { return {a.x >= b.x, a.y >= b.y}; }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float2 vmax(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }

}  // namespace vndf
