// Extended-precision recomputation of the cap sampler's half vector for the
// rare ill-conditioned samples.
//
// In FP32 the half vector h = c + i (Sec. 3.3) is accurate to a few ulp of its
// O(1) summands, and the unstretch v = M^-T h divides that rounding by |v|.
// For samples whose condition number
//   kappa = |(ax (|c.x| + |i.x|), ay (|c.y| + |i.y|), h.z)| / |v|
// (or its unstretched analogue for the pdf's |h|) is large, the kernel
// recomputes c and i as unevaluated sums of two floats (double-float
// arithmetic: products split exactly with fma, sums with Knuth's two-sum;
// Dekker 1971, Knuth TAOCP vol. 2 sec. 4.2.2) and rounds h once at the end.
// Everything downstream of h is well conditioned, so the FP32 pipeline then
// resumes unchanged.  Only FP32 arithmetic units are used (GB300 runs FP64 at a
// small fraction of the FP32 rate).
#pragma once
#include <cuda_runtime.h>

namespace vndf {

struct df {
  float hi, lo;  // value = hi + lo, |lo| <= ulp(hi) / 2
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  const df s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = df_two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return df_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = df_two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return df_fast_two_sum(p.hi, p.lo);
}

// sin(pi r) and cos(pi r) for |r| <= 1/4 as double-floats: Taylor series to
// r^13 (sin) and r^14 (cos); the first omitted terms are below 2.1e-14 on
// |pi r| <= pi/4.  Coefficients are (-1)^k pi^n / n! split into hi + lo floats.
// The three highest terms are summed in single precision (their share is below
// 2^-24 of the low-order part), the rest in double-float.
__device__ __forceinline__ void df_sincospi_reduced(float r, df& s, df& c) {
  // sin(pi r) / r: pi, -pi^3/3!, pi^5/5!, -pi^7/7!, pi^9/9!, -pi^11/11!, pi^13/13!
  // (each split as hi = float(c), lo = float(c - hi) from the FP64 value)
  const df S1{3.1415927410125732f, -8.742277657347586e-08f};
  const df S3{-5.167712688446045f, -9.160392266949202e-08f};
  const df S5{2.550163984298706f, 5.557863858030032e-08f};
  const df S7{-0.5992645025253296f, -2.6795461849360436e-08f};
  constexpr float S9 = 0.08214588463306427f, S11 = -0.00737043097615242f, S13 = 0.0004663027939386666f;
  // cos(pi r): 1, -pi^2/2!, pi^4/4!, -pi^6/6!, pi^8/8!, -pi^10/10!, pi^12/12!, -pi^14/14!
  const df C2{-4.934802055358887f, -1.451857940537593e-07f};
  const df C4{4.058712005615234f, 1.2080153055649134e-07f};
  const df C6{-1.3352627754211426f, 6.566553523157381e-09f};
  const df C8{0.23533062636852264f, 3.990370700535095e-09f};
  constexpr float C10 = -0.025806890800595284f, C12 = 0.001929574296809733f, C14 = -0.00010463810758665204f;
  const df z = df_two_prod(r, r);  // r^2 exactly
  // sin
  float ts = fmaf(z.hi, S13, S11);
  ts = fmaf(z.hi, ts, S9);
  df ps = df_add(df_mul(df{ts, 0.f}, z), S7);
  ps = df_add(df_mul(ps, z), S5);
  ps = df_add(df_mul(ps, z), S3);
  ps = df_add(df_mul(ps, z), S1);
  s = df_mul_f(ps, r);
  // cos
  float tc = fmaf(z.hi, C14, C12);
  tc = fmaf(z.hi, tc, C10);
  df pc = df_add(df_mul(df{tc, 0.f}, z), C8);
  pc = df_add(df_mul(pc, z), C6);
  pc = df_add(df_mul(pc, z), C4);
  pc = df_add(df_mul(pc, z), C2);
  c = df_add_f(df_mul(pc, z), 1.f);
}

// h = c + i for the cap sampler, with c and i carried in double-float and h
// rounded once (same formulas as cap_half_vector).  Also returns a = 1 + i.z.
template <bool EXT = false>
__device__ __forceinline__ void cap_half_vector_precise(float wx, float wy, float wz, float ax, float ay, float u1,
                                                       float u2, float& hx, float& hy, float& hz, float& a_out) {
  // i = s / |s|, s = (ax wx, ay wy, wz): exact products, one Newton step on rsqrt
  const df sx = df_two_prod(ax, wx), sy = df_two_prod(ay, wy), sz = df_two_prod(wz, 1.f);
  const df l2 = df_add(df_add(df_mul(sx, sx), df_mul(sy, sy)), df_two_prod(wz, wz));
  const float r0 = rsqrtf(l2.hi);
  const df t = df_mul_f(df_mul_f(l2, r0), r0);              // l2 r0^2 ~ 1
  const df res = df_add_f(df{-t.hi, -t.lo}, 1.f);            // 1 - l2 r0^2
  const df rr = df_fast_two_sum(r0, 0.5f * r0 * res.hi);     // r0 (1 + res / 2)
  const df ix = df_mul(sx, rr), iy = df_mul(sy, rr), iz = df_mul(sz, rr);
  // sin^2 = u2 (2 a (1 - u2) + u2 (i.x^2 + i.y^2)), a = 1 + i.z
  const df rho2 = df_add(df_mul(ix, ix), df_mul(iy, iy));
  df a = df_add_f(iz, 1.f);
  if constexpr (EXT) {
    if (iz.hi < 0.f) {
      // a = rho2 / (1 - i.z): quotient q, then one correction (rho2 - q d) / d
      const df d = df_add_f(df{-iz.hi, -iz.lo}, 1.f);
      const float q = rho2.hi / d.hi;
      const df qd = df_mul_f(d, q);
      const df r = df_add(rho2, df{-qd.hi, -qd.lo});
      a = df_fast_two_sum(q, r.hi / d.hi);
    }
  }
  const float om = 1.f - u2;  // exact
  const df S = df_add(df_mul_f(a, 2.f * om), df_mul_f(rho2, u2));
  const df sin2 = df_mul_f(S, u2);
  const float s0 = sqrtf(sin2.hi);
  const float corr = s0 > 0.f ? (fmaf(-s0, s0, sin2.hi) + sin2.lo) / (2.f * s0) : 0.f;
  const df st = df_fast_two_sum(s0, corr);
  // azimuth: x = 2 u1, exact reduction to r = x - j/2, quadrant by j
  const float x = 2.f * u1;
  const float j = rintf(2.f * x);
  const float r = fmaf(-0.5f, j, x);
  df sr, cr;
  df_sincospi_reduced(r, sr, cr);
  const int k = static_cast<int>(j) & 3;
  df sp = (k & 1) ? cr : sr;
  df cp = (k & 1) ? sr : cr;
  if (k & 2) sp = df{-sp.hi, -sp.lo};
  if ((k + 1) & 2) cp = df{-cp.hi, -cp.lo};
  const df hxd = df_add(df_mul(st, cp), ix);
  const df hyd = df_add(df_mul(st, sp), iy);
  hx = hxd.hi;
  hy = hyd.hi;
  hz = df_mul_f(a, om).hi;
  a_out = a.hi;
}

}  // namespace vndf
