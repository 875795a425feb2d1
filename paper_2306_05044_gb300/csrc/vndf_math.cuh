// FP32 device math of the GGX visible-normal samplers and the VNDF density.
//
// Notation follows Dupuy & Benyoub (HPG 2023).  M = diag(1/ax, 1/ay, 1) maps the
// unit hemisphere onto the GGX ellipsoid (Sec. 2, "Definition").  Per sample:
//   i = M^-1 wi / |M^-1 wi|                     (Sec. 2, step (1))
//   cap sampler:  c uniform on z in (-i.z, 1],   h = c + i   (Sec. 3.3)
//   prior sampler: Heitz 2018 cross-section sampler, h unit  (Sec. 2, step (2))
//   v = M^-T h = (ax hx, ay hy, hz),  wm = v / |v|           (Sec. 2, step (3))
//
// Density.  Eq. 1 gives D_vis(wm) = D_vis_std(h/|h|, i) |det M^T| / |M^T wm|^3
// with D_vis_std = max(h.i/|h|, 0) / (pi (1 + i.z)/2) (Eqs. 2-4).  Since
// M^T wm = h/|v|, |M^T wm| = |h|/|v|, and
//   pdf = 2 max(h.i, 0) |v|^3 / (pi ax ay (1 + i.z) |h|^3).
// For the cap sampler |h|^2 = 2 (1 + c.i) and h.i = |h|^2 / 2, so
//   pdf = |v|^3 / (pi ax ay (1 + i.z) |h|^2).
// Evaluating the density from (h, v) instead of from the rounded float wm keeps
// its relative error at a few ulp even at alpha = 1e-3, where d log D / d angle
// is of order 1/alpha.
//
// Rounding.  With a = 1 + i.z, the cap height z = (1 - u2) a - i.z satisfies
//   1 - z = u2 a,   1 + z = 2 (1 - u2) + u2 (1 - i.z),   1 - i.z = (i.x^2 + i.y^2) / a,
// so sin^2 = (1 - z)(1 + z) = u2 (2 a (1 - u2) + u2 (i.x^2 + i.y^2)) is a sum of
// non-negative terms, and h.z = z + i.z = (1 - u2) a is a single product (1 - u2
// is exact for 24-bit uniforms).  Neither cancels, unlike 1 - z^2 near the bottom
// of the cap (z -> -1 when i.z -> 1).  The azimuth is evaluated as sin/cos(pi x)
// at x = 2 u1, which is exact, so no rounding of 2 pi u1 enters the angle.  What remains is the
// rounding of the O(1) summands of h.x and h.y, which the unstretch divides by
// |v|: the error is a few ulp times
//   kappa = |(ax (|c.x| + |i.x|), ay (|c.y| + |i.y|), h.z)| / |v|.
#pragma once
#include <cstdint>

#include "pair.cuh"
#include "precise.cuh"

namespace vndf {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kMethodCap = 0;
constexpr int kMethodPolar = 1;
// The cap sampler on the extended domain: incident directions below the
// horizon too.  Nothing in Sec. 3.2-3.3 or Eq. 4 needs wi.z > 0: the cap
// z in (-i.z, 1] and sigma_std = (1 + i.z)/2 hold for every i.z > -1, and the
// samples are the normals with wm.z > 0 that face wi.  For i.z < 0 the value
// a = 1 + i.z is formed as (i.x^2 + i.y^2) / (1 - i.z), which does not cancel.
constexpr int kMethodCapExt = 2;
// Smallest a = 1 + i.z of the extended domain: the stretched direction at
// least about 1.4e-6 rad from straight down.  Below it the cap has shrunk to a
// point and the inputs take the fallback.
constexpr float kMinCapA = 0x1p-40f;

template <int METHOD>
constexpr bool is_cap() { return METHOD == kMethodCap || METHOD == kMethodCapExt; }

__device__ __forceinline__ bool finite_f(float x) { return fabsf(x) < __int_as_float(0x7f800000); }

// Square root by the PTX sqrt.approx.f32 instruction: one instruction instead
// of the correctly rounded sequence; measured on GB300 within 0.944 ulp of the
// exact root over every float in [1, 4) and 2^24 random floats in
// [2^-100, 2^100] (the correctly rounded root is within 0.5 ulp).
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Reciprocal by the PTX rcp.approx.ftz.f32 instruction (documented maximum error
// 1 ulp; subnormal inputs and results flush to zero): one MUFU instruction with
// no subnormal fix-up, for operands that the callers keep in the normal range.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The same as function objects, for applying them lane by lane (pair.cuh's vmap).
struct SqrtFast {
  __device__ __forceinline__ float operator()(float x) const { return sqrt_fast(x); }
};
struct RcpFast {
  __device__ __forceinline__ float operator()(float x) const { return rcp_fast(x); }
};
struct RsqrtF {
  __device__ __forceinline__ float operator()(float x) const { return rsqrtf(x); }
};

// sin(pi x) and cos(pi x) for finite x (used with x = 2 u1, the azimuth in
// half turns).  Reduction: j = rint(2x), r = x - j/2 in [-1/4, 1/4]; for
// x in [0, 2] the subtraction is exact (Sterbenz).  sin(pi r) and cos(pi r)
// come from their Taylor series (odd terms to r^9, even terms to r^10; the
// first omitted terms are below 2.5e-9 on |pi r| <= pi/4), evaluated by Horner
// with fma; the quadrant identities sin(pi (r + k/2)) = {s, c, -s, -c},
// cos(pi (r + k/2)) = {c, -s, -c, s} are exact.  Absolute error <= 1.5 * 2^-24
// over all 2^24 uniforms (checked against FP64 sin and cos).
// (Written for float or, with the packed FP32x2 operations of pair.cuh, for a
// float2 of two independent arguments; both give the same bits per lane.)
__device__ __forceinline__ void sincospi_quadrant(float j, float ps, float pc, float& s, float& c) {
  const int k = static_cast<int>(j) & 3;
  const float a = (k & 1) ? pc : ps;
  const float b = (k & 1) ? ps : pc;
  s = (k & 2) ? -a : a;
  c = ((k + 1) & 2) ? -b : b;
}
__device__ __forceinline__ void sincospi_quadrant(float2 j, float2 ps, float2 pc, float2& s, float2& c) {
  sincospi_quadrant(j.x, ps.x, pc.x, s.x, c.x);
  sincospi_quadrant(j.y, ps.y, pc.y, s.y, c.y);
}
struct RintTwice {
  __device__ __forceinline__ float operator()(float x) const { return rintf(2.f * x); }
};

template <typename V>
__device__ __forceinline__ void sincospi_taylor(V x, V& s, V& c) {
  constexpr float S1 = 3.14159265358979323846f;     //  pi
  constexpr float S3 = -5.16771278004997003f;       // -pi^3 / 3!
  constexpr float S5 = 2.55016403987734549f;        //  pi^5 / 5!
  constexpr float S7 = -0.599264529320792077f;      // -pi^7 / 7!
  constexpr float S9 = 0.0821458866111282288f;      //  pi^9 / 9!
  constexpr float C2 = -4.93480220054467931f;       // -pi^2 / 2!
  constexpr float C4 = 4.05871212641676822f;        //  pi^4 / 4!
  constexpr float C6 = -1.33526276885458949f;       // -pi^6 / 6!
  constexpr float C8 = 0.235330630358893200f;       //  pi^8 / 8!
  constexpr float C10 = -0.0258068913900140009f;    // -pi^10 / 10!
  const V j = vmap(RintTwice{}, x);
  const V r = vfma(splat<V>(-0.5f), j, x);
  const V r2 = vmul(r, r);
  V ps = vfma(r2, splat<V>(S9), splat<V>(S7));
  ps = vfma(r2, ps, splat<V>(S5));
  ps = vfma(r2, ps, splat<V>(S3));
  ps = vfma(r2, ps, splat<V>(S1));
  ps = vmul(ps, r);
  V pc = vfma(r2, splat<V>(C10), splat<V>(C8));
  pc = vfma(r2, pc, splat<V>(C6));
  pc = vfma(r2, pc, splat<V>(C4));
  pc = vfma(r2, pc, splat<V>(C2));
  pc = vfma(r2, pc, splat<V>(1.f));
  sincospi_quadrant(j, ps, pc, s, c);
}

// Domain of the method: wi.z > 0, alphas > 0, everything finite (NaN fails every test).
__device__ __forceinline__ bool in_domain(float wx, float wy, float wz, float ax, float ay) {
  return (wz > 0.f) & (ax > 0.f) & (ay > 0.f) & finite_f(wx) & finite_f(wy) & finite_f(wz) &
         finite_f(ax) & finite_f(ay);
}

// The part of the extended domain known before stretching (alphas > 0, all
// finite); a >= kMinCapA is tested once a is formed (a NaN a fails it).
__device__ __forceinline__ bool in_domain_ext_inputs(float wx, float wy, float wz, float ax, float ay) {
  return (ax > 0.f) & (ay > 0.f) & finite_f(wx) & finite_f(wy) & finite_f(wz) & finite_f(ax) & finite_f(ay);
}

__device__ __forceinline__ bool2 in_domain(float2 wx, float2 wy, float2 wz, float2 ax, float2 ay) {
  return {in_domain(wx.x, wy.x, wz.x, ax.x, ay.x), in_domain(wx.y, wy.y, wz.y, ax.y, ay.y)};
}
__device__ __forceinline__ bool2 in_domain_ext_inputs(float2 wx, float2 wy, float2 wz, float2 ax, float2 ay) {
  return {in_domain_ext_inputs(wx.x, wy.x, wz.x, ax.x, ay.x), in_domain_ext_inputs(wx.y, wy.y, wz.y, ax.y, ay.y)};
}

// With both roughnesses 1 (UnitAlpha) only the direction is tested.
__device__ __forceinline__ bool in_domain(float wx, float wy, float wz, UnitAlpha, UnitAlpha) {
  return (wz > 0.f) & finite_f(wx) & finite_f(wy) & finite_f(wz);
}
__device__ __forceinline__ bool in_domain_ext_inputs(float wx, float wy, float wz, UnitAlpha, UnitAlpha) {
  return finite_f(wx) & finite_f(wy) & finite_f(wz);
}
__device__ __forceinline__ bool2 in_domain(float2 wx, float2 wy, float2 wz, UnitAlpha u, UnitAlpha) {
  return {in_domain(wx.x, wy.x, wz.x, u, u), in_domain(wx.y, wy.y, wz.y, u, u)};
}
__device__ __forceinline__ bool2 in_domain_ext_inputs(float2 wx, float2 wy, float2 wz, UnitAlpha u, UnitAlpha) {
  return {in_domain_ext_inputs(wx.x, wy.x, wz.x, u, u), in_domain_ext_inputs(wx.y, wy.y, wz.y, u, u)};
}

// A (the roughness type) is V, or UnitAlpha for the hemisphere configuration.
template <int METHOD, typename V, typename A>
__device__ __forceinline__ Mask<V> in_domain_m(V wx, V wy, V wz, A ax, A ay) {
  if constexpr (METHOD == kMethodCapExt)
    return in_domain_ext_inputs(wx, wy, wz, ax, ay);
  else
    return in_domain(wx, wy, wz, ax, ay);
}

// The samplers below are written for V = float (one sample) or V = float2 (two
// independent samples, one per half, on the packed FP32x2 operations of
// pair.cuh).  Every operation is explicit, so both widths round every lane the
// same way and give the same bits.
template <typename V>
struct StretchedV {
  V x, y, z;  // i = M^-1 wi / |M^-1 wi|
  V a;        // 1 + i.z rounded once, as fma(wi.z, 1 / |M^-1 wi|, 1)
};
using Stretched = StretchedV<float>;

// a is formed by one fma rather than as 1 + (the rounded i.z): an add whose
// operand is a packed product used nowhere else may be fused into an fma by the
// assembler, which would round the two widths differently.
template <typename V, typename A>
__device__ __forceinline__ StretchedV<V> stretch(V wx, V wy, V wz, A ax, A ay) {
  const V sx = vmul(ax, wx), sy = vmul(ay, wy);
  const V r = vmap(RsqrtF{}, vfma(sx, sx, vfma(sy, sy, vmul(wz, wz))));
  return {vmul(sx, r), vmul(sy, r), vmul(wz, r), vfma(wz, r, splat<V>(1.f))};
}

// Spherical-cap hemisphere sample: returns h = c + i (unnormalised).  With
// EXT, i.z may be negative and a = 1 + i.z is formed without cancellation.
template <bool EXT = false, typename V>
__device__ __forceinline__ void cap_half_vector(const StretchedV<V>& i, V u1, V u2, V& hx, V& hy, V& hz, V& a) {
  const V rho2 = vfma(i.x, i.x, vmul(i.y, i.y));  // 1 - i.z^2
  // both variants take the stretch's a above the horizon, so they agree bit for bit there
  const V a_up = i.a;
  if constexpr (EXT)  // 1 - i.z in [1, 2]
    a = vsel(vge(i.z, splat<V>(0.f)), a_up, vmul(rho2, vmap(RcpFast{}, vsub(splat<V>(1.f), i.z))));
  else
    a = a_up;
  const V om = vsub(splat<V>(1.f), u2);
  const V sin2 = vmul(u2, vfma(vmul(splat<V>(2.f), a), om, vmul(u2, rho2)));  // (1 - z)(1 + z)
  const V st = vmap(SqrtFast{}, sin2);
  V sp, cp;
  sincospi_taylor(vmul(splat<V>(2.f), u1), sp, cp);
  hx = vfma(st, cp, i.x);
  hy = vfma(st, sp, i.y);
  hz = vmul(om, a);  // z + i.z
}

// Heitz 2018 cross-section sampler (Sec. 2 step (2)): returns a unit hemisphere
// normal h.  The construction of that method (basis (w1, w2, i), a uniform point
// (t1, t2) on the unit disk, the far half compressed by s = (1 + i.z)/2, lifted
// onto the hemisphere along i), with the rounding care the cap sampler gets:
// every quantity that cancels near the rim of the disk is rewritten exactly,
//   1 - t1^2     = (1 - u2) + u2 sin^2(phi)                       (= q^2),
//   q -/+ t2o    = (1 - u2) / (q +/- t2o)      (t2o = sqrt(u2) sin(phi); q^2 - t2o^2 = 1 - u2),
//   1 - s        = (i.x^2 + i.y^2) / (2 (1 + i.z)),
//   1 - t1^2 - t2^2 = (q - t2)(q + t2) = s (q - t2o) (2 (1 - s) q + s (q + t2o)),
// so all factors are sums of non-negative terms.
template <typename V>
__device__ __forceinline__ void polar_disk_normal(const StretchedV<V>& i, V u1, V u2, V& hx, V& hy, V& hz) {
  const V tmp = vfma(i.x, i.x, vmul(i.y, i.y));
  // w1 = (-i.y, i.x, 0) / |.|, or (1, 0, 0) at the pole
  const Mask<V> tilted = vgt(tmp, splat<V>(0.f));
  const V r0 = vmap(RsqrtF{}, tmp);
  const V w1x = vsel(tilted, vmul(vneg(i.y), r0), splat<V>(1.f));
  const V w1y = vsel(tilted, vmul(i.x, r0), splat<V>(0.f));
  // w2 = i x w1 (w1.z = 0)
  const V w2x = vmul(vneg(i.z), w1y);
  const V w2y = vmul(i.z, w1x);
  const V w2z = vfma(i.x, w1y, vmul(vneg(i.y), w1x));
  V sp, cp;
  sincospi_taylor(vmul(splat<V>(2.f), u1), sp, cp);
  const V r = vmap(SqrtFast{}, u2);
  const V t1 = vmul(r, cp);
  const V t2o = vmul(r, sp);
  const V om = vsub(splat<V>(1.f), u2);
  const V q = vmap(SqrtFast{}, vfma(vmul(u2, sp), sp, om));  // sqrt(1 - t1^2)
  const V a = vadd(splat<V>(1.f), i.z);
  const V s = vmul(splat<V>(0.5f), a);
  const V oms = vmul(vmul(splat<V>(0.5f), tmp), vmap(RcpFast{}, a));  // 1 - s
  const Mask<V> pos = vge(t2o, splat<V>(0.f));
  const V big = vsel(pos, vadd(q, t2o), vsub(q, t2o));  // no cancellation either way
  const V small = vmul(om, vmap(RcpFast{}, big));       // the other one of q -/+ t2o
  const V qm = vsel(pos, small, big);                   // q - t2o
  const V qp = vsel(pos, big, small);                   // q + t2o
  const V t2 = vfma(oms, q, vmul(s, t2o));
  const V ti = vmap(SqrtFast{}, vmul(vmul(s, qm), vfma(vmul(splat<V>(2.f), oms), q, vmul(s, qp))));
  hx = vfma(t1, w1x, vfma(t2, w2x, vmul(ti, i.x)));
  hy = vfma(t1, w1y, vfma(t2, w2y, vmul(ti, i.y)));
  hz = vfma(t2, w2z, vmul(ti, i.z));
}

// Threshold on the condition number above which a cap sample is recomputed in
// double-float (cap_half_vector_precise): with it every sample meets 4e-6 rad
// for wm and 1e-5 relative for the pdf with margin (the pdf's error grows like
// 3 kappa + 2 kappa_h ulps, the angle's like kappa); about 7e-4 of the
// anisotropic workload's samples take that path.
constexpr float kRescueKappa = 24.f;

// The FP32 tail of a sample: unstretch h, normalise, and (if PDF) the fused density.
template <int METHOD, bool PDF, typename V, typename A>
__device__ __forceinline__ void finish_sample(const StretchedV<V>& i, A ax, A ay, V hx, V hy, V hz, V a, V& mx,
                                              V& my, V& mz, V& pdf) {
  const V vx = vmul(ax, hx), vy = vmul(ay, hy), vz = hz;
  const V vv = vfma(vx, vx, vfma(vy, vy, vmul(vz, vz)));
  const V rv = vmap(RsqrtF{}, vv);
  mx = vmul(vx, rv);
  my = vmul(vy, rv);
  mz = vmul(vz, rv);
  if constexpr (PDF) {
    const V nv = vmul(vv, rv);  // |v|
    const V rden = vmap(RcpFast{}, vmul(vmul(vmul(splat<V>(kPi), ax), ay), a));
    if constexpr (is_cap<METHOD>()) {
      // |v|^3 / (pi ax ay a |h|^2) as (|v|^2 / |h|^2) |v| / (pi ax ay a): |v|^2 / |h|^2 lies
      // between min(ax, ay, 1)^2 and max(ax, ay, 1)^2, so no factor leaves the FP32 range,
      // whereas |v|^3 underflows once |v| < 2e-13 (tiny roughness together with the
      // extended domain's smallest cap heights a)
      const V hh = vfma(hx, hx, vfma(hy, hy, vmul(hz, hz)));
      pdf = vmul(vmul(vmul(vv, vmap(RcpFast{}, hh)), nv), rden);
    } else {
      const V hi = vmax(vfma(hx, i.x, vfma(hy, i.y, vmul(hz, i.z))), splat<V>(0.f));
      pdf = vmul(vmul(vmul(vmul(splat<V>(2.f), hi), vv), nv), rden);
    }
  }
}

// One sample (V = float) or two (V = float2) of Sec. 2 steps (1)-(3) with the
// chosen hemisphere sampler and, if PDF, the fused density.  Out-of-domain
// inputs give wm = (0,0,1), pdf = 0.  With PRECISE (cap sampler only) the
// returned mask flags ill-conditioned samples whose results must be replaced
// by sample_one_precise; the check costs a few FP32 operations and keeps the
// rare slow path out of the unrolled loop.
template <int METHOD, bool PDF, bool PRECISE = false, typename V, typename A>
__device__ __forceinline__ Mask<V> sample_one(V wx, V wy, V wz, A ax, A ay, V u1, V u2, V& mx, V& my, V& mz,
                                              V& pdf) {
  Mask<V> ok = in_domain_m<METHOD>(wx, wy, wz, ax, ay);
  const StretchedV<V> i = stretch(wx, wy, wz, ax, ay);
  V hx, hy, hz, a;
  if constexpr (is_cap<METHOD>()) {
    cap_half_vector<METHOD == kMethodCapExt>(i, u1, u2, hx, hy, hz, a);
    if constexpr (METHOD == kMethodCapExt) ok &= vge(a, splat<V>(kMinCapA));
  } else {
    polar_disk_normal(i, u1, u2, hx, hy, hz);
    a = vadd(splat<V>(1.f), i.z);
  }
  finish_sample<METHOD, PDF>(i, ax, ay, hx, hy, hz, a, mx, my, mz, pdf);
  Mask<V> bad{};
  if constexpr (PRECISE && is_cap<METHOD>()) {
    // |c.x| + |i.x| etc. bound the rounding of h; compare it with |v| and |h|
    const V sx = vadd(vabs(vsub(hx, i.x)), vabs(i.x)), sy = vadd(vabs(vsub(hy, i.y)), vabs(i.y));
    const V vx = vmul(ax, hx), vy = vmul(ay, hy);
    const V hz2 = vmul(hz, hz);
    const V vv = vfma(vx, vx, vfma(vy, vy, hz2));
    const V ksx = vmul(ax, sx), ksy = vmul(ay, sy);
    const V k2 = vfma(ksx, ksx, vfma(ksy, ksy, hz2));
    // both tests whether or not the pdf is wanted, so the normals do not depend on it
    const V kh2 = vfma(sx, sx, vfma(sy, sy, hz2));
    const V K2 = splat<V>(kRescueKappa * kRescueKappa);
    bad = vgt(k2, vmul(K2, vv)) | vgt(kh2, vmul(K2, vfma(hx, hx, vfma(hy, hy, hz2))));
    bad &= ok;
  }
  mx = vsel(ok, mx, splat<V>(0.f));
  my = vsel(ok, my, splat<V>(0.f));
  mz = vsel(ok, mz, splat<V>(1.f));
  if constexpr (PDF) pdf = vsel(ok, pdf, splat<V>(0.f));
  return bad;
}

// Lanes k, k + 1 of a thread's four samples as one pair, and back.
__device__ __forceinline__ float2 lanes(const float (&v)[4], int k) { return make_float2(v[k], v[k + 1]); }
__device__ __forceinline__ void set_lanes(float (&v)[4], int k, float2 x) {
  v[k] = x.x;
  v[k + 1] = x.y;
}

// A thread's four consecutive samples, computed as two packed pairs; returns the
// rescue flags of sample_one (PRECISE) as bits 0..3.
template <int METHOD, bool PDF>
__device__ __forceinline__ unsigned sample_four(const float (&X)[4], const float (&Y)[4], const float (&Z)[4],
                                                const float (&AX)[4], const float (&AY)[4], const float (&U1)[4],
                                                const float (&U2)[4], float (&MX)[4], float (&MY)[4],
                                                float (&MZ)[4], float (&P)[4]) {
  unsigned rescue = 0;
#pragma unroll
  for (int k = 0; k < 4; k += 2) {
    float2 mx, my, mz, p;
    const bool2 b = sample_one<METHOD, PDF, true>(lanes(X, k), lanes(Y, k), lanes(Z, k), lanes(AX, k), lanes(AY, k),
                                                  lanes(U1, k), lanes(U2, k), mx, my, mz, p);
    set_lanes(MX, k, mx);
    set_lanes(MY, k, my);
    set_lanes(MZ, k, mz);
    if constexpr (PDF) set_lanes(P, k, p);
    rescue |= (unsigned(b.x) << k) | (unsigned(b.y) << (k + 1));
  }
  return rescue;
}

// The cap sample recomputed with its half vector in double-float (in-domain
// inputs only); returns (wm.x, wm.y, wm.z, pdf).  Not inlined, and returning by
// value, so that the rare path neither bloats nor spills the FP32 path.
template <bool PDF, bool EXT = false>
__device__ __noinline__ float4 sample_one_precise(float wx, float wy, float wz, float ax, float ay, float u1,
                                                  float u2) {
  float hx, hy, hz, a;
  cap_half_vector_precise<EXT>(wx, wy, wz, ax, ay, u1, u2, hx, hy, hz, a);
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  finish_sample<kMethodCap, PDF>(Stretched{0.f, 0.f, 0.f}, ax, ay, hx, hy, hz, a, r.x, r.y, r.z, r.w);
  return r;
}

// Density of a given normal (Eq. 1 through the App. A forms of D and G1):
// 2 max(0, wi.wm) / (pi ax ay (|M^-1 wi| + wi.z) Q^2), Q = mx^2/ax^2 + my^2/ay^2 + mz^2.
// |M^-1 wi| + wi.z is twice the projected area of the microsurface seen from
// wi (unit wi); with EXT (incident directions below the horizon) it is formed
// as (sx^2 + sy^2) / (|M^-1 wi| - wi.z) when wi.z < 0, which does not cancel.
template <bool EXT = false>
__device__ __forceinline__ float pdf_of_normal(float wx, float wy, float wz, float ax, float ay,
                                               float mx, float my, float mz) {
  bool ok = (EXT ? in_domain_ext_inputs(wx, wy, wz, ax, ay) : in_domain(wx, wy, wz, ax, ay)) & (mz > 0.f);
  const float sx = ax * wx, sy = ay * wy;
  const float l = sqrt_fast(fmaf(sx, sx, fmaf(sy, sy, wz * wz)));
  float lw = l + wz;
  if constexpr (EXT) {
    if (wz < 0.f) lw = fmaf(sx, sx, sy * sy) / (l - wz);
    ok &= lw >= kMinCapA * l;  // a = 1 + i.z = lw / l
  }
  const float qx = mx * rcp_fast(ax), qy = my * rcp_fast(ay);
  const float q = fmaf(qx, qx, fmaf(qy, qy, mz * mz));
  const float d = fmaxf(fmaf(wx, mx, fmaf(wy, my, wz * mz)), 0.f);
  // (ax q)(ay q) rather than ax ay q^2: q grows like 1 / alpha^2 away from the peak
  const float p = 2.f * d * rcp_fast(kPi * lw * (ax * q) * (ay * q));
  return ok ? p : 0.f;
}

}  // namespace vndf
