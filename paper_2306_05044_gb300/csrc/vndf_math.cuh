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

template <int METHOD>
__device__ __forceinline__ bool in_domain_m(float wx, float wy, float wz, float ax, float ay) {
  if constexpr (METHOD == kMethodCapExt)
    return in_domain_ext_inputs(wx, wy, wz, ax, ay);
  else
    return in_domain(wx, wy, wz, ax, ay);
}

struct Stretched {
  float x, y, z;  // i = M^-1 wi / |M^-1 wi|
};

__device__ __forceinline__ Stretched stretch(float wx, float wy, float wz, float ax, float ay) {
  const float sx = ax * wx, sy = ay * wy;
  const float l2 = fmaf(sx, sx, fmaf(sy, sy, wz * wz));
  const float r = rsqrtf(l2);
  return {sx * r, sy * r, wz * r};
}

// Spherical-cap hemisphere sample: returns h = c + i (unnormalised).  With
// EXT, i.z may be negative and a = 1 + i.z is formed without cancellation.
template <bool EXT = false>
__device__ __forceinline__ void cap_half_vector(const Stretched& i, float u1, float u2,
                                                float& hx, float& hy, float& hz, float& a) {
  const float rho2 = fmaf(i.x, i.x, i.y * i.y);                 // 1 - i.z^2
  // an explicit add, never contracted with the stretch's product into an fma:
  // both variants then round a the same way and agree bit for bit above the horizon
  const float a_up = __fadd_rn(1.f, i.z);
  if constexpr (EXT)
    a = i.z >= 0.f ? a_up : rho2 * rcp_fast(1.f - i.z);  // 1 - i.z in [1, 2]
  else
    a = a_up;
  const float sin2 = u2 * fmaf(2.f * a, 1.f - u2, u2 * rho2);  // (1 - z)(1 + z)
  const float st = sqrt_fast(sin2);
  float sp, cp;
  sincospi_taylor(2.f * u1, sp, cp);
  hx = fmaf(st, cp, i.x);
  hy = fmaf(st, sp, i.y);
  hz = (1.f - u2) * a;                  // z + i.z
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
__device__ __forceinline__ void polar_disk_normal(const Stretched& i, float u1, float u2,
                                                  float& hx, float& hy, float& hz) {
  const float tmp = fmaf(i.x, i.x, i.y * i.y);
  float w1x = 1.f, w1y = 0.f;
  if (tmp > 0.f) {
    const float r = rsqrtf(tmp);
    w1x = -i.y * r;
    w1y = i.x * r;
  }
  // w2 = i x w1 (w1.z = 0)
  const float w2x = -i.z * w1y;
  const float w2y = i.z * w1x;
  const float w2z = fmaf(i.x, w1y, -i.y * w1x);
  float sp, cp;
  sincospi_taylor(2.f * u1, sp, cp);
  const float r = sqrt_fast(u2);
  const float t1 = r * cp;
  const float t2o = r * sp;
  const float om = 1.f - u2;
  const float q = sqrt_fast(fmaf(u2 * sp, sp, om));  // sqrt(1 - t1^2)
  const float a = 1.f + i.z;
  const float s = 0.5f * a;
  const float oms = 0.5f * tmp * rcp_fast(a);      // 1 - s
  const bool pos = t2o >= 0.f;
  const float big = pos ? q + t2o : q - t2o;        // no cancellation either way
  const float small = om * rcp_fast(big);           // the other one of q -/+ t2o
  const float qm = pos ? small : big;               // q - t2o
  const float qp = pos ? big : small;               // q + t2o
  const float t2 = fmaf(oms, q, s * t2o);
  const float ti = sqrt_fast(s * qm * fmaf(2.f * oms, q, s * qp));
  hx = fmaf(t1, w1x, fmaf(t2, w2x, ti * i.x));
  hy = fmaf(t1, w1y, fmaf(t2, w2y, ti * i.y));
  hz = fmaf(t2, w2z, ti * i.z);
}

// Threshold on the condition number above which a cap sample is recomputed in
// double-float (cap_half_vector_precise): with it every sample meets 4e-6 rad
// for wm and 1e-5 relative for the pdf with margin (the pdf's error grows like
// 3 kappa + 2 kappa_h ulps, the angle's like kappa); about 7e-4 of the
// anisotropic workload's samples take that path.
constexpr float kRescueKappa = 24.f;

// The FP32 tail of a sample: unstretch h, normalise, and (if PDF) the fused density.
template <int METHOD, bool PDF>
__device__ __forceinline__ void finish_sample(const Stretched& i, float ax, float ay, float hx, float hy, float hz,
                                              float a, float& mx, float& my, float& mz, float& pdf) {
  const float vx = ax * hx, vy = ay * hy, vz = hz;
  const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  const float rv = rsqrtf(vv);
  mx = vx * rv;
  my = vy * rv;
  mz = vz * rv;
  if constexpr (PDF) {
    const float nv = vv * rv;  // |v|
    if constexpr (is_cap<METHOD>()) {
      // |v|^3 / (pi ax ay a |h|^2) as (|v|^2 / |h|^2) |v| / (pi ax ay a): |v|^2 / |h|^2 lies
      // between min(ax, ay, 1)^2 and max(ax, ay, 1)^2, so no factor leaves the FP32 range,
      // whereas |v|^3 underflows once |v| < 2e-13 (tiny roughness together with the
      // extended domain's smallest cap heights a)
      const float hh = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
      pdf = (vv * rcp_fast(hh)) * nv * rcp_fast(kPi * ax * ay * a);
    } else {
      const float hi = fmaxf(fmaf(hx, i.x, fmaf(hy, i.y, hz * i.z)), 0.f);
      pdf = 2.f * hi * vv * nv * rcp_fast(kPi * ax * ay * a);
    }
  }
}

// One sample of Sec. 2 steps (1)-(3) with the chosen hemisphere sampler and,
// if PDF, the fused density.  Out-of-domain inputs give wm = (0,0,1), pdf = 0.
// With PRECISE (cap sampler only) the return value flags an ill-conditioned
// sample whose result must be replaced by sample_one_precise; the check costs a
// few FP32 operations and keeps the rare slow path out of the unrolled loop.
template <int METHOD, bool PDF, bool PRECISE = false>
__device__ __forceinline__ bool sample_one(float wx, float wy, float wz, float ax, float ay,
                                           float u1, float u2,
                                           float& mx, float& my, float& mz, float& pdf) {
  bool ok = in_domain_m<METHOD>(wx, wy, wz, ax, ay);
  const Stretched i = stretch(wx, wy, wz, ax, ay);
  float hx, hy, hz, a;
  if constexpr (is_cap<METHOD>()) {
    cap_half_vector<METHOD == kMethodCapExt>(i, u1, u2, hx, hy, hz, a);
    if constexpr (METHOD == kMethodCapExt) ok &= a >= kMinCapA;
  } else {
    polar_disk_normal(i, u1, u2, hx, hy, hz);
    a = 1.f + i.z;
  }
  finish_sample<METHOD, PDF>(i, ax, ay, hx, hy, hz, a, mx, my, mz, pdf);
  bool bad = false;
  if constexpr (PRECISE && is_cap<METHOD>()) {
    // |c.x| + |i.x| etc. bound the rounding of h; compare it with |v| and |h|
    const float sx = fabsf(hx - i.x) + fabsf(i.x), sy = fabsf(hy - i.y) + fabsf(i.y);
    const float vx = ax * hx, vy = ay * hy;
    const float vv = fmaf(vx, vx, fmaf(vy, vy, hz * hz));
    const float k2 = fmaf(ax * sx, ax * sx, fmaf(ay * sy, ay * sy, hz * hz));
    // both tests whether or not the pdf is wanted, so the normals do not depend on it
    const float kh2 = fmaf(sx, sx, fmaf(sy, sy, hz * hz));
    bad = (k2 > kRescueKappa * kRescueKappa * vv) |
          (kh2 > kRescueKappa * kRescueKappa * fmaf(hx, hx, fmaf(hy, hy, hz * hz)));
    bad &= ok;
  }
  if (!ok) {
    mx = 0.f;
    my = 0.f;
    mz = 1.f;
    if constexpr (PDF) pdf = 0.f;
  }
  return bad;
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
