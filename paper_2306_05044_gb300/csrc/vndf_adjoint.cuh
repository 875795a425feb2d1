// Reverse-mode derivative of the spherical-cap sampler and its fused pdf with
// the uniforms held fixed (reparameterised gradients).  The paper defines the
// forward map only (Sec. 2 steps (1)-(3), Sec. 3.3, Eq. 1); this file is its
// hand-written adjoint.  The forward is recomputed in registers (with the
// same formulas as sample_one<cap>, but cheaper reciprocal and square-root
// forms since this kernel is bound by instruction issue, not memory), and the
// chain rule is applied backwards:
//
//   s   = (ax wx, ay wy, wz),  r = |s|^-1,  i = s r,  a = 1 + i.z
//   S   = 2 a (1 - u2) + u2 (i.x^2 + i.y^2),  st = sqrt(u2 S)        (sin theta)
//   h   = (st cos phi + i.x, st sin phi + i.y, (1 - u2) a)
//   v   = (ax h.x, ay h.y, h.z),  wm = v / |v|
//   pdf = |v|^3 / (pi ax ay a |h|^2)
//
// Singular points: st = sqrt(u2 S) is differentiated through S with
// d st / dS = u2 / (2 st) = sqrt(u2) / (2 sqrt(S)), finite because
// S >= 2 (1 - u2) >= 2^-23 for the 24-bit uniforms (u2 <= 1 - 2^-24) and taken
// as exactly 0 at u2 = 0.  |v| and
// |h| are bounded below by h.z = (1 - u2) a > 0.  No clamp sits on the
// differentiated path.  Out-of-domain samples return zero gradients (their
// output is the constant fallback).
#pragma once
#include "vndf_math.cuh"

namespace vndf {

struct Grad5 {
  float wx, wy, wz, ax, ay;
};

// Adjoint of (wm, pdf) for one sample.  gmx, gmy, gmz: adjoint of wm; gpdf:
// adjoint of pdf; glog: adjoint of log(pdf).  Also returns the forward values.
// With PDF_TERMS = false the pdf adjoints are taken as zero at compile time and
// the returned pdf is not computed (0).  With EXT, the extended domain of
// kMethodCapExt (incident directions below the horizon): a = 1 + i.z is then
// formed as (i.x^2 + i.y^2) / (1 - i.z) when i.z < 0, and da / di.z = 1 either way.
template <bool PDF_TERMS = true, bool EXT = false>
__device__ __forceinline__ Grad5 cap_backward_one(float wx, float wy, float wz, float ax, float ay, float u1,
                                                  float u2, float gmx, float gmy, float gmz, float gpdf,
                                                  float glog, float& mx, float& my, float& mz, float& pdf) {
  bool ok = EXT ? in_domain_ext_inputs(wx, wy, wz, ax, ay) : in_domain(wx, wy, wz, ax, ay);
  // ---- forward (as in sample_one<cap>)
  const float sx = ax * wx, sy = ay * wy;
  const float l2 = fmaf(sx, sx, fmaf(sy, sy, wz * wz));
  const float r = rsqrtf(l2);
  const float ix = sx * r, iy = sy * r, iz = wz * r;
  const float rho2 = fmaf(ix, ix, iy * iy);
  const float a_up = __fadd_rn(1.f, iz);
  float a = a_up;
  if constexpr (EXT) {
    if (iz < 0.f) a = rho2 * rcp_fast(1.f - iz);
    ok &= a >= kMinCapA;
  }
  const float om = 1.f - u2;
  const float S = fmaf(2.f * a, om, u2 * rho2);
  // st = sqrt(u2 S) and d st / dS = u2 / (2 st) from one rsqrt; both are 0 at u2 = 0
  const float q = u2 * S;
  const float rq = rsqrtf(q);
  const float st = u2 > 0.f ? q * rq : 0.f;
  const float u2rq = u2 > 0.f ? u2 * rq : 0.f;
  float sp, cp;
  sincospi_taylor(2.f * u1, sp, cp);
  const float hx = fmaf(st, cp, ix), hy = fmaf(st, sp, iy), hz = om * a;
  const float vx = ax * hx, vy = ay * hy, vz = hz;
  const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  const float rv = rsqrtf(vv);
  mx = vx * rv;
  my = vy * rv;
  mz = vz * rv;
  const float hh = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
  // two reciprocals, of a |h|^2 and of pi ax ay, give 1/hh, 1/a, 1/ax, 1/ay and the pdf
  // (|v|^2 / (a |h|^2)) (|v| / (pi ax ay)), each factor within the FP32 range where the
  // full product a |h|^2 ax ay, or |v|^3, would not be (tiny roughness together with the
  // extended domain's smallest a)
  float rhh = 0.f, ra = 0.f, rax = 0.f, ray = 0.f, glp = 0.f;
  pdf = 0.f;
  if constexpr (PDF_TERMS) {
    const float rah = rcp_fast(a * hh);
    const float rxy = rcp_fast(kPi * ax * ay);
    pdf = (vv * rah) * ((vv * rv) * rxy);
    rhh = a * rah;
    ra = hh * rah;
    const float q2 = kPi * rxy;
    rax = ay * q2;
    ray = ax * q2;
    glp = fmaf(gpdf, pdf, glog);  // adjoint of log pdf
  }

  // ---- reverse
  // log pdf = 1.5 log vv - log pi - log ax - log ay - log a - log hh
  const float g_vv = 1.5f * glp * rv * rv;
  float g_ax = -glp * rax;
  float g_ay = -glp * ray;
  float g_a = -glp * ra;
  const float g_hh = -glp * rhh;
  // wm = v / |v|
  const float gdot = fmaf(gmx, mx, fmaf(gmy, my, gmz * mz));
  const float g_vx = fmaf(fmaf(-mx, gdot, gmx), rv, 2.f * vx * g_vv);
  const float g_vy = fmaf(fmaf(-my, gdot, gmy), rv, 2.f * vy * g_vv);
  const float g_vz = fmaf(fmaf(-mz, gdot, gmz), rv, 2.f * vz * g_vv);
  // v = (ax hx, ay hy, hz), hh = |h|^2
  const float g_hx = fmaf(2.f * hx, g_hh, ax * g_vx);
  const float g_hy = fmaf(2.f * hy, g_hh, ay * g_vy);
  const float g_hz = fmaf(2.f * hz, g_hh, g_vz);
  g_ax = fmaf(hx, g_vx, g_ax);
  g_ay = fmaf(hy, g_vy, g_ay);
  // h = (st cp + ix, st sp + iy, om a)
  const float g_st = fmaf(cp, g_hx, sp * g_hy);
  float g_ix = g_hx, g_iy = g_hy;
  g_a = fmaf(om, g_hz, g_a);
  // st = sqrt(u2 S)
  const float g_S = 0.5f * u2rq * g_st;
  // S = 2 a om + u2 rho2
  g_a = fmaf(2.f * om, g_S, g_a);
  const float g_rho2 = u2 * g_S;
  g_ix = fmaf(2.f * ix, g_rho2, g_ix);
  g_iy = fmaf(2.f * iy, g_rho2, g_iy);
  // a = 1 + iz
  const float g_iz = g_a;
  // i = s / |s|: g_s = (g_i - i (i . g_i)) / |s|.  Its z part is written as
  // g_iz (1 - i.z^2) - i.z (i.x g_ix + i.y g_iy) with 1 - i.z^2 = i.x^2 + i.y^2:
  // near straight down, g_iz grows like 1 / (1 + i.z) and the plain form cancels.
  const float gxy = fmaf(g_ix, ix, g_iy * iy);
  const float idot = fmaf(g_iz, iz, gxy);
  const float g_sx = fmaf(-ix, idot, g_ix) * r;
  const float g_sy = fmaf(-iy, idot, g_iy) * r;
  const float g_sz = fmaf(g_iz, rho2, -iz * gxy) * r;
  // s = (ax wx, ay wy, wz)
  Grad5 g;
  g.wx = ax * g_sx;
  g.wy = ay * g_sy;
  g.wz = g_sz;
  g.ax = fmaf(wx, g_sx, g_ax);
  g.ay = fmaf(wy, g_sy, g_ay);
  if (!ok) {
    g = Grad5{0.f, 0.f, 0.f, 0.f, 0.f};
    mx = 0.f;
    my = 0.f;
    mz = 1.f;
    pdf = 0.f;
  }
  return g;
}

}  // namespace vndf
