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

template <typename V>
struct Grad5V {
  V wx, wy, wz, ax, ay;
};
using Grad5 = Grad5V<float>;

// Adjoint of (wm, pdf) for one sample (V = float) or two (V = float2, on the
// packed FP32x2 operations; both widths give the same bits).  gmx, gmy, gmz:
// adjoint of wm; gpdf: adjoint of pdf; glog: adjoint of log(pdf).  Also returns
// the forward values.  With PDF_TERMS = false the pdf adjoints are taken as
// zero at compile time and the returned pdf is not computed (0).  With EXT, the
// extended domain of kMethodCapExt (incident directions below the horizon):
// a = 1 + i.z is then formed as (i.x^2 + i.y^2) / (1 - i.z) when i.z < 0, and
// da / di.z = 1 either way.
template <bool PDF_TERMS = true, bool EXT = false, typename V>
__device__ __forceinline__ Grad5V<V> cap_backward_one(V wx, V wy, V wz, V ax, V ay, V u1, V u2, V gmx, V gmy, V gmz,
                                                      V gpdf, V glog, V& mx, V& my, V& mz, V& pdf) {
  const V zero = splat<V>(0.f), one = splat<V>(1.f), two = splat<V>(2.f);
  Mask<V> ok;
  if constexpr (EXT)
    ok = in_domain_ext_inputs(wx, wy, wz, ax, ay);
  else
    ok = in_domain(wx, wy, wz, ax, ay);
  // ---- forward (as in sample_one<cap>)
  const V sx = vmul(ax, wx), sy = vmul(ay, wy);
  const V l2 = vfma(sx, sx, vfma(sy, sy, vmul(wz, wz)));
  const V r = vmap(RsqrtF{}, l2);
  const V ix = vmul(sx, r), iy = vmul(sy, r), iz = vmul(wz, r);
  const V rho2 = vfma(ix, ix, vmul(iy, iy));
  V a = vfma(wz, r, one);  // 1 + i.z rounded once, as in the sampler
  if constexpr (EXT) {
    a = vsel(vgt(zero, iz), vmul(rho2, vmap(RcpFast{}, vsub(one, iz))), a);
    ok &= vge(a, splat<V>(kMinCapA));
  }
  const V om = vsub(one, u2);
  const V S = vfma(vmul(two, a), om, vmul(u2, rho2));
  // st = sqrt(u2 S) and d st / dS = u2 / (2 st) from one rsqrt; both are 0 at u2 = 0
  const V q = vmul(u2, S);
  const V rq = vmap(RsqrtF{}, q);
  const Mask<V> upos = vgt(u2, zero);
  const V st = vsel(upos, vmul(q, rq), zero);
  const V u2rq = vsel(upos, vmul(u2, rq), zero);
  V sp, cp;
  sincospi_taylor(vmul(two, u1), sp, cp);
  const V hx = vfma(st, cp, ix), hy = vfma(st, sp, iy), hz = vmul(om, a);
  const V vx = vmul(ax, hx), vy = vmul(ay, hy), vz = hz;
  const V vv = vfma(vx, vx, vfma(vy, vy, vmul(vz, vz)));
  const V rv = vmap(RsqrtF{}, vv);
  mx = vmul(vx, rv);
  my = vmul(vy, rv);
  mz = vmul(vz, rv);
  const V hh = vfma(hx, hx, vfma(hy, hy, vmul(hz, hz)));
  // two reciprocals, of a |h|^2 and of pi ax ay, give 1/hh, 1/a, 1/ax, 1/ay and the pdf
  // (|v|^2 / (a |h|^2)) (|v| / (pi ax ay)), each factor within the FP32 range where the
  // full product a |h|^2 ax ay, or |v|^3, would not be (tiny roughness together with the
  // extended domain's smallest a)
  V rhh = zero, ra = zero, rax = zero, ray = zero, nglp = zero;  // nglp = -(adjoint of log pdf)
  pdf = zero;
  if constexpr (PDF_TERMS) {
    const V rah = vmap(RcpFast{}, vmul(a, hh));
    const V rxy = vmap(RcpFast{}, vmul(vmul(splat<V>(kPi), ax), ay));
    pdf = vmul(vmul(vv, rah), vmul(vmul(vv, rv), rxy));
    rhh = vmul(a, rah);
    ra = vmul(hh, rah);
    const V q2 = vmul(splat<V>(kPi), rxy);
    rax = vmul(ay, q2);
    ray = vmul(ax, q2);
    nglp = vneg(vfma(gpdf, pdf, glog));
  }

  // ---- reverse
  // log pdf = 1.5 log vv - log pi - log ax - log ay - log a - log hh
  const V g_vv = vmul(vmul(vmul(splat<V>(-1.5f), nglp), rv), rv);
  V g_ax = vmul(nglp, rax);
  V g_ay = vmul(nglp, ray);
  V g_a = vmul(nglp, ra);
  const V g_hh = vmul(nglp, rhh);
  // wm = v / |v|
  const V ngdot = vneg(vfma(gmx, mx, vfma(gmy, my, vmul(gmz, mz))));
  const V g_vx = vfma(vfma(mx, ngdot, gmx), rv, vmul(vmul(two, vx), g_vv));
  const V g_vy = vfma(vfma(my, ngdot, gmy), rv, vmul(vmul(two, vy), g_vv));
  const V g_vz = vfma(vfma(mz, ngdot, gmz), rv, vmul(vmul(two, vz), g_vv));
  // v = (ax hx, ay hy, hz), hh = |h|^2
  const V g_hx = vfma(vmul(two, hx), g_hh, vmul(ax, g_vx));
  const V g_hy = vfma(vmul(two, hy), g_hh, vmul(ay, g_vy));
  const V g_hz = vfma(vmul(two, hz), g_hh, g_vz);
  g_ax = vfma(hx, g_vx, g_ax);
  g_ay = vfma(hy, g_vy, g_ay);
  // h = (st cp + ix, st sp + iy, om a)
  const V g_st = vfma(cp, g_hx, vmul(sp, g_hy));
  V g_ix = g_hx, g_iy = g_hy;
  g_a = vfma(om, g_hz, g_a);
  // st = sqrt(u2 S)
  const V g_S = vmul(vmul(splat<V>(0.5f), u2rq), g_st);
  // S = 2 a om + u2 rho2
  g_a = vfma(vmul(two, om), g_S, g_a);
  const V g_rho2 = vmul(u2, g_S);
  g_ix = vfma(vmul(two, ix), g_rho2, g_ix);
  g_iy = vfma(vmul(two, iy), g_rho2, g_iy);
  // a = 1 + iz
  const V g_iz = g_a;
  // i = s / |s|: g_s = (g_i - i (i . g_i)) / |s|.  Its z part is written as
  // g_iz (1 - i.z^2) - i.z (i.x g_ix + i.y g_iy) with 1 - i.z^2 = i.x^2 + i.y^2:
  // near straight down, g_iz grows like 1 / (1 + i.z) and the plain form cancels.
  const V gxy = vfma(g_ix, ix, vmul(g_iy, iy));
  const V nidot = vneg(vfma(g_iz, iz, gxy));
  const V g_sx = vmul(vfma(ix, nidot, g_ix), r);
  const V g_sy = vmul(vfma(iy, nidot, g_iy), r);
  const V g_sz = vmul(vfma(g_iz, rho2, vmul(iz, vneg(gxy))), r);
  // s = (ax wx, ay wy, wz); out-of-domain samples: zero gradients and the fallback outputs
  Grad5V<V> g;
  g.wx = vsel(ok, vmul(ax, g_sx), zero);
  g.wy = vsel(ok, vmul(ay, g_sy), zero);
  g.wz = vsel(ok, g_sz, zero);
  g.ax = vsel(ok, vfma(wx, g_sx, g_ax), zero);
  g.ay = vsel(ok, vfma(wy, g_sy, g_ay), zero);
  mx = vsel(ok, mx, zero);
  my = vsel(ok, my, zero);
  mz = vsel(ok, mz, one);
  pdf = vsel(ok, pdf, zero);
  return g;
}

}  // namespace vndf
