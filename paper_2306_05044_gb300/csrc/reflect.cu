// Reflection-BSDF sampling with the spherical-cap VNDF sampler: the step a
// renderer takes right after drawing a visible normal (App. A, "Importance
// Sampling Using the GGX VNDF"):
//   wm  ~ D_vis(., wi)                           (Sec. 2 steps (1)-(3), Sec. 3.3)
//   wo  = 2 (wi.wm) wm - wi                      (Eq. reflect)
//   PDF = G1(wm, wi) D(wm) / (4 cos theta_i)     (App. A, with the Jacobian of Eq. jacobian)
//   weight = f_r(wo, wi) |cos theta_o| / PDF = F(wi.wm) G2 / G1(wi)   (App. A, Eq. rendering_mc, L = 1)
// with Schlick's Fresnel and the height-correlated G2 (zero when wo is below
// the surface).  Everything is written from the sampler's hemisphere
// quantities (h = c + i, v = M^-T h, L = |M^-1 wi|) so that nothing cancels:
//   wi.wm = L |h|^2 / (2 |wi| |v|)               (because i.h = |h|^2 / 2 on the cap),
//   PDF   = |wi| |v|^4 / (2 pi ax ay L (1 + i.z) |h|^4)
//   (D(wm) = |v|^4 / (pi ax ay |h|^4) and G1 / (4 cos theta_i) = |wi| / (2 L (1 + i.z))).
// Samples whose half vector is ill-conditioned get it recomputed in
// double-float, as in vndf_sample (queued per warp and redone 32 at a time).
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"
#include "rescue.cuh"
#include "staging.cuh"
#include "vndf_math.cuh"

// 1: ill-conditioned samples queued per warp and redone 32 at a time (rescue.cuh); 0: in place.
#ifndef VNDF_RESCUE_BATCHED
#define VNDF_RESCUE_BATCHED 1
#endif
// Grid of the streaming kernel: at most this many waves of 8 CTAs per SM.
#ifndef VNDF_REFL_WAVES
#define VNDF_REFL_WAVES 4
#endif

namespace vndf {

constexpr int kReflBlock = 256;

struct ReflArgs {
  const float *wx, *wy, *wz, *ax, *ay, *u1, *u2;
  float f0;
  float *ox, *oy, *oz, *pdf, *weight;
  Rng rng;
};

// Half vector (hx, hy, hz) and a = 1 + i.z of an ill-conditioned sample, in double-float.
__device__ __noinline__ float4 half_vector_precise(float wx, float wy, float wz, float ax, float ay, float u1,
                                                   float u2) {
  float4 r;
  cap_half_vector_precise(wx, wy, wz, ax, ay, u1, u2, r.x, r.y, r.z, r.w);
  return r;
}

template <typename V>
struct ReflectedV {
  V ox, oy, oz, pdf, weight;
};
using Reflected = ReflectedV<float>;

// One reflected sample (V = float) or two (V = float2, on the packed FP32x2
// operations; both widths give the same bits).  With PRECISE_H (one sample
// only) the half vector comes from the double-float path; otherwise from FP32,
// and *bad reports whether it was ill-conditioned (the caller then redoes the
// sample with PRECISE_H).
template <bool PRECISE_H, typename V>
__device__ __forceinline__ ReflectedV<V> reflect_one(V wx, V wy, V wz, V ax, V ay, V u1, V u2, float f0,
                                                     Mask<V>* bad) {
  const Mask<V> ok = in_domain(wx, wy, wz, ax, ay);
  const V sx = vmul(ax, wx), sy = vmul(ay, wy);
  const V l2 = vfma(sx, sx, vfma(sy, sy, vmul(wz, wz)));
  const V rl = vmap(RsqrtF{}, l2);
  const StretchedV<V> i{vmul(sx, rl), vmul(sy, rl), vmul(wz, rl), vfma(wz, rl, splat<V>(1.f))};
  V hx, hy, hz, a;
  if constexpr (PRECISE_H) {
    static_assert(sizeof(V) == sizeof(float), "the double-float path takes one sample");
    const float4 p = half_vector_precise(wx, wy, wz, ax, ay, u1, u2);
    hx = p.x;
    hy = p.y;
    hz = p.z;
    a = p.w;
  } else {
    cap_half_vector(i, u1, u2, hx, hy, hz, a);
    // the condition check of sample_one<cap, PDF, PRECISE>
    const V cx = vadd(vabs(vsub(hx, i.x)), vabs(i.x)), cy = vadd(vabs(vsub(hy, i.y)), vabs(i.y));
    const V vx = vmul(ax, hx), vy = vmul(ay, hy);
    const V hz2 = vmul(hz, hz);
    const V vv = vfma(vx, vx, vfma(vy, vy, hz2));
    const V kx = vmul(ax, cx), ky = vmul(ay, cy);
    const V k2 = vfma(kx, kx, vfma(ky, ky, hz2));
    const V kh2 = vfma(cx, cx, vfma(cy, cy, hz2));
    const V hh = vfma(hx, hx, vfma(hy, hy, hz2));
    const V K2 = splat<V>(kRescueKappa * kRescueKappa);
    *bad = ok & (vgt(k2, vmul(K2, vv)) | vgt(kh2, vmul(K2, hh)));
  }
  const V vx = vmul(ax, hx), vy = vmul(ay, hy), vz = hz;
  const V vv = vfma(vx, vx, vfma(vy, vy, vmul(vz, vz)));
  const V rv = vmap(RsqrtF{}, vv);
  const V mx = vmul(vx, rv), my = vmul(vy, rv), mz = vmul(vz, rv);
  const V hh = vfma(hx, hx, vfma(hy, hy, vmul(hz, hz)));
  const V rw = vmap(RsqrtF{}, vfma(wx, wx, vfma(wy, wy, vmul(wz, wz))));  // 1 / |wi|
  const V L = vmul(l2, rl);
  const V ux = vmul(wx, rw), uy = vmul(wy, rw), uz = vmul(wz, rw);  // unit wi
  const V d = vmul(vmul(vmul(vmul(splat<V>(0.5f), L), hh), rv), rw);  // wi.wm without cancellation
  const V d2 = vmul(splat<V>(2.f), d);
  ReflectedV<V> r;
  r.ox = vfma(d2, mx, vneg(ux));
  r.oy = vfma(d2, my, vneg(uy));
  r.oz = vfma(d2, mz, vneg(uz));
  // PDF = |wi| |v|^4 / (2 pi ax ay L a |h|^4)
  V den = vmul(vmul(vmul(splat<V>(2.f * kPi), ax), ay), L);
  den = vmul(vmul(vmul(vmul(den, a), hh), hh), rw);
  r.pdf = vmul(vmul(vv, vv), vmap(RcpFast{}, den));
  // weight = F G2 / G1(wi) with G2 / G1 = (L_u + z_u) z_o / ((L_u + z_u) z_o + z_u P_o / (L_o + z_o))
  const V A = vfma(L, rw, uz);  // |M^-1 wi_unit| + wi_unit.z
  const V px = vmul(ax, r.ox), py = vmul(ay, r.oy);
  const V po = vfma(px, px, vmul(py, py));
  const V lo = vmap(SqrtFast{}, vfma(r.oz, r.oz, po));
  const V num = vmul(A, r.oz);
  const V g = vmul(num, vmap(RcpFast{}, vfma(vmul(uz, po), vmap(RcpFast{}, vadd(lo, r.oz)), num)));
  const V t = vsub(splat<V>(1.f), d);
  const V t2 = vmul(t, t);
  const V fr = vfma(splat<V>(1.f - f0), vmul(vmul(t2, t2), t), splat<V>(f0));
  r.weight = vsel(vgt(r.oz, splat<V>(0.f)), vmul(fr, g), splat<V>(0.f));
  // out-of-domain inputs: wo = (0, 0, 1), pdf = weight = 0
  r.ox = vsel(ok, r.ox, splat<V>(0.f));
  r.oy = vsel(ok, r.oy, splat<V>(0.f));
  r.oz = vsel(ok, r.oz, splat<V>(1.f));
  r.pdf = vsel(ok, r.pdf, splat<V>(0.f));
  r.weight = vsel(ok, r.weight, splat<V>(0.f));
  return r;
}

template <bool PHILOX, bool ISO>
__device__ __forceinline__ void refl_stage(const ReflArgs& a, int64_t e, float4* slot) {
  cp_async16(slot + 0 * kReflBlock, a.wx + e);
  cp_async16(slot + 1 * kReflBlock, a.wy + e);
  cp_async16(slot + 2 * kReflBlock, a.wz + e);
  cp_async16(slot + 3 * kReflBlock, a.ax + e);
  int k = 4;
  if constexpr (!ISO) cp_async16(slot + (k++) * kReflBlock, a.ay + e);
  if constexpr (!PHILOX) {
    cp_async16(slot + (k++) * kReflBlock, a.u1 + e);
    cp_async16(slot + (k++) * kReflBlock, a.u2 + e);
  }
}

// Four samples per thread per grid-stride step (two packed pairs), inputs staged two steps deep;
// ill-conditioned samples are queued per warp and redone 32 at a time (rescue.cuh).  Two CTAs per SM:
// the register file then holds both pairs' reflection and weight arithmetic without spilling (124
// registers); measured at 2^28 with weights, 1633 us against 1653 us at three CTAs (80 registers, 16-28
// bytes of spills) and 1670 us at four.
template <bool PHILOX, bool ISO>
__global__ void __launch_bounds__(kReflBlock, 2) reflect_pipe_kernel(ReflArgs a, int64_t n4) {
  pdl_trigger();
  pdl_wait();
  constexpr int NS = streams_in<PHILOX, ISO>();
  extern __shared__ float4 smem_r[];  // [2][NS][kReflBlock], then one rescue queue per warp
  RescueQueue* const queues = reinterpret_cast<RescueQueue*>(smem_r + 2 * NS * kReflBlock);
  RescueQueue& rq = queues[threadIdx.x >> 5];
  int pending = 0;  // warp-uniform
  const int64_t stride = int64_t(gridDim.x) * kReflBlock;
  const int64_t q0 = int64_t(blockIdx.x) * kReflBlock + threadIdx.x;
  const int64_t w0 = q0 - (threadIdx.x & 31);
  float4* mine = smem_r + threadIdx.x;
  if (q0 < n4) refl_stage<PHILOX, ISO>(a, 4 * q0, mine);
  cp_async_commit();
  auto redo = [&](int64_t i) {  // sample i recomputed from its inputs in global memory
    const float ax = a.ax[i], ay = ISO ? ax : a.ay[i];
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(i), u1, u2);
    } else {
      u1 = a.u1[i];
      u2 = a.u2[i];
    }
    const Reflected r = reflect_one<true>(a.wx[i], a.wy[i], a.wz[i], ax, ay, u1, u2, a.f0, nullptr);
    a.ox[i] = r.ox;
    a.oy[i] = r.oy;
    a.oz[i] = r.oz;
    if (a.pdf) a.pdf[i] = r.pdf;
    if (a.weight) a.weight[i] = r.weight;
  };
  constexpr bool kBatched = VNDF_RESCUE_BATCHED;
  int slot = 0;
  for (int64_t q = q0, qw = w0; kBatched ? qw < n4 : q < n4; q += stride, qw += stride) {
    const bool active = !kBatched || q < n4;
    if (q + stride < n4) refl_stage<PHILOX, ISO>(a, 4 * (q + stride), mine + (slot ^ 1) * NS * kReflBlock);
    cp_async_commit();
    cp_async_wait<1>();
    const float4* cur = mine + slot * NS * kReflBlock;
    slot ^= 1;
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4];
    *reinterpret_cast<float4*>(X) = cur[0 * kReflBlock];
    *reinterpret_cast<float4*>(Y) = cur[1 * kReflBlock];
    *reinterpret_cast<float4*>(Z) = cur[2 * kReflBlock];
    *reinterpret_cast<float4*>(AX) = cur[3 * kReflBlock];
    *reinterpret_cast<float4*>(AY) = ISO ? cur[3 * kReflBlock] : cur[4 * kReflBlock];
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = cur[(ISO ? 4 : 5) * kReflBlock];
      *reinterpret_cast<float4*>(U2) = cur[(ISO ? 5 : 6) * kReflBlock];
    }
    float OX[4], OY[4], OZ[4], P[4], Wt[4];
    unsigned rescue = 0;
#pragma unroll
    for (int k = 0; k < 4; k += 2) {  // two packed pairs
      bool2 bad;
      const ReflectedV<float2> r = reflect_one<false>(lanes(X, k), lanes(Y, k), lanes(Z, k), lanes(AX, k),
                                                      lanes(AY, k), lanes(U1, k), lanes(U2, k), a.f0, &bad);
      set_lanes(OX, k, r.ox);
      set_lanes(OY, k, r.oy);
      set_lanes(OZ, k, r.oz);
      set_lanes(P, k, r.pdf);
      set_lanes(Wt, k, r.weight);
      rescue |= (unsigned(bad.x) << k) | (unsigned(bad.y) << (k + 1));
    }
    if constexpr (!kBatched) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (rescue & (1u << k)) {  // rare: redone in place
          const Reflected r =
              reflect_one<true>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k], a.f0, static_cast<bool*>(nullptr));
          OX[k] = r.ox;
          OY[k] = r.oy;
          OZ[k] = r.oz;
          P[k] = r.pdf;
          Wt[k] = r.weight;
        }
    }
    if (active) {
      st_stream(a.ox + e, *reinterpret_cast<float4*>(OX));
      st_stream(a.oy + e, *reinterpret_cast<float4*>(OY));
      st_stream(a.oz + e, *reinterpret_cast<float4*>(OZ));
      if (a.pdf) st_stream(a.pdf + e, *reinterpret_cast<float4*>(P));
      if (a.weight) st_stream(a.weight + e, *reinterpret_cast<float4*>(Wt));
    } else {
      rescue = 0;
    }
    if (kBatched && __any_sync(0xffffffffu, rescue != 0)) {  // rare
#pragma unroll
      for (int k = 0; k < 4; ++k) rescue_push(rq, pending, (rescue >> k) & 1u, e + k);
      rescue_drain(rq, pending, false, redo);
    }
  }
  if constexpr (kBatched) rescue_drain_cta(queues, pending, redo);
  cp_async_wait<0>();
}

template <bool PHILOX, bool ISO>
__global__ void __launch_bounds__(kReflBlock) reflect_scalar_kernel(ReflArgs a, int64_t begin, int64_t n) {
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kReflBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kReflBlock + threadIdx.x; e < n; e += stride) {
    const float ax = a.ax[e];
    const float ay = ISO ? ax : a.ay[e];
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(e), u1, u2);
    } else {
      u1 = a.u1[e];
      u2 = a.u2[e];
    }
    bool bad;
    Reflected r = reflect_one<false>(a.wx[e], a.wy[e], a.wz[e], ax, ay, u1, u2, a.f0, &bad);
    if (bad) r = reflect_one<true>(a.wx[e], a.wy[e], a.wz[e], ax, ay, u1, u2, a.f0, nullptr);
    a.ox[e] = r.ox;
    a.oy[e] = r.oy;
    a.oz[e] = r.oz;
    if (a.pdf) a.pdf[e] = r.pdf;
    if (a.weight) a.weight[e] = r.weight;
  }
}

template <bool PHILOX, bool ISO>
int launch_reflect(const ReflArgs& a, int64_t n, bool vec, cudaStream_t s) {
  int64_t done = 0;
  if (vec && n / 4 > 0) {
    const int64_t n4 = n / 4;
    constexpr size_t smem =
        size_t(2) * streams_in<PHILOX, ISO>() * kReflBlock * 16 + (kReflBlock / 32) * sizeof(RescueQueue);
    if (!ensure_dynamic_smem<reflect_pipe_kernel<PHILOX, ISO>>(smem)) return VNDF_ERR_CUDA;
    if (!launch_pdl(reflect_pipe_kernel<PHILOX, ISO>, grid_for(n4, kReflBlock, 8, VNDF_REFL_WAVES), kReflBlock, smem,
                    s, a, n4))
      return VNDF_ERR_CUDA;
    done = 4 * n4;
  }
  if (done < n)
    if (!launch_pdl(reflect_scalar_kernel<PHILOX, ISO>, grid_for(n - done, kReflBlock, 8, 32), kReflBlock, 0, s, a,
                    done, n))
      return VNDF_ERR_CUDA;
  return launch_status();
}

}  // namespace vndf

using namespace vndf;

extern "C" int vndf_sample_reflection(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                      const float* alpha_x, const float* alpha_y, const float* u1, const float* u2,
                                      uint64_t seed, uint64_t counter_base, uint32_t stream_id, float f0,
                                      float* wo_x, float* wo_y, float* wo_z, float* pdf, float* weight,
                                      void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !wo_x || !wo_y || !wo_z) return VNDF_ERR_NULL;
  if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wo_x, wo_y, wo_z, pdf, weight))
    return VNDF_ERR_ALIGN;
  if (aliased({wo_x, wo_y, wo_z, pdf, weight}, {wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2})) return VNDF_ERR_ARG;
  if (const int f = pre_launch("vndf_sample_reflection")) return f;
  const ReflArgs a{wi_x, wi_y, wi_z, alpha_x, alpha_y, u1,     u2,
                   f0,   wo_x, wo_y, wo_z,    pdf,     weight, make_rng(seed, counter_base, stream_id)};
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wo_x, wo_y, wo_z, pdf, weight);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (u1) return alpha_y ? launch_reflect<false, false>(a, n, vec, s) : launch_reflect<false, true>(a, n, vec, s);
  return alpha_y ? launch_reflect<true, false>(a, n, vec, s) : launch_reflect<true, true>(a, n, vec, s);
}
