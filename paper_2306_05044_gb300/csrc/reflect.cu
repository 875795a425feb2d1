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
#ifndef VNDF_SAMPLE_WAVES
#define VNDF_SAMPLE_WAVES 4
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

struct Reflected {
  float ox, oy, oz, pdf, weight;
};

// One reflected sample.  With PRECISE_H the half vector comes from the
// double-float path; otherwise from FP32, and *bad reports whether it was
// ill-conditioned (the caller then redoes the sample with PRECISE_H).
template <bool PRECISE_H>
__device__ __forceinline__ Reflected reflect_one(float wx, float wy, float wz, float ax, float ay, float u1,
                                                 float u2, float f0, bool* bad) {
  const bool ok = in_domain(wx, wy, wz, ax, ay);
  const float sx = ax * wx, sy = ay * wy;
  const float l2 = fmaf(sx, sx, fmaf(sy, sy, wz * wz));
  const float rl = rsqrtf(l2);
  const Stretched i{sx * rl, sy * rl, wz * rl, fmaf(wz, rl, 1.f)};
  float hx, hy, hz, a;
  if constexpr (PRECISE_H) {
    const float4 p = half_vector_precise(wx, wy, wz, ax, ay, u1, u2);
    hx = p.x;
    hy = p.y;
    hz = p.z;
    a = p.w;
  } else {
    cap_half_vector(i, u1, u2, hx, hy, hz, a);
    // the condition check of sample_one<cap, PDF, PRECISE>
    const float cx = fabsf(hx - i.x) + fabsf(i.x), cy = fabsf(hy - i.y) + fabsf(i.y);
    const float vx = ax * hx, vy = ay * hy;
    const float vv = fmaf(vx, vx, fmaf(vy, vy, hz * hz));
    const float k2 = fmaf(ax * cx, ax * cx, fmaf(ay * cy, ay * cy, hz * hz));
    const float kh2 = fmaf(cx, cx, fmaf(cy, cy, hz * hz));
    const float hh = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
    *bad = ok & ((k2 > kRescueKappa * kRescueKappa * vv) | (kh2 > kRescueKappa * kRescueKappa * hh));
  }
  const float vx = ax * hx, vy = ay * hy, vz = hz;
  const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  const float rv = rsqrtf(vv);
  const float mx = vx * rv, my = vy * rv, mz = vz * rv;
  const float hh = fmaf(hx, hx, fmaf(hy, hy, hz * hz));
  const float wn2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
  const float rw = rsqrtf(wn2);                      // 1 / |wi|
  const float L = l2 * rl;
  const float ux = wx * rw, uy = wy * rw, uz = wz * rw;  // unit wi
  const float d = 0.5f * L * hh * rv * rw;           // wi.wm without cancellation
  Reflected r;
  r.ox = fmaf(2.f * d, mx, -ux);
  r.oy = fmaf(2.f * d, my, -uy);
  r.oz = fmaf(2.f * d, mz, -uz);
  // PDF = |wi| |v|^4 / (2 pi ax ay L a |h|^4)
  r.pdf = vv * vv * rcp_fast(2.f * kPi * ax * ay * L * a * hh * hh * rw);
  // weight = F G2 / G1(wi) with G2 / G1 = (L_u + z_u) z_o / ((L_u + z_u) z_o + z_u P_o / (L_o + z_o))
  const float A = fmaf(L, rw, uz);                   // |M^-1 wi_unit| + wi_unit.z
  const float px = ax * r.ox, py = ay * r.oy;
  const float po = fmaf(px, px, py * py);
  const float lo = sqrt_fast(fmaf(r.oz, r.oz, po));
  const float num = A * r.oz;
  const float g = num * rcp_fast(fmaf(uz * po, rcp_fast(lo + r.oz), num));
  const float t = 1.f - d;
  const float t2 = t * t;
  const float fr = fmaf(1.f - f0, t2 * t2 * t, f0);
  r.weight = r.oz > 0.f ? fr * g : 0.f;
  if (!ok) r = Reflected{0.f, 0.f, 1.f, 0.f, 0.f};
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

// Four samples per thread per grid-stride step, inputs staged two steps deep;
// ill-conditioned samples are queued per warp and redone 32 at a time (rescue.cuh).
template <bool PHILOX, bool ISO>
__global__ void __launch_bounds__(kReflBlock, 3) reflect_pipe_kernel(ReflArgs a, int64_t n4) {
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
    for (int k = 0; k < 4; ++k) {
      bool bad;
      Reflected r = reflect_one<false>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k], a.f0, &bad);
      if (!kBatched && bad) r = reflect_one<true>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k], a.f0, nullptr);
      rescue |= unsigned(bad) << k;
      OX[k] = r.ox;
      OY[k] = r.oy;
      OZ[k] = r.oz;
      P[k] = r.pdf;
      Wt[k] = r.weight;
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
    if (!launch_pdl(reflect_pipe_kernel<PHILOX, ISO>, grid_for(n4, kReflBlock, 8, VNDF_SAMPLE_WAVES), kReflBlock, smem,
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
