// vndf_sample_hemisphere: the spherical-cap sampler of Sec. 3.3 on its own,
// i.e. visible normals of the hemisphere configuration (D_std = 1/pi, Eq. 3)
// seen from a direction wi, normalised (the normalisation Sec. 3.3 says a
// stand-alone use needs) and with the density of Eq. 2.  With alpha = 1 the
// GGX NDF is D_std and M is the identity, so this is the extended-domain cap
// sampler of vndf_math.cuh with both roughnesses fixed to 1 (UnitAlpha: the
// products with them vanish at compile time), and the kernel streams 12 bytes
// in and 16 out per sample (Philox mode).  Ill-conditioned samples (|h| small against its
// summands) are redone in double-float as in vndf_sample, batched per warp.
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
#ifndef VNDF_HEMI_WAVES
#define VNDF_HEMI_WAVES 4
#endif

namespace vndf {

constexpr int kHemiBlock = 256;

struct HemiArgs {
  const float *wx, *wy, *wz, *u1, *u2;
  float *mx, *my, *mz, *pdf;
  Rng rng;
};

template <bool PHILOX>
__host__ __device__ constexpr int hemi_streams_in() { return PHILOX ? 3 : 5; }

template <bool PHILOX>
__device__ __forceinline__ void hemi_stage(const HemiArgs& a, int64_t e, float4* slot) {
  cp_async16(slot + 0 * kHemiBlock, a.wx + e);
  cp_async16(slot + 1 * kHemiBlock, a.wy + e);
  cp_async16(slot + 2 * kHemiBlock, a.wz + e);
  if constexpr (!PHILOX) {
    cp_async16(slot + 3 * kHemiBlock, a.u1 + e);
    cp_async16(slot + 4 * kHemiBlock, a.u2 + e);
  }
}

// One sample; returns (wm, pdf), the double-float path taken when needed.
template <bool PDF>
__device__ __forceinline__ float4 hemi_one(float wx, float wy, float wz, float u1, float u2) {
  float4 r;
  if (sample_one<kMethodCapExt, PDF, true>(wx, wy, wz, UnitAlpha{}, UnitAlpha{}, u1, u2, r.x, r.y, r.z, r.w))
    r = sample_one_precise<PDF, true>(wx, wy, wz, 1.f, 1.f, u1, u2);
  return r;
}

// Four samples per thread per grid-stride step, inputs staged two steps deep
// in shared memory with per-thread cp.async copies (no barriers); flagged
// samples are queued per warp and redone 32 at a time (rescue.cuh).
template <bool PHILOX, bool PDF>
__global__ void __launch_bounds__(kHemiBlock, 3) hemi_pipe_kernel(HemiArgs a, int64_t n4) {
  pdl_trigger();
  pdl_wait();
  constexpr int NS = hemi_streams_in<PHILOX>();
  extern __shared__ float4 smem_h[];  // [2][NS][kHemiBlock], then one rescue queue per warp
  RescueQueue* const queues = reinterpret_cast<RescueQueue*>(smem_h + 2 * NS * kHemiBlock);
  RescueQueue& rq = queues[threadIdx.x >> 5];
  int pending = 0;  // warp-uniform
  const int64_t stride = int64_t(gridDim.x) * kHemiBlock;
  const int64_t q0 = int64_t(blockIdx.x) * kHemiBlock + threadIdx.x;
  const int64_t w0 = q0 - (threadIdx.x & 31);
  float4* mine = smem_h + threadIdx.x;
  if (q0 < n4) hemi_stage<PHILOX>(a, 4 * q0, mine);
  cp_async_commit();
  auto redo = [&](int64_t i) {  // sample i recomputed from its inputs in global memory
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(i), u1, u2);
    } else {
      u1 = a.u1[i];
      u2 = a.u2[i];
    }
    const float4 r = sample_one_precise<PDF, true>(a.wx[i], a.wy[i], a.wz[i], 1.f, 1.f, u1, u2);
    a.mx[i] = r.x;
    a.my[i] = r.y;
    a.mz[i] = r.z;
    if constexpr (PDF) a.pdf[i] = r.w;
  };
  constexpr bool kBatched = VNDF_RESCUE_BATCHED;
  int slot = 0;
  for (int64_t q = q0, qw = w0; kBatched ? qw < n4 : q < n4; q += stride, qw += stride) {
    const bool active = !kBatched || q < n4;
    if (q + stride < n4) hemi_stage<PHILOX>(a, 4 * (q + stride), mine + (slot ^ 1) * NS * kHemiBlock);
    cp_async_commit();
    cp_async_wait<1>();
    const float4* cur = mine + slot * NS * kHemiBlock;
    slot ^= 1;
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], U1[4], U2[4];
    *reinterpret_cast<float4*>(X) = cur[0 * kHemiBlock];
    *reinterpret_cast<float4*>(Y) = cur[1 * kHemiBlock];
    *reinterpret_cast<float4*>(Z) = cur[2 * kHemiBlock];
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = cur[3 * kHemiBlock];
      *reinterpret_cast<float4*>(U2) = cur[4 * kHemiBlock];
    }
    float MX[4], MY[4], MZ[4], P[4];
    unsigned rescue = 0;
#pragma unroll
    for (int k = 0; k < 4; k += 2) {  // two packed pairs
      float2 mx, my, mz, p;
      const bool2 b = sample_one<kMethodCapExt, PDF, true>(lanes(X, k), lanes(Y, k), lanes(Z, k), UnitAlpha{},
                                                           UnitAlpha{}, lanes(U1, k), lanes(U2, k), mx, my, mz, p);
      set_lanes(MX, k, mx);
      set_lanes(MY, k, my);
      set_lanes(MZ, k, mz);
      if constexpr (PDF) set_lanes(P, k, p);
      rescue |= (unsigned(b.x) << k) | (unsigned(b.y) << (k + 1));
    }
    if constexpr (!kBatched) {
      if (rescue) {  // rare: redone in place
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (rescue & (1u << k)) {
            const float4 r = sample_one_precise<PDF, true>(X[k], Y[k], Z[k], 1.f, 1.f, U1[k], U2[k]);
            MX[k] = r.x;
            MY[k] = r.y;
            MZ[k] = r.z;
            P[k] = r.w;
          }
      }
    }
    if (active) {
      st_stream(a.mx + e, *reinterpret_cast<float4*>(MX));
      st_stream(a.my + e, *reinterpret_cast<float4*>(MY));
      st_stream(a.mz + e, *reinterpret_cast<float4*>(MZ));
      if constexpr (PDF) st_stream(a.pdf + e, *reinterpret_cast<float4*>(P));
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

template <bool PHILOX, bool PDF>
__global__ void __launch_bounds__(kHemiBlock) hemi_scalar_kernel(HemiArgs a, int64_t begin, int64_t n) {
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kHemiBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kHemiBlock + threadIdx.x; e < n; e += stride) {
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(e), u1, u2);
    } else {
      u1 = a.u1[e];
      u2 = a.u2[e];
    }
    const float4 r = hemi_one<PDF>(a.wx[e], a.wy[e], a.wz[e], u1, u2);
    a.mx[e] = r.x;
    a.my[e] = r.y;
    a.mz[e] = r.z;
    if constexpr (PDF) a.pdf[e] = r.w;
  }
}

template <bool PHILOX, bool PDF>
int launch_hemi(const HemiArgs& a, int64_t n, bool vec, cudaStream_t s) {
  int64_t done = 0;
  if (vec && n / 4 > 0) {
    const int64_t n4 = n / 4;
    constexpr size_t smem =
        size_t(2) * hemi_streams_in<PHILOX>() * kHemiBlock * 16 + (kHemiBlock / 32) * sizeof(RescueQueue);
    if (!ensure_dynamic_smem<hemi_pipe_kernel<PHILOX, PDF>>(smem)) return VNDF_ERR_CUDA;
    if (!launch_pdl(hemi_pipe_kernel<PHILOX, PDF>, grid_for(n4, kHemiBlock, 8, VNDF_HEMI_WAVES), kHemiBlock, smem, s,
                    a, n4))
      return VNDF_ERR_CUDA;
    done = 4 * n4;
  }
  if (done < n)
    if (!launch_pdl(hemi_scalar_kernel<PHILOX, PDF>, grid_for(n - done, kHemiBlock, 8, 32), kHemiBlock, 0, s, a, done,
                    n))
      return VNDF_ERR_CUDA;
  return launch_status();
}

}  // namespace vndf

using namespace vndf;

extern "C" int vndf_sample_hemisphere(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                      const float* u1, const float* u2, uint64_t seed, uint64_t counter_base,
                                      uint32_t stream_id, float* wm_x, float* wm_y, float* wm_z, float* pdf,
                                      void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !wm_x || !wm_y || !wm_z) return VNDF_ERR_NULL;
  if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
  if (!all_aligned4(wi_x, wi_y, wi_z, u1, u2, wm_x, wm_y, wm_z, pdf)) return VNDF_ERR_ALIGN;
  if (aliased({wm_x, wm_y, wm_z, pdf}, {wi_x, wi_y, wi_z, u1, u2})) return VNDF_ERR_ARG;
  if (const int f = pre_launch("vndf_sample_hemisphere")) return f;
  const HemiArgs a{wi_x, wi_y, wi_z, u1, u2, wm_x, wm_y, wm_z, pdf, make_rng(seed, counter_base, stream_id)};
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, u1, u2, wm_x, wm_y, wm_z, pdf);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (u1) return pdf ? launch_hemi<false, true>(a, n, vec, s) : launch_hemi<false, false>(a, n, vec, s);
  return pdf ? launch_hemi<true, true>(a, n, vec, s) : launch_hemi<true, false>(a, n, vec, s);
}
