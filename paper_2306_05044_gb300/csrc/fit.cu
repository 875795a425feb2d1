// One optimisation step of a roughness map through reparameterised
// spherical-cap samples (forward, adjoint and Adam in two launches that a
// CUDA graph can capture together).
//
// Per texel t (one CTA), with S samples drawn as in vndf_sample (Sec. 2 steps
// (1)-(3), Sec. 3.3) from Philox stream stream_id + t at global indices
// counter_base + (step - 1) S + j:
//   m_t   = (1/S) sum_j wm_tj                                  (lobe mean)
//   L     = (1 / 3N) sum_t |m_t - target_t|^2                   (MSE; N texels in the whole map)
//   g_t   = dL/d(ax_t, ay_t) = (2 / 3N S) sum_j (m_t - target_t) . d wm_tj / d alpha
//   Adam (Kingma & Ba 2015) with bias correction at the 1-based step, then
//   alpha is projected onto [alpha_min, alpha_max].
// The step counter lives in device memory: the finishing kernel adds one, so
// replaying a captured graph advances the optimisation.  Every sum runs in a
// fixed order (per-thread sample order, fixed warp/block trees, texels in
// index order), so a run is bit-reproducible and can be checkpointed by
// saving alpha, the Adam moments and the step counter.
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"
#include "vndf_adjoint.cuh"

namespace vndf {

constexpr int kFitBlock = 256;

struct FitArgs {
  int32_t nt, ns;
  int32_t n_total;  // texels of the whole map (normalisation of the loss and its gradient)
  const float *wx, *wy, *wz, *tx, *ty, *tz;
  float *ax, *ay, *mx, *my, *vx, *vy;
  int64_t* step;
  float lr, b1, b2, eps, amin, amax;
  Rng rng;  // rng.stream: stream id of texel 0
  float* texel_loss;
  float* loss;
};

__device__ __forceinline__ float warp_sum_fit(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum of three values; the result is returned to every thread.
__device__ __forceinline__ float3 block_sum3(float3 v, float (*sm)[kFitBlock / 32]) {
  v.x = warp_sum_fit(v.x);
  v.y = warp_sum_fit(v.y);
  v.z = warp_sum_fit(v.z);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sm[0][w] = v.x;
    sm[1][w] = v.y;
    sm[2][w] = v.z;
  }
  __syncthreads();
  float3 r;
  r.x = warp_sum_fit(l < kFitBlock / 32 ? sm[0][l] : 0.f);
  r.y = warp_sum_fit(l < kFitBlock / 32 ? sm[1][l] : 0.f);
  r.z = warp_sum_fit(l < kFitBlock / 32 ? sm[2][l] : 0.f);
  __syncthreads();
  return r;  // identical in every warp (same inputs, same tree)
}

// 4 CTAs per SM (at most 64 registers): keeping the uniforms between the passes would otherwise
// take the kernel to 74 registers and 3 CTAs.
__global__ void __launch_bounds__(kFitBlock, 4) fit_kernel(FitArgs a) {
  __shared__ float sm[3][kFitBlock / 32];
  const int64_t step = *a.step + 1;  // 1-based step performed by this launch
  Rng r = a.rng;
  r.base = a.rng.base + uint64_t(step - 1) * uint64_t(a.ns);
  const float inv_s = 1.f / float(a.ns);
  const float gscale = 2.f / (3.f * float(a.n_total));
  for (int32_t t = blockIdx.x; t < a.nt; t += gridDim.x) {
    const float wx = a.wx[t], wy = a.wy[t], wz = a.wz[t];
    const float ax = a.ax[t], ay = a.ay[t];
    Rng rt = r;
    rt.stream = a.rng.stream + uint32_t(t);
    // When every thread has at most one group of 4 samples (S <= 4 x block), the uniforms of the
    // forward pass are kept in registers for the adjoint pass instead of being drawn again.
    const bool one_group = a.ns <= 4 * kFitBlock;
    float ku1[4] = {0.f, 0.f, 0.f, 0.f}, ku2[4] = {0.f, 0.f, 0.f, 0.f};
    // ---- forward: lobe mean
    float3 sum = make_float3(0.f, 0.f, 0.f);
    for (int32_t j0 = 4 * threadIdx.x; j0 < a.ns; j0 += 4 * kFitBlock) {
      float u1[4], u2[4];
      uniforms2(rt, uint64_t(j0), u1[0], u2[0], u1[1], u2[1]);
      uniforms2(rt, uint64_t(j0 + 2), u1[2], u2[2], u1[3], u2[3]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ku1[k] = u1[k];
        ku2[k] = u2[k];
      }
#pragma unroll
      for (int k = 0; k < 4; k += 2) {  // two packed pairs, added in sample order
        float2 mx, my, mz, p;
        sample_one<kMethodCap, false>(splat<float2>(wx), splat<float2>(wy), splat<float2>(wz), splat<float2>(ax),
                                      splat<float2>(ay), lanes(u1, k), lanes(u2, k), mx, my, mz, p);
        if (j0 + k < a.ns) {
          sum.x += mx.x;
          sum.y += my.x;
          sum.z += mz.x;
        }
        if (j0 + k + 1 < a.ns) {
          sum.x += mx.y;
          sum.y += my.y;
          sum.z += mz.y;
        }
      }
    }
    const float3 m = block_sum3(sum, sm);
    const float dx = m.x * inv_s - a.tx[t], dy = m.y * inv_s - a.ty[t], dz = m.z * inv_s - a.tz[t];
    // ---- adjoint of the lobe mean: every sample sees g_wm = (2 / 3T)(m - target) / S
    const float gx = gscale * dx * inv_s, gy = gscale * dy * inv_s, gz = gscale * dz * inv_s;
    float3 ga = make_float3(0.f, 0.f, 0.f);
    for (int32_t j0 = 4 * threadIdx.x; j0 < a.ns; j0 += 4 * kFitBlock) {
      float u1[4], u2[4];
      if (one_group) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          u1[k] = ku1[k];
          u2[k] = ku2[k];
        }
      } else {
        uniforms2(rt, uint64_t(j0), u1[0], u2[0], u1[1], u2[1]);
        uniforms2(rt, uint64_t(j0 + 2), u1[2], u2[2], u1[3], u2[3]);
      }
#pragma unroll
      for (int k = 0; k < 4; k += 2) {  // two packed pairs, added in sample order
        float2 mx, my, mz, p;
        const Grad5V<float2> g = cap_backward_one<false>(
            splat<float2>(wx), splat<float2>(wy), splat<float2>(wz), splat<float2>(ax), splat<float2>(ay),
            lanes(u1, k), lanes(u2, k), splat<float2>(gx), splat<float2>(gy), splat<float2>(gz), splat<float2>(0.f),
            splat<float2>(0.f), mx, my, mz, p);
        if (j0 + k < a.ns) {
          ga.x += g.ax.x;
          ga.y += g.ay.x;
        }
        if (j0 + k + 1 < a.ns) {
          ga.x += g.ax.y;
          ga.y += g.ay.y;
        }
      }
    }
    const float3 g = block_sum3(ga, sm);
    if (threadIdx.x == 0) {
      const float c1 = 1.f - powf(a.b1, float(step));
      const float c2 = 1.f - powf(a.b2, float(step));
      const float mx = fmaf(a.b1, a.mx[t], (1.f - a.b1) * g.x);
      const float my = fmaf(a.b1, a.my[t], (1.f - a.b1) * g.y);
      const float vx = fmaf(a.b2, a.vx[t], (1.f - a.b2) * g.x * g.x);
      const float vy = fmaf(a.b2, a.vy[t], (1.f - a.b2) * g.y * g.y);
      const float nx = ax - a.lr * (mx / c1) / (sqrtf(vx / c2) + a.eps);
      const float ny = ay - a.lr * (my / c1) / (sqrtf(vy / c2) + a.eps);
      a.mx[t] = mx;
      a.my[t] = my;
      a.vx[t] = vx;
      a.vy[t] = vy;
      a.ax[t] = fminf(fmaxf(nx, a.amin), a.amax);
      a.ay[t] = fminf(fmaxf(ny, a.amin), a.amax);
      a.texel_loss[t] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    }
  }
}

// Loss = sum of texel losses (texel order, fixed tree) / 3N; then advance the step counter.
__global__ void __launch_bounds__(1024) fit_finish_kernel(FitArgs a) {
  __shared__ float sm[32];
  float v = 0.f;
  // thread t sums texels t, t + 1024, ... in order (coalesced loads, 16 in flight), then a fixed tree
#pragma unroll 16
  for (int32_t t = threadIdx.x; t < a.nt; t += 1024) v += a.texel_loss[t];
  v = warp_sum_fit(v);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s = warp_sum_fit(sm[threadIdx.x]);
    if (threadIdx.x == 0) {
      if (a.loss) *a.loss = s / (3.f * float(a.n_total));
      *a.step += 1;
    }
  }
}

}  // namespace vndf

using namespace vndf;

extern "C" size_t vndf_fit_workspace_bytes(int32_t n_texels) {
  return n_texels > 0 ? size_t(n_texels) * sizeof(float) : 0;
}

extern "C" int vndf_fit_step(int32_t n_texels, int32_t n_texels_total, int32_t samples_per_texel,
                             const float* wi_x, const float* wi_y,
                             const float* wi_z, const float* target_x, const float* target_y, const float* target_z,
                             float* alpha_x, float* alpha_y, float* adam_m_x, float* adam_m_y, float* adam_v_x,
                             float* adam_v_y, int64_t* step, float lr, float beta1, float beta2, float eps,
                             float alpha_min, float alpha_max, uint64_t seed, uint64_t counter_base,
                             uint32_t stream_id, float* loss, void* workspace, size_t workspace_bytes,
                             void* cuda_stream) {
  if (n_texels < 0 || samples_per_texel < 1 || samples_per_texel > (1 << 20)) return VNDF_ERR_SIZE;
  if (n_texels_total != 0 && n_texels_total < n_texels) return VNDF_ERR_SIZE;
  if (n_texels == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !target_x || !target_y || !target_z || !alpha_x || !alpha_y || !adam_m_x ||
      !adam_m_y || !adam_v_x || !adam_v_y || !step)
    return VNDF_ERR_NULL;
  if (!(alpha_min > 0.f) || !(alpha_max >= alpha_min) || !(lr >= 0.f) || !(eps >= 0.f) || !(beta1 >= 0.f) ||
      !(beta1 < 1.f) || !(beta2 >= 0.f) || !(beta2 < 1.f))
    return VNDF_ERR_ARG;
  if (!workspace || workspace_bytes < vndf_fit_workspace_bytes(n_texels)) return VNDF_ERR_WORKSPACE;
  if (!all_aligned4(wi_x, wi_y, wi_z, target_x, target_y, target_z, alpha_x, alpha_y, adam_m_x, adam_m_y,
                    adam_v_x, adam_v_y, loss, workspace) ||
      !aligned(step, 8))
    return VNDF_ERR_ALIGN;
  // alpha and the Adam moments are read and updated in place; each must be an array of its own
  if (aliased({alpha_x, alpha_y, adam_m_x, adam_m_y, adam_v_x, adam_v_y, step, loss, workspace},
              {wi_x, wi_y, wi_z, target_x, target_y, target_z}))
    return VNDF_ERR_ARG;
  if (const int f = pre_launch("vndf_fit_step", true)) return f;
  FitArgs a{n_texels, samples_per_texel, n_texels_total ? n_texels_total : n_texels,
            wi_x,     wi_y,     wi_z,     target_x,  target_y, target_z,
            alpha_x,  alpha_y,           adam_m_x, adam_m_y, adam_v_x, adam_v_y,  step,     lr,
            beta1,    beta2,             eps,      alpha_min, alpha_max, make_rng(seed, counter_base, stream_id),
            static_cast<float*>(workspace), loss};
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const unsigned grid = grid_for(int64_t(n_texels) * kFitBlock, kFitBlock, 8, 64);
  fit_kernel<<<grid, kFitBlock, 0, s>>>(a);
  fit_finish_kernel<<<1, 1024, 0, s>>>(a);
  return launch_status();
}
