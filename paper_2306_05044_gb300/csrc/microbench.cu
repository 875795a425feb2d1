// The paper's GPU benchmark protocol (Sec. 4, "GPU Synthetic Benchmark": the
// sampler called 64 times per lane) as a CUDA kernel: every lane draws its own
// incident direction and roughness in registers, samples `samples_per_lane`
// normals with the chosen hemisphere sampler and its fused pdf, and writes only
// the four sums (sum wm.x, sum wm.y, sum wm.z, sum pdf).  Memory traffic is 16
// bytes per lane, so the time measures the samplers' arithmetic, which is what
// the paper compares between the spherical-cap and the cross-section sampler.
//
// Per-lane inputs, from Philox4x32-10 block (l mod 2^32, l >> 32, 0xffffffff, 0)
// with key = seed (words w0..w3 as 24-bit uniforms v0..v3):
//   cos(theta_i) = 1e-4 + (1 - 1e-4) v0,  phi_i = 2 pi v1,
//   alpha_x = 1e-3^(1 - v2),  alpha_y = 1e-3^(1 - v3)   (log-uniform in [1e-3, 1]).
// Sample j of lane l uses the sampling layout of vndf_sample with stream 0 and
// global index l * samples_per_lane + j.
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"
#include "vndf_math.cuh"

namespace vndf {

constexpr int kMicroBlock = 256;

template <int METHOD, bool PRECISE>
__global__ void __launch_bounds__(kMicroBlock) microbench_kernel(int64_t lanes, int32_t spl, Rng r, float4* out) {
  const int64_t stride = int64_t(gridDim.x) * kMicroBlock;
  for (int64_t l = int64_t(blockIdx.x) * kMicroBlock + threadIdx.x; l < lanes; l += stride) {
    const uint4 w = philox4x32_10(make_uint4(uint32_t(l), uint32_t(uint64_t(l) >> 32), 0xffffffffu, 0u), r.k0, r.k1);
    const float ct = fmaf(1.f - 1e-4f, word_to_unit(w.x), 1e-4f);
    float sp, cp;
    sincospi_taylor(2.f * word_to_unit(w.y), sp, cp);
    const float st = sqrtf(fmaxf(fmaf(-ct, ct, 1.f), 0.f));
    const float wx = st * cp, wy = st * sp, wz = ct;
    constexpr float kLn1e3 = -6.90775527898213705f;  // ln(1e-3)
    const float ax = __expf(kLn1e3 * (1.f - word_to_unit(w.z)));
    const float ay = __expf(kLn1e3 * (1.f - word_to_unit(w.w)));
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint64_t j0 = uint64_t(l) * uint64_t(spl);
    for (int32_t j = 0; j < spl; j += 2) {
      float a1, a2, b1, b2;
      uniforms2(r, j0 + uint64_t(j), a1, a2, b1, b2);
      // the two samples as one packed pair (same bits as two single-sample calls)
      float2 m2x, m2y, m2z, p2;
      const bool2 rr = sample_one<METHOD, true, PRECISE>(splat<float2>(wx), splat<float2>(wy), splat<float2>(wz),
                                                         splat<float2>(ax), splat<float2>(ay), make_float2(a1, b1),
                                                         make_float2(a2, b2), m2x, m2y, m2z, p2);
      float mx = m2x.x, my = m2y.x, mz = m2z.x, p = p2.x, nx = m2x.y, ny = m2y.y, nz = m2z.y, q = p2.y;
      const bool ra = rr.x, rb = rr.y;
      if constexpr (METHOD == kMethodCap && PRECISE) {
        if (ra) {
          const float4 r = sample_one_precise<true>(wx, wy, wz, ax, ay, a1, a2);
          mx = r.x;
          my = r.y;
          mz = r.z;
          p = r.w;
        }
        if (rb) {
          const float4 r = sample_one_precise<true>(wx, wy, wz, ax, ay, b1, b2);
          nx = r.x;
          ny = r.y;
          nz = r.z;
          q = r.w;
        }
      }
      acc.x += mx;
      acc.y += my;
      acc.z += mz;
      acc.w += p;
      if (j + 1 < spl) {
        acc.x += nx;
        acc.y += ny;
        acc.z += nz;
        acc.w += q;
      }
    }
    out[l] = acc;
  }
}

}  // namespace vndf

using namespace vndf;

extern "C" int vndf_microbench(int64_t lanes, int32_t samples_per_lane, int method, int precise, uint64_t seed,
                               float* sums, void* cuda_stream) {
  if (lanes < 0 || lanes >= (int64_t(1) << 40) || samples_per_lane < 1 || samples_per_lane > (1 << 20))
    return VNDF_ERR_SIZE;
  if (method != VNDF_METHOD_SPHERICAL_CAP && method != VNDF_METHOD_POLAR_DISK) return VNDF_ERR_METHOD;
  if (lanes == 0) return VNDF_OK;
  if (!sums) return VNDF_ERR_NULL;
  if (!aligned(sums, 16)) return VNDF_ERR_ALIGN;
  if (const int f = pre_launch("vndf_microbench")) return f;
  const Rng r = make_rng(seed, 0, 0);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const unsigned grid = grid_for(lanes, kMicroBlock, 8, 16);
  float4* out = reinterpret_cast<float4*>(sums);
  if (method == VNDF_METHOD_SPHERICAL_CAP && precise)
    microbench_kernel<kMethodCap, true><<<grid, kMicroBlock, 0, s>>>(lanes, samples_per_lane, r, out);
  else if (method == VNDF_METHOD_SPHERICAL_CAP)
    microbench_kernel<kMethodCap, false><<<grid, kMicroBlock, 0, s>>>(lanes, samples_per_lane, r, out);
  else
    microbench_kernel<kMethodPolar, false><<<grid, kMicroBlock, 0, s>>>(lanes, samples_per_lane, r, out);
  return launch_status();
}
