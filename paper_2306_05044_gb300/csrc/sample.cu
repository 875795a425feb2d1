// Streaming kernels of the sampling hot path: vndf_rng_uniform, vndf_sample,
// vndf_pdf.  One thread handles four consecutive samples with 128-bit loads and
// stores of every structure-of-arrays stream (coalesced: a warp moves 512
// contiguous bytes per array); a scalar kernel covers the n % 4 tail and
// unaligned buffers with the same per-sample function, so results do not
// depend on the path taken.
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"
#include "vndf_math.cuh"

namespace vndf {

constexpr int kBlock = 256;

struct SampleArgs {
  const float *wx, *wy, *wz, *ax, *ay, *u1, *u2;
  float *mx, *my, *mz, *pdf;
  Rng rng;
};

template <int METHOD, bool PHILOX, bool ISO, bool PDF>
__global__ void __launch_bounds__(kBlock) sample_vec4_kernel(SampleArgs a, int64_t n4) {
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t q = int64_t(blockIdx.x) * kBlock + threadIdx.x; q < n4; q += stride) {
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4];
    *reinterpret_cast<float4*>(X) = ld_stream(a.wx + e);
    *reinterpret_cast<float4*>(Y) = ld_stream(a.wy + e);
    *reinterpret_cast<float4*>(Z) = ld_stream(a.wz + e);
    *reinterpret_cast<float4*>(AX) = ld_stream(a.ax + e);
    if constexpr (ISO) {
      *reinterpret_cast<float4*>(AY) = *reinterpret_cast<float4*>(AX);
    } else {
      *reinterpret_cast<float4*>(AY) = ld_stream(a.ay + e);
    }
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = ld_stream(a.u1 + e);
      *reinterpret_cast<float4*>(U2) = ld_stream(a.u2 + e);
    }
    float MX[4], MY[4], MZ[4], P[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      sample_one<METHOD, PDF>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k], MX[k], MY[k], MZ[k], P[k]);
    st_stream(a.mx + e, *reinterpret_cast<float4*>(MX));
    st_stream(a.my + e, *reinterpret_cast<float4*>(MY));
    st_stream(a.mz + e, *reinterpret_cast<float4*>(MZ));
    if constexpr (PDF) st_stream(a.pdf + e, *reinterpret_cast<float4*>(P));
  }
}

template <int METHOD, bool PHILOX, bool ISO, bool PDF>
__global__ void __launch_bounds__(kBlock) sample_scalar_kernel(SampleArgs a, int64_t begin, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kBlock + threadIdx.x; e < n; e += stride) {
    const float ax = a.ax[e];
    const float ay = ISO ? ax : a.ay[e];
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(e), u1, u2);
    } else {
      u1 = a.u1[e];
      u2 = a.u2[e];
    }
    float mx, my, mz, p;
    sample_one<METHOD, PDF>(a.wx[e], a.wy[e], a.wz[e], ax, ay, u1, u2, mx, my, mz, p);
    a.mx[e] = mx;
    a.my[e] = my;
    a.mz[e] = mz;
    if constexpr (PDF) a.pdf[e] = p;
  }
}

template <int METHOD, bool PHILOX, bool ISO, bool PDF>
int launch_sample(const SampleArgs& a, int64_t n, bool vec, cudaStream_t s) {
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    if (n4 > 0) {
      sample_vec4_kernel<METHOD, PHILOX, ISO, PDF><<<grid_for(n4, kBlock, 8, 32), kBlock, 0, s>>>(a, n4);
      done = 4 * n4;
    }
  }
  if (done < n)
    sample_scalar_kernel<METHOD, PHILOX, ISO, PDF>
        <<<grid_for(n - done, kBlock, 8, 32), kBlock, 0, s>>>(a, done, n);
  return launch_status();
}

template <int METHOD, bool PHILOX, bool ISO>
int dispatch_pdf(const SampleArgs& a, int64_t n, bool vec, cudaStream_t s) {
  return a.pdf ? launch_sample<METHOD, PHILOX, ISO, true>(a, n, vec, s)
               : launch_sample<METHOD, PHILOX, ISO, false>(a, n, vec, s);
}

template <int METHOD, bool PHILOX>
int dispatch_iso(const SampleArgs& a, int64_t n, bool vec, cudaStream_t s) {
  return a.ay ? dispatch_pdf<METHOD, PHILOX, false>(a, n, vec, s)
              : dispatch_pdf<METHOD, PHILOX, true>(a, n, vec, s);
}

template <int METHOD>
int dispatch_rng(const SampleArgs& a, int64_t n, bool vec, cudaStream_t s) {
  return a.u1 ? dispatch_iso<METHOD, false>(a, n, vec, s) : dispatch_iso<METHOD, true>(a, n, vec, s);
}

// ---------------------------------------------------------------- uniforms
__global__ void __launch_bounds__(kBlock) rng_vec4_kernel(Rng r, float* u1, float* u2, int64_t n4) {
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t q = int64_t(blockIdx.x) * kBlock + threadIdx.x; q < n4; q += stride) {
    float U1[4], U2[4];
    uniforms4(r, uint64_t(4 * q), U1, U2);
    st_stream(u1 + 4 * q, *reinterpret_cast<float4*>(U1));
    st_stream(u2 + 4 * q, *reinterpret_cast<float4*>(U2));
  }
}

__global__ void __launch_bounds__(kBlock) rng_scalar_kernel(Rng r, float* u1, float* u2, int64_t begin,
                                                            int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kBlock + threadIdx.x; e < n; e += stride) {
    float a, b;
    uniforms1(r, uint64_t(e), a, b);
    u1[e] = a;
    u2[e] = b;
  }
}

// ---------------------------------------------------------------- pdf
template <bool ISO>
__global__ void __launch_bounds__(kBlock) pdf_vec4_kernel(const float* wx, const float* wy, const float* wz,
                                                          const float* ax, const float* ay, const float* mx,
                                                          const float* my, const float* mz, float* pdf,
                                                          int64_t n4) {
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t q = int64_t(blockIdx.x) * kBlock + threadIdx.x; q < n4; q += stride) {
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], MX[4], MY[4], MZ[4], P[4];
    *reinterpret_cast<float4*>(X) = ld_stream(wx + e);
    *reinterpret_cast<float4*>(Y) = ld_stream(wy + e);
    *reinterpret_cast<float4*>(Z) = ld_stream(wz + e);
    *reinterpret_cast<float4*>(AX) = ld_stream(ax + e);
    if constexpr (ISO) {
      *reinterpret_cast<float4*>(AY) = *reinterpret_cast<float4*>(AX);
    } else {
      *reinterpret_cast<float4*>(AY) = ld_stream(ay + e);
    }
    *reinterpret_cast<float4*>(MX) = ld_stream(mx + e);
    *reinterpret_cast<float4*>(MY) = ld_stream(my + e);
    *reinterpret_cast<float4*>(MZ) = ld_stream(mz + e);
#pragma unroll
    for (int k = 0; k < 4; ++k) P[k] = pdf_of_normal(X[k], Y[k], Z[k], AX[k], AY[k], MX[k], MY[k], MZ[k]);
    st_stream(pdf + e, *reinterpret_cast<float4*>(P));
  }
}

template <bool ISO>
__global__ void __launch_bounds__(kBlock) pdf_scalar_kernel(const float* wx, const float* wy, const float* wz,
                                                            const float* ax, const float* ay, const float* mx,
                                                            const float* my, const float* mz, float* pdf,
                                                            int64_t begin, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kBlock + threadIdx.x; e < n; e += stride) {
    const float a = ax[e];
    pdf[e] = pdf_of_normal(wx[e], wy[e], wz[e], a, ISO ? a : ay[e], mx[e], my[e], mz[e]);
  }
}

template <bool ISO>
int launch_pdf(int64_t n, const float* wx, const float* wy, const float* wz, const float* ax, const float* ay,
               const float* mx, const float* my, const float* mz, float* pdf, bool vec, cudaStream_t s) {
  int64_t done = 0;
  if (vec && n / 4 > 0) {
    const int64_t n4 = n / 4;
    pdf_vec4_kernel<ISO><<<grid_for(n4, kBlock, 8, 32), kBlock, 0, s>>>(wx, wy, wz, ax, ay, mx, my, mz, pdf, n4);
    done = 4 * n4;
  }
  if (done < n)
    pdf_scalar_kernel<ISO><<<grid_for(n - done, kBlock, 8, 32), kBlock, 0, s>>>(wx, wy, wz, ax, ay, mx, my, mz,
                                                                                  pdf, done, n);
  return launch_status();
}

}  // namespace vndf

using namespace vndf;

extern "C" int vndf_rng_uniform(int64_t n, uint64_t seed, uint64_t counter_base, uint32_t stream_id, float* u1,
                                float* u2, void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (n == 0) return VNDF_OK;
  if (!u1 || !u2) return VNDF_ERR_NULL;
  if (!all_aligned4(u1, u2)) return VNDF_ERR_ALIGN;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const Rng r = make_rng(seed, counter_base, stream_id);
  int64_t done = 0;
  if (all_aligned16(u1, u2) && n / 4 > 0) {
    const int64_t n4 = n / 4;
    rng_vec4_kernel<<<grid_for(n4, kBlock, 8, 32), kBlock, 0, s>>>(r, u1, u2, n4);
    done = 4 * n4;
  }
  if (done < n) rng_scalar_kernel<<<grid_for(n - done, kBlock, 8, 32), kBlock, 0, s>>>(r, u1, u2, done, n);
  return launch_status();
}

extern "C" int vndf_sample(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                           const float* alpha_x, const float* alpha_y, const float* u1, const float* u2,
                           uint64_t seed, uint64_t counter_base, uint32_t stream_id, int method, float* wm_x,
                           float* wm_y, float* wm_z, float* pdf, void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (method != VNDF_METHOD_SPHERICAL_CAP && method != VNDF_METHOD_POLAR_DISK) return VNDF_ERR_METHOD;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !wm_x || !wm_y || !wm_z) return VNDF_ERR_NULL;
  if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf)) return VNDF_ERR_ALIGN;
  SampleArgs a{wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf,
               make_rng(seed, counter_base, stream_id)};
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return method == VNDF_METHOD_SPHERICAL_CAP ? dispatch_rng<kMethodCap>(a, n, vec, s)
                                             : dispatch_rng<kMethodPolar>(a, n, vec, s);
}

extern "C" int vndf_pdf(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z, const float* alpha_x,
                        const float* alpha_y, const float* wm_x, const float* wm_y, const float* wm_z, float* pdf,
                        void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !wm_x || !wm_y || !wm_z || !pdf) return VNDF_ERR_NULL;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf)) return VNDF_ERR_ALIGN;
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return alpha_y ? launch_pdf<false>(n, wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf, vec, s)
                 : launch_pdf<true>(n, wi_x, wi_y, wi_z, alpha_x, alpha_x, wm_x, wm_y, wm_z, pdf, vec, s);
}
