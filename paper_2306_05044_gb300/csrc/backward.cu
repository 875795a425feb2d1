// Adjoint kernels of the spherical-cap sampler (reparameterised gradients):
//   vndf_sample_backward        generic vector-Jacobian product of (wm, pdf)
//   vndf_sample_loss_backward   fused forward + loss + adjoint for
//                               loss = sum_i (c_i . wm_i + log pdf_i)
// Both recompute the forward in registers (no stored tape) and share the
// per-sample adjoint in vndf_adjoint.cuh.  The fused kernel reduces the loss
// per fixed 128-sample group (one warp, four samples per lane, shuffle tree;
// no block barrier), and a one-block kernel sums the group partials in index
// order, so the loss is bit-reproducible and independent of the grid.
#include <cuda_runtime.h>

#include "common.cuh"
#include "philox.cuh"
#include "staging.cuh"
#include "vndf_adjoint.cuh"

// Staged kernels: 1 = full chunks go through backward_pipe_kernel / loss_backward_pipe_kernel; their
// grids (at most this many waves of 8 CTAs per SM, of which 3 are resident) and resident CTAs per SM.
// Measured on GB300 (fused at 2^24 / 2^26 samples, generic at 2^24): 1 wave 141.7 / 539.1 / 146.2 us,
// 4 waves 141.7 / 529.5 / 139.4, 8 waves 147.7 / 525.5 / 137.6, 16 waves 158.0 / 528.0 / 145.6.
#ifndef VNDF_BWD_STAGED
#define VNDF_BWD_STAGED 1
#endif
#ifndef VNDF_BWD_WAVES
#define VNDF_BWD_WAVES 8
#endif
#ifndef VNDF_LOSS_WAVES
#define VNDF_LOSS_WAVES 4
#endif
#ifndef VNDF_BWD_MIN_BLOCKS
#define VNDF_BWD_MIN_BLOCKS 3
#endif
// 1 = the loss's partial-sum kernel is a programmatic dependent launch of the loss kernel before it:
// it is launched while that kernel runs and waits (in hardware) for its completion before reading.
#ifndef VNDF_LOSS_PDL
#define VNDF_LOSS_PDL 1
#endif

namespace vndf {

constexpr int kBwdBlock = 256;
constexpr int kChunk = 4 * kBwdBlock;  // samples per block iteration
constexpr int kGroup = 128;            // samples per loss partial (one warp)

struct BwdArgs {
  const float *wx, *wy, *wz, *ax, *ay, *u1, *u2;
  const float *gmx, *gmy, *gmz, *gp;  // adjoints (generic) or c (fused: gmx..gmz)
  float *gwx, *gwy, *gwz, *gax, *gay;
  Rng rng;
};

__device__ __forceinline__ void load4(const float* p, int64_t e, float (&d)[4]) {
  *reinterpret_cast<float4*>(d) = ld_stream(p + e);
}
__device__ __forceinline__ void store4(float* p, int64_t e, const float (&d)[4]) {
  st_stream(p + e, *reinterpret_cast<const float4*>(d));
}

template <bool PHILOX, bool ISO, bool EXT>
__global__ void __launch_bounds__(kBwdBlock, 3) backward_vec4_kernel(BwdArgs a, int64_t n4) {
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kBwdBlock;
  for (int64_t q = int64_t(blockIdx.x) * kBwdBlock + threadIdx.x; q < n4; q += stride) {
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4];
    float GX[4] = {0.f, 0.f, 0.f, 0.f}, GY[4] = {0.f, 0.f, 0.f, 0.f}, GZ[4] = {0.f, 0.f, 0.f, 0.f};
    float GP[4] = {0.f, 0.f, 0.f, 0.f};
    load4(a.wx, e, X);
    load4(a.wy, e, Y);
    load4(a.wz, e, Z);
    load4(a.ax, e, AX);
    if constexpr (ISO) {
#pragma unroll
      for (int k = 0; k < 4; ++k) AY[k] = AX[k];
    } else {
      load4(a.ay, e, AY);
    }
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      load4(a.u1, e, U1);
      load4(a.u2, e, U2);
    }
    if (a.gmx) {
      load4(a.gmx, e, GX);
      load4(a.gmy, e, GY);
      load4(a.gmz, e, GZ);
    }
    if (a.gp) load4(a.gp, e, GP);
    float OWX[4], OWY[4], OWZ[4], OAX[4], OAY[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float mx, my, mz, pdf;
      const Grad5 g = cap_backward_one<true, EXT>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k], GX[k], GY[k],
                                                  GZ[k], GP[k], 0.f, mx, my, mz, pdf);
      OWX[k] = g.wx;
      OWY[k] = g.wy;
      OWZ[k] = g.wz;
      OAX[k] = ISO ? g.ax + g.ay : g.ax;
      OAY[k] = g.ay;
    }
    if (a.gwx) {
      store4(a.gwx, e, OWX);
      store4(a.gwy, e, OWY);
      store4(a.gwz, e, OWZ);
    }
    if (a.gax) store4(a.gax, e, OAX);
    if (!ISO && a.gay) store4(a.gay, e, OAY);
  }
}

template <bool PHILOX, bool ISO, bool EXT>
__global__ void __launch_bounds__(kBwdBlock) backward_scalar_kernel(BwdArgs a, int64_t begin, int64_t n) {
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kBwdBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kBwdBlock + threadIdx.x; e < n; e += stride) {
    const float ax = a.ax[e];
    const float ay = ISO ? ax : a.ay[e];
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(e), u1, u2);
    } else {
      u1 = a.u1[e];
      u2 = a.u2[e];
    }
    const float gx = a.gmx ? a.gmx[e] : 0.f, gy = a.gmx ? a.gmy[e] : 0.f, gz = a.gmx ? a.gmz[e] : 0.f;
    float mx, my, mz, pdf;
    const Grad5 g = cap_backward_one<true, EXT>(a.wx[e], a.wy[e], a.wz[e], ax, ay, u1, u2, gx, gy, gz,
                                     a.gp ? a.gp[e] : 0.f, 0.f, mx, my, mz, pdf);
    if (a.gwx) {
      a.gwx[e] = g.wx;
      a.gwy[e] = g.wy;
      a.gwz[e] = g.wz;
    }
    if (a.gax) a.gax[e] = ISO ? vadd(g.ax, g.ay) : g.ax;
    if (!ISO && a.gay) a.gay[e] = g.ay;
  }
}

// The generic adjoint over full 4-sample groups with 16-byte aligned streams: each
// thread's next group is staged in shared memory with cp.async while the current
// one is computed (per-thread copies, no barrier).  The optional adjoint inputs
// g_wm and g_pdf are staged only when given (warp-uniform flags); slot k of the
// layout is stream k in the order wi xyz, alpha_x, [alpha_y], [u1, u2], [g_wm xyz],
// [g_pdf].  Same per-sample function, so the same bits as backward_vec4_kernel.
template <bool PHILOX, bool ISO>
__host__ __device__ constexpr int bwd_fixed_streams() { return 4 + (ISO ? 0 : 1) + (PHILOX ? 0 : 2); }

template <bool PHILOX, bool ISO>
__device__ __forceinline__ void bwd_stage(const BwdArgs& a, int64_t e, float4* slot, bool has_g, bool has_p) {
  int k = 0;
  cp_async16(slot + (k++) * kBwdBlock, a.wx + e);
  cp_async16(slot + (k++) * kBwdBlock, a.wy + e);
  cp_async16(slot + (k++) * kBwdBlock, a.wz + e);
  cp_async16(slot + (k++) * kBwdBlock, a.ax + e);
  if constexpr (!ISO) cp_async16(slot + (k++) * kBwdBlock, a.ay + e);
  if constexpr (!PHILOX) {
    cp_async16(slot + (k++) * kBwdBlock, a.u1 + e);
    cp_async16(slot + (k++) * kBwdBlock, a.u2 + e);
  }
  if (has_g) {
    cp_async16(slot + (k++) * kBwdBlock, a.gmx + e);
    cp_async16(slot + (k++) * kBwdBlock, a.gmy + e);
    cp_async16(slot + (k++) * kBwdBlock, a.gmz + e);
  }
  if (has_p) cp_async16(slot + k * kBwdBlock, a.gp + e);
}

template <bool PHILOX, bool ISO, bool EXT>
__global__ void __launch_bounds__(kBwdBlock, VNDF_BWD_MIN_BLOCKS) backward_pipe_kernel(BwdArgs a, int64_t n4) {
  pdl_trigger();
  pdl_wait();
  constexpr int kFixed = bwd_fixed_streams<PHILOX, ISO>();
  const bool has_g = a.gmx != nullptr, has_p = a.gp != nullptr;
  const int ns = kFixed + (has_g ? 3 : 0) + (has_p ? 1 : 0);
  extern __shared__ float4 smem_b[];  // [2][ns][kBwdBlock]
  const int64_t stride = int64_t(gridDim.x) * kBwdBlock;
  const int64_t q0 = int64_t(blockIdx.x) * kBwdBlock + threadIdx.x;
  float4* mine = smem_b + threadIdx.x;
  if (q0 < n4) bwd_stage<PHILOX, ISO>(a, 4 * q0, mine, has_g, has_p);
  cp_async_commit();
  int slot = 0;
  for (int64_t q = q0; q < n4; q += stride) {
    if (q + stride < n4) bwd_stage<PHILOX, ISO>(a, 4 * (q + stride), mine + (slot ^ 1) * ns * kBwdBlock, has_g, has_p);
    cp_async_commit();
    cp_async_wait<1>();
    const float4* cur = mine + slot * ns * kBwdBlock;
    slot ^= 1;
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4];
    float GX[4] = {0.f, 0.f, 0.f, 0.f}, GY[4] = {0.f, 0.f, 0.f, 0.f}, GZ[4] = {0.f, 0.f, 0.f, 0.f};
    float GP[4] = {0.f, 0.f, 0.f, 0.f};
    int k = 0;
    *reinterpret_cast<float4*>(X) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(Y) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(Z) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(AX) = cur[(k++) * kBwdBlock];
    if constexpr (ISO) {
      *reinterpret_cast<float4*>(AY) = *reinterpret_cast<float4*>(AX);
    } else {
      *reinterpret_cast<float4*>(AY) = cur[(k++) * kBwdBlock];
    }
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = cur[(k++) * kBwdBlock];
      *reinterpret_cast<float4*>(U2) = cur[(k++) * kBwdBlock];
    }
    if (has_g) {
      *reinterpret_cast<float4*>(GX) = cur[(k++) * kBwdBlock];
      *reinterpret_cast<float4*>(GY) = cur[(k++) * kBwdBlock];
      *reinterpret_cast<float4*>(GZ) = cur[(k++) * kBwdBlock];
    }
    if (has_p) *reinterpret_cast<float4*>(GP) = cur[k * kBwdBlock];
    float OWX[4], OWY[4], OWZ[4], OAX[4], OAY[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float mx, my, mz, pdf;
      const Grad5 g = cap_backward_one<true, EXT>(X[j], Y[j], Z[j], AX[j], AY[j], U1[j], U2[j], GX[j], GY[j],
                                                  GZ[j], GP[j], 0.f, mx, my, mz, pdf);
      OWX[j] = g.wx;
      OWY[j] = g.wy;
      OWZ[j] = g.wz;
      OAX[j] = ISO ? g.ax + g.ay : g.ax;
      OAY[j] = g.ay;
    }
    if (a.gwx) {
      store4(a.gwx, e, OWX);
      store4(a.gwy, e, OWY);
      store4(a.gwz, e, OWZ);
    }
    if (a.gax) store4(a.gax, e, OAX);
    if (!ISO && a.gay) store4(a.gay, e, OAY);
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- fused loss + adjoint
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order (warp butterflies, then warp 0 over the warp sums).
template <int BLOCK>
__device__ __forceinline__ float block_sum(float v, float* smem) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) smem[w] = v;
  __syncthreads();
  float r = 0.f;
  if (w == 0) {
    r = l < BLOCK / 32 ? smem[l] : 0.f;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

template <bool PHILOX, bool ISO, bool VEC>
__global__ void __launch_bounds__(kBwdBlock, 3) loss_backward_kernel(BwdArgs a, int64_t n, int64_t ch0,
                                                                  int64_t chunks, float* partials,
                                                                  unsigned* sum_counter) {
  pdl_wait();
  if (sum_counter && blockIdx.x == 0 && threadIdx.x == 0) *sum_counter = 0u;  // read by sum_partials_kernel
#if VNDF_LOSS_PDL
  asm volatile("griddepcontrol.launch_dependents;");  // the sum kernel may be scheduled; it waits for us
#endif
  for (int64_t ch = ch0 + blockIdx.x; ch < chunks; ch += gridDim.x) {
    const int64_t e = ch * kChunk + 4 * int64_t(threadIdx.x);
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4], CX[4], CY[4], CZ[4];
    const bool full = VEC && e + 3 < n;
    if (full) {
      load4(a.wx, e, X);
      load4(a.wy, e, Y);
      load4(a.wz, e, Z);
      load4(a.ax, e, AX);
      if constexpr (ISO) {
#pragma unroll
        for (int k = 0; k < 4; ++k) AY[k] = AX[k];
      } else {
        load4(a.ay, e, AY);
      }
      load4(a.gmx, e, CX);
      load4(a.gmy, e, CY);
      load4(a.gmz, e, CZ);
      if constexpr (!PHILOX) {
        load4(a.u1, e, U1);
        load4(a.u2, e, U2);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool in = e + k < n;
        X[k] = in ? a.wx[e + k] : 0.f;
        Y[k] = in ? a.wy[e + k] : 0.f;
        Z[k] = in ? a.wz[e + k] : 0.f;  // wz = 0: out of domain, contributes nothing
        AX[k] = in ? a.ax[e + k] : 1.f;
        AY[k] = ISO ? AX[k] : (in ? a.ay[e + k] : 1.f);
        CX[k] = in ? a.gmx[e + k] : 0.f;
        CY[k] = in ? a.gmy[e + k] : 0.f;
        CZ[k] = in ? a.gmz[e + k] : 0.f;
        if constexpr (!PHILOX) {
          U1[k] = in ? a.u1[e + k] : 0.f;
          U2[k] = in ? a.u2[e + k] : 0.f;
        }
      }
    }
    if constexpr (PHILOX) {
      if (full) {
        uniforms4(a.rng, uint64_t(e), U1, U2);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) uniforms1(a.rng, uint64_t(e + k), U1[k], U2[k]);
      }
    }
    float OWX[4], OWY[4], OWZ[4], OAX[4], OAY[4];
    float local = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float mx, my, mz, pdf;
      const Grad5 g = cap_backward_one(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k], CX[k], CY[k], CZ[k], 0.f,
                                       1.f, mx, my, mz, pdf);
      const bool ok = pdf > 0.f;
      local += ok ? fmaf(CX[k], mx, fmaf(CY[k], my, fmaf(CZ[k], mz, __logf(pdf)))) : 0.f;
      OWX[k] = g.wx;
      OWY[k] = g.wy;
      OWZ[k] = g.wz;
      OAX[k] = ISO ? g.ax + g.ay : g.ax;
      OAY[k] = g.ay;
    }
    if (full) {
      if (a.gwx) {
        store4(a.gwx, e, OWX);
        store4(a.gwy, e, OWY);
        store4(a.gwz, e, OWZ);
      }
      if (a.gax) store4(a.gax, e, OAX);
      if (!ISO && a.gay) store4(a.gay, e, OAY);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (e + k < n) {
          if (a.gwx) {
            a.gwx[e + k] = OWX[k];
            a.gwy[e + k] = OWY[k];
            a.gwz[e + k] = OWZ[k];
          }
          if (a.gax) a.gax[e + k] = OAX[k];
          if (!ISO && a.gay) a.gay[e + k] = OAY[k];
        }
      }
    }
    // one partial per warp (128 samples); groups past n are never read
    const float w = warp_sum(local);
    const int64_t grp = ch * (kChunk / kGroup) + (threadIdx.x >> 5);
    if ((threadIdx.x & 31) == 0 && grp * kGroup < n) partials[grp] = w;
  }
}

template <bool PHILOX, bool ISO>
__host__ __device__ constexpr int loss_streams_in() { return 7 + (ISO ? 0 : 1) + (PHILOX ? 0 : 2); }

// This thread's 16-byte slice of every input stream of chunk ch, copied to shared memory.
template <bool PHILOX, bool ISO>
__device__ __forceinline__ void loss_stage(const BwdArgs& a, int64_t e, float4* slot) {
  int k = 0;
  cp_async16(slot + (k++) * kBwdBlock, a.wx + e);
  cp_async16(slot + (k++) * kBwdBlock, a.wy + e);
  cp_async16(slot + (k++) * kBwdBlock, a.wz + e);
  cp_async16(slot + (k++) * kBwdBlock, a.ax + e);
  if constexpr (!ISO) cp_async16(slot + (k++) * kBwdBlock, a.ay + e);
  cp_async16(slot + (k++) * kBwdBlock, a.gmx + e);
  cp_async16(slot + (k++) * kBwdBlock, a.gmy + e);
  cp_async16(slot + (k++) * kBwdBlock, a.gmz + e);
  if constexpr (!PHILOX) {
    cp_async16(slot + (k++) * kBwdBlock, a.u1 + e);
    cp_async16(slot + (k++) * kBwdBlock, a.u2 + e);
  }
}

// The fused kernel over the full chunks [0, chunks), 16-byte aligned streams: each
// thread's slice of the next chunk is staged in shared memory with cp.async while
// the current one is computed (per-thread copies, no barrier).  Partials are those
// of loss_backward_kernel, so the loss does not depend on which kernel ran.
template <bool PHILOX, bool ISO>
__global__ void __launch_bounds__(kBwdBlock, VNDF_BWD_MIN_BLOCKS) loss_backward_pipe_kernel(BwdArgs a, int64_t chunks,
                                                                       float* partials, unsigned* sum_counter) {
  constexpr int NS = loss_streams_in<PHILOX, ISO>();
  pdl_wait();
  if (blockIdx.x == 0 && threadIdx.x == 0) *sum_counter = 0u;  // read by sum_partials_kernel
  extern __shared__ float4 smem_l[];  // [2][NS][kBwdBlock]
  float4* mine = smem_l + threadIdx.x;
  if (int64_t(blockIdx.x) < chunks)
    loss_stage<PHILOX, ISO>(a, int64_t(blockIdx.x) * kChunk + 4 * threadIdx.x, mine);
  cp_async_commit();
  int slot = 0;
  for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
    const int64_t e = ch * kChunk + 4 * int64_t(threadIdx.x);
#if VNDF_LOSS_PDL
    // the sum kernel may be scheduled once every CTA is in its last chunk (not earlier: its waiting CTAs
    // would hold CTA slots this grid still needs)
    if (ch + gridDim.x >= chunks) asm volatile("griddepcontrol.launch_dependents;");
#endif
    if (ch + gridDim.x < chunks)
      loss_stage<PHILOX, ISO>(a, e + int64_t(gridDim.x) * kChunk, mine + (slot ^ 1) * NS * kBwdBlock);
    cp_async_commit();
    cp_async_wait<1>();
    const float4* cur = mine + slot * NS * kBwdBlock;
    slot ^= 1;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4], CX[4], CY[4], CZ[4];
    int k = 0;
    *reinterpret_cast<float4*>(X) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(Y) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(Z) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(AX) = cur[(k++) * kBwdBlock];
    if constexpr (ISO) {
      *reinterpret_cast<float4*>(AY) = *reinterpret_cast<float4*>(AX);
    } else {
      *reinterpret_cast<float4*>(AY) = cur[(k++) * kBwdBlock];
    }
    *reinterpret_cast<float4*>(CX) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(CY) = cur[(k++) * kBwdBlock];
    *reinterpret_cast<float4*>(CZ) = cur[(k++) * kBwdBlock];
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = cur[(k++) * kBwdBlock];
      *reinterpret_cast<float4*>(U2) = cur[(k++) * kBwdBlock];
    }
    float OWX[4], OWY[4], OWZ[4], OAX[4], OAY[4];
    float local = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float mx, my, mz, pdf;
      const Grad5 g = cap_backward_one(X[j], Y[j], Z[j], AX[j], AY[j], U1[j], U2[j], CX[j], CY[j], CZ[j], 0.f,
                                       1.f, mx, my, mz, pdf);
      const bool ok = pdf > 0.f;
      local += ok ? fmaf(CX[j], mx, fmaf(CY[j], my, fmaf(CZ[j], mz, __logf(pdf)))) : 0.f;
      OWX[j] = g.wx;
      OWY[j] = g.wy;
      OWZ[j] = g.wz;
      OAX[j] = ISO ? g.ax + g.ay : g.ax;
      OAY[j] = g.ay;
    }
    if (a.gwx) {
      store4(a.gwx, e, OWX);
      store4(a.gwy, e, OWY);
      store4(a.gwz, e, OWZ);
    }
    if (a.gax) store4(a.gax, e, OAX);
    if (!ISO && a.gay) store4(a.gay, e, OAY);
    const float w = warp_sum(local);
    if ((threadIdx.x & 31) == 0) partials[ch * (kChunk / kGroup) + (threadIdx.x >> 5)] = w;
  }
  cp_async_wait<0>();
}

// The loss partials are summed in two fixed levels.  Segment b holds partials
// [b * kSegPartials, (b + 1) * kSegPartials); a CTA adds a segment in a fixed order
// (thread t takes t, t + kSumBlock, ... in turn, then a fixed tree) and stores the
// segment sum; the CTA that finishes last (a counter that the loss kernel zeroed
// before any CTA here started) adds the segment sums the same way.  The order
// depends only on n, so the loss is bit-reproducible for a given n, and the work
// is spread over many SMs instead of one.
constexpr int kSegPartials = 2048;
constexpr int kSumBlock = 256;

__host__ __device__ inline int64_t loss_segments(int64_t groups) {
  return (groups + kSegPartials - 1) / kSegPartials;
}

__global__ void __launch_bounds__(kSumBlock) sum_partials_kernel(const float* partials, int64_t m, float* seg,
                                                                 int64_t nseg, unsigned* counter, float* out) {
  __shared__ float smem[32];
  __shared__ bool last;
  // as a programmatic dependent launch: wait until the loss kernel before it has completed and its
  // writes are visible (returns at once after an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int64_t b = blockIdx.x; b < nseg; b += gridDim.x) {
    const int64_t j0 = b * kSegPartials, j1 = j0 + kSegPartials < m ? j0 + kSegPartials : m;
    float v = 0.f;
#pragma unroll 8
    for (int64_t j = j0 + threadIdx.x; j < j1; j += kSumBlock) v += partials[j];
    const float t = block_sum<kSumBlock>(v, smem);
    if (threadIdx.x == 0) seg[b] = t;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {  // uniform over the block
    __threadfence();
    float w = 0.f;
    for (int64_t k = threadIdx.x; k < nseg; k += kSumBlock) w += __ldcg(seg + k);
    const float t = block_sum<kSumBlock>(w, smem);
    if (threadIdx.x == 0) *out = t;
  }
}

template <bool PHILOX, bool ISO, bool EXT>
int launch_backward(const BwdArgs& a, int64_t n, bool vec, cudaStream_t s) {
  int64_t done = 0;
  if (vec && n / 4 > 0) {
    const int64_t n4 = n / 4;
    if (VNDF_BWD_STAGED && n4 >= int64_t(16) * 3 * sm_count() * kBwdBlock) {
      // staged kernel for large calls (as for the fused loss); the limit is set for the widest layout
      constexpr size_t smem_max = size_t(2) * (bwd_fixed_streams<PHILOX, ISO>() + 4) * kBwdBlock * 16;
      if (!ensure_dynamic_smem<backward_pipe_kernel<PHILOX, ISO, EXT>>(smem_max)) return VNDF_ERR_CUDA;
      const int ns = bwd_fixed_streams<PHILOX, ISO>() + (a.gmx ? 3 : 0) + (a.gp ? 1 : 0);
      if (!launch_pdl(backward_pipe_kernel<PHILOX, ISO, EXT>, grid_for(n4, kBwdBlock, 8, VNDF_BWD_WAVES), kBwdBlock,
                      size_t(2) * ns * kBwdBlock * 16, s, a, n4))
        return VNDF_ERR_CUDA;
    } else if (!launch_pdl(backward_vec4_kernel<PHILOX, ISO, EXT>, grid_for(n4, kBwdBlock, 8, 32), kBwdBlock, 0, s,
                           a, n4)) {
      return VNDF_ERR_CUDA;
    }
    done = 4 * n4;
  }
  if (done < n && !launch_pdl(backward_scalar_kernel<PHILOX, ISO, EXT>, grid_for(n - done, kBwdBlock, 8, 32),
                              kBwdBlock, 0, s, a, done, n))
    return VNDF_ERR_CUDA;
  return launch_status();
}

// Loss workspace: the group partials, then the segment sums, then the counter.
struct LossWorkspace {
  float* partials;
  float* seg;
  unsigned* counter;
};

inline LossWorkspace loss_workspace(void* ws, int64_t n) {
  const int64_t groups = (n + kGroup - 1) / kGroup;
  float* p = static_cast<float*>(ws);
  return LossWorkspace{p, p + groups, reinterpret_cast<unsigned*>(p + groups + loss_segments(groups))};
}

template <bool PHILOX, bool ISO>
int launch_loss(const BwdArgs& a, int64_t n, bool vec, const LossWorkspace& w, float* loss, cudaStream_t s) {
  float* partials = w.partials;
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  const int64_t groups = (n + kGroup - 1) / kGroup;
  // the staged kernel pays off once every resident CTA gets many chunks (measured: slower at 2^22
  // samples, 6 % faster at 2^24); results are the same bits either way
  const int64_t full = n / kChunk;
  if (vec && VNDF_BWD_STAGED && full >= int64_t(16) * 3 * sm_count()) {
    // full chunks through the staged kernel, the ragged last chunk (if any) through the plain one
    {
      constexpr size_t smem = size_t(2) * loss_streams_in<PHILOX, ISO>() * kBwdBlock * 16;
      if (!ensure_dynamic_smem<loss_backward_pipe_kernel<PHILOX, ISO>>(smem)) return VNDF_ERR_CUDA;
      if (!launch_pdl(loss_backward_pipe_kernel<PHILOX, ISO>, grid_for(full * kBwdBlock, kBwdBlock, 8, VNDF_LOSS_WAVES),
                      kBwdBlock, smem, s, a, full, partials, w.counter))
        return VNDF_ERR_CUDA;
    }
    if (full < chunks)
      loss_backward_kernel<PHILOX, ISO, true><<<1, kBwdBlock, 0, s>>>(a, n, full, chunks, partials, nullptr);
  } else {
    const unsigned grid = grid_for(chunks * kBwdBlock, kBwdBlock, 8, 16);
    const bool ok = vec ? launch_pdl(loss_backward_kernel<PHILOX, ISO, true>, grid, kBwdBlock, 0, s, a, n, 0, chunks,
                                     partials, w.counter)
                        : launch_pdl(loss_backward_kernel<PHILOX, ISO, false>, grid, kBwdBlock, 0, s, a, n, 0, chunks,
                                     partials, w.counter);
    if (!ok) return VNDF_ERR_CUDA;
  }
  const int64_t nseg = loss_segments(groups);
  const unsigned sgrid = static_cast<unsigned>(nseg < 65535 ? nseg : 65535);
#if VNDF_LOSS_PDL
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sgrid);
  cfg.blockDim = dim3(kSumBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const float* cpartials = partials;
  if (cudaLaunchKernelEx(&cfg, sum_partials_kernel, cpartials, groups, w.seg, nseg, w.counter, loss) != cudaSuccess)
    return VNDF_ERR_CUDA;
#else
  sum_partials_kernel<<<sgrid, kSumBlock, 0, s>>>(partials, groups, w.seg, nseg, w.counter, loss);
#endif
  return launch_status();
}

}  // namespace vndf

using namespace vndf;

namespace vndf {
template <bool EXT>
int backward_entry(const char* name, int64_t n, const float* wi_x, const float* wi_y, const float* wi_z, const float* alpha_x,
                   const float* alpha_y, const float* u1, const float* u2, uint64_t seed, uint64_t counter_base,
                   uint32_t stream_id, const float* g_wm_x, const float* g_wm_y, const float* g_wm_z,
                   const float* g_pdf, float* g_wi_x, float* g_wi_y, float* g_wi_z, float* g_alpha_x,
                   float* g_alpha_y, void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x) return VNDF_ERR_NULL;
  if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
  const int gwm_count = (g_wm_x != nullptr) + (g_wm_y != nullptr) + (g_wm_z != nullptr);
  const int gwi_count = (g_wi_x != nullptr) + (g_wi_y != nullptr) + (g_wi_z != nullptr);
  if (gwm_count != 0 && gwm_count != 3) return VNDF_ERR_ARG;
  if (gwi_count != 0 && gwi_count != 3) return VNDF_ERR_ARG;
  if (alpha_y == nullptr && g_alpha_y != nullptr) return VNDF_ERR_ARG;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, g_wm_x, g_wm_y, g_wm_z, g_pdf, g_wi_x, g_wi_y,
                    g_wi_z, g_alpha_x, g_alpha_y))
    return VNDF_ERR_ALIGN;
  if (aliased({g_wi_x, g_wi_y, g_wi_z, g_alpha_x, g_alpha_y},
              {wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, g_wm_x, g_wm_y, g_wm_z, g_pdf}))
    return VNDF_ERR_ARG;
  if (const int f = pre_launch(name)) return f;
  BwdArgs a{wi_x,   wi_y,   wi_z,   alpha_x, alpha_y,   u1,        u2,       g_wm_x,
            g_wm_y, g_wm_z, g_pdf,  g_wi_x,  g_wi_y,    g_wi_z,    g_alpha_x, g_alpha_y,
            make_rng(seed, counter_base, stream_id)};
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, g_wm_x, g_wm_y, g_wm_z, g_pdf,
                                 g_wi_x, g_wi_y, g_wi_z, g_alpha_x, g_alpha_y);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (u1)
    return alpha_y ? launch_backward<false, false, EXT>(a, n, vec, s)
                   : launch_backward<false, true, EXT>(a, n, vec, s);
  return alpha_y ? launch_backward<true, false, EXT>(a, n, vec, s) : launch_backward<true, true, EXT>(a, n, vec, s);
}
}  // namespace vndf

extern "C" int vndf_sample_backward(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                    const float* alpha_x, const float* alpha_y, const float* u1, const float* u2,
                                    uint64_t seed, uint64_t counter_base, uint32_t stream_id, const float* g_wm_x,
                                    const float* g_wm_y, const float* g_wm_z, const float* g_pdf, float* g_wi_x,
                                    float* g_wi_y, float* g_wi_z, float* g_alpha_x, float* g_alpha_y,
                                    void* cuda_stream) {
  return backward_entry<false>("vndf_sample_backward", n, wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, seed,
                               counter_base, stream_id, g_wm_x, g_wm_y, g_wm_z, g_pdf, g_wi_x, g_wi_y, g_wi_z,
                               g_alpha_x, g_alpha_y, cuda_stream);
}

extern "C" int vndf_sample_backward_extended(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                             const float* alpha_x, const float* alpha_y, const float* u1,
                                             const float* u2, uint64_t seed, uint64_t counter_base,
                                             uint32_t stream_id, const float* g_wm_x, const float* g_wm_y,
                                             const float* g_wm_z, const float* g_pdf, float* g_wi_x, float* g_wi_y,
                                             float* g_wi_z, float* g_alpha_x, float* g_alpha_y, void* cuda_stream) {
  return backward_entry<true>("vndf_sample_backward_extended", n, wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, seed,
                              counter_base, stream_id, g_wm_x, g_wm_y, g_wm_z, g_pdf, g_wi_x, g_wi_y, g_wi_z,
                              g_alpha_x, g_alpha_y, cuda_stream);
}

extern "C" size_t vndf_loss_workspace_bytes(int64_t n) {
  if (n <= 0) return 0;
  const int64_t groups = (n + kGroup - 1) / kGroup;
  return size_t(groups + loss_segments(groups) + 1) * sizeof(float);
}

extern "C" int vndf_sample_loss_backward(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                         const float* alpha_x, const float* alpha_y, const float* c_x,
                                         const float* c_y, const float* c_z, const float* u1, const float* u2,
                                         uint64_t seed, uint64_t counter_base, uint32_t stream_id, float* g_wi_x,
                                         float* g_wi_y, float* g_wi_z, float* g_alpha_x, float* g_alpha_y,
                                         float* loss, void* workspace, size_t workspace_bytes,
                                         void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (!loss) return VNDF_ERR_NULL;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (n == 0) return cudaMemsetAsync(loss, 0, sizeof(float), s) == cudaSuccess ? VNDF_OK : VNDF_ERR_CUDA;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !c_x || !c_y || !c_z) return VNDF_ERR_NULL;
  if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
  const int gwi_count = (g_wi_x != nullptr) + (g_wi_y != nullptr) + (g_wi_z != nullptr);
  if (gwi_count != 0 && gwi_count != 3) return VNDF_ERR_ARG;
  if (alpha_y == nullptr && g_alpha_y != nullptr) return VNDF_ERR_ARG;
  if (!workspace || workspace_bytes < vndf_loss_workspace_bytes(n)) return VNDF_ERR_WORKSPACE;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, c_x, c_y, c_z, u1, u2, g_wi_x, g_wi_y, g_wi_z,
                    g_alpha_x, g_alpha_y, loss, workspace))
    return VNDF_ERR_ALIGN;
  if (aliased({g_wi_x, g_wi_y, g_wi_z, g_alpha_x, g_alpha_y, loss, workspace},
              {wi_x, wi_y, wi_z, alpha_x, alpha_y, c_x, c_y, c_z, u1, u2}))
    return VNDF_ERR_ARG;
  if (const int f = pre_launch("vndf_sample_loss_backward", true)) return f;
  BwdArgs a{wi_x, wi_y,   wi_z,   alpha_x, alpha_y,   u1,        u2,       c_x,
            c_y,  c_z,    nullptr, g_wi_x, g_wi_y,    g_wi_z,    g_alpha_x, g_alpha_y,
            make_rng(seed, counter_base, stream_id)};
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, c_x, c_y, c_z, u1, u2, g_wi_x, g_wi_y,
                                 g_wi_z, g_alpha_x, g_alpha_y);
  const LossWorkspace w = loss_workspace(workspace, n);
  if (u1)
    return alpha_y ? launch_loss<false, false>(a, n, vec, w, loss, s)
                   : launch_loss<false, true>(a, n, vec, w, loss, s);
  return alpha_y ? launch_loss<true, false>(a, n, vec, w, loss, s)
                 : launch_loss<true, true>(a, n, vec, w, loss, s);
}
