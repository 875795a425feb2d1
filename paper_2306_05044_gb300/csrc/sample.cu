// Streaming kernels of the sampling hot path: vndf_rng_uniform, vndf_sample,
// vndf_pdf.  One thread handles four consecutive samples with 128-bit loads and
// stores of every structure-of-arrays stream (coalesced: a warp moves 512
// contiguous bytes per array); a scalar kernel covers the n % 4 tail and
// unaligned buffers with the same per-sample function, so results do not
// depend on the path taken.
#include <cuda_runtime.h>

#include "common.cuh"
#include "staging.cuh"
#include "philox.cuh"
#include "rescue.cuh"
#include "vndf_math.cuh"

// Launch shape of the streaming sampler (compile-time, so the shape can be
// tuned per build without a runtime switch).
#ifndef VNDF_SAMPLE_BLOCK
#define VNDF_SAMPLE_BLOCK 256
#endif
#ifndef VNDF_SAMPLE_MIN_BLOCKS
#define VNDF_SAMPLE_MIN_BLOCKS 3
#endif
// Grid of the staged streaming kernel: at most this many waves of 8 CTAs per SM (3 are resident), per
// method.  Measured at 2^28 samples on GB300 (launches alone, packed-pair kernels): cap 16 / 20 / 24 / 28 /
// 32 waves 1405 / 1394 / 1389 / 1382 / 1390 us; prior 6 / 8 / 10 / 12 / 16 waves 1425 / 1428 / 1430 / 1432 /
// 1436 us; extended domain 20 / 28 / 32 / 36 / 40 waves 1488 / 1451 / 1465 / 1494 / 1495 us.  Smaller CTA
// shares balance the tail and let each CTA's final recomputation of its ill-conditioned samples overlap
// other CTAs' streaming; the prior sampler recomputes nothing and prefers longer runs.  Calls below about
// 2^27 samples take the small-call grid instead (about four groups per thread).
#ifndef VNDF_SAMPLE_WAVES
#define VNDF_SAMPLE_WAVES 28
#endif
#ifndef VNDF_SAMPLE_WAVES_EXT
#define VNDF_SAMPLE_WAVES_EXT 28
#endif
#ifndef VNDF_SAMPLE_WAVES_POLAR
#define VNDF_SAMPLE_WAVES_POLAR 6
#endif
#ifndef VNDF_SAMPLE_PREFETCH
#define VNDF_SAMPLE_PREFETCH 1
#endif
#ifndef VNDF_SAMPLE_STAGES
#define VNDF_SAMPLE_STAGES 2
#endif
#ifndef VNDF_SAMPLE_MIN_ITERS
#define VNDF_SAMPLE_MIN_ITERS 4
#endif
// 1 = vndf_sample's kernels are programmatic dependent launches (common.cuh: launch_pdl).
#ifndef VNDF_SAMPLE_PDL
#define VNDF_SAMPLE_PDL 1
#endif
// Ill-conditioned samples: 1 = queued per warp and redone 32 at a time
// (rescue.cuh); 0 = each redone in place by its own lane.
#ifndef VNDF_RESCUE_BATCHED
#define VNDF_RESCUE_BATCHED 1
#endif

namespace vndf {

constexpr int kBlock = 256;
constexpr int kSampleBlock = VNDF_SAMPLE_BLOCK;

struct SampleArgs {
  const float *wx, *wy, *wz, *ax, *ay, *u1, *u2;
  float *mx, *my, *mz, *pdf;
  Rng rng;
};

// Inputs of one 4-sample group (128-bit loads of every stream).
struct Group4 {
  float4 x, y, z, ax, ay, u1, u2;
};

template <bool PHILOX, bool ISO>
__device__ __forceinline__ void load_group(const SampleArgs& a, int64_t e, Group4& g) {
  g.x = ld_stream(a.wx + e);
  g.y = ld_stream(a.wy + e);
  g.z = ld_stream(a.wz + e);
  g.ax = ld_stream(a.ax + e);
  if constexpr (!ISO) g.ay = ld_stream(a.ay + e);
  if constexpr (!PHILOX) {
    g.u1 = ld_stream(a.u1 + e);
    g.u2 = ld_stream(a.u2 + e);
  }
}

// Grid-stride loop over 4-sample groups.  The loads of the thread's next group
// are issued before the current group is computed (software pipelining), so a
// warp keeps one group of loads in flight while its arithmetic runs.
template <int METHOD, bool PHILOX, bool ISO, bool PDF>
__global__ void __launch_bounds__(kSampleBlock, VNDF_SAMPLE_MIN_BLOCKS) sample_vec4_kernel(SampleArgs a, int64_t n4) {
  const int64_t stride = int64_t(gridDim.x) * kSampleBlock;
  int64_t q = int64_t(blockIdx.x) * kSampleBlock + threadIdx.x;
  Group4 next;
  if (q < n4) load_group<PHILOX, ISO>(a, 4 * q, next);
  for (; q < n4; q += stride) {
    const Group4 cur = next;
    if (VNDF_SAMPLE_PREFETCH && q + stride < n4) load_group<PHILOX, ISO>(a, 4 * (q + stride), next);
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4];
    *reinterpret_cast<float4*>(X) = cur.x;
    *reinterpret_cast<float4*>(Y) = cur.y;
    *reinterpret_cast<float4*>(Z) = cur.z;
    *reinterpret_cast<float4*>(AX) = cur.ax;
    *reinterpret_cast<float4*>(AY) = ISO ? cur.ax : cur.ay;
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = cur.u1;
      *reinterpret_cast<float4*>(U2) = cur.u2;
    }
    float MX[4], MY[4], MZ[4], P[4];
    unsigned rescue = sample_four<METHOD, PDF>(X, Y, Z, AX, AY, U1, U2, MX, MY, MZ, P);
    if constexpr (is_cap<METHOD>()) {
      if (rescue) {  // rare: ill-conditioned samples redone in double-float
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (rescue & (1u << k)) {
            const float4 r =
                sample_one_precise<PDF, METHOD == kMethodCapExt>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k]);
            MX[k] = r.x;
            MY[k] = r.y;
            MZ[k] = r.z;
            P[k] = r.w;
          }
      }
    }
    st_stream(a.mx + e, *reinterpret_cast<float4*>(MX));
    st_stream(a.my + e, *reinterpret_cast<float4*>(MY));
    st_stream(a.mz + e, *reinterpret_cast<float4*>(MZ));
    if constexpr (PDF) st_stream(a.pdf + e, *reinterpret_cast<float4*>(P));
    if (!VNDF_SAMPLE_PREFETCH && q + stride < n4) load_group<PHILOX, ISO>(a, 4 * (q + stride), next);
  }
}

template <bool PHILOX, bool ISO>
__device__ __forceinline__ void stage_group(const SampleArgs& a, int64_t e, float4* slot) {
  // slot[k * kSampleBlock] is stream k of this thread's group
  cp_async16(slot + 0 * kSampleBlock, a.wx + e);
  cp_async16(slot + 1 * kSampleBlock, a.wy + e);
  cp_async16(slot + 2 * kSampleBlock, a.wz + e);
  cp_async16(slot + 3 * kSampleBlock, a.ax + e);
  int k = 4;
  if constexpr (!ISO) cp_async16(slot + (k++) * kSampleBlock, a.ay + e);
  if constexpr (!PHILOX) {
    cp_async16(slot + (k++) * kSampleBlock, a.u1 + e);
    cp_async16(slot + (k++) * kSampleBlock, a.u2 + e);
  }
}

template <int METHOD, bool PHILOX, bool ISO, bool PDF>
__global__ void __launch_bounds__(kSampleBlock, VNDF_SAMPLE_MIN_BLOCKS) sample_pipe_kernel(SampleArgs a, int64_t n4) {
  pdl_trigger();
  pdl_wait();
  constexpr int S = VNDF_SAMPLE_STAGES;
  constexpr int NS = streams_in<PHILOX, ISO>();
  extern __shared__ float4 smem[];  // [S][NS][kSampleBlock], then one rescue queue per warp
  RescueQueue* const queues = reinterpret_cast<RescueQueue*>(smem + S * NS * kSampleBlock);
  RescueQueue& rq = queues[threadIdx.x >> 5];
  int pending = 0;  // warp-uniform
  const int64_t stride = int64_t(gridDim.x) * kSampleBlock;
  const int64_t q0 = int64_t(blockIdx.x) * kSampleBlock + threadIdx.x;
  const int64_t w0 = q0 - (threadIdx.x & 31);  // first group of this warp: the loop runs warp-uniformly
  float4* mine = smem + threadIdx.x;
#pragma unroll
  for (int st = 0; st < S - 1; ++st) {
    const int64_t q = q0 + st * stride;
    if (q < n4) stage_group<PHILOX, ISO>(a, 4 * q, mine + st * NS * kSampleBlock);
    cp_async_commit();  // one group per stage, possibly empty, keeps the count uniform
  }
  auto redo = [&](int64_t i) {  // sample i recomputed from its inputs in global memory
    const float ax = a.ax[i], ay = ISO ? ax : a.ay[i];
    float u1, u2;
    if constexpr (PHILOX) {
      uniforms1(a.rng, uint64_t(i), u1, u2);
    } else {
      u1 = a.u1[i];
      u2 = a.u2[i];
    }
    const float4 r = sample_one_precise<PDF, METHOD == kMethodCapExt>(a.wx[i], a.wy[i], a.wz[i], ax, ay, u1, u2);
    a.mx[i] = r.x;
    a.my[i] = r.y;
    a.mz[i] = r.z;
    if constexpr (PDF) a.pdf[i] = r.w;
  };
  constexpr bool kBatched = is_cap<METHOD>() && VNDF_RESCUE_BATCHED;
  int slot = 0;
  // batched: the loop runs warp-uniformly (ballots need every lane); otherwise per thread
  for (int64_t q = q0, qw = w0; kBatched ? qw < n4 : q < n4; q += stride, qw += stride) {
    const bool active = !kBatched || q < n4;  // false only for the tail lanes of the last step
    const int64_t qn = q + (S - 1) * stride;
    if (qn < n4) stage_group<PHILOX, ISO>(a, 4 * qn, mine + ((slot + S - 1) % S) * NS * kSampleBlock);
    cp_async_commit();
    cp_async_wait<S - 1>();  // this thread's copies for q have landed
    const float4* cur = mine + slot * NS * kSampleBlock;
    const int64_t e = 4 * q;
    float X[4], Y[4], Z[4], AX[4], AY[4], U1[4], U2[4];
    *reinterpret_cast<float4*>(X) = cur[0 * kSampleBlock];
    *reinterpret_cast<float4*>(Y) = cur[1 * kSampleBlock];
    *reinterpret_cast<float4*>(Z) = cur[2 * kSampleBlock];
    *reinterpret_cast<float4*>(AX) = cur[3 * kSampleBlock];
    *reinterpret_cast<float4*>(AY) = ISO ? cur[3 * kSampleBlock] : cur[4 * kSampleBlock];
    if constexpr (PHILOX) {
      uniforms4(a.rng, uint64_t(e), U1, U2);
    } else {
      *reinterpret_cast<float4*>(U1) = cur[(ISO ? 4 : 5) * kSampleBlock];
      *reinterpret_cast<float4*>(U2) = cur[(ISO ? 5 : 6) * kSampleBlock];
    }
    slot = (slot + 1) % S;
    float MX[4], MY[4], MZ[4], P[4];
    unsigned rescue = sample_four<METHOD, PDF>(X, Y, Z, AX, AY, U1, U2, MX, MY, MZ, P);
    if constexpr (is_cap<METHOD>() && !kBatched) {
      if (rescue) {  // rare: ill-conditioned samples redone in double-float, in place
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (rescue & (1u << k)) {
            const float4 r =
                sample_one_precise<PDF, METHOD == kMethodCapExt>(X[k], Y[k], Z[k], AX[k], AY[k], U1[k], U2[k]);
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
    }
    if constexpr (kBatched) {
      // rare: ill-conditioned samples are queued and redone in double-float, 32 at a time
      if (!active) rescue = 0;
      if (__any_sync(0xffffffffu, rescue != 0)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) rescue_push(rq, pending, (rescue >> k) & 1u, e + k);
        rescue_drain(rq, pending, false, redo);
      }
    }
  }
  if constexpr (kBatched) rescue_drain_cta(queues, pending, redo);
  cp_async_wait<0>();
}

template <int METHOD, bool PHILOX, bool ISO, bool PDF>
__global__ void __launch_bounds__(kBlock) sample_scalar_kernel(SampleArgs a, int64_t begin, int64_t n) {
  pdl_trigger();
  pdl_wait();
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
    const float wx = a.wx[e], wy = a.wy[e], wz = a.wz[e];
    if (sample_one<METHOD, PDF, true>(wx, wy, wz, ax, ay, u1, u2, mx, my, mz, p)) {
      const float4 r = sample_one_precise<PDF, METHOD == kMethodCapExt>(wx, wy, wz, ax, ay, u1, u2);
      mx = r.x;
      my = r.y;
      mz = r.z;
      p = r.w;
    }
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
      // small calls: about VNDF_SAMPLE_MIN_ITERS groups per thread (so the staging overlaps; one fewer
      // up to 2^21 samples, where the grid then fills all three CTA slots of every SM), in whole
      // multiples of the SM count so that every SM runs the same number of CTAs.  Measured in a CUDA
      // graph at 2^20 samples: 456 CTAs 6.86 us, 304 CTAs 7.10, 256 CTAs 7.8; at 2^22 (eager) three
      // groups per thread took 30.45 us against 30.22 with four, at 2^24 103.4 against 100.5.
      unsigned grid = grid_for(n4, kSampleBlock, 2048 / kSampleBlock,
                               METHOD == kMethodCapExt  ? VNDF_SAMPLE_WAVES_EXT
                               : METHOD == kMethodPolar ? VNDF_SAMPLE_WAVES_POLAR
                                                        : VNDF_SAMPLE_WAVES);
      const int64_t iters = VNDF_SAMPLE_MIN_ITERS - (n4 <= (int64_t(1) << 19) ? 1 : 0);
      if (iters > 1) {
        const int64_t per_iters = (n4 + int64_t(kSampleBlock) * iters - 1) / (int64_t(kSampleBlock) * iters);
        const int64_t sms = sm_count();
        const int64_t g = (per_iters + sms - 1) / sms * sms;
        if (g < int64_t(grid)) grid = unsigned(g);
      }
      if constexpr (VNDF_SAMPLE_STAGES >= 2) {
        constexpr size_t smem = size_t(VNDF_SAMPLE_STAGES) * streams_in<PHILOX, ISO>() * kSampleBlock * 16 +
                                (kSampleBlock / 32) * sizeof(RescueQueue);
        if (!ensure_dynamic_smem<sample_pipe_kernel<METHOD, PHILOX, ISO, PDF>>(smem)) return VNDF_ERR_CUDA;
        if (VNDF_SAMPLE_PDL) {
          if (!launch_pdl(sample_pipe_kernel<METHOD, PHILOX, ISO, PDF>, grid, kSampleBlock, smem, s, a, n4))
            return VNDF_ERR_CUDA;
        } else {
          sample_pipe_kernel<METHOD, PHILOX, ISO, PDF><<<grid, kSampleBlock, smem, s>>>(a, n4);
        }
      } else {
        sample_vec4_kernel<METHOD, PHILOX, ISO, PDF><<<grid, kSampleBlock, 0, s>>>(a, n4);
      }
      done = 4 * n4;
    }
  }
  if (done < n) {
    const unsigned grid = grid_for(n - done, kBlock, 8, 32);
    if (VNDF_SAMPLE_PDL) {
      if (!launch_pdl(sample_scalar_kernel<METHOD, PHILOX, ISO, PDF>, grid, kBlock, 0, s, a, done, n))
        return VNDF_ERR_CUDA;
    } else {
      sample_scalar_kernel<METHOD, PHILOX, ISO, PDF><<<grid, kBlock, 0, s>>>(a, done, n);
    }
  }
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

// ---------------------------------------------------------------- recomputation count
// How many samples vndf_sample recomputes in double-float for these inputs: the same per-sample
// function and condition test, the results discarded, the flags counted (ballot per warp, one atomic).
template <int METHOD, bool PHILOX, bool ISO>
__global__ void __launch_bounds__(kBlock) rescue_count_kernel(SampleArgs a, int64_t n, unsigned long long* count) {
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  unsigned long long mine = 0;
  for (int64_t e = int64_t(blockIdx.x) * kBlock + threadIdx.x; e < n; e += stride) {
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
    mine += sample_one<METHOD, false, true>(a.wx[e], a.wy[e], a.wz[e], ax, ay, u1, u2, mx, my, mz, p) ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

template <int METHOD>
int launch_rescue_count(const SampleArgs& a, int64_t n, unsigned long long* count, cudaStream_t s) {
  const unsigned grid = grid_for(n, kBlock, 8, 8);
  if (a.u1) {
    return (a.ay ? launch_pdl(rescue_count_kernel<METHOD, false, false>, grid, kBlock, 0, s, a, n, count)
                 : launch_pdl(rescue_count_kernel<METHOD, false, true>, grid, kBlock, 0, s, a, n, count))
               ? launch_status()
               : VNDF_ERR_CUDA;
  }
  return (a.ay ? launch_pdl(rescue_count_kernel<METHOD, true, false>, grid, kBlock, 0, s, a, n, count)
               : launch_pdl(rescue_count_kernel<METHOD, true, true>, grid, kBlock, 0, s, a, n, count))
             ? launch_status()
             : VNDF_ERR_CUDA;
}

// ---------------------------------------------------------------- uniforms
__global__ void __launch_bounds__(kBlock) rng_vec4_kernel(Rng r, float* u1, float* u2, int64_t n4) {
  pdl_trigger();
  pdl_wait();
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
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kBlock + threadIdx.x; e < n; e += stride) {
    float a, b;
    uniforms1(r, uint64_t(e), a, b);
    u1[e] = a;
    u2[e] = b;
  }
}

// ---------------------------------------------------------------- pdf
template <bool ISO, bool EXT>
__global__ void __launch_bounds__(kBlock) pdf_vec4_kernel(const float* wx, const float* wy, const float* wz,
                                                          const float* ax, const float* ay, const float* mx,
                                                          const float* my, const float* mz, float* pdf,
                                                          int64_t n4) {
  pdl_trigger();
  pdl_wait();
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
    for (int k = 0; k < 4; ++k) P[k] = pdf_of_normal<EXT>(X[k], Y[k], Z[k], AX[k], AY[k], MX[k], MY[k], MZ[k]);
    st_stream(pdf + e, *reinterpret_cast<float4*>(P));
  }
}

template <bool ISO, bool EXT>
__global__ void __launch_bounds__(kBlock) pdf_scalar_kernel(const float* wx, const float* wy, const float* wz,
                                                            const float* ax, const float* ay, const float* mx,
                                                            const float* my, const float* mz, float* pdf,
                                                            int64_t begin, int64_t n) {
  pdl_trigger();
  pdl_wait();
  const int64_t stride = int64_t(gridDim.x) * kBlock;
  for (int64_t e = begin + int64_t(blockIdx.x) * kBlock + threadIdx.x; e < n; e += stride) {
    const float a = ax[e];
    pdf[e] = pdf_of_normal<EXT>(wx[e], wy[e], wz[e], a, ISO ? a : ay[e], mx[e], my[e], mz[e]);
  }
}

template <bool ISO, bool EXT>
int launch_pdf(int64_t n, const float* wx, const float* wy, const float* wz, const float* ax, const float* ay,
               const float* mx, const float* my, const float* mz, float* pdf, bool vec, cudaStream_t s) {
  int64_t done = 0;
  if (vec && n / 4 > 0) {
    const int64_t n4 = n / 4;
    if (!launch_pdl(pdf_vec4_kernel<ISO, EXT>, grid_for(n4, kBlock, 8, 32), kBlock, 0, s, wx, wy, wz, ax, ay, mx, my,
                    mz, pdf, n4))
      return VNDF_ERR_CUDA;
    done = 4 * n4;
  }
  if (done < n && !launch_pdl(pdf_scalar_kernel<ISO, EXT>, grid_for(n - done, kBlock, 8, 32), kBlock, 0, s, wx, wy,
                              wz, ax, ay, mx, my, mz, pdf, done, n))
    return VNDF_ERR_CUDA;
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
  if (aliased({u1, u2}, {})) return VNDF_ERR_ARG;
  if (const int f = pre_launch("vndf_rng_uniform")) return f;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const Rng r = make_rng(seed, counter_base, stream_id);
  int64_t done = 0;
  if (all_aligned16(u1, u2) && n / 4 > 0) {
    const int64_t n4 = n / 4;
    if (!launch_pdl(rng_vec4_kernel, grid_for(n4, kBlock, 8, 32), kBlock, 0, s, r, u1, u2, n4)) return VNDF_ERR_CUDA;
    done = 4 * n4;
  }
  if (done < n && !launch_pdl(rng_scalar_kernel, grid_for(n - done, kBlock, 8, 32), kBlock, 0, s, r, u1, u2, done, n))
    return VNDF_ERR_CUDA;
  return launch_status();
}

extern "C" int vndf_sample(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                           const float* alpha_x, const float* alpha_y, const float* u1, const float* u2,
                           uint64_t seed, uint64_t counter_base, uint32_t stream_id, int method, float* wm_x,
                           float* wm_y, float* wm_z, float* pdf, void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (method != VNDF_METHOD_SPHERICAL_CAP && method != VNDF_METHOD_POLAR_DISK &&
      method != VNDF_METHOD_SPHERICAL_CAP_EXTENDED)
    return VNDF_ERR_METHOD;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !wm_x || !wm_y || !wm_z) return VNDF_ERR_NULL;
  if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf)) return VNDF_ERR_ALIGN;
  if (aliased({wm_x, wm_y, wm_z, pdf}, {wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2})) return VNDF_ERR_ARG;
  if (const int f = pre_launch("vndf_sample")) return f;
  SampleArgs a{wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf,
               make_rng(seed, counter_base, stream_id)};
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, wm_x, wm_y, wm_z, pdf);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (method == VNDF_METHOD_SPHERICAL_CAP) return dispatch_rng<kMethodCap>(a, n, vec, s);
  if (method == VNDF_METHOD_POLAR_DISK) return dispatch_rng<kMethodPolar>(a, n, vec, s);
  return dispatch_rng<kMethodCapExt>(a, n, vec, s);
}

extern "C" int vndf_rescue_count(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                 const float* alpha_x, const float* alpha_y, const float* u1, const float* u2,
                                 uint64_t seed, uint64_t counter_base, uint32_t stream_id, int method,
                                 unsigned long long* count, void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (method != VNDF_METHOD_SPHERICAL_CAP && method != VNDF_METHOD_POLAR_DISK &&
      method != VNDF_METHOD_SPHERICAL_CAP_EXTENDED)
    return VNDF_ERR_METHOD;
  if (!count) return VNDF_ERR_NULL;
  if (!aligned(count, 8)) return VNDF_ERR_ALIGN;
  if (n > 0) {
    if (!wi_x || !wi_y || !wi_z || !alpha_x) return VNDF_ERR_NULL;
    if ((u1 == nullptr) != (u2 == nullptr)) return VNDF_ERR_ARG;
    if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2)) return VNDF_ERR_ALIGN;
    if (aliased({count}, {wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2})) return VNDF_ERR_ARG;
  }
  if (const int f = pre_launch("vndf_rescue_count")) return f;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) return VNDF_ERR_CUDA;
  if (n == 0 || method == VNDF_METHOD_POLAR_DISK) return VNDF_OK;  // the prior sampler has no such path
  const SampleArgs a{wi_x,    wi_y,    wi_z,    alpha_x, alpha_y, u1, u2, nullptr, nullptr, nullptr, nullptr,
                     make_rng(seed, counter_base, stream_id)};
  return method == VNDF_METHOD_SPHERICAL_CAP ? launch_rescue_count<kMethodCap>(a, n, count, s)
                                             : launch_rescue_count<kMethodCapExt>(a, n, count, s);
}

template <bool EXT>
int pdf_entry(const char* name, int64_t n, const float* wi_x, const float* wi_y, const float* wi_z, const float* alpha_x,
              const float* alpha_y, const float* wm_x, const float* wm_y, const float* wm_z, float* pdf,
              void* cuda_stream) {
  if (n < 0 || n >= kMaxN) return VNDF_ERR_SIZE;
  if (n == 0) return VNDF_OK;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !wm_x || !wm_y || !wm_z || !pdf) return VNDF_ERR_NULL;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf)) return VNDF_ERR_ALIGN;
  if (aliased({pdf}, {wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z})) return VNDF_ERR_ARG;
  if (const int f = pre_launch(name)) return f;
  const bool vec = all_aligned16(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf);
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return alpha_y ? launch_pdf<false, EXT>(n, wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf, vec, s)
                 : launch_pdf<true, EXT>(n, wi_x, wi_y, wi_z, alpha_x, alpha_x, wm_x, wm_y, wm_z, pdf, vec, s);
}

extern "C" int vndf_pdf(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z, const float* alpha_x,
                        const float* alpha_y, const float* wm_x, const float* wm_y, const float* wm_z, float* pdf,
                        void* cuda_stream) {
  return pdf_entry<false>("vndf_pdf", n, wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf, cuda_stream);
}

extern "C" int vndf_pdf_extended(int64_t n, const float* wi_x, const float* wi_y, const float* wi_z,
                                 const float* alpha_x, const float* alpha_y, const float* wm_x, const float* wm_y,
                                 const float* wm_z, float* pdf, void* cuda_stream) {
  return pdf_entry<true>("vndf_pdf_extended", n, wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf, cuda_stream);
}
