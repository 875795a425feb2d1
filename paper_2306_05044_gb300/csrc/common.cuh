// Host-side helpers shared by the libvndf entry points: argument checks,
// device properties and launch shapes, and the streaming load/store forms.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "vndf.h"

namespace vndf {

constexpr int64_t kMaxN = int64_t(1) << 62;

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Every non-NULL pointer must be 4-byte aligned.
template <typename... P>
inline bool all_aligned4(P... p) {
  return (... && (p == nullptr || aligned(p, 4)));
}

// Every non-NULL pointer 16-byte aligned: the float4 path may be taken.
template <typename... P>
inline bool all_aligned16(P... p) {
  return (... && (p == nullptr || aligned(p, 16)));
}

// Multiprocessor count of the current device (cached per device; several host
// threads may ask at once, and all of them store the same value).
inline int sm_count() {
  static std::atomic<int> cache[64];  // zero-initialised (static storage)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// Grid for a grid-stride loop over `work` items with `block` threads per CTA:
// at most `waves` resident waves of `per_sm` CTAs on every SM.
inline unsigned grid_for(int64_t work, int block, int per_sm, int waves) {
  const int64_t need = (work + block - 1) / block;
  const int64_t cap = int64_t(sm_count()) * per_sm * waves;
  const int64_t g = need < cap ? need : cap;
  return static_cast<unsigned>(g < 1 ? 1 : g);
}

inline int launch_status() { return cudaGetLastError() == cudaSuccess ? VNDF_OK : VNDF_ERR_CUDA; }

// Streaming (evict-first) 128-bit loads and stores: every byte is touched once.
__device__ __forceinline__ float4 ld_stream(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st_stream(float* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }

}  // namespace vndf
