// Host-side helpers shared by the libvndf entry points: argument checks,
// device properties and launch shapes, and the streaming load/store forms.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <initializer_list>

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
// threads may ask at once, and all of them store the same value).  0 when the
// device or its attribute cannot be queried: nothing is assumed about the part.
inline int sm_count() {
  static std::atomic<int> cache[64];  // zero-initialised (static storage)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
  int v = dev < 64 ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 0;
    if (dev < 64) cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// Host-side fault injection (status.cu), for testing how callers handle the
// library's error returns without making any GPU fail.  The environment
// variable VNDF_FAULT = "<kind>" or "<kind>@<entry point name>" makes the
// named entry point (every one, without a name) return, after its argument
// checks and before it enqueues any work:
//   launch     VNDF_ERR_CUDA, as if a kernel launch had failed;
//   align      VNDF_ERR_ALIGN, as if a pointer were misaligned;
//   workspace  VNDF_ERR_WORKSPACE, only in entry points that take a workspace.
// Unset or empty: VNDF_OK (no effect).
int injected_fault(const char* entry, bool takes_workspace);

// Status of an entry point just before it enqueues work: an injected fault,
// else VNDF_ERR_CUDA when the current device cannot be queried (launch shapes
// are sized from its multiprocessor count), else VNDF_OK.
inline int pre_launch(const char* entry, bool takes_workspace = false) {
  const int f = injected_fault(entry, takes_workspace);
  if (f != VNDF_OK) return f;
  return sm_count() > 0 ? VNDF_OK : VNDF_ERR_CUDA;
}

// True when a non-NULL output pointer equals another output pointer or an
// input pointer.  Outputs must not overlap inputs (a kernel may write an
// output before it has read every input it needs); exact equality is the
// overlap that can be detected from pointers alone.
inline bool aliased(std::initializer_list<const void*> outs, std::initializer_list<const void*> ins) {
  for (auto o = outs.begin(); o != outs.end(); ++o) {
    if (*o == nullptr) continue;
    for (auto p = outs.begin(); p != o; ++p)
      if (*p == *o) return true;
    for (const void* i : ins)
      if (i == *o) return true;
  }
  return false;
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

// Programmatic dependent launch.  A kernel launched with launch_pdl may be scheduled before the work ahead
// of it in the stream has finished: its CTAs become resident once every CTA of the kernel ahead has
// signalled pdl_trigger (or exited), and each first waits in hardware (pdl_wait) until that kernel has
// completed and its writes are visible.  Every kernel launched this way calls pdl_wait before it reads an
// input or writes an output, so results are those of an ordinary launch: what it hides is the launch
// latency between back-to-back calls (measured: 2^22 samples 32.2 -> 30.2 us per call).  While the stream
// is being captured into a CUDA graph the launch is an ordinary one: inside a graph the early-resident
// CTAs measured slower (2^20 samples 7.1 -> 9.9 us per replayed launch).  After an ordinary launch
// pdl_wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline bool launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &capture) != cudaSuccess) return false;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = capture == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...) == cudaSuccess;
}

// Streaming (evict-first) 128-bit loads and stores: every byte is touched once.
__device__ __forceinline__ float4 ld_stream(const float* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st_stream(float* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }

}  // namespace vndf
