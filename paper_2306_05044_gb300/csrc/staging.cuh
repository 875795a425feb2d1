// Per-thread shared-memory staging for the streaming kernels: each thread
// copies its own next 16-byte group of every input stream with cp.async
// (asynchronous global->shared copies, cached in L2 only) and later reads back
// only what it copied, so the only synchronisation is the per-thread
// cp.async.wait_group: no barrier and no spin.  This keeps a group of loads in
// flight per thread without holding registers for it.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

namespace vndf {

// Raise KERNEL's dynamic shared-memory limit to `bytes` on the current device,
// once per (kernel, device): the attribute belongs to the device's copy of the
// kernel, so a process that uses several GPUs sets it on each.  Thread-safe;
// returns false if the CUDA call fails.
template <auto KERNEL>
inline bool ensure_dynamic_smem(size_t bytes) {
  static std::atomic<uint64_t> done{0};  // bit d: set on device d (devices 0..63)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return true;
  if (cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) != cudaSuccess)
    return false;
  if (bit) done.fetch_or(bit, std::memory_order_release);
  return true;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <bool PHILOX, bool ISO>
__host__ __device__ constexpr int streams_in() { return 4 + (ISO ? 0 : 1) + (PHILOX ? 0 : 2); }

}  // namespace vndf
