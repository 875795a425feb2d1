// Deferred, warp-batched recomputation of ill-conditioned samples.
//
// A streaming kernel flags the few samples whose FP32 half vector is
// ill-conditioned and redoes them in double-float.  Done in place, one flagged
// lane stalls its 31 neighbours for the whole slow path; on inputs where a few
// per mille of the samples are flagged (incident directions below the horizon at
// low roughness), a third of all warp steps would carry one.  Instead each warp
// queues its flagged samples (inputs and index) in shared memory and, once 32
// are waiting, recomputes them together, one per lane, overwriting the FP32
// results already stored.  Results do not depend on when a sample is
// recomputed, so they are the same as with the in-place path.
//
// Both calls are warp-collective: every lane of the warp makes them, with
// warp-uniform `count`.  __syncwarp orders this warp's earlier global stores
// (the FP32 group results) before the recomputed ones.
#pragma once
#include <cstdint>

namespace vndf {

// 31 entries can wait while a round of 32 lanes pushes one sample each.
constexpr int kRescueCap = 64;

template <int NF>
struct RescueQueue {
  float v[NF][kRescueCap];
  int64_t idx[kRescueCap];
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Queue this lane's sample if `flag`; count grows by the number of flagged lanes.
template <int NF>
__device__ __forceinline__ void rescue_push(RescueQueue<NF>& q, int& count, bool flag, const float (&v)[NF],
                                            int64_t idx) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (flag) {
    const int pos = count + __popc(m & lanemask_lt());
#pragma unroll
    for (int f = 0; f < NF; ++f) q.v[f][pos] = v[f];
    q.idx[pos] = idx;
  }
  count += __popc(m);
}

// While 32 or more samples wait (with `all`, while any wait), each lane takes
// one from the top of the queue and calls fn(v, idx).
template <int NF, class Fn>
__device__ __forceinline__ void rescue_drain(RescueQueue<NF>& q, int& count, bool all, Fn&& fn) {
  const int lane = threadIdx.x & 31;
  while (count >= 32 || (all && count > 0)) {
    __syncwarp();
    const int take = count < 32 ? count : 32;
    const int base = count - take;
    if (lane < take) {
      float v[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) v[f] = q.v[f][base + lane];
      fn(v, q.idx[base + lane]);
    }
    count = base;
    __syncwarp();
  }
}

}  // namespace vndf
