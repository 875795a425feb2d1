// Deferred, warp-batched recomputation of ill-conditioned samples.
//
// A streaming kernel flags the few samples whose FP32 half vector is
// ill-conditioned and redoes them in double-float.  Done in place, one flagged
// lane stalls its 31 neighbours for the whole slow path; on inputs where a few
// per mille of the samples are flagged (incident directions below the horizon at
// low roughness), a third of all warp steps would carry one.  Instead each warp
// queues the indices of its flagged samples in shared memory and, once 32 are
// waiting, recomputes them together, one per lane: the lane reloads the
// sample's inputs (rare, so from L2 or HBM at no measurable cost) and
// overwrites the FP32 results already stored.  A sample's result does not
// depend on when it is recomputed, so results equal the in-place path's.
//
// Both calls are warp-collective: every lane of the warp makes them, with a
// warp-uniform `count`.  __syncwarp orders this warp's earlier global stores
// (the FP32 group results) before the recomputed ones.
#pragma once
#include <cstdint>

namespace vndf {

// 31 indices can wait while a step of 32 lanes x 4 samples pushes up to 128.
constexpr int kRescueCap = 160;

struct RescueQueue {
  int64_t idx[kRescueCap];
};

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Queue this lane's sample index if `flag`; count grows by the number of flagged lanes.
__device__ __forceinline__ void rescue_push(RescueQueue& q, int& count, bool flag, int64_t idx) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (flag) q.idx[count + __popc(m & lanemask_lt())] = idx;
  count += __popc(m);
}

// While 32 or more samples wait (with `all`, while any wait), each lane takes
// one index from the top of the queue and calls fn(idx).
template <class Fn>
__device__ __forceinline__ void rescue_drain(RescueQueue& q, int& count, bool all, Fn&& fn) {
  const int lane = threadIdx.x & 31;
  while (count >= 32 || (all && count > 0)) {
    __syncwarp();
    const int take = count < 32 ? count : 32;
    const int base = count - take;
    if (lane < take) fn(q.idx[base + lane]);
    count = base;
    __syncwarp();
  }
}

}  // namespace vndf
