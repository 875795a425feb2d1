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
//
// What is left in the queues when the warps finish (fewer than 32 per warp;
// a warp of a 2^28-sample launch flags only a few to a few dozen samples in
// all) is recomputed by the whole CTA at once (rescue_drain_cta): one
// barrier, then every thread takes entries of the concatenated queues in turn,
// so a handful of flagged samples no longer costs each warp a full pass of the
// slow path with one or two lanes active.
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

// CTA-collective (every thread of the block, after its warp's last push):
// the entries left in all warps' queues, recomputed by all threads of the
// block.  `queues` is the block's array of per-warp queues, `count` this
// warp's (warp-uniform) number of waiting entries.  The barrier orders every
// warp's earlier global stores before the recomputed ones, which another warp
// of the block may now write.
template <class Fn>
__device__ __forceinline__ void rescue_drain_cta(RescueQueue* queues, int count, Fn&& fn) {
  __shared__ int s_count[32];
  const int warps = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) s_count[threadIdx.x >> 5] = count;
  __syncthreads();
  int total = 0;
  for (int w = 0; w < warps; ++w) total += s_count[w];
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int w = 0, k = e;
    while (k >= s_count[w]) k -= s_count[w++];  // ends: e < total
    fn(queues[w].idx[k]);
  }
}

}  // namespace vndf
