// Batched directional albedo of the GGX microfacet BRDF, estimated with the
// spherical-cap VNDF sampler: for every query q (incident direction wi_q,
// roughness alpha_q, sample count N_q)
//   E_q = (1 / N_q) sum_j f_r(wo_j, wi) |cos theta_o| / PDF(wo_j)        (App. A, Eq. rendering_mc, L = 1)
// where wm_j is drawn from the VNDF (Sec. 2, Sec. 3.3), wo_j = 2 (wm.wi) wm - wi
// (Eq. reflect) and PDF = G1 D / (4 cos theta_i) (App. A).  The D and G1 terms
// cancel, leaving the weight F(wi.wm) G2 / G1(wi) (zero when wo is below the
// surface), with Schlick's Fresnel and the height-correlated G2 of App. A:
//   G2 / G1(wi) = (L_i + z_i) z_o / ((L_i + z_i) z_o + z_i P_o / (L_o + z_o)),
//   L_k = |M^-1 w_k|,  P_o = ax^2 wo.x^2 + ay^2 wo.y^2  (so L_o - z_o = P_o / (L_o + z_o) without cancellation).
//
// Work decomposition (ragged counts in one launch):
// * Samples of a query are cut into groups of 256 consecutive samples; lane l of
//   the warp that owns a group sums samples 8l .. 8l+7 in order, then the warp
//   adds the 32 lane sums with a fixed butterfly.  That order is a property of
//   the data, not of the launch, so E is bit-identical for every launch shape.
// * An item is `groups_per_item` consecutive groups of one query.  A one-block
//   prologue computes per-query item counts and their exclusive scan; each warp
//   of the persistent kernel (only as many CTAs as the SMs hold at once) then
//   takes a contiguous run of about total / W items (W = warps in the grid) on
//   its own, with no block barrier, and writes one partial per group.  When it
//   leaves a query it adds the number of that query's items it did to the
//   query's counter; the warp whose addition completes the query sums the
//   query's group partials (fixed lane-strided order + butterfly) into E_q.
// * Nothing waits on anything: completion is detected with an atomic counter
//   per query (fence, then atomicAdd), so no warp ever spins.  The one barrier
//   is at CTA start, after the item offsets are copied into shared memory.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "common.cuh"
#include "philox.cuh"
#include "vndf_math.cuh"

namespace vndf {

constexpr int kGroupSamples = 256;  // samples per reduction group (one warp)
constexpr int kLaneSamples = 8;     // consecutive samples per lane
constexpr int kAlbedoMaxWarps = 20;  // warps per CTA at most (the kernel's launch bound)
// Up to this many item offsets (nq + 1) are copied into each CTA's shared
// memory (48 KB, the default dynamic limit), so that finding an item's query
// costs shared-memory rather than L2 latency; larger batches search in place.
constexpr int32_t kCachedOffsets = 12288;

struct AlbedoArgs {
  const float *wx, *wy, *wz, *ax, *ay;
  const int32_t* ns;
  int32_t nq;
  int32_t gmax;  // group slots per query (ceil(max_samples / 256))
  int32_t max_n;
  int32_t groups_per_item;
  float f0;
  Rng rng;  // rng.stream is the stream id of query 0
  float* E;
  int32_t* ctl;     // [0] reserved (0), [1] total items, [2 .. 2+nq] item offsets, then done[nq]
  float* partials;  // nq * gmax group sums
};

__host__ __device__ inline size_t albedo_ctl_ints(int32_t nq) { return 3 + 2 * size_t(nq); }
__host__ __device__ inline size_t albedo_partials_offset(int32_t nq) {
  return (albedo_ctl_ints(nq) * 4 + 255) / 256 * 256;
}

// ---------------------------------------------------------------- prologue
__global__ void __launch_bounds__(1024) albedo_prologue_kernel(AlbedoArgs a) {
  __shared__ int32_t warp_tot[32];
  const int t = threadIdx.x;
  const int32_t per = (a.nq + 1023) / 1024;
  const int32_t q0 = min(a.nq, t * per), q1 = min(a.nq, q0 + per);
  int32_t* offsets = a.ctl + 2;
  int32_t* done = a.ctl + 3 + a.nq;
  int32_t local = 0;
  // a query outside the sampler's domain (wi.z <= 0, alpha <= 0, non-finite) or with a count outside
  // [0, max] gets no work and E = NaN; its item count is parked in offsets[q] until the scan is known
  for (int32_t q = q0; q < q1; ++q) {
    const int32_t n = a.ns[q];
    const float ax = a.ax[q], ay = a.ay ? a.ay[q] : ax;
    const bool valid = n >= 0 && n <= a.max_n && in_domain(a.wx[q], a.wy[q], a.wz[q], ax, ay);
    const int32_t groups = valid ? (n + kGroupSamples - 1) / kGroupSamples : 0;
    const int32_t items = (groups + a.groups_per_item - 1) / a.groups_per_item;
    offsets[q] = items;
    local += items;
    done[q] = 0;
    if (!valid) a.E[q] = __int_as_float(0x7fc00000);  // NaN
    else if (n == 0) a.E[q] = 0.f;
  }
  // exclusive scan of the per-thread totals (fixed order)
  int32_t incl = local;
  const int lane = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int32_t x = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    warp_tot[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  int32_t run = (w > 0 ? warp_tot[w - 1] : 0) + incl - local;
  for (int32_t q = q0; q < q1; ++q) {
    const int32_t items = offsets[q];  // written above by this thread
    offsets[q] = run;
    run += items;
  }
  if (t == 1023) {
    offsets[a.nq] = run;
    a.ctl[1] = run;
    a.ctl[0] = 0;
  }
}

// ---------------------------------------------------------------- sample weight
struct QueryConst {
  float ux, uy, uz;  // unit wi
  float ax, ay;
  Stretched i;       // M^-1 wi / |M^-1 wi|
  float A;           // L_i + z_i for the unit wi
};

__device__ __forceinline__ QueryConst query_const(const AlbedoArgs& a, int32_t q) {
  QueryConst c;
  const float wx = a.wx[q], wy = a.wy[q], wz = a.wz[q];
  c.ax = a.ax[q];
  c.ay = a.ay ? a.ay[q] : c.ax;
  const float rn = rsqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
  c.ux = wx * rn;
  c.uy = wy * rn;
  c.uz = wz * rn;
  const float sx = c.ax * c.ux, sy = c.ay * c.uy;
  const float l2 = fmaf(sx, sx, fmaf(sy, sy, c.uz * c.uz));
  const float rl = rsqrtf(l2);
  c.i = Stretched{sx * rl, sy * rl, c.uz * rl, fmaf(c.uz, rl, 1.f)};
  c.A = l2 * rl + c.uz;
  return c;
}

// Estimator terms of two samples (u1, u2 of each in the halves of a float2):
// F G2 / G1(wi), or 0 when wo is below the surface.  The cap sample is the
// sampler's own (cap_half_vector); the FP32 fma / mul / add run as packed pairs
// (pair.cuh), every lane rounded as in the one-sample form of the same steps;
// square roots, reciprocals and the final select per lane.
__device__ __forceinline__ float2 albedo_weight2(const QueryConst& c, float f0, float2 u1, float2 u2) {
  using V = float2;
  // the cap sample of Sec. 3.3 for both samples, h = (hx, hy, hz)
  const StretchedV<V> i{splat<V>(c.i.x), splat<V>(c.i.y), splat<V>(c.i.z), splat<V>(c.i.a)};
  V hx, hy, hz, a;
  cap_half_vector(i, u1, u2, hx, hy, hz, a);
  // wm = v / |v| with v = (ax hx, ay hy, hz), and wo = 2 (wi.wm) wm - wi
  const V vx = vmul(splat<V>(c.ax), hx), vy = vmul(splat<V>(c.ay), hy);
  const V rv = vmap(RsqrtF{}, vfma(vx, vx, vfma(vy, vy, vmul(hz, hz))));
  const V mx = vmul(vx, rv), my = vmul(vy, rv), mz = vmul(hz, rv);
  const V d = vfma(mx, splat<V>(c.ux), vfma(my, splat<V>(c.uy), vmul(mz, splat<V>(c.uz))));  // wi.wm > 0
  const V d2 = vadd(d, d);
  const V ox = vfma(d2, mx, splat<V>(-c.ux));
  const V oy = vfma(d2, my, splat<V>(-c.uy));
  const V oz = vfma(d2, mz, splat<V>(-c.uz));
  // G2 / G1(wi) = A oz / (A oz + uz P_o / (L_o + oz))
  const V sx = vmul(splat<V>(c.ax), ox), sy = vmul(splat<V>(c.ay), oy);
  const V po = vfma(sx, sx, vmul(sy, sy));
  const V lo = vmap(SqrtFast{}, vfma(oz, oz, po));
  const V num = vmul(splat<V>(c.A), oz);
  const V den = vfma(vmul(splat<V>(c.uz), po), vmap(RcpFast{}, vadd(lo, oz)), num);
  const V g = vmul(num, vmap(RcpFast{}, den));
  // Schlick's Fresnel at wi.wm
  const V t = vsub(splat<V>(1.f), d);
  const V t2 = vmul(t, t);
  const V fr = vfma(splat<V>(1.f - f0), vmul(vmul(t2, t2), t), splat<V>(f0));
  const V w = vmul(fr, g);
  return make_float2(oz.x > 0.f ? w.x : 0.f, oz.y > 0.f ? w.y : 0.f);
}

__device__ __forceinline__ float warp_tree(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- persistent kernel
// The item's query: the last q with offsets[q] <= item (every lane runs the same search).
__device__ __forceinline__ int32_t item_query(const int32_t* offsets, int32_t nq, int32_t item) {
  int32_t lo = 0, hi = nq - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One CTA of up to 20 warps per SM (86 registers): a lane computes its eight uniforms and then its four
// packed weight pairs side by side, which the register file of 2 x 16 warps (64 each) could not hold
// (4096-query grid, graph replays: 183 us at 20 warps, 187 at 16 with 116 registers, 195 at 32 warps).
__global__ void __launch_bounds__(32 * kAlbedoMaxWarps, 1) albedo_kernel(AlbedoArgs a) {
  extern __shared__ int32_t s_offsets[];
  const int lane = threadIdx.x & 31;
  const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
  const int32_t* offsets = a.ctl + 2;
  if (a.nq + 1 <= kCachedOffsets) {  // uniform over the block
    for (int32_t i = threadIdx.x; i <= a.nq; i += blockDim.x) s_offsets[i] = offsets[i];
    __syncthreads();
    offsets = s_offsets;
  }
  int32_t* done = a.ctl + 3 + a.nq;
  const int32_t total = a.ctl[1];
  // Each warp takes a contiguous run of items, the runs differing in length by at most one
  // item: the warps finish together, and the query changes only at the run's query
  // boundaries, so its search, its per-query constants and its completion count are paid
  // once per query and run, not per item.
  const int64_t w = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int32_t it0 = int32_t(w * total / warps), it1 = int32_t((w + 1) * total / warps);
  if (it0 >= it1) return;
  int32_t q = item_query(offsets, a.nq, it0);
  int32_t n = a.ns[q];
  int32_t groups = (n + kGroupSamples - 1) / kGroupSamples;
  QueryConst c = query_const(a, q);
  Rng r = a.rng;
  r.stream = a.rng.stream + uint32_t(q);
  int32_t mine = 0;  // items of query q done by this warp since the last count
  // Adds this warp's items of query q to its completion count; the warp whose addition
  // completes the query sums the query's group partials (fixed order) into E_q.
  auto finish = [&]() {
    int32_t last = 0;
    if (lane == 0) {
      __threadfence();
      const int32_t items_q = offsets[q + 1] - offsets[q];
      last = atomicAdd(done + q, mine) + mine == items_q;
    }
    if (__shfl_sync(0xffffffffu, last, 0)) {
      __threadfence();
      float sum = 0.f;
      for (int32_t g = lane; g < groups; g += 32) sum += __ldcg(a.partials + size_t(q) * a.gmax + g);
      sum = warp_tree(sum);
      if (lane == 0) a.E[q] = sum / float(n);
    }
    mine = 0;
  };
  for (int32_t item = it0; item < it1; ++item) {
    if (offsets[q + 1] <= item) {  // next query with items (queries without items are skipped)
      finish();
      do {
        ++q;
      } while (offsets[q + 1] <= item);
      n = a.ns[q];
      groups = (n + kGroupSamples - 1) / kGroupSamples;
      c = query_const(a, q);
      r.stream = a.rng.stream + uint32_t(q);
    }
    const int32_t k = item - offsets[q];
    const int32_t g_end = min(groups, (k + 1) * a.groups_per_item);
    for (int32_t g = k * a.groups_per_item; g < g_end; ++g) {
      const int32_t j0 = g * kGroupSamples + lane * kLaneSamples;
      float acc = 0.f;
      // all of the lane's uniforms first, then all of its weights: independent Philox chains and
      // independent weight chains side by side (same terms, same order of the sum)
      float U1[kLaneSamples], U2[kLaneSamples];
#pragma unroll
      for (int s = 0; s < kLaneSamples; s += 2) uniforms2(r, uint64_t(j0 + s), U1[s], U2[s], U1[s + 1], U2[s + 1]);
      if ((g + 1) * kGroupSamples <= n) {  // a full group (warp-uniform): no per-sample bound
#pragma unroll
        for (int s = 0; s < kLaneSamples; s += 2) {
          const float2 w = albedo_weight2(c, a.f0, make_float2(U1[s], U1[s + 1]),
                                          make_float2(U2[s], U2[s + 1]));
          acc += w.x;
          acc += w.y;
        }
      } else {
#pragma unroll
        for (int s = 0; s < kLaneSamples; s += 2) {
          const float2 w = albedo_weight2(c, a.f0, make_float2(U1[s], U1[s + 1]),
                                          make_float2(U2[s], U2[s + 1]));
          acc += j0 + s < n ? w.x : 0.f;
          acc += j0 + s + 1 < n ? w.y : 0.f;
        }
      }
      acc = warp_tree(acc);
      if (lane == 0) a.partials[size_t(q) * a.gmax + g] = acc;
    }
    ++mine;
  }
  finish();
}

// ---------------------------------------------------------------- launch configuration
struct AlbedoConfig {
  int32_t block_warps, groups_per_item, ctas_per_sm;
};

bool config_ok(const AlbedoConfig& c) {
  return c.block_warps >= 1 && c.block_warps <= kAlbedoMaxWarps && c.groups_per_item >= 1 && c.groups_per_item <= 256 &&
         c.ctas_per_sm >= 1 && c.ctas_per_sm <= 32;
}

// Per-device tuned configuration (set by vndf_albedo_autotune), else the default.
std::mutex g_tune_mutex;
AlbedoConfig g_tuned[64];
bool g_has_tuned[64] = {false};

constexpr AlbedoConfig kDefaultConfig{20, 2, 1};

AlbedoConfig current_config() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (dev >= 0 && dev < 64 && g_has_tuned[dev]) return g_tuned[dev];
  return kDefaultConfig;
}

size_t albedo_smem(const AlbedoArgs& a) {
  return a.nq + 1 <= kCachedOffsets ? size_t(a.nq + 1) * sizeof(int32_t) : 0;
}

// CTAs of block_warps warps that one SM holds at once (at least 1).
int albedo_resident(const AlbedoArgs& a, int32_t block_warps) {
  int resident = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, albedo_kernel, 32 * block_warps, albedo_smem(a)) !=
          cudaSuccess ||
      resident < 1)
    resident = 1;
  return resident;
}

int launch_albedo(AlbedoArgs a, const AlbedoConfig& c, cudaStream_t s) {
  a.groups_per_item = c.groups_per_item;
  albedo_prologue_kernel<<<1, 1024, 0, s>>>(a);
  const size_t smem = albedo_smem(a);
  // Every CTA must be resident from the start: the item runs are cut for the whole grid, and
  // a CTA that waited for a free slot would finish its run after the others.
  const int resident = albedo_resident(a, c.block_warps);
  const int ctas = c.ctas_per_sm < resident ? c.ctas_per_sm : resident;
  const unsigned grid = static_cast<unsigned>(sm_count() * ctas);
  albedo_kernel<<<grid, 32 * c.block_warps, smem, s>>>(a);
  return launch_status();
}

}  // namespace vndf

using namespace vndf;

namespace vndf {
// Work items, their offsets and the item total are int32: every group slot of
// the batch (n_queries x ceil(max / 256), which bounds the items) must have an
// index below 2^31.
inline bool albedo_fits_int32(int32_t n_queries, int32_t max_samples) {
  const int64_t gmax = (int64_t(max_samples) + kGroupSamples - 1) / kGroupSamples;
  return int64_t(n_queries) * gmax < (int64_t(1) << 31);
}
}  // namespace vndf

extern "C" size_t vndf_albedo_workspace_bytes(int32_t n_queries, int32_t max_samples_per_query) {
  if (n_queries <= 0 || max_samples_per_query < 0 || max_samples_per_query > (1 << 30)) return 0;
  if (!albedo_fits_int32(n_queries, max_samples_per_query)) return 0;
  const size_t gmax = (size_t(max_samples_per_query) + kGroupSamples - 1) / kGroupSamples;
  return albedo_partials_offset(n_queries) + size_t(n_queries) * gmax * sizeof(float);
}

namespace vndf {
// Checks of everything but the workspace.
int albedo_validate_args(int32_t n_queries, const float* wi_x, const float* wi_y, const float* wi_z,
                         const float* alpha_x, const float* alpha_y, const int32_t* n_samples, int32_t max_samples,
                         float* E) {
  if (n_queries < 0 || max_samples < 0 || max_samples > (1 << 30)) return VNDF_ERR_SIZE;
  if (n_queries == 0) return VNDF_OK;
  if (!albedo_fits_int32(n_queries, max_samples)) return VNDF_ERR_SIZE;
  if (!wi_x || !wi_y || !wi_z || !alpha_x || !n_samples || !E) return VNDF_ERR_NULL;
  if (!all_aligned4(wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, E)) return VNDF_ERR_ALIGN;
  if (aliased({E}, {wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples})) return VNDF_ERR_ARG;
  return VNDF_OK;
}

int albedo_validate(int32_t n_queries, const float* wi_x, const float* wi_y, const float* wi_z, const float* alpha_x,
                    const float* alpha_y, const int32_t* n_samples, int32_t max_samples, float* E,
                    void* workspace, size_t workspace_bytes) {
  const int st = albedo_validate_args(n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples, E);
  if (st != VNDF_OK || n_queries == 0) return st;
  if (!workspace || workspace_bytes < vndf_albedo_workspace_bytes(n_queries, max_samples))
    return VNDF_ERR_WORKSPACE;
  if (!aligned(workspace, 256)) return VNDF_ERR_ALIGN;
  if (aliased({E, workspace}, {wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples})) return VNDF_ERR_ARG;
  return VNDF_OK;
}

AlbedoArgs albedo_args(int32_t n_queries, const float* wi_x, const float* wi_y, const float* wi_z,
                       const float* alpha_x, const float* alpha_y, const int32_t* n_samples, int32_t max_samples,
                       float f0, uint64_t seed, uint64_t counter_base, uint32_t stream_id, float* E,
                       void* workspace) {
  AlbedoArgs a;
  a.wx = wi_x;
  a.wy = wi_y;
  a.wz = wi_z;
  a.ax = alpha_x;
  a.ay = alpha_y;
  a.ns = n_samples;
  a.nq = n_queries;
  a.max_n = max_samples;
  a.gmax = (max_samples + kGroupSamples - 1) / kGroupSamples;
  a.groups_per_item = 1;
  a.f0 = f0;
  a.rng = make_rng(seed, counter_base, stream_id);
  a.E = E;
  a.ctl = static_cast<int32_t*>(workspace);
  a.partials = reinterpret_cast<float*>(static_cast<char*>(workspace) + albedo_partials_offset(n_queries));
  return a;
}
}  // namespace vndf

namespace vndf {
// vndf_albedo_batched after its argument checks and with the name under which
// an injected fault is looked up (the no-allocation variant runs the same path).
int albedo_batched_entry(const char* name, int32_t n_queries, const float* wi_x, const float* wi_y,
                         const float* wi_z, const float* alpha_x, const float* alpha_y, const int32_t* n_samples,
                         int32_t max_samples_per_query, float f0, uint64_t seed, uint64_t counter_base,
                         uint32_t stream_id, float* E, void* workspace, size_t workspace_bytes,
                         const int32_t* config, bool takes_workspace, void* cuda_stream) {
  const int st = albedo_validate(n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples,
                                 max_samples_per_query, E, workspace, workspace_bytes);
  if (st != VNDF_OK || n_queries == 0) return st;
  AlbedoConfig c = current_config();
  if (config) {
    c = AlbedoConfig{config[0], config[1], config[2]};
    if (!config_ok(c)) return VNDF_ERR_ARG;
  }
  if (const int f = pre_launch(name, takes_workspace)) return f;
  const AlbedoArgs a = albedo_args(n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples,
                                   max_samples_per_query, f0, seed, counter_base, stream_id, E, workspace);
  return launch_albedo(a, c, static_cast<cudaStream_t>(cuda_stream));
}
}  // namespace vndf

extern "C" int vndf_albedo_batched(int32_t n_queries, const float* wi_x, const float* wi_y, const float* wi_z,
                                   const float* alpha_x, const float* alpha_y, const int32_t* n_samples,
                                   int32_t max_samples_per_query, float f0, uint64_t seed, uint64_t counter_base,
                                   uint32_t stream_id, float* E, void* workspace, size_t workspace_bytes,
                                   const int32_t* config, void* cuda_stream) {
  return albedo_batched_entry("vndf_albedo_batched", n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples,
                              max_samples_per_query, f0, seed, counter_base, stream_id, E, workspace,
                              workspace_bytes, config, true, cuda_stream);
}

extern "C" int vndf_albedo_autotune(int32_t n_queries, const float* wi_x, const float* wi_y, const float* wi_z,
                                    const float* alpha_x, const float* alpha_y, const int32_t* n_samples,
                                    int32_t max_samples_per_query, float f0, uint64_t seed,
                                    uint64_t counter_base, uint32_t stream_id, float* E, void* workspace,
                                    size_t workspace_bytes, int32_t* best_config, float* best_ms,
                                    void* cuda_stream) {
  const int st = albedo_validate(n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples,
                                 max_samples_per_query, E, workspace, workspace_bytes);
  if (st != VNDF_OK) return st;
  if (n_queries == 0) return VNDF_ERR_SIZE;
  if (const int f = pre_launch("vndf_albedo_autotune", true)) return f;
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  AlbedoArgs a = albedo_args(n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples_per_query, f0,
                             seed, counter_base, stream_id, E, workspace);
  static const int32_t warps[] = {4, 8, 16, kAlbedoMaxWarps};
  static const int32_t gpis[] = {1, 2, 4};
  static const int32_t ctas[] = {1, 2, 4, 8, 16};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return VNDF_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return VNDF_ERR_CUDA;
  }
  AlbedoConfig best = kDefaultConfig;
  float best_t = INFINITY;
  int rc = VNDF_OK;
  for (int32_t w : warps) {
    const int resident = albedo_resident(a, w);
    for (int32_t g : gpis) {
      int32_t prev = 0;
      for (int32_t c : ctas) {
        const int32_t eff = c < resident ? c : resident;  // the CTAs per SM the launch gets
        if (eff == prev) continue;                         // the same launch as the last one timed
        prev = eff;
        const AlbedoConfig cfg{w, g, eff};
        rc = launch_albedo(a, cfg, s);  // warm-up
        if (rc != VNDF_OK) break;
        float t = INFINITY;
        for (int rep = 0; rep < 10; ++rep) {  // best of 10: the configurations lie within a few per cent
          cudaEventRecord(e0, s);
          rc = launch_albedo(a, cfg, s);
          cudaEventRecord(e1, s);
          if (rc != VNDF_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = VNDF_ERR_CUDA;
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          t = fminf(t, ms);
        }
        if (rc != VNDF_OK) break;
        if (t < best_t) {
          best_t = t;
          best = cfg;
        }
      }
      if (rc != VNDF_OK) break;
    }
    if (rc != VNDF_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != VNDF_OK) return rc;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (dev >= 0 && dev < 64) {
      g_tuned[dev] = best;
      g_has_tuned[dev] = true;
    }
  }
  if (best_config) {
    best_config[0] = best.block_warps;
    best_config[1] = best.groups_per_item;
    best_config[2] = best.ctas_per_sm;
  }
  if (best_ms) *best_ms = best_t;
  return VNDF_OK;
}

extern "C" int vndf_albedo_set_config(const int32_t* config) {
  if (config && !config_ok(AlbedoConfig{config[0], config[1], config[2]})) return VNDF_ERR_ARG;
  if (const int f = injected_fault("vndf_albedo_set_config", false)) return f;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return VNDF_ERR_CUDA;
  if (dev >= 64) return config ? VNDF_ERR_SIZE : VNDF_OK;  // configurations are kept for devices 0..63
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_has_tuned[dev] = config != nullptr;
  if (config) g_tuned[dev] = AlbedoConfig{config[0], config[1], config[2]};
  return VNDF_OK;
}

extern "C" int vndf_albedo_get_config(int32_t* config) {
  if (!config) return VNDF_ERR_NULL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return VNDF_ERR_CUDA;
  bool set = false;
  AlbedoConfig c = kDefaultConfig;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (dev < 64 && g_has_tuned[dev]) {
      c = g_tuned[dev];
      set = true;
    }
  }
  config[0] = c.block_warps;
  config[1] = c.groups_per_item;
  config[2] = c.ctas_per_sm;
  return set ? 1 : 0;
}

// ---------------------------------------------------------------- no-allocation variant
// Some callers cannot hand the library a workspace: code on a renderer's
// per-frame path, where a cudaMalloc would synchronise the device and stall the
// frame, or a plugin that only receives the pointers a host application chose
// to give it and owns no allocator.  For them, vndf_albedo_batched_noalloc runs
// the same two kernels with the scratch held in this fixed device array instead
// of a caller workspace.  The array exists on every GPU that loads the library
// and stays allocated until the process exits.
static __device__ __align__(256) unsigned char g_albedo_scratch[VNDF_ALBEDO_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mutex;
void* g_scratch_ptr[64] = {nullptr};

// Device address of g_albedo_scratch on the current device.  Host code may not
// use the symbol's name as a pointer (on the host it is only a stand-in), so
// the address is looked up once per device, with that device current, and cached.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VNDF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_albedo_scratch) != cudaSuccess || p == nullptr) return VNDF_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return VNDF_OK;
}
}  // namespace

extern "C" int vndf_albedo_batched_noalloc(int32_t n_queries, const float* wi_x, const float* wi_y,
                                           const float* wi_z, const float* alpha_x, const float* alpha_y,
                                           const int32_t* n_samples, int32_t max_samples_per_query, float f0,
                                           uint64_t seed, uint64_t counter_base, uint32_t stream_id, float* E,
                                           const int32_t* config, void* cuda_stream) {
  const int st = albedo_validate_args(n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples,
                                      max_samples_per_query, E);
  if (st != VNDF_OK || n_queries == 0) return st;
  if (vndf_albedo_workspace_bytes(n_queries, max_samples_per_query) > VNDF_ALBEDO_NOALLOC_SCRATCH_BYTES)
    return VNDF_ERR_SIZE;
  if (config && !config_ok(AlbedoConfig{config[0], config[1], config[2]})) return VNDF_ERR_ARG;
  if (const int f = injected_fault("vndf_albedo_batched_noalloc", false)) return f;
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != VNDF_OK) return rc;
  // The prologue kernel rewrites every control word the persistent kernel reads,
  // and each group partial is written before it is read, so what an earlier call
  // left in the array never leaks into this one.
  return albedo_batched_entry("vndf_albedo_batched_noalloc", n_queries, wi_x, wi_y, wi_z, alpha_x, alpha_y,
                              n_samples, max_samples_per_query, f0, seed, counter_base, stream_id, E, scratch,
                              VNDF_ALBEDO_NOALLOC_SCRATCH_BYTES, config, false, cuda_stream);
}
