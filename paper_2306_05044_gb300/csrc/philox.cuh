// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.2 / Table 2) and the
// mapping of a sample's global index to its two uniforms.
//
// Layout (the paper asks only for u1, u2 in [0, 1), Sec. 2): sample g reads
// block b = g >> 1 with counter (b lo, b hi, stream_id, 0) and key (seed lo,
// seed hi); even g takes words (0, 1), odd g words (2, 3).  u = (w >> 8) 2^-24.
#pragma once
#include <cstdint>

namespace vndf {

struct Rng {
  uint32_t k0, k1;     // key words
  uint64_t base;       // global index of sample 0
  uint32_t stream;     // counter word 2
};

__host__ __device__ inline Rng make_rng(uint64_t seed, uint64_t counter_base, uint32_t stream_id) {
  Rng r;
  r.k0 = static_cast<uint32_t>(seed);
  r.k1 = static_cast<uint32_t>(seed >> 32);
  r.base = counter_base;
  r.stream = stream_id;
  return r;
}

// Ten rounds: two 32x32->64 products with the published multipliers, the word
// permutation, and the Weyl key schedule with the published increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(const Rng& r, uint64_t block) {
  return philox4x32_10(make_uint4(static_cast<uint32_t>(block), static_cast<uint32_t>(block >> 32),
                                  r.stream, 0u),
                       r.k0, r.k1);
}

// (w >> 8) * 2^-24: exact in float32, in [0, 1 - 2^-24].
__device__ __forceinline__ float word_to_unit(uint32_t w) {
  return __uint2float_rn(w >> 8) * 5.9604644775390625e-8f;
}

// Uniforms of one sample with local index i (one Philox call).
__device__ __forceinline__ void uniforms1(const Rng& r, uint64_t i, float& u1, float& u2) {
  const uint64_t g = r.base + i;
  const uint4 w = philox_block(r, g >> 1);
  const bool odd = (g & 1u) != 0;
  u1 = word_to_unit(odd ? w.z : w.x);
  u2 = word_to_unit(odd ? w.w : w.y);
}

// Uniforms of samples i0 .. i0+3 (i0 a multiple of 4): two Philox calls when the
// first global index is even, three when it is odd.  Each block index is taken
// from its own global index (mod 2^64), so a batch may straddle the wrap.
__device__ __forceinline__ void uniforms4(const Rng& r, uint64_t i0, float (&u1)[4], float (&u2)[4]) {
  const uint64_t g0 = r.base + i0;
  if ((g0 & 1u) == 0) {
    const uint4 a = philox_block(r, g0 >> 1);
    const uint4 b = philox_block(r, (g0 + 2) >> 1);
    u1[0] = word_to_unit(a.x); u2[0] = word_to_unit(a.y);
    u1[1] = word_to_unit(a.z); u2[1] = word_to_unit(a.w);
    u1[2] = word_to_unit(b.x); u2[2] = word_to_unit(b.y);
    u1[3] = word_to_unit(b.z); u2[3] = word_to_unit(b.w);
  } else {
    const uint4 a = philox_block(r, g0 >> 1);
    const uint4 b = philox_block(r, (g0 + 1) >> 1);
    const uint4 c = philox_block(r, (g0 + 3) >> 1);
    u1[0] = word_to_unit(a.z); u2[0] = word_to_unit(a.w);
    u1[1] = word_to_unit(b.x); u2[1] = word_to_unit(b.y);
    u1[2] = word_to_unit(b.z); u2[2] = word_to_unit(b.w);
    u1[3] = word_to_unit(c.x); u2[3] = word_to_unit(c.y);
  }
}

// Uniforms of samples j0, j0+1 (j0 even): one Philox call when the global index
// of j0 is even, two when it is odd.
__device__ __forceinline__ void uniforms2(const Rng& r, uint64_t j0, float& a1, float& a2, float& b1, float& b2) {
  const uint64_t g0 = r.base + j0;
  if ((g0 & 1u) == 0) {
    const uint4 w = philox_block(r, g0 >> 1);
    a1 = word_to_unit(w.x);
    a2 = word_to_unit(w.y);
    b1 = word_to_unit(w.z);
    b2 = word_to_unit(w.w);
  } else {
    const uint4 w = philox_block(r, g0 >> 1);
    const uint4 x = philox_block(r, (g0 + 1) >> 1);
    a1 = word_to_unit(w.z);
    a2 = word_to_unit(w.w);
    b1 = word_to_unit(x.x);
    b2 = word_to_unit(x.y);
  }
}

}  // namespace vndf
