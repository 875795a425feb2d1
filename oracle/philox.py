"""Philox4x32-10 counter-based generator, FP64 oracle side (test infrastructure).

The paper only asks for two uniform numbers u1, u2 in [0, 1) per sample
(Sec. 2, "Importance Sampling"); it names no generator.  The generator used
on both sides of this project is Philox4x32-10 as published by Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
(SC'11, Sec. 3.2 and Table 2): a 128-bit counter, a 64-bit key, ten rounds
of two 32x32->64 multiplies with the published multipliers, a fixed word
permutation and a Weyl-sequence key schedule with the published increments.

This file is part of the oracle: plain, slow, vectorised numpy, written from
that description, sharing nothing with the CUDA path.  Only tests, the smoke
entry and the CPU baseline leg of the bench may import it.

Counter layout (a reading: the paper is silent on it):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (b & 0xffffffff, b >> 32, stream_id, 0),  b = g >> 1
where g = counter_base + i is the global index of sample i.  One Philox block
yields four words; the even sample of a pair takes words (0, 1) and the odd
sample takes words (2, 3).  The first word of a sample gives u1, the second u2,
each as (x >> 8) * 2^-24, which is exact in FP32 and FP64 and lies in
[0, 1 - 2^-24].
"""
import numpy as np

# SC'11, Table 2 / Sec. 3.2: round multipliers and key increments for Philox4x32.
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)  # golden ratio
PHILOX_W1 = np.uint32(0xBB67AE85)  # sqrt(3) - 1
ROUNDS = 10

_MASK32 = np.uint64(0xFFFFFFFF)


def _mulhilo(m, x):
    """32x32 -> 64-bit product split into (hi, lo) 32-bit words."""
    p = m * x.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & _MASK32).astype(np.uint32)


def philox4x32_10(counter, key):
    """Apply ten Philox rounds.

    counter: uint32 array of shape (4, N) (words x0..x3).
    key:     uint32 array of shape (2,) or (2, N).
    Returns a uint32 array of shape (4, N).
    """
    x0, x1, x2, x3 = (np.asarray(counter[j], dtype=np.uint32).copy() for j in range(4))
    k0 = np.asarray(key[0], dtype=np.uint32).copy()
    k1 = np.asarray(key[1], dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for r in range(ROUNDS):
            hi0, lo0 = _mulhilo(PHILOX_M0, x0)
            hi1, lo1 = _mulhilo(PHILOX_M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
            if r + 1 < ROUNDS:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
    return np.stack([x0, x1, x2, x3])


def seed_key(seed):
    """64-bit seed -> Philox key words (lo, hi)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)


def block_counters(block_index, stream_id):
    """Counters (b lo, b hi, stream_id, 0) for an array of 64-bit block indices."""
    b = np.asarray(block_index, dtype=np.uint64)
    lo = (b & _MASK32).astype(np.uint32)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    sid = np.broadcast_to(np.asarray(stream_id, dtype=np.uint64) & _MASK32, b.shape).astype(np.uint32)
    return np.stack([lo, hi, sid, np.zeros_like(lo)])


def word_to_unit(x):
    """uint32 word -> uniform in [0, 1 - 2^-24], exact in FP64: (x >> 8) * 2^-24."""
    return (np.asarray(x, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


def sample_words(seed, counter_base, stream_id, n):
    """The two 32-bit words (w1, w2) drawn by samples i = 0..n-1.

    Sample i has global index g = counter_base + i (mod 2^64) and reads block g >> 1.
    """
    g = (np.uint64(int(counter_base) & 0xFFFFFFFFFFFFFFFF) + np.arange(n, dtype=np.uint64))
    out = philox4x32_10(block_counters(g >> np.uint64(1), stream_id), seed_key(seed))
    odd = (g & np.uint64(1)).astype(bool)
    w1 = np.where(odd, out[2], out[0])
    w2 = np.where(odd, out[3], out[1])
    return w1, w2


def uniforms_at(seed, counter_base, stream_id, index):
    """(u1, u2) in FP64 of the samples with the given local indices (any order)."""
    g = np.uint64(int(counter_base) & 0xFFFFFFFFFFFFFFFF) + np.asarray(index, dtype=np.uint64)
    out = philox4x32_10(block_counters(g >> np.uint64(1), stream_id), seed_key(seed))
    odd = (g & np.uint64(1)).astype(bool)
    return word_to_unit(np.where(odd, out[2], out[0])), word_to_unit(np.where(odd, out[3], out[1]))


def sample_uniforms(seed, counter_base, stream_id, n):
    """(u1, u2) in FP64 for samples i = 0..n-1 (both exactly representable in FP32)."""
    w1, w2 = sample_words(seed, counter_base, stream_id, n)
    return word_to_unit(w1), word_to_unit(w2)
