"""Pins for the oracle's Philox4x32-10 and its u-mapping.

The generator itself is checked against NVIDIA's cuRAND host-side
Philox4x32-10 generator (a separate implementation of the same published
algorithm, run as a library on the CPU).  cuRAND's host generator lays its
output out as word k = 4 * (65536 * x0 + s) + j of block (x0, 0, s, 0), so
comparing against it exercises the round function, the key schedule, the key
words and counter words 0, 1 and 2.  Counter word 3 is always 0 in this
project's layout.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

from oracle import philox

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("offset", [0, 4 * 65536 * 3 + 4 * 17, (1 << 50), (7 << 50) + 4 * 65000])
def test_philox_matches_curand_host_generator(seed, offset):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    n = 4096
    ref = _curand_words(lib, seed, offset, n)
    k = offset + np.arange(n, dtype=np.uint64)
    blk = k // np.uint64(4)
    x0_full = blk // np.uint64(65536)
    ctr = np.stack([(x0_full & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                    (x0_full >> np.uint64(32)).astype(np.uint32),
                    (blk % np.uint64(65536)).astype(np.uint32),
                    np.zeros(n, np.uint32)])
    out = philox.philox4x32_10(ctr, philox.seed_key(seed))
    word = (k % np.uint64(4)).astype(np.int64)
    mine = out[word, np.arange(n)]
    np.testing.assert_array_equal(mine, ref)


def test_uniforms_exact_in_fp32_and_in_range():
    u1, u2 = philox.sample_uniforms(7, 0, 3, 1 << 16)
    for u in (u1, u2):
        assert np.all(u.astype(np.float32).astype(np.float64) == u)
        assert u.min() >= 0.0 and u.max() <= 1.0 - 2.0 ** -24


def test_uniform_mapping_extremes():
    assert philox.word_to_unit(np.uint32(0)) == 0.0
    assert philox.word_to_unit(np.uint32(0xFFFFFFFF)) == 1.0 - 2.0 ** -24
    assert philox.word_to_unit(np.uint32(0x80000000)) == 0.5


@pytest.mark.parametrize("base", [0, 1, 2, 3, (1 << 32) - 1, (1 << 64) - 5])
def test_stream_is_a_function_of_global_index(base):
    """Shifting the counter base by k shifts the sample stream by k samples."""
    n = 257
    a1, a2 = philox.sample_uniforms(99, base, 5, n + 8)
    for k in (1, 2, 3, 8):
        b1, b2 = philox.sample_uniforms(99, (base + k) % (1 << 64), 5, n)
        np.testing.assert_array_equal(a1[k:k + n], b1)
        np.testing.assert_array_equal(a2[k:k + n], b2)


def test_pair_words_are_distinct_and_streams_differ():
    w1, w2 = philox.sample_words(1, 0, 0, 1 << 14)
    assert np.all(w1[0::2] != w1[1::2])
    assert np.all(w2[0::2] != w2[1::2])
    v1, _ = philox.sample_words(1, 0, 1, 1 << 14)
    assert np.mean(v1 == w1) < 1e-3


def test_uniforms_statistically_uniform():
    from scipy import stats
    u1, u2 = philox.sample_uniforms(2024, 0, 0, 1 << 17)
    assert stats.kstest(u1, "uniform").pvalue > 1e-3
    assert stats.kstest(u2, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(u1, u2)[0, 1]) < 0.02


def test_uniforms_at_matches_contiguous_stream():
    a1, a2 = philox.sample_uniforms(5, 3, 9, 1000)
    idx = np.array([0, 1, 2, 17, 500, 999, 998])
    b1, b2 = philox.uniforms_at(5, 3, 9, idx)
    np.testing.assert_array_equal(a1[idx], b1)
    np.testing.assert_array_equal(a2[idx], b2)
