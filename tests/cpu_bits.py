"""Inputs and digests for the cross-ISA check of the host sampler (vndf_cpu_sample).

The host sampler's FP32 path is built with -ffp-contract=off and every fused
multiply-add written as an explicit std::fma, so with IEEE square roots and
divides it must give the same bits on x86-64 (scalar; fma is a library call)
and on AArch64 (vectorised NEON).  This module draws a fixed input set with
integer Philox words and IEEE float32 additions and multiplications only, so
the inputs themselves are bit-identical on every host, and hashes the
sampler's outputs.  The record in tests/host_bits/ holds the digests of the
x86-64 build; it is not a parity reference (parity is checked against the
FP64 oracle in tests/test_cpu_sampler.py), only a record of one ISA's bits
against which the other's are compared.
"""
import hashlib
import os

import numpy as np

from oracle import philox

RECORD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_bits", "cpu_sampler_x86_64.txt")
N = (1 << 16) + 3
CASES = (("cap", 0), ("cap_extended", 0), ("polar", 0))


def _unit(words):
    """uint32 words -> float32 in [0, 1 - 2^-24], exact."""
    return ((words >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)


def inputs(extended):
    """wi with components in [-1, 1) (z in (0, 1] above the horizon, else [-1, 1)), alpha in [1e-3, 1 + 1e-3),
    u on the 2^-24 grid; every value formed from Philox words by exact or single IEEE float32 operations."""
    f32 = np.float32
    a1, a2 = philox.sample_words(101, 0, 0, N)
    b1, b2 = philox.sample_words(101, 0, 1, N)
    c1, c2 = philox.sample_words(101, 0, 2, N)
    two, one, eps = f32(2), f32(1), f32(2.0 ** -24)
    wx = _unit(a1) * two - one
    wy = _unit(a2) * two - one
    wz = _unit(b1) * two - one if extended else _unit(b1) + eps
    ax = _unit(b2) + f32(1e-3)
    ay = _unit(c1) + f32(1e-3)
    u1, u2 = _unit(c2), _unit(philox.sample_words(101, 0, 3, N)[0])
    return [np.ascontiguousarray(t, dtype=np.float32) for t in (wx, wy, wz, ax, ay, u1, u2)]


def digest(arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<f4").tobytes())
    return h.hexdigest()


def current(vndf):
    """{"inputs_upper": ..., "inputs_extended": ..., "<method>": ...} for this host's build."""
    out = {"inputs_upper": digest(inputs(False)), "inputs_extended": digest(inputs(True))}
    for method, precise in CASES:
        x = inputs(method == "cap_extended")
        out[method] = digest(vndf.vndf_cpu_sample(*x, method=method, precise=bool(precise), threads=4))
    return out


def read_record():
    with open(RECORD) as fh:
        return dict(line.split()[:2] for line in fh if line.strip() and not line.startswith("#"))
