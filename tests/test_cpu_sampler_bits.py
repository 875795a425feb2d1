"""The host sampler's FP32 path gives the same bits on x86-64 and on AArch64.

The library is built with -ffp-contract=off and writes every fused
multiply-add explicitly, so the x86-64 build (scalar, fma by library call) and
the AArch64 build (NEON vector loop) must agree bit for bit.  The digests of
the x86-64 build's outputs on fixed, ISA-independent inputs are recorded in
tests/host_bits/ (a record of bits, not a parity reference); this test
recomputes them with the build of the host it runs on.  It runs in the CPU
suite and, marked gpu, on the GPU's host, which is where the paper's CPU
protocol is timed.
"""
import platform

import pytest

import cpu_bits


@pytest.fixture(scope="module")
def v():
    from paper_2306_05044_gb300 import _build
    _build.build()
    import paper_2306_05044_gb300 as lib
    lib.load()
    return lib


@pytest.mark.parametrize("suite", ["cpu", pytest.param("gpu_host", marks=pytest.mark.gpu)])
def test_host_sampler_bits_match_the_x86_64_record(v, suite):
    rec = cpu_bits.read_record()
    got = cpu_bits.current(v)
    # the inputs are formed by integer Philox and single IEEE float32 operations: the same on every host
    assert got["inputs_upper"] == rec["inputs_upper"]
    assert got["inputs_extended"] == rec["inputs_extended"]
    diff = [m for m, _ in cpu_bits.CASES if got[m] != rec[m]]
    assert diff == [], f"{platform.machine()} build differs from the x86-64 record for {diff}"
