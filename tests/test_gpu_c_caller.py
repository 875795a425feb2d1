"""The C ABI used from a plain C program (no Python, no torch on the calling side).

tests/c_caller/vndf_c_caller.c allocates device buffers with the CUDA runtime,
calls vndf_sample (in-kernel Philox, fused density) and vndf_pdf, checks the
documented argument errors, and writes inputs and outputs to a file; this test
compiles it against include/vndf.h and libvndf.so, runs it, and compares its
results with the FP64 oracle at the tolerances of tests/parity.py.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

import parity
from oracle import philox

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def caller(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path_factory.mktemp("c_caller") / "vndf_c_caller")
    lib_dir = os.path.join(ROOT, "paper_2306_05044_gb300")
    cmd = [nvcc, "-x", "c++", os.path.join(ROOT, "tests", "c_caller", "vndf_c_caller.c"), "-o", exe,
           "-I", os.path.join(ROOT, "include"), "-L", lib_dir, "-lvndf", "-Xlinker", f"-rpath={lib_dir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_caller_matches_the_oracle(caller, tmp_path):
    n = (1 << 18) + 3
    out = str(tmp_path / "samples.bin")
    r = subprocess.run([caller, str(n), out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    raw = open(out, "rb").read()
    assert int(np.frombuffer(raw[:8], "<i8")[0]) == n
    a = np.frombuffer(raw[8:], "<f4").reshape(10, n)
    wi, ax, ay, wm, pdf, pdf2 = a[0:3], a[3], a[4], a[5:8], a[8], a[9]
    u1, u2 = philox.sample_uniforms(7, 3, 1, n)  # seed 7, counter base 3, stream 1 as in the C program
    st = parity.compare_cap(wm, pdf, u1, u2, wi, ax, ay, strict=True)
    print("C caller:", st)
    assert st["tail_angle_frac"] == 0.0 and st["tail_pdf_frac"] == 0.0
    # the density of the sampled normals, recomputed from the FP32 normals, agrees with the fused one to the
    # precision FP32 normals allow (about angle error x 4 / alpha)
    rel = np.abs(pdf2.astype(np.float64) / pdf - 1)
    assert np.median(rel) < 1e-5
