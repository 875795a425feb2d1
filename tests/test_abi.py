"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every function that include/*.h declares, and
reject bad arguments on the host with the documented status codes before it
touches the GPU (so these calls are safe without one).
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(vndf_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2306_05044_gb300 import _build
    _build.build()
    import paper_2306_05044_gb300 as v
    return v.load()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("vndf_sample", "vndf_pdf", "vndf_rng_uniform", "vndf_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []


def test_binding_signatures_cover_header(lib):
    import paper_2306_05044_gb300 as v
    assert set(_declared()) <= set(v.SIGNATURES)


def test_status_strings(lib):
    import paper_2306_05044_gb300 as v
    assert v.status_string(0) == "ok"
    for code in range(-7, 0):
        assert v.status_string(code) not in ("ok", "unknown status")
    assert v.status_string(-99) == "unknown status"
    assert v.vndf_abi_version() == 3


FAKE = 0x10000  # 16-byte aligned host value; never dereferenced on the error paths


def _sample(lib, n=8, method=0, ptrs=None, u=(None, None), ay=FAKE):
    p = ptrs or [FAKE] * 3
    return lib.vndf_sample(n, p[0], p[1], p[2], FAKE, ay, u[0], u[1], 0, 0, 0, method,
                           FAKE, FAKE, FAKE, FAKE, None)


def test_sample_rejects_bad_arguments(lib):
    assert _sample(lib, n=-1) == -2
    assert _sample(lib, n=1 << 62) == -2
    assert _sample(lib, method=5) == -4
    assert _sample(lib, ptrs=[None, FAKE, FAKE]) == -1
    assert _sample(lib, ptrs=[FAKE + 2, FAKE, FAKE]) == -3
    assert _sample(lib, u=(FAKE, None)) == -7
    assert _sample(lib, n=0) == 0  # n = 0 is a no-op and launches nothing


def test_rng_and_pdf_reject_bad_arguments(lib):
    assert lib.vndf_rng_uniform(-3, 1, 0, 0, FAKE, FAKE, None) == -2
    assert lib.vndf_rng_uniform(4, 1, 0, 0, None, FAKE, None) == -1
    assert lib.vndf_rng_uniform(4, 1, 0, 0, FAKE + 1, FAKE, None) == -3
    assert lib.vndf_pdf(-1, FAKE, FAKE, FAKE, FAKE, None, FAKE, FAKE, FAKE, FAKE, None) == -2
    assert lib.vndf_pdf(4, FAKE, FAKE, FAKE, FAKE, None, FAKE, FAKE, FAKE, None, None) == -1
    assert lib.vndf_pdf(0, FAKE, FAKE, FAKE, FAKE, None, FAKE, FAKE, FAKE, FAKE, None) == 0


def test_extended_entry_points_reject_bad_arguments(lib):
    assert _sample(lib, method=3) == -4
    assert _sample(lib, method=2, n=-1) == -2
    assert _sample(lib, method=2, ptrs=[FAKE, None, FAKE]) == -1
    assert lib.vndf_pdf_extended(-1, FAKE, FAKE, FAKE, FAKE, None, FAKE, FAKE, FAKE, FAKE, None) == -2
    assert lib.vndf_pdf_extended(4, FAKE, FAKE, FAKE, None, None, FAKE, FAKE, FAKE, FAKE, None) == -1
    assert lib.vndf_pdf_extended(4, FAKE, FAKE, FAKE + 2, FAKE, None, FAKE, FAKE, FAKE, FAKE, None) == -3
    hemi = lambda n, wx=FAKE, u1=None, u2=None, mx=FAKE: lib.vndf_sample_hemisphere(  # noqa: E731
        n, wx, FAKE, FAKE, u1, u2, 0, 0, 0, mx, FAKE, FAKE, FAKE, None)
    assert hemi(-1) == -2
    assert hemi(1 << 62) == -2
    assert hemi(4, wx=None) == -1
    assert hemi(4, mx=None) == -1
    assert hemi(4, u1=FAKE) == -7
    assert hemi(4, wx=FAKE + 1) == -3
    assert hemi(0, wx=None) == 0


def test_binding_fails_loudly_without_gpu_tensors(lib):
    import torch

    import paper_2306_05044_gb300 as v
    x = torch.zeros(8)
    with pytest.raises(ValueError):
        v.vndf_sample(x, x, x, x)


def test_albedo_rejects_bad_arguments(lib):
    ws_need = lib.vndf_albedo_workspace_bytes(16, 1000)
    assert ws_need > 0
    assert lib.vndf_albedo_workspace_bytes(0, 1000) == 0
    args = lambda nq, ws, wsb, cfg=None, mx=1000: (nq, FAKE, FAKE, FAKE, FAKE, None, FAKE, mx, 0.04, 1, 0, 0,  # noqa: E731
                                                   FAKE, ws, wsb, cfg, None)
    assert lib.vndf_albedo_batched(*args(0, None, 0)) == 0
    assert lib.vndf_albedo_batched(*args(-1, FAKE, ws_need)) == -2
    assert lib.vndf_albedo_batched(*args(16, None, ws_need)) == -5
    assert lib.vndf_albedo_batched(*args(16, FAKE, ws_need - 1)) == -5
    assert lib.vndf_albedo_batched(*args(16, FAKE + 16, ws_need)) == -3  # workspace not 256-byte aligned
    import ctypes
    bad = (ctypes.c_int32 * 3)(0, 1, 1)
    assert lib.vndf_albedo_batched(*args(16, FAKE, ws_need, bad)) == -7
