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
    E = FAKE + 0x100  # the output must not alias the inputs
    args = lambda nq, ws, wsb, cfg=None, mx=1000: (nq, FAKE, FAKE, FAKE, FAKE, None, FAKE, mx, 0.04, 1, 0, 0,  # noqa: E731
                                                   E, ws, wsb, cfg, None)
    assert lib.vndf_albedo_batched(*args(0, None, 0)) == 0
    assert lib.vndf_albedo_batched(*args(-1, FAKE, ws_need)) == -2
    assert lib.vndf_albedo_batched(*args(16, None, ws_need)) == -5
    assert lib.vndf_albedo_batched(*args(16, FAKE, ws_need - 1)) == -5
    assert lib.vndf_albedo_batched(*args(16, FAKE + 16, ws_need)) == -3  # workspace not 256-byte aligned
    import ctypes
    bad = (ctypes.c_int32 * 3)(0, 1, 1)
    assert lib.vndf_albedo_batched(*args(16, FAKE, ws_need, bad)) == -7


def _ptrs(k):
    """k distinct, 16-byte aligned fake addresses (never dereferenced: every call below returns before it
    touches the GPU)."""
    return [FAKE + 0x1000 * (j + 1) for j in range(k)]


no_gpu = pytest.mark.skipif(__import__("torch").cuda.is_available(),
                            reason="valid-looking fake pointers must never reach a launch on a GPU machine")


def _entry_calls(lib):
    """One call per GPU entry point, every pointer distinct and aligned, so that only an injected fault (or the
    missing device) can stop it; name -> (thunk, takes a workspace)."""
    p = _ptrs(40)
    ws_loss = lib.vndf_loss_workspace_bytes(64)
    ws_alb = lib.vndf_albedo_workspace_bytes(16, 1000)
    ws_fit = lib.vndf_fit_workspace_bytes(16)
    cfg = (ctypes.c_int32 * 3)(8, 1, 8)
    return {
        "vndf_rng_uniform": (lambda: lib.vndf_rng_uniform(64, 1, 0, 0, p[0], p[1], None), False),
        "vndf_sample": (lambda: lib.vndf_sample(64, p[0], p[1], p[2], p[3], p[4], None, None, 0, 0, 0, 0,
                                                p[5], p[6], p[7], p[8], None), False),
        "vndf_pdf": (lambda: lib.vndf_pdf(64, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8], None), False),
        "vndf_pdf_extended": (lambda: lib.vndf_pdf_extended(64, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7],
                                                            p[8], None), False),
        "vndf_sample_reflection": (lambda: lib.vndf_sample_reflection(64, p[0], p[1], p[2], p[3], p[4], None, None,
                                                                      0, 0, 0, 0.04, p[5], p[6], p[7], p[8], p[9],
                                                                      None), False),
        "vndf_sample_hemisphere": (lambda: lib.vndf_sample_hemisphere(64, p[0], p[1], p[2], None, None, 0, 0, 0,
                                                                      p[5], p[6], p[7], p[8], None), False),
        "vndf_sample_backward": (lambda: lib.vndf_sample_backward(64, p[0], p[1], p[2], p[3], p[4], None, None, 0, 0,
                                                                  0, p[5], p[6], p[7], p[8], p[9], p[10], p[11],
                                                                  p[12], p[13], None), False),
        "vndf_sample_backward_extended": (lambda: lib.vndf_sample_backward_extended(
            64, p[0], p[1], p[2], p[3], p[4], None, None, 0, 0, 0, p[5], p[6], p[7], p[8], p[9], p[10], p[11],
            p[12], p[13], None), False),
        "vndf_sample_loss_backward": (lambda: lib.vndf_sample_loss_backward(
            64, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], None, None, 0, 0, 0, p[9], p[10], p[11], p[12],
            p[13], p[14], p[15], ws_loss, None), True),
        "vndf_albedo_batched": (lambda: lib.vndf_albedo_batched(16, p[0], p[1], p[2], p[3], None, p[4], 1000, 0.04,
                                                                1, 0, 0, p[5], p[6], ws_alb, cfg, None), True),
        "vndf_albedo_batched_noalloc": (lambda: lib.vndf_albedo_batched_noalloc(
            16, p[0], p[1], p[2], p[3], None, p[4], 1000, 0.04, 1, 0, 0, p[5], cfg, None), False),
        "vndf_fit_step": (lambda: lib.vndf_fit_step(16, 0, 64, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8],
                                                    p[9], p[10], p[11], p[12], 1e-2, 0.9, 0.999, 1e-8, 1e-3, 1.0,
                                                    1, 0, 0, p[13], p[14], ws_fit, None), True),
        "vndf_microbench": (lambda: lib.vndf_microbench(64, 8, 0, 0, 1, p[0], None), False),
        "vndf_rescue_count": (lambda: lib.vndf_rescue_count(64, p[0], p[1], p[2], p[3], p[4], None, None, 0, 0, 0, 0,
                                                            p[5], None), False),
        "vndf_albedo_set_config": (lambda: lib.vndf_albedo_set_config(cfg), False),
    }


@no_gpu
def test_injected_faults_return_their_status_before_any_launch(lib, monkeypatch):
    """VNDF_FAULT makes every GPU entry point return the injected status after its argument checks and
    before it enqueues work (host-side injection; no GPU is made to fail)."""
    calls = _entry_calls(lib)
    for kind, status in (("launch", -6), ("align", -3)):
        monkeypatch.setenv("VNDF_FAULT", kind)
        for name, (call, _) in calls.items():
            assert call() == status, (kind, name)
    monkeypatch.setenv("VNDF_FAULT", "workspace")
    for name, (call, takes_ws) in calls.items():
        if takes_ws:
            assert call() == -5, name
    # a named entry point only: the others go on to the device query, which fails here (no GPU)
    monkeypatch.setenv("VNDF_FAULT", "align@vndf_pdf")
    assert calls["vndf_pdf"][0]() == -3
    assert calls["vndf_pdf_extended"][0]() == -6
    # argument errors still come first
    monkeypatch.setenv("VNDF_FAULT", "launch")
    assert lib.vndf_pdf(-1, *_ptrs(9), None) == -2
    assert lib.vndf_pdf(4, *_ptrs(8), None, None) == -1


@no_gpu
def test_missing_device_is_a_cuda_error_not_an_assumed_part(lib, monkeypatch):
    """Without a device the multiprocessor count cannot be queried: every GPU entry point returns
    VNDF_ERR_CUDA instead of sizing its grid for an assumed part (no launch is attempted)."""
    monkeypatch.delenv("VNDF_FAULT", raising=False)
    for name, (call, _) in _entry_calls(lib).items():
        assert call() == -6, name


def test_outputs_aliasing_inputs_are_rejected(lib):
    """An output pointer equal to an input pointer or to another output is VNDF_ERR_ARG (checked on the host
    before anything is enqueued)."""
    p = _ptrs(20)
    wi = p[0:3]
    assert lib.vndf_sample(64, *wi, p[3], p[4], None, None, 0, 0, 0, 0, wi[0], p[6], p[7], p[8], None) == -7
    assert lib.vndf_sample(64, *wi, p[3], p[4], p[9], p[10], 0, 0, 0, 0, p[5], p[6], p[7], p[10], None) == -7
    assert lib.vndf_sample(64, *wi, p[3], p[4], None, None, 0, 0, 0, 0, p[5], p[5], p[7], p[8], None) == -7
    assert lib.vndf_sample(64, *wi, p[3], p[4], None, None, 0, 0, 0, 2, p[5], p[6], p[7], p[3], None) == -7
    assert lib.vndf_rng_uniform(64, 1, 0, 0, p[0], p[0], None) == -7
    assert lib.vndf_pdf(64, *wi, p[3], p[4], p[5], p[6], p[7], p[7], None) == -7
    assert lib.vndf_pdf_extended(64, *wi, p[3], None, p[5], p[6], p[7], wi[2], None) == -7
    assert lib.vndf_sample_reflection(64, *wi, p[3], p[4], None, None, 0, 0, 0, 0.04, p[5], p[6], p[7], p[8],
                                      p[4], None) == -7
    assert lib.vndf_sample_hemisphere(64, *wi, None, None, 0, 0, 0, p[5], p[6], wi[1], p[8], None) == -7
    assert lib.vndf_sample_backward(64, *wi, p[3], p[4], None, None, 0, 0, 0, p[5], p[6], p[7], p[8], p[9],
                                    p[10], p[11], p[3], p[13], None) == -7
    assert lib.vndf_sample_backward_extended(64, *wi, p[3], p[4], None, None, 0, 0, 0, p[5], p[6], p[7], p[8],
                                             p[9], p[10], p[11], p[12], p[5], None) == -7
    ws = lib.vndf_loss_workspace_bytes(64)
    assert lib.vndf_sample_loss_backward(64, *wi, p[3], p[4], p[5], p[6], p[7], None, None, 0, 0, 0, p[9],
                                         p[10], p[11], p[12], p[13], p[13], p[15], ws, None) == -7
    wsa = lib.vndf_albedo_workspace_bytes(16, 1000)
    assert lib.vndf_albedo_batched(16, *wi, p[3], None, p[4], 1000, 0.04, 1, 0, 0, wi[0], p[6], wsa, None,
                                   None) == -7
    assert lib.vndf_albedo_batched(16, *wi, p[3], None, p[4], 1000, 0.04, 1, 0, 0, p[5], p[5], wsa, None,
                                   None) == -7
    wsf = lib.vndf_fit_workspace_bytes(16)
    assert lib.vndf_fit_step(16, 0, 64, *wi, p[3], p[4], p[5], p[6], p[7], p[8], p[6], p[10], p[11], p[12], 1e-2,
                             0.9, 0.999, 1e-8, 1e-3, 1.0, 1, 0, 0, p[13], p[14], wsf, None) == -7
    assert lib.vndf_fit_step(16, 0, 64, *wi, p[3], p[4], p[5], p[0], p[7], p[8], p[9], p[10], p[11], p[12], 1e-2,
                             0.9, 0.999, 1e-8, 1e-3, 1.0, 1, 0, 0, p[13], p[14], wsf, None) == -7
    assert lib.vndf_cpu_sample(64, *wi, p[3], p[4], p[5], p[6], 0, 0, p[7], p[8], p[6], None, 1) == -7


def test_albedo_batches_past_int32_group_indices_are_rejected(lib):
    """Work items and their offsets are int32: a batch whose group slots (n_queries x ceil(max / 256)) reach
    2^31 is a size error, and its workspace size is reported as 0."""
    big = 1 << 30  # 2^22 groups per query
    assert lib.vndf_albedo_workspace_bytes(511, big) > 0
    assert lib.vndf_albedo_workspace_bytes(512, big) == 0
    p = _ptrs(8)
    args = lambda nq, ws, wsb: (nq, p[0], p[1], p[2], p[3], None, p[4], big, 0.04, 1, 0, 0, p[5], ws, wsb,  # noqa: E731
                                None, None)
    assert lib.vndf_albedo_batched(*args(512, p[6], 1 << 62)) == -2
    assert lib.vndf_albedo_batched_noalloc(512, p[0], p[1], p[2], p[3], None, p[4], big, 0.04, 1, 0, 0, p[5],
                                           None, None) == -2
    assert lib.vndf_albedo_batched_noalloc(16, p[0], p[1], p[2], p[3], None, p[4], big, 0.04, 1, 0, 0, p[5],
                                           None, None) == -2  # beyond the fixed scratch array


def test_rescue_count_rejects_bad_arguments(lib):
    p = _ptrs(8)
    call = lambda n=64, wx=p[0], method=0, count=p[5], u=(None, None): lib.vndf_rescue_count(  # noqa: E731
        n, wx, p[1], p[2], p[3], p[4], u[0], u[1], 0, 0, 0, method, count, None)
    assert call(n=-1) == -2
    assert call(method=9) == -4
    assert call(count=None) == -1
    assert call(count=p[5] + 4) == -3
    assert call(wx=None) == -1
    assert call(u=(p[6], None)) == -7
    assert call(count=p[0]) == -7  # the count aliases an input
