"""Python binding of libvndf: spherical-cap GGX visible-normal sampling on GB300.

Dupuy & Benyoub, "Sampling Visible GGX Normals with Spherical Caps" (HPG 2023).
The functions here carry the names of the C entry points declared in
``include/vndf.h`` and only marshal arguments: they check tensor placement and
dtype, allocate outputs with torch when none are given, pass raw device
pointers and the current CUDA stream, and turn a negative status into
``VndfError``.  Every step of the computation runs in libvndf's CUDA kernels;
there is no fallback.  Importing works without a GPU, but every call needs
the compiled library (``__graft_entry__.build()``) and a CUDA device.
"""
import ctypes
import os

import torch

_PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG_DIR, "libvndf.so")

METHODS = {"cap": 0, "spherical_cap": 0, "polar": 1, "polar_disk": 1, "cap_extended": 2,
           "spherical_cap_extended": 2}

VNDF_OK = 0
_P = ctypes.c_void_p
_F = ctypes.c_float
_I32 = ctypes.c_int32
_U32 = ctypes.c_uint32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/vndf.h
SIGNATURES = {
    "vndf_abi_version": (ctypes.c_int, []),
    "vndf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "vndf_pointer_device_accessible": (ctypes.c_int, [_P]),
    "vndf_rng_uniform": (ctypes.c_int, [_I64, _U64, _U64, _U32, _P, _P, _P]),
    "vndf_sample": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _U64, _U64, _U32, ctypes.c_int,
                                   _P, _P, _P, _P, _P]),
    "vndf_rescue_count": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _U64, _U64, _U32, ctypes.c_int, _P, _P]),
    "vndf_pdf": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vndf_pdf_extended": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vndf_sample_hemisphere": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _U64, _U64, _U32, _P, _P, _P, _P, _P]),
    "vndf_sample_reflection": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _U64, _U64, _U32, _F,
                                              _P, _P, _P, _P, _P, _P]),
    "vndf_sample_backward": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _U64, _U64, _U32,
                                            _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vndf_sample_backward_extended": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _U64, _U64, _U32,
                                            _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "vndf_loss_workspace_bytes": (_SZ, [_I64]),
    "vndf_sample_loss_backward": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _U64, _U64, _U32,
                                                 _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "vndf_albedo_workspace_bytes": (_SZ, [_I32, _I32]),
    "vndf_albedo_batched": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, _P, _I32, _F, _U64, _U64, _U32, _P, _P, _SZ,
                                           _P, _P]),
    "vndf_albedo_autotune": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, _P, _I32, _F, _U64, _U64, _U32, _P, _P, _SZ,
                                            _P, _P, _P]),
    "vndf_albedo_set_config": (ctypes.c_int, [_P]),
    "vndf_albedo_get_config": (ctypes.c_int, [_P]),
    "vndf_fit_workspace_bytes": (_SZ, [_I32]),
    "vndf_fit_step": (ctypes.c_int, [_I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _F, _F,
                                     _F, _F, _F, _F, _U64, _U64, _U32, _P, _P, _SZ, _P]),
    "vndf_microbench": (ctypes.c_int, [_I64, _I32, ctypes.c_int, ctypes.c_int, _U64, _P, _P]),
    "vndf_cpu_sample": (ctypes.c_int, [_I64, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                       ctypes.c_int]),
    "vndf_albedo_batched_noalloc": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, _P, _I32, _F, _U64, _U64, _U32, _P,
                                                   _P, _P]),
}


class VndfError(RuntimeError):
    """A libvndf entry point returned a negative status."""

    def __init__(self, func, status):
        self.status = status
        super().__init__(f"{func}: {status_string(status)} (status {status})")


_lib = None


def load():
    """Load libvndf.so (built in-tree) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvndf.so is not built at {LIB_PATH}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status):
    return load().vndf_status_string(int(status)).decode()


def vndf_abi_version():
    return load().vndf_abi_version()


def vndf_pointer_device_accessible(t):
    """True when the current CUDA device can dereference the tensor's memory (device, or mapped pinned host)."""
    st = load().vndf_pointer_device_accessible(t.data_ptr())
    if st < 0:
        raise VndfError("vndf_pointer_device_accessible", st)
    return st == 1


def _check(func, status):
    if status != VNDF_OK:
        raise VndfError(func, status)


def _ptr(t, name, dtype=torch.float32):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda and not (torch.cuda.is_available() and t.is_pinned() and vndf_pointer_device_accessible(t)):
        raise ValueError(f"{name} must live on a CUDA device (or in pinned host memory the device can address)")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream, device):
    if stream is None:
        stream = torch.cuda.current_stream(device if device.type == "cuda" else None)
    return ctypes.c_void_p(stream.cuda_stream)


def _out(t, n, like):
    """Output buffer: the given tensor, else device memory beside `like`, else pinned host memory when
    `like` itself is pinned host memory the device can address."""
    if t is not None:
        return t
    if like.is_cuda:
        return torch.empty(n, dtype=torch.float32, device=like.device)
    _ptr(like, "input")  # raises unless `like` is device-addressable pinned host memory
    return torch.empty(n, dtype=torch.float32, pin_memory=True)


def _method(method):
    if isinstance(method, int):
        return method
    try:
        return METHODS[method]
    except KeyError:
        raise ValueError(f"unknown method {method!r}") from None


def vndf_rng_uniform(n, seed, counter_base=0, stream_id=0, u1=None, u2=None, device=None, stream=None):
    """The (u1, u2) that vndf_sample draws in Philox mode for samples 0..n-1."""
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if u1 is None:
        u1 = torch.empty(n, dtype=torch.float32, device=device)
    if u2 is None:
        u2 = torch.empty(n, dtype=torch.float32, device=device)
    st = load().vndf_rng_uniform(int(n), int(seed) & (2**64 - 1), int(counter_base) & (2**64 - 1),
                                 int(stream_id) & 0xFFFFFFFF, _ptr(u1, "u1"), _ptr(u2, "u2"),
                                 _stream(stream, u1.device))
    _check("vndf_rng_uniform", st)
    return u1, u2


def vndf_sample(wi_x, wi_y, wi_z, alpha_x, alpha_y=None, u1=None, u2=None, seed=0, counter_base=0,
                stream_id=0, method="cap", wm_x=None, wm_y=None, wm_z=None, pdf=None, with_pdf=True,
                n=None, stream=None):
    """Sample wm (and its pdf) for every element; see vndf_sample in include/vndf.h.

    alpha_y=None means isotropic; u1=u2=None means in-kernel Philox with
    (seed, counter_base, stream_id).  Returns (wm_x, wm_y, wm_z, pdf or None).
    """
    n = wi_x.numel() if n is None else int(n)
    wm_x = _out(wm_x, n, wi_x)
    wm_y = _out(wm_y, n, wi_x)
    wm_z = _out(wm_z, n, wi_x)
    if with_pdf:
        pdf = _out(pdf, n, wi_x)
    else:
        pdf = None
    st = load().vndf_sample(
        n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(alpha_x, "alpha_x"),
        _ptr(alpha_y, "alpha_y"), _ptr(u1, "u1"), _ptr(u2, "u2"), int(seed) & (2**64 - 1),
        int(counter_base) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF, _method(method),
        _ptr(wm_x, "wm_x"), _ptr(wm_y, "wm_y"), _ptr(wm_z, "wm_z"), _ptr(pdf, "pdf"),
        _stream(stream, wi_x.device))
    _check("vndf_sample", st)
    return wm_x, wm_y, wm_z, pdf


def vndf_rescue_count(wi_x, wi_y, wi_z, alpha_x, alpha_y=None, u1=None, u2=None, seed=0, counter_base=0,
                      stream_id=0, method="cap", count=None, n=None, stream=None):
    """Number of samples vndf_sample recomputes in double-float for these arguments (a device int64 tensor of
    one element, or ``count`` if given); see vndf_rescue_count in include/vndf.h."""
    n = wi_x.numel() if n is None else int(n)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=wi_x.device)
    st = load().vndf_rescue_count(
        n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(alpha_x, "alpha_x"),
        _ptr(alpha_y, "alpha_y"), _ptr(u1, "u1"), _ptr(u2, "u2"), int(seed) & (2**64 - 1),
        int(counter_base) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF, _method(method),
        _ptr(count, "count", torch.int64), _stream(stream, wi_x.device))
    _check("vndf_rescue_count", st)
    return count


def vndf_sample_reflection(wi_x, wi_y, wi_z, alpha_x, alpha_y=None, u1=None, u2=None, seed=0, counter_base=0,
                           stream_id=0, f0=0.04, wo_x=None, wo_y=None, wo_z=None, pdf=None, weight=None,
                           with_pdf=True, with_weight=True, n=None, stream=None):
    """Reflected direction, its pdf and the BRDF weight per sample; see vndf_sample_reflection in include/vndf.h.

    Returns (wo_x, wo_y, wo_z, pdf or None, weight or None)."""
    n = wi_x.numel() if n is None else int(n)
    wo_x, wo_y, wo_z = (_out(t, n, wi_x) for t in (wo_x, wo_y, wo_z))
    pdf = _out(pdf, n, wi_x) if with_pdf else None
    weight = _out(weight, n, wi_x) if with_weight else None
    st = load().vndf_sample_reflection(
        n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(alpha_x, "alpha_x"),
        _ptr(alpha_y, "alpha_y"), _ptr(u1, "u1"), _ptr(u2, "u2"), int(seed) & (2**64 - 1),
        int(counter_base) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF, float(f0), _ptr(wo_x, "wo_x"),
        _ptr(wo_y, "wo_y"), _ptr(wo_z, "wo_z"), _ptr(pdf, "pdf"), _ptr(weight, "weight"),
        _stream(stream, wi_x.device))
    _check("vndf_sample_reflection", st)
    return wo_x, wo_y, wo_z, pdf, weight


def vndf_pdf(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf=None, n=None, stream=None,
             extended=False):
    """GGX VNDF density of the given normals; see vndf_pdf (and, with extended=True,
    vndf_pdf_extended) in include/vndf.h."""
    n = wi_x.numel() if n is None else int(n)
    pdf = _out(pdf, n, wi_x)
    name = "vndf_pdf_extended" if extended else "vndf_pdf"
    st = getattr(load(), name)(n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"),
                               _ptr(alpha_x, "alpha_x"), _ptr(alpha_y, "alpha_y"), _ptr(wm_x, "wm_x"),
                               _ptr(wm_y, "wm_y"), _ptr(wm_z, "wm_z"), _ptr(pdf, "pdf"),
                               _stream(stream, wi_x.device))
    _check(name, st)
    return pdf


def vndf_pdf_extended(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf=None, n=None, stream=None):
    """vndf_pdf on the extended domain (wi below the horizon too); see include/vndf.h."""
    return vndf_pdf(wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf, n, stream, extended=True)


def vndf_sample_hemisphere(wi_x, wi_y, wi_z, u1=None, u2=None, seed=0, counter_base=0, stream_id=0, wm_x=None,
                           wm_y=None, wm_z=None, pdf=None, with_pdf=True, n=None, stream=None):
    """Stand-alone hemisphere sampler (Sec. 3.3, normalised, Eq. 2 density); see include/vndf.h.

    Returns (wm_x, wm_y, wm_z, pdf or None)."""
    n = wi_x.numel() if n is None else int(n)
    wm_x, wm_y, wm_z = (_out(t, n, wi_x) for t in (wm_x, wm_y, wm_z))
    pdf = _out(pdf, n, wi_x) if with_pdf else None
    st = load().vndf_sample_hemisphere(
        n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(u1, "u1"), _ptr(u2, "u2"),
        int(seed) & (2**64 - 1), int(counter_base) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF,
        _ptr(wm_x, "wm_x"), _ptr(wm_y, "wm_y"), _ptr(wm_z, "wm_z"), _ptr(pdf, "pdf"), _stream(stream, wi_x.device))
    _check("vndf_sample_hemisphere", st)
    return wm_x, wm_y, wm_z, pdf


def vndf_sample_backward(wi_x, wi_y, wi_z, alpha_x, alpha_y=None, u1=None, u2=None, seed=0, counter_base=0,
                         stream_id=0, g_wm_x=None, g_wm_y=None, g_wm_z=None, g_pdf=None, want_wi=True,
                         want_alpha=True, n=None, stream=None, extended=False, outputs=None):
    """Gradients of (wm, pdf) w.r.t. (wi, alpha) for fixed u; see vndf_sample_backward (and, with
    extended=True, vndf_sample_backward_extended) in include/vndf.h.

    Returns (g_wi_x, g_wi_y, g_wi_z, g_alpha_x, g_alpha_y); entries not requested are None.
    With alpha_y=None (isotropic) g_alpha_x holds d/d alpha and g_alpha_y is None.  ``outputs`` may
    pass preallocated (g_wi_x, g_wi_y, g_wi_z, g_alpha_x, g_alpha_y); those not requested are ignored.
    """
    n = wi_x.numel() if n is None else int(n)
    given = list(outputs) if outputs is not None else [None] * 5
    g_wi = [_out(given[k], n, wi_x) for k in range(3)] if want_wi else [None, None, None]
    g_ax = _out(given[3], n, wi_x) if want_alpha else None
    g_ay = _out(given[4], n, wi_x) if (want_alpha and alpha_y is not None) else None
    name = "vndf_sample_backward_extended" if extended else "vndf_sample_backward"
    st = getattr(load(), name)(
        n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(alpha_x, "alpha_x"),
        _ptr(alpha_y, "alpha_y"), _ptr(u1, "u1"), _ptr(u2, "u2"), int(seed) & (2**64 - 1),
        int(counter_base) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF, _ptr(g_wm_x, "g_wm_x"),
        _ptr(g_wm_y, "g_wm_y"), _ptr(g_wm_z, "g_wm_z"), _ptr(g_pdf, "g_pdf"), _ptr(g_wi[0], "g_wi_x"),
        _ptr(g_wi[1], "g_wi_y"), _ptr(g_wi[2], "g_wi_z"), _ptr(g_ax, "g_alpha_x"), _ptr(g_ay, "g_alpha_y"),
        _stream(stream, wi_x.device))
    _check(name, st)
    return g_wi[0], g_wi[1], g_wi[2], g_ax, g_ay


def vndf_sample_backward_extended(*args, **kwargs):
    """vndf_sample_backward on the extended domain (wi below the horizon too); see include/vndf.h."""
    return vndf_sample_backward(*args, extended=True, **kwargs)


def vndf_loss_workspace_bytes(n):
    return int(load().vndf_loss_workspace_bytes(int(n)))


def vndf_sample_loss_backward(wi_x, wi_y, wi_z, alpha_x, alpha_y, c_x, c_y, c_z, u1=None, u2=None, seed=0,
                              counter_base=0, stream_id=0, workspace=None, outputs=None, n=None, stream=None):
    """Fused forward + loss + adjoint of loss = sum(c . wm + log pdf); returns (loss, g_wi_x, g_wi_y, g_wi_z,
    g_alpha_x, g_alpha_y).  ``outputs`` may pass preallocated (loss, g_wi_x, g_wi_y, g_wi_z, g_alpha_x,
    g_alpha_y); ``workspace`` a uint8 device tensor of at least vndf_loss_workspace_bytes(n) bytes."""
    n = wi_x.numel() if n is None else int(n)
    if outputs is None:
        outputs = (torch.empty(1, dtype=torch.float32, device=wi_x.device),
                   *(_out(None, n, wi_x) for _ in range(4)),
                   _out(None, n, wi_x) if alpha_y is not None else None)
    loss, gx, gy, gz, gax, gay = outputs
    need = vndf_loss_workspace_bytes(n)
    if workspace is None:
        workspace = torch.empty(max(need, 4), dtype=torch.uint8, device=wi_x.device)
    st = load().vndf_sample_loss_backward(
        n, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(alpha_x, "alpha_x"),
        _ptr(alpha_y, "alpha_y"), _ptr(c_x, "c_x"), _ptr(c_y, "c_y"), _ptr(c_z, "c_z"), _ptr(u1, "u1"),
        _ptr(u2, "u2"), int(seed) & (2**64 - 1), int(counter_base) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF,
        _ptr(gx, "g_wi_x"), _ptr(gy, "g_wi_y"), _ptr(gz, "g_wi_z"), _ptr(gax, "g_alpha_x"),
        _ptr(gay, "g_alpha_y"), _ptr(loss, "loss"), _ptr(workspace, "workspace", torch.uint8),
        int(workspace.numel()), _stream(stream, wi_x.device))
    _check("vndf_sample_loss_backward", st)
    return loss, gx, gy, gz, gax, gay


def vndf_albedo_workspace_bytes(n_queries, max_samples_per_query):
    return int(load().vndf_albedo_workspace_bytes(int(n_queries), int(max_samples_per_query)))


def _albedo_common(wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples_per_query, E, workspace):
    nq = wi_x.numel()
    if E is None:
        E = torch.empty(nq, dtype=torch.float32, device=wi_x.device)
    need = vndf_albedo_workspace_bytes(nq, max_samples_per_query)
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=wi_x.device)
    args = (nq, _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"), _ptr(alpha_x, "alpha_x"),
            _ptr(alpha_y, "alpha_y"), _ptr(n_samples, "n_samples", torch.int32), int(max_samples_per_query))
    return E, workspace, args


def vndf_albedo_batched(wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples_per_query=65536, f0=0.04,
                        seed=3, counter_base=0, stream_id=0, E=None, workspace=None, config=None, stream=None):
    """Per-query directional albedo; see vndf_albedo_batched in include/vndf.h.  config: None or
    (warps per CTA, groups per item, CTAs per SM)."""
    E, workspace, args = _albedo_common(wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples_per_query, E,
                                        workspace)
    cfg = None if config is None else (ctypes.c_int32 * 3)(*[int(c) for c in config])
    st = load().vndf_albedo_batched(*args, float(f0), int(seed) & (2**64 - 1), int(counter_base) & (2**64 - 1),
                                    int(stream_id) & 0xFFFFFFFF, _ptr(E, "E"), _ptr(workspace, "workspace",
                                                                                   torch.uint8),
                                    int(workspace.numel()), cfg, _stream(stream, wi_x.device))
    _check("vndf_albedo_batched", st)
    return E


def vndf_albedo_set_config(config):
    """Set (or, with None, reset) the launch configuration config=None albedo calls use on the current device."""
    cfg = None if config is None else (ctypes.c_int32 * 3)(*[int(c) for c in config])
    _check("vndf_albedo_set_config", load().vndf_albedo_set_config(cfg))


def vndf_albedo_get_config():
    """(configuration a config=None albedo call uses on the current device, whether it was set or tuned)."""
    cfg = (ctypes.c_int32 * 3)()
    st = load().vndf_albedo_get_config(cfg)
    if st < 0:
        raise VndfError("vndf_albedo_get_config", st)
    return tuple(cfg), st == 1


def tune_cache_key(device_name, sm_count, n_queries, max_samples_per_query):
    """Key of an albedo autotune result: the device (name and multiprocessor count) and the batch's size class
    (query count rounded up to a power of two, and the per-query bound)."""
    bucket = 1 << max(0, int(n_queries) - 1).bit_length()
    return f"{device_name}|sm{int(sm_count)}|nq{bucket}|max{int(max_samples_per_query)}"


def tune_cache_lookup(path, key):
    """The cached ((warps, groups, ctas), ms) for key, or None (missing or unreadable file, unknown key)."""
    import json
    try:
        with open(path) as fh:
            entry = json.load(fh).get(key)
    except (OSError, ValueError, AttributeError):
        return None
    if not entry:
        return None
    return tuple(int(c) for c in entry["config"]), float(entry["ms"])


def tune_cache_store(path, key, config, ms):
    """Add or replace key in the JSON cache file, written to a temporary file and renamed into place."""
    import json
    try:
        with open(path) as fh:
            data = json.load(fh)
        if not isinstance(data, dict):
            data = {}
    except (OSError, ValueError):
        data = {}
    data[key] = {"config": [int(c) for c in config], "ms": float(ms)}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def vndf_albedo_autotune(wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples_per_query=65536, f0=0.04,
                         seed=3, counter_base=0, stream_id=0, E=None, workspace=None, stream=None, cache=None):
    """Pick and remember the fastest albedo launch configuration; returns ((warps, groups, ctas), ms).

    With ``cache`` (a JSON file path), a configuration stored there for this device and batch size class is
    set without timing (vndf_albedo_set_config); otherwise the configurations are timed and the result is
    stored for the next process.  E is not computed on a cache hit."""
    key = None
    if cache is not None:
        props = torch.cuda.get_device_properties(wi_x.device)
        key = tune_cache_key(props.name, props.multi_processor_count, wi_x.numel(), max_samples_per_query)
        hit = tune_cache_lookup(cache, key)
        if hit is not None:
            with torch.cuda.device(wi_x.device):
                vndf_albedo_set_config(hit[0])
            return hit
    E, workspace, args = _albedo_common(wi_x, wi_y, wi_z, alpha_x, alpha_y, n_samples, max_samples_per_query, E,
                                        workspace)
    best = (ctypes.c_int32 * 3)()
    ms = ctypes.c_float()
    st = load().vndf_albedo_autotune(*args, float(f0), int(seed) & (2**64 - 1), int(counter_base) & (2**64 - 1),
                                     int(stream_id) & 0xFFFFFFFF, _ptr(E, "E"),
                                     _ptr(workspace, "workspace", torch.uint8), int(workspace.numel()), best,
                                     ctypes.byref(ms), _stream(stream, wi_x.device))
    _check("vndf_albedo_autotune", st)
    if key is not None:
        tune_cache_store(cache, key, tuple(best), ms.value)
    return tuple(best), ms.value


def vndf_fit_workspace_bytes(n_texels):
    return int(load().vndf_fit_workspace_bytes(int(n_texels)))


def vndf_fit_step(state, wi_x, wi_y, wi_z, target_x, target_y, target_z, samples_per_texel=1024, lr=1e-2,
                  beta1=0.9, beta2=0.999, eps=1e-8, alpha_min=1e-3, alpha_max=1.0, seed=5, counter_base=0,
                  stream_id=0, loss=None, workspace=None, stream=None, n_texels_total=0):
    """One fitting step in place; see vndf_fit_step in include/vndf.h.

    state: dict of device tensors alpha_x, alpha_y, m_x, m_y, v_x, v_y (float32, one per texel) and
    step (int64, one element).  n_texels_total: the whole map's texel count when these texels are a part
    of it (pass stream_id = the part's first texel); 0 means this call's count.  Returns the loss tensor
    (one float, before the update) or None.
    """
    nt = wi_x.numel()
    if workspace is None:
        workspace = torch.empty(max(vndf_fit_workspace_bytes(nt), 4), dtype=torch.uint8, device=wi_x.device)
    st = load().vndf_fit_step(
        nt, int(n_texels_total), int(samples_per_texel), _ptr(wi_x, "wi_x"), _ptr(wi_y, "wi_y"), _ptr(wi_z, "wi_z"),
        _ptr(target_x, "target_x"), _ptr(target_y, "target_y"), _ptr(target_z, "target_z"),
        _ptr(state["alpha_x"], "alpha_x"), _ptr(state["alpha_y"], "alpha_y"), _ptr(state["m_x"], "m_x"),
        _ptr(state["m_y"], "m_y"), _ptr(state["v_x"], "v_x"), _ptr(state["v_y"], "v_y"),
        _ptr(state["step"], "step", torch.int64), float(lr), float(beta1), float(beta2), float(eps),
        float(alpha_min), float(alpha_max), int(seed) & (2**64 - 1), int(counter_base) & (2**64 - 1),
        int(stream_id) & 0xFFFFFFFF, _ptr(loss, "loss"), _ptr(workspace, "workspace", torch.uint8),
        int(workspace.numel()), _stream(stream, wi_x.device))
    _check("vndf_fit_step", st)
    return loss


def fit_state(alpha_x, alpha_y):
    """Fresh optimiser state for vndf_fit_step (copies of the initial maps, zero moments, step 0)."""
    z = torch.zeros_like(alpha_x)
    return {"alpha_x": alpha_x.clone(), "alpha_y": alpha_y.clone(), "m_x": z.clone(), "m_y": z.clone(),
            "v_x": z.clone(), "v_y": z.clone(),
            "step": torch.zeros(1, dtype=torch.int64, device=alpha_x.device)}


def vndf_microbench(lanes, samples_per_lane=64, method="cap", seed=1, sums=None, precise=True, device=None,
                    stream=None):
    """The paper's 64-samples-per-lane protocol; returns the (lanes, 4) sums tensor."""
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    if sums is None:
        sums = torch.empty(lanes, 4, dtype=torch.float32, device=device)
    st = load().vndf_microbench(int(lanes), int(samples_per_lane), _method(method), int(bool(precise)),
                                int(seed) & (2**64 - 1),
                                _ptr(sums, "sums"), _stream(stream, sums.device))
    _check("vndf_microbench", st)
    return sums


def vndf_cpu_sample(wi_x, wi_y, wi_z, alpha_x, alpha_y, u1, u2, method="cap", with_pdf=True, threads=0,
                    out=None, precise=False):
    """Host-CPU sampler on numpy float32 arrays; see vndf_cpu_sample in include/vndf.h.

    ``out`` optionally gives preallocated contiguous float32 outputs (wm_x, wm_y, wm_z, pdf).
    Returns (wm_x, wm_y, wm_z, pdf or None) as numpy arrays."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (wi_x, wi_y, wi_z, alpha_x)]
    ay = None if alpha_y is None else np.ascontiguousarray(alpha_y, dtype=np.float32)
    us = [np.ascontiguousarray(a, dtype=np.float32) for a in (u1, u2)]
    n = arrs[0].size
    if out is None:
        out = [np.empty(n, dtype=np.float32) for _ in range(4 if with_pdf else 3)]
    else:
        out = list(out)[:4 if with_pdf else 3]
        for o in out:
            if o.dtype != np.float32 or not o.flags.c_contiguous or o.size != n:
                raise ValueError("vndf_cpu_sample: outputs must be contiguous float32 arrays of the input size")
    p = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    st = load().vndf_cpu_sample(n, *(p(a) for a in arrs), p(ay), p(us[0]), p(us[1]), _method(method),
                                int(bool(precise)), p(out[0]), p(out[1]), p(out[2]), p(out[3]) if with_pdf else None,
                                int(threads))
    _check("vndf_cpu_sample", st)
    return out[0], out[1], out[2], (out[3] if with_pdf else None)
