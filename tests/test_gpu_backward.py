"""GPU parity of the adjoint kernels against the oracle's complex-step derivatives.

The reference gradient is the oracle's vector-Jacobian product (oracle.grad,
complex step through Sec. 2 / Sec. 3.3 / Eq. 1 in FP64), pinned against
central differences on the CPU; one test also takes FP64 central differences of
the oracle's forward map as the reference directly.  Per sample the error is measured against the
largest reference component, e = max_k |g_k - r_k| / max_k |r_k|.  Like the
forward, the adjoint inherits the conditioning of h = c + i, so a small tail
of ill-conditioned samples is reported rather than bounded by a flat limit.
"""
import numpy as np
import pytest
import torch

import parity
import workloads
from oracle import grad, philox, vndf as ovndf

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _errors(gpu, ref):
    scale = np.abs(ref).max(axis=0)
    return np.abs(gpu - ref).max(axis=0) / np.maximum(scale, 1e-30)


def _check_errors(e, label):
    print(f"{label}: median {np.median(e):.2e} p99.9 {np.quantile(e, 0.999):.2e} max {e.max():.2e} "
          f"frac>1e-3 {(e > 1e-3).mean():.2e}")
    assert np.median(e) < 1e-5
    assert np.quantile(e, 0.999) < 1e-3


@pytest.mark.parametrize("iso,explicit", [(False, False), (True, False), (False, True)])
def test_backward_matches_complex_step(v, iso, explicit):
    n = (1 << 16) + 3
    d = workloads.adjoint_2e24(n=n, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(9)
    gwm = [torch.randn(n, generator=g, device=DEV) for _ in range(3)]
    gp = torch.randn(n, generator=g, device=DEV)
    ay = None if iso else d["alpha_y"]
    if explicit:
        u1n, u2n = philox.sample_uniforms(123, 0, 0, n)
        u1 = torch.as_tensor(u1n.astype(np.float32), device=DEV)
        u2 = torch.as_tensor(u2n.astype(np.float32), device=DEV)
        kw = dict(u1=u1, u2=u2)
    else:
        u1n, u2n = philox.sample_uniforms(4, 5, 0, n)
        kw = dict(seed=4, counter_base=5)
    gx, gy, gz, gax, gay = v.vndf_sample_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], ay,
                                                  g_wm_x=gwm[0], g_wm_y=gwm[1], g_wm_z=gwm[2], g_pdf=gp, **kw)
    wi = np.stack([_np(d[k]) for k in ("wi_x", "wi_y", "wi_z")])
    axn = _np(d["alpha_x"])
    ayn = axn if iso else _np(d["alpha_y"])
    rwi, rax, ray = grad.vjp(u1n, u2n, wi, axn, ayn, np.stack([_np(t) for t in gwm]), _np(gp), isotropic=iso)
    if iso:
        ref = np.concatenate([rwi, rax[None]])
        got = np.stack([_np(gx), _np(gy), _np(gz), _np(gax)])
        assert gay is None
    else:
        ref = np.concatenate([rwi, rax[None], ray[None]])
        got = np.stack([_np(gx), _np(gy), _np(gz), _np(gax), _np(gay)])
    _check_errors(_errors(got, ref), f"backward iso={iso} explicit={explicit}")
    # the sampler is invariant to the scale of wi
    gw = got[:3]
    hom = np.abs((gw * wi).sum(0)) / (np.sqrt((gw ** 2).sum(0)) * np.sqrt((wi ** 2).sum(0)) + 1e-30)
    assert np.quantile(hom, 0.999) < 1e-3


@pytest.mark.parametrize("ext", [False, True])
def test_backward_matches_central_differences(v, ext):
    """The adjoint against FP64 central finite differences of the oracle's forward map, a referee
    independent of the complex step: g . J with J[k] = (f(x + s e_k) - f(x - s e_k)) / 2s,
    s = 1e-6 max(1, |x_k|).  Extended: wi on the whole sphere.  The differences lose accuracy where
    the step reaches a singularity, so the samples within 1e-2 of a = 1 + i.z = 0 are left to the
    complex-step tests, as are those on which the FP64 forward itself is weak."""
    n = 8195
    d = (workloads.sphere_stream if ext else workloads.adjoint_2e24)(n=n, seed=21, device=DEV)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
    wi = np.stack([_np(d[k]) for k in keys[:3]])
    ax, ay = _np(d["alpha_x"]), _np(d["alpha_y"])
    u1, u2 = philox.sample_uniforms(31, 0, 0, n)
    ok = ovndf.in_domain(wi, ax, ay, ext)
    rng = np.random.default_rng(8)
    gw = rng.standard_normal((3, n))
    with np.errstate(all="ignore"):
        _, pdf = ovndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, extended=ext)
        gp = np.where(ok, rng.standard_normal(n) / pdf, 0.0)  # pdf and wm terms of comparable size
    gw32, gp32 = gw.astype(np.float32), gp.astype(np.float32)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=DEV)  # noqa: E731
    out = v.vndf_sample_backward(*(d[k] for k in keys), u1=t(u1), u2=t(u2), g_wm_x=t(gw32[0]), g_wm_y=t(gw32[1]),
                                 g_wm_z=t(gw32[2]), g_pdf=t(gp32), extended=ext)
    got = np.stack([_np(x) for x in out])
    assert np.isfinite(got).all() and np.all(got[:, ~ok] == 0.0)
    keep = ok & (parity.one_plus_zi(wi, ax, ay) >= 1e-2) & ~parity.fp64_weak(u2, wi, ax, ay)
    idx = np.flatnonzero(keep)
    assert idx.size > (0.6 if ext else 0.99) * n  # sphere: 75 % kept (small alpha pushes i.z to -1)
    with np.errstate(all="ignore"):
        jac = grad.jacobian_central_difference(u1[idx], u2[idx], wi[:, idx], ax[idx], ay[idx], extended=ext)
    g = np.concatenate([gw32.astype(np.float64), gp32.astype(np.float64)[None]])[:, idx]
    ref = np.einsum("ion,on->in", jac, g)
    _check_errors(_errors(got[:, idx], ref), f"backward vs central differences ext={ext}")


def test_backward_optional_outputs_and_inputs(v):
    n = 4099
    d = workloads.adjoint_2e24(n=n, seed=40, device=DEV)
    gp = torch.ones(n, device=DEV)
    full = v.vndf_sample_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=1, g_pdf=gp)
    only_a = v.vndf_sample_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=1,
                                    g_pdf=gp, want_wi=False)
    assert only_a[0] is None
    assert torch.equal(full[3], only_a[3]) and torch.equal(full[4], only_a[4])
    # no adjoint at all: zero gradients
    z = v.vndf_sample_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=1)
    for t in z:
        assert torch.count_nonzero(t) == 0


def test_fused_loss_matches_oracle(v):
    n = (1 << 20) + 7
    d = workloads.adjoint_2e24(n=n, device=DEV)
    loss, gx, gy, gz, gax, gay = v.vndf_sample_loss_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"],
                                                             d["alpha_y"], d["c_x"], d["c_y"], d["c_z"], seed=4)
    loss2 = v.vndf_sample_loss_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], d["c_x"],
                                        d["c_y"], d["c_z"], seed=4)[0]
    assert torch.equal(loss, loss2)  # deterministic
    u1, u2 = philox.sample_uniforms(4, 0, 0, n)
    wi = np.stack([_np(d[k]) for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = _np(d["alpha_x"]), _np(d["alpha_y"])
    c = np.stack([_np(d[k]) for k in ("c_x", "c_y", "c_z")])
    wm, pdf = ovndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay)
    terms = ovndf.dot(c, wm) + np.log(pdf)
    ref = terms.sum()
    got = float(loss.item())
    print(f"loss gpu {got:.8e} oracle {ref:.8e} rel {abs(got / ref - 1):.2e}")
    assert abs(got - ref) <= 1e-5 * np.abs(terms).sum()
    # gradients on a subset: g_wm = c, g_pdf = 1 / pdf
    idx = np.arange(0, n, 97)
    rwi, rax, ray = grad.vjp(u1[idx], u2[idx], wi[:, idx], ax[idx], ay[idx], c[:, idx], 1.0 / pdf[idx])
    ref_g = np.concatenate([rwi, rax[None], ray[None]])
    got_g = np.stack([_np(t)[idx] for t in (gx, gy, gz, gax, gay)])
    _check_errors(_errors(got_g, ref_g), "fused loss gradients")


def test_fused_loss_ragged_and_unaligned(v):
    """Tail chunks and the scalar path give the same per-sample gradients as the generic backward."""
    n = 3001
    d = workloads.adjoint_2e24(n=n + 1, seed=41, device=DEV)
    sl = {k: t[1:].clone()[:n] for k, t in d.items()}  # clone -> aligned
    un = {k: t[1:n + 1] for k, t in d.items()}          # view offset by one float -> unaligned
    for src in (sl, un):
        loss, gx, gy, gz, gax, gay = v.vndf_sample_loss_backward(
            src["wi_x"], src["wi_y"], src["wi_z"], src["alpha_x"], src["alpha_y"], src["c_x"], src["c_y"],
            src["c_z"], seed=8, n=n)
        _, _, _, pdf = v.vndf_sample(src["wi_x"], src["wi_y"], src["wi_z"], src["alpha_x"], src["alpha_y"],
                                     seed=8, n=n)
        ref = v.vndf_sample_backward(src["wi_x"], src["wi_y"], src["wi_z"], src["alpha_x"], src["alpha_y"],
                                     seed=8, g_wm_x=src["c_x"].contiguous(), g_wm_y=src["c_y"].contiguous(),
                                     g_wm_z=src["c_z"].contiguous(), g_pdf=1.0 / pdf, n=n)
        for a, b in zip((gx, gy, gz, gax, gay), ref):
            torch.testing.assert_close(a[:n], b[:n], rtol=1e-4, atol=1e-6)


def test_fused_loss_staged_path(v):
    """Above 16 x 3 x SMs full chunks the fused loss runs the shared-memory-staged kernel (plus the plain
    kernel on a ragged last chunk): per-sample gradients equal, bit for bit, those of small calls that take
    the plain kernel, and the loss equals the FP64 sum of the same per-sample terms."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 16 * 3 * sms * 1024 + 517
    d = workloads.adjoint_2e24(n=n, seed=43, device=DEV)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y", "c_x", "c_y", "c_z")
    big = v.vndf_sample_loss_backward(*(d[k] for k in keys), seed=8)
    for start, m in ((0, 3000), (n // 2 + 5, 1025), (n - 2000, 2000)):
        part = v.vndf_sample_loss_backward(*(d[k][start:start + m].contiguous() for k in keys), seed=8,
                                           counter_base=start)
        for a, b in zip(big[1:], part[1:]):
            assert torch.equal(a[start:start + m], b)
    wx, wy, wz, pdf = v.vndf_sample(*(d[k] for k in keys[:5]), seed=8)
    terms = (d["c_x"].double() * wx.double() + d["c_y"].double() * wy.double() + d["c_z"].double() * wz.double()
             + torch.log(pdf.double()))
    ref = terms.sum().item()
    assert abs(big[0].item() - ref) <= 1e-5 * terms.abs().sum().item()


@pytest.mark.parametrize("inputs", ["both", "g_wm", "g_pdf"])
def test_generic_backward_staged_path(v, inputs):
    """Above 16 x 3 x SMs x 256 groups the generic adjoint runs the shared-memory-staged kernel: its
    gradients equal, bit for bit, those of small calls that take the plain kernel, for every
    combination of the optional adjoint inputs."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 16 * 3 * sms * 1024 + 517
    d = workloads.adjoint_2e24(n=n, seed=44, device=DEV)
    gp = torch.rand(n, device=DEV, generator=torch.Generator(device=DEV).manual_seed(5))
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")

    def call(sl, base):
        g = {} if inputs == "g_pdf" else {"g_wm_x": d["c_x"][sl], "g_wm_y": d["c_y"][sl], "g_wm_z": d["c_z"][sl]}
        if inputs != "g_wm":
            g["g_pdf"] = gp[sl]
        return v.vndf_sample_backward(*(d[k][sl] for k in keys), seed=6, counter_base=base, **g)

    big = call(slice(0, n), 0)
    for start, m in ((0, 3000), (n // 2 + 7, 1029), (n - 2000, 2000)):
        part = call(slice(start, start + m), start)
        for a, b in zip(big, part):
            assert torch.equal(a[start:start + m], b)


def test_autograd_function(v):
    from paper_2306_05044_gb300.autograd import vndf_sample_autograd
    n = 5000
    d = workloads.adjoint_2e24(n=n, seed=42, device=DEV)
    leaves = {k: d[k].clone().requires_grad_(True) for k in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")}
    wm_x, wm_y, wm_z, pdf = vndf_sample_autograd(leaves["wi_x"], leaves["wi_y"], leaves["wi_z"],
                                                 leaves["alpha_x"], leaves["alpha_y"], seed=3, counter_base=10)
    loss = (d["c_x"] * wm_x + d["c_y"] * wm_y + d["c_z"] * wm_z).sum() + torch.log(pdf).sum()
    loss.backward()
    ref = v.vndf_sample_loss_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], d["c_x"],
                                      d["c_y"], d["c_z"], seed=3, counter_base=10)
    for k, r in zip(("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y"), ref[1:]):
        torch.testing.assert_close(leaves[k].grad, r, rtol=1e-4, atol=1e-5)


@pytest.mark.slow
def test_full_size_fused_loss_sampled(v):
    """The 2^24-sample fused forward+adjoint launch, checked on sampled gradients."""
    n = 1 << 24
    d = workloads.adjoint_2e24(n=n, device=DEV)
    loss, gx, gy, gz, gax, gay = v.vndf_sample_loss_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"],
                                                             d["alpha_y"], d["c_x"], d["c_y"], d["c_z"], seed=4)
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([np.arange(64), n - 1 - np.arange(64), rng.integers(0, n, 1 << 14)]))
    ti = torch.as_tensor(idx, device=DEV)
    pick = lambda t: t.index_select(0, ti).cpu().numpy().astype(np.float64)  # noqa: E731
    wi = np.stack([pick(d[k]) for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = pick(d["alpha_x"]), pick(d["alpha_y"])
    c = np.stack([pick(d[k]) for k in ("c_x", "c_y", "c_z")])
    u1, u2 = philox.uniforms_at(4, 0, 0, idx)
    _, pdf = ovndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay)
    rwi, rax, ray = grad.vjp(u1, u2, wi, ax, ay, c, 1.0 / pdf)
    ref = np.concatenate([rwi, rax[None], ray[None]])
    got = np.stack([pick(t) for t in (gx, gy, gz, gax, gay)])
    _check_errors(_errors(got, ref), "full-size fused gradients")
    assert np.isfinite(loss.item())


def _tiled(blk, n, period):
    """Device copies of blk's arrays tiled to length n, written slice by slice (no torch kernel
    runs over more than `period` elements)."""
    out = {}
    for k, t in blk.items():
        x = torch.empty(n, dtype=torch.float32, device=DEV)
        for s0 in range(0, n, period):
            m = min(period, n - s0)
            x[s0:s0 + m].copy_(t[:m])
        out[k] = x
    return out


@pytest.mark.slow
def test_adjoints_beyond_int32(v):
    """The fused forward+loss+adjoint and the generic adjoint over one call of 2^31 + 4101 samples
    (about 112 GB): 64-bit element indices, Philox counters and loss-partial indices past 2^31.
    The inputs tile a 2^20 + 3 block.  The loss workspace is filled with NaN first, so a partial
    that no warp wrote would show; every partial is finite, the loss equals their sum, the partials
    of 128-sample groups at the 2^31 boundary, the end and random places equal the oracle's sums of
    the same terms, and the gradients there match the oracle's complex-step products."""
    n = (1 << 31) + 4101
    free, _ = torch.cuda.mem_get_info()
    if free < 130 * (1 << 30):
        pytest.skip(f"needs about 120 GB of free device memory, {free / 2**30:.0f} GB free")
    period = (1 << 20) + 3
    blk = workloads.adjoint_2e24(n=period, seed=42, device=DEV)
    d = _tiled(blk, n, period)
    blk_np = {k: t.cpu().numpy().astype(np.float64) for k, t in blk.items()}
    nbytes = v.vndf_loss_workspace_bytes(n)
    ws = torch.full(((nbytes + 3) // 4,), float("nan"), dtype=torch.float32, device=DEV)
    loss, gx, gy, gz, gax, gay = v.vndf_sample_loss_backward(
        d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], d["c_x"], d["c_y"], d["c_z"], seed=5,
        counter_base=7, workspace=ws.view(torch.uint8))
    torch.cuda.synchronize()
    groups = (n + 127) // 128
    partials = ws[:groups].cpu().numpy().astype(np.float64)
    assert np.isfinite(partials).all()
    got = float(loss.item())
    assert abs(got - partials.sum()) <= 1e-6 * np.abs(partials).sum()
    rng = np.random.default_rng(2)
    gsel = np.unique(np.concatenate([[0, (1 << 31) // 128 - 1, (1 << 31) // 128, groups - 1],
                                     rng.integers(0, groups, 60)]))
    idx = np.concatenate([np.arange(128 * g, min(128 * g + 128, n)) for g in gsel])

    def gather(t):
        return np.concatenate([t[128 * int(g):min(128 * int(g) + 128, n)].cpu().numpy() for g in gsel])

    wi = np.stack([blk_np[k][idx % period] for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = blk_np["alpha_x"][idx % period], blk_np["alpha_y"][idx % period]
    c = np.stack([blk_np[k][idx % period] for k in ("c_x", "c_y", "c_z")])
    u1, u2 = philox.uniforms_at(5, 7, 0, idx)
    wm, pdf = ovndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay)
    terms = ovndf.dot(c, wm) + np.log(pdf)
    # partials of the selected groups against the oracle's sums of the same 128 terms
    bounds = np.cumsum([0] + [min(128 * int(g) + 128, n) - 128 * int(g) for g in gsel])
    for j, g in enumerate(gsel):
        t = terms[bounds[j]:bounds[j + 1]]
        assert abs(partials[g] - t.sum()) <= 1e-5 * np.abs(t).sum(), (g, partials[g], t.sum())
    rwi, rax, ray = grad.vjp(u1, u2, wi, ax, ay, c, 1.0 / pdf)
    ref = np.concatenate([rwi, rax[None], ray[None]])
    got_g = np.stack([gather(t).astype(np.float64) for t in (gx, gy, gz, gax, gay)])
    _check_errors(_errors(got_g, ref), "fused gradients beyond int32")
    del gx, gy, gz, gax, gay, ws
    torch.cuda.empty_cache()
    # the generic adjoint with g_wm = c and no density term, over the same inputs
    gx, gy, gz, gax, gay = v.vndf_sample_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"],
                                                  seed=5, counter_base=7, g_wm_x=d["c_x"], g_wm_y=d["c_y"],
                                                  g_wm_z=d["c_z"])
    torch.cuda.synchronize()
    rwi, rax, ray = grad.vjp(u1, u2, wi, ax, ay, c, np.zeros_like(pdf))
    ref = np.concatenate([rwi, rax[None], ray[None]])
    got_g = np.stack([gather(t).astype(np.float64) for t in (gx, gy, gz, gax, gay)])
    _check_errors(_errors(got_g, ref), "generic gradients beyond int32")
    del d, gx, gy, gz, gax, gay
    torch.cuda.empty_cache()
