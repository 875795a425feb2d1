"""GPU parity of the extended domain (incident directions below the horizon) and of the
stand-alone hemisphere sampler, through the C ABI, against the FP64 oracle and, where
1 + z_i' is below 1e-9, the 50-digit reference.

Inputs: the sphere workload (wi uniform on the whole sphere, alphas log-uniform in
[1e-3, 1]) at sizes that span many CTAs and a ragged tail, explicit edge cases, and the
full 2^28-sample workload in the bench's launch on sampled outputs.
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


def _np(*ts):
    return [t.detach().cpu().numpy() for t in ts]


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


KEYS = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")


@pytest.mark.parametrize("n,base", [((1 << 20) + 5, 0), ((1 << 18) + 2, 9)])
def test_extended_sphere_workload(v, n, base):
    d = workloads.sphere_stream(n=n, device=DEV)
    wx, wy, wz, pdf = v.vndf_sample(*(d[k] for k in KEYS), seed=4, counter_base=base, method="cap_extended")
    u1, u2 = philox.sample_uniforms(4, base, 0, n)
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"]))
    ax, ay = _np(d["alpha_x"], d["alpha_y"])
    wm = np.stack(_np(wx, wy, wz))
    p = pdf.cpu().numpy()
    st = parity.compare_cap(wm, p, u1, u2, wi, ax, ay, extended=True)
    st.update(parity.compare_cap_mp(wm, p, u1, u2, wi, ax, ay))
    print("sphere", n, base, st)
    # a handful of directions stretch to within 2^-40 of straight down; compare_cap has checked
    # that both sides agree on them and that the GPU returned the exact fallback
    assert st["out_of_domain"] <= 16
    assert (wm[2] > 0).all()


def test_extended_equals_cap_above_horizon(v):
    """For wi.z > 0 the extended method is the cap sampler bit for bit; below it the cap method
    returns its fallback."""
    n = 100003
    d = workloads.sphere_stream(n=n, seed=41, device=DEV)
    a = v.vndf_sample(*(d[k] for k in KEYS), seed=6, method="cap")
    b = v.vndf_sample(*(d[k] for k in KEYS), seed=6, method="cap_extended")
    up = d["wi_z"] > 0
    for x, y in zip(a, b):
        assert torch.equal(x[up], y[up])
    assert torch.all(a[2][~up] == 1.0) and torch.all(a[3][~up] == 0.0)
    assert torch.all(b[3][~up] > 0.0)


def test_extended_path_and_split_independent(v):
    n = 30001
    d = workloads.sphere_stream(n=n + 1, seed=42, device=DEV)
    full = v.vndf_sample(*(d[k][:n] for k in KEYS), seed=5, counter_base=3, method="cap_extended")
    shifted = {k: torch.cat([d[k][:1], d[k][:n]]) for k in KEYS}
    s = v.vndf_sample(*(shifted[k][1:] for k in KEYS), seed=5, counter_base=3, method="cap_extended", n=n)
    for x, y in zip(full, s):
        assert torch.equal(x, y)


def test_extended_edges(v):
    """Straight down, just inside and just outside 1 + z_i' >= 2^-40, grazing, NaN, alpha <= 0,
    the extremes of u, alpha = 1e-3 below the horizon."""
    nan = float("nan")
    wx = [0.0, 1e-5, 1e-7, 1.0, nan, 0.3, 0.6, 0.6, 0.8, 0.5, 2e-6]
    wy = [0.0, 0.0, 0.0, 0.0, 0.1, 0.1, 0.0, 0.0, 0.0, -0.5, 0.0]
    wz = [-1.0, -1.0, -1.0, 0.0, -0.5, -0.5, -0.8, -0.8, -0.6, -0.7, -1.0]
    ax = [1.0, 1.0, 1.0, 0.5, 0.5, 0.0, 1e-3, 1.0, 1e-3, 0.02, 1.0]
    ay = [1.0, 1.0, 1.0, 0.5, 0.5, 0.5, 1e-3, 1e-3, 1.0, 0.7, 1.0]
    u1 = [0.3, 0.3, 0.3, 0.0, 0.3, 0.3, 0.0, 0.5, 0.99, 0.25, 0.6]
    u2 = [0.7, 0.7, 0.7, 0.0, 0.7, 0.7, 1 - 2 ** -24, 0.0, 0.5, 0.999, 0.1]
    t = [_dev(x) for x in (wx, wy, wz, ax, ay, u1, u2)]
    mx, my, mz, pdf = v.vndf_sample(*t[:5], t[5], t[6], method="cap_extended")
    wm = np.stack(_np(mx, my, mz))
    p = pdf.cpu().numpy()
    wi = np.array([wx, wy, wz], np.float32)
    args = (np.array(u1, np.float32), np.array(u2, np.float32), wi, np.array(ax, np.float32),
            np.array(ay, np.float32))
    st = parity.compare_cap(wm, p, *args, extended=True)
    st.update(parity.compare_cap_mp(wm, p, *args))
    print("edges", st)
    assert st["out_of_domain"] == 4  # straight down, 1 + z_i' = 5e-15, NaN, alpha = 0
    # 1 + z_i' = 5e-11 and 2e-12, and the two u2 = 0 samples (their cap point is the pole, sin(theta) = 0,
    # which FP64 forms from 1 - z^2 at its resolution)
    assert st["n_mp"] == 4
    assert np.all(np.isfinite(p)) and np.all(wm[2][p > 0] > 0)


def test_pdf_extended_at_given_normals(v):
    n = (1 << 18) + 1
    d = workloads.sphere_stream(n=n, seed=43, device=DEV)
    wx, wy, wz, fused = v.vndf_sample(*(d[k] for k in KEYS), seed=8, method="cap_extended")
    p = v.vndf_pdf(*(d[k] for k in KEYS), wx, wy, wz, extended=True)
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"])).astype(np.float64)
    wm = np.stack(_np(wx, wy, wz)).astype(np.float64)
    ax, ay = (t.astype(np.float64) for t in _np(d["alpha_x"], d["alpha_y"]))
    ref = ovndf.vndf_pdf(wm, wi, ax, ay, extended=True)
    keep = parity.one_plus_zi(wi, ax, ay) >= parity.A_MP
    rel = np.abs(p.cpu().numpy() / ref - 1.0)[keep]
    # wi.wm cancels near the visibility boundary, and 1/(|M^-1 wi| + wi.z) is formed from a
    # quotient when wi.z < 0: bound by the condition of the dot product plus a few ulp
    kd = ((np.abs(wi * wm).sum(0) / np.abs(ovndf.dot(wi, wm))) / np.sqrt(ovndf.dot(wi, wi)))[keep]
    bound = np.maximum(1e-5, parity.K_ULP * (kd + 8.0) * parity.EPS32)
    assert np.all(rel <= bound), rel.max()
    # the upper-domain entry keeps its fallback below the horizon and agrees above it
    q = v.vndf_pdf(*(d[k] for k in KEYS), wx, wy, wz).cpu().numpy()
    up = wi[2] > 0
    assert np.all(q[~up] == 0.0)
    np.testing.assert_allclose(q[up], p.cpu().numpy()[up], rtol=2e-6)


def test_hemisphere_sampler(v):
    """Stand-alone hemisphere sampler (any wi length, whole sphere) against the oracle's
    sample_hemisphere (normalised half vector, Eq. 2 density)."""
    n = (1 << 20) + 7
    d = workloads.hemisphere_stream(n=n, device=DEV)
    wx, wy, wz, pdf = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], seed=9)
    u1, u2 = philox.sample_uniforms(9, 0, 0, n)
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"])).astype(np.float64)
    one = np.ones(n)
    wm = np.stack(_np(wx, wy, wz))
    st = parity.compare_cap(wm, pdf.cpu().numpy(), u1, u2, wi, one, one, extended=True)
    st.update(parity.compare_cap_mp(wm, pdf.cpu().numpy(), u1, u2, wi, one, one))
    print("hemisphere", st)
    keep = ~parity.fp64_weak(u2, wi, one, one)
    ref, pref = ovndf.sample_hemisphere(u1, u2, wi)
    ang = parity.angle_between(wm.astype(np.float64)[:, keep], ref[:, keep])
    assert ang.max() <= parity.ANGLE_TOL
    # Eq. 2 at the float normal: 2 max(0, wi.wm) / (pi (1 + wi.z)); the fused value avoids the dot
    rel = np.abs(pdf.cpu().numpy()[keep] / pref[keep] - 1.0)
    assert np.quantile(rel, 0.999) < 1e-5


def test_hemisphere_equals_ggx_at_alpha_one(v):
    """With alpha_x = alpha_y = 1 the GGX sampler is the hemisphere sampler: same bits."""
    n = 65537
    d = workloads.hemisphere_stream(n=n, seed=44, device=DEV)
    ones = torch.ones(n, device=DEV)
    a = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], ones, ones, seed=3, method="cap_extended")
    b = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], seed=3)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    c = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], seed=3, with_pdf=False)
    assert c[3] is None
    for x, y in zip(b[:3], c[:3]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9])
def test_hemisphere_tiny_and_explicit_u(v, n):
    d = workloads.hemisphere_stream(n=n, seed=45, device=DEV)
    u1, u2 = philox.sample_uniforms(2, 0, 0, n)
    a = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], _dev(u1), _dev(u2))
    b = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], seed=2)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.slow
def test_full_size_sphere_stream_sampled(v):
    """2^28 samples of the sphere workload in one call (the bench's launch), checked on sampled
    outputs and both ends."""
    n = 1 << 28
    d = workloads.sphere_stream(n=n, device=DEV)
    out = v.vndf_sample(*(d[k] for k in KEYS), seed=2, method="cap_extended")
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([np.arange(1024), n - 1 - np.arange(1024), rng.integers(0, n, 1 << 16)]))
    ti = torch.as_tensor(idx, device=DEV)
    wi = np.stack([d[k].index_select(0, ti).cpu().numpy() for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = (d[k].index_select(0, ti).cpu().numpy() for k in ("alpha_x", "alpha_y"))
    wm = np.stack([o.index_select(0, ti).cpu().numpy() for o in out[:3]])
    pdf = out[3].index_select(0, ti).cpu().numpy()
    u1, u2 = philox.uniforms_at(2, 0, 0, idx)
    st = parity.compare_cap(wm, pdf, u1, u2, wi, ax, ay, extended=True)
    st.update(parity.compare_cap_mp(wm, pdf, u1, u2, wi, ax, ay))
    print("full size sphere sampled", st)
    del d, out
    torch.cuda.empty_cache()


def _sphere_adjoint_inputs(n, seed):
    """The sphere workload with roughness kept >= 1e-2 (where FP32 gradients have a useful condition)."""
    d = workloads.sphere_stream(n=n, seed=seed, device=DEV)
    for k in ("alpha_x", "alpha_y"):
        d[k] = torch.clamp(d[k], min=1e-2).contiguous()
    return d


@pytest.mark.parametrize("iso", [False, True])
def test_backward_extended_matches_complex_step(v, iso):
    """vndf_sample_backward_extended against the oracle's complex-step vector-Jacobian product on the
    extended domain (about half the samples below the horizon)."""
    n = (1 << 13) + 3
    d = _sphere_adjoint_inputs(n, 51)
    ay = None if iso else d["alpha_y"]
    g = torch.randn(4, n, device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    got = v.vndf_sample_backward_extended(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], ay, seed=12,
                                          g_wm_x=g[0].contiguous(), g_wm_y=g[1].contiguous(),
                                          g_wm_z=g[2].contiguous(), g_pdf=g[3].contiguous())
    u1, u2 = philox.sample_uniforms(12, 0, 0, n)
    wi = np.stack([d[k].cpu().numpy().astype(np.float64) for k in ("wi_x", "wi_y", "wi_z")])
    ax = d["alpha_x"].cpu().numpy().astype(np.float64)
    ayn = ax if iso else d["alpha_y"].cpu().numpy().astype(np.float64)
    gn = g.cpu().numpy().astype(np.float64)
    keep = parity.one_plus_zi(wi, ax, ayn) >= 1e-6  # where the FP64 oracle is itself accurate
    rwi, rax, ray = grad.vjp(u1, u2, wi, ax, ayn, gn[:3], gn[3], isotropic=iso, extended=True)
    ref = np.concatenate([rwi, rax[None]] + ([] if iso else [ray[None]]))
    outs = [got[0], got[1], got[2], got[3]] + ([] if iso else [got[4]])
    mine = np.stack([t.cpu().numpy().astype(np.float64) for t in outs])
    scale = np.abs(ref).max(axis=0)
    e = (np.abs(mine - ref).max(axis=0) / np.maximum(scale, 1e-30))[keep]
    print(f"extended adjoint iso={iso}: median {np.median(e):.2e} p99.9 {np.quantile(e, 0.999):.2e} "
          f"max {e.max():.2e} below-horizon {(wi[2] < 0).mean():.2f}")
    assert (wi[2][keep] < 0).mean() > 0.3
    assert np.median(e) < 1e-5
    assert np.quantile(e, 0.999) < 1e-3


def test_backward_extended_equals_upper_above_horizon(v):
    """Above the horizon the extended adjoint is the upper-hemisphere adjoint bit for bit; below it the
    upper one returns zero gradients."""
    n = 20001
    d = _sphere_adjoint_inputs(n, 52)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
    gpdf = torch.rand(n, device=DEV, generator=torch.Generator(device=DEV).manual_seed(4))
    a = v.vndf_sample_backward(*(d[k] for k in keys), seed=3, g_pdf=gpdf)
    b = v.vndf_sample_backward_extended(*(d[k] for k in keys), seed=3, g_pdf=gpdf)
    up = d["wi_z"] > 0
    for x, y in zip(a, b):
        assert torch.equal(x[up], y[up])
        assert torch.all(x[~up] == 0)
    assert torch.any(b[2][~up] != 0)


def test_autograd_extended(v):
    """The autograd wrapper with extended=True reaches the extended adjoint."""
    from paper_2306_05044_gb300.autograd import vndf_sample_autograd
    n = 4099
    d = _sphere_adjoint_inputs(n, 53)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
    leaves = {k: d[k].clone().requires_grad_(True) for k in keys}
    wm_x, wm_y, wm_z, pdf = vndf_sample_autograd(*(leaves[k] for k in keys), seed=5, extended=True)
    c = torch.randn(3, n, device=DEV, generator=torch.Generator(device=DEV).manual_seed(6))
    (c[0] * wm_x + c[1] * wm_y + c[2] * wm_z + pdf).sum().backward()
    ref = v.vndf_sample_backward_extended(*(d[k] for k in keys), seed=5, g_wm_x=c[0].contiguous(),
                                          g_wm_y=c[1].contiguous(), g_wm_z=c[2].contiguous(),
                                          g_pdf=torch.ones(n, device=DEV))
    for k, r in zip(keys, ref):
        assert torch.equal(leaves[k].grad, r)
