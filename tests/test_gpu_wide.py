"""Stress inputs through every sampling entry point, through the C ABI.

The wide workload puts wi on the whole sphere with lengths 1e-3 to 1e3, the
roughness anywhere in 1e-5 to 10 (independently per axis) and the uniforms on
the 2^-24 grid with 1 % at the ends and quarter points of [0, 1).  Checks:
every output finite; the exact fallback outside each entry point's domain; the
flat 4e-6 rad / 1e-5 bounds inside the accuracy contract and the
condition-scaled bound outside it (tests/parity.py); extended-domain samples on
which the FP64 oracle itself is weak checked against the 50-digit reference;
the density of given normals and the hemisphere and reflection samplers on the
same inputs against the oracle.
"""
import numpy as np
import pytest
import torch

import parity
import workloads
from oracle import microfacet, vndf as ovndf

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KEYS = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


@pytest.fixture(scope="module")
def wide():
    d = workloads.wide_stream(n=(1 << 18) + 3, seed=19, device=DEV)
    h = {k: t.cpu().numpy().astype(np.float64) for k, t in d.items()}
    return d, h


def _np(*ts):
    return [t.cpu().numpy().astype(np.float64) for t in ts]


@pytest.mark.parametrize("kind", ["cap", "cap_extended"])
def test_sampler_on_wide_inputs(v, wide, kind):
    d, h = wide
    out = v.vndf_sample(*(d[k] for k in KEYS), u1=d["u1"], u2=d["u2"], method=kind)
    wm = np.stack(_np(*out[:3]))
    pdf = _np(out[3])[0]
    assert np.isfinite(wm).all() and np.isfinite(pdf).all()
    wi = np.stack([h["wi_x"], h["wi_y"], h["wi_z"]])
    ext = kind == "cap_extended"
    st = parity.compare_cap(wm, pdf, h["u1"], h["u2"], wi, h["alpha_x"], h["alpha_y"], strict=True, extended=ext)
    if ext:
        st.update(parity.compare_cap_mp(wm, pdf, h["u1"], h["u2"], wi, h["alpha_x"], h["alpha_y"], limit=300))
    print("wide", kind, st)
    # the density of the sampled normals, through the density entry point, against the oracle's Eq. 1
    # (extended: where FP64 forms 1 + z_i' accurately)
    p = v.vndf_pdf(*(d[k] for k in KEYS), *out[:3], extended=ext)
    pg = _np(p)[0]
    assert np.isfinite(pg).all()
    ref = ovndf.vndf_pdf(wm, wi, h["alpha_x"], h["alpha_y"], ext)
    ok = ovndf.in_domain(wi, h["alpha_x"], h["alpha_y"], ext)
    assert np.all(pg[~ok] == 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        keep = ok & (parity.one_plus_zi(wi, h["alpha_x"], h["alpha_y"]) >= parity.A_MP)
        kd = (np.abs(wi * wm).sum(0) / np.abs(ovndf.dot(wi, wm))) / np.sqrt(ovndf.dot(wi, wi))
        rel = np.abs(pg / ref - 1.0)
    bound = np.maximum(parity.PDF_TOL, parity.K_ULP * (kd + 8.0) * parity.EPS32)
    bad = np.flatnonzero(keep & ~(rel <= bound))
    assert bad.size == 0, (bad[:5], rel[bad[:5]], bound[bad[:5]])


def test_hemisphere_on_wide_inputs(v, wide):
    d, h = wide
    out = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], u1=d["u1"], u2=d["u2"])
    wm = np.stack(_np(*out[:3]))
    pdf = _np(out[3])[0]
    assert np.isfinite(wm).all() and np.isfinite(pdf).all()
    wi = np.stack([h["wi_x"], h["wi_y"], h["wi_z"]])
    one = np.ones(wi.shape[1])
    st = parity.compare_cap(wm, pdf, h["u1"], h["u2"], wi, one, one, strict=True, extended=True)
    st.update(parity.compare_cap_mp(wm, pdf, h["u1"], h["u2"], wi, one, one, limit=300))
    print("wide hemisphere", st)


def test_reflection_on_wide_inputs(v, wide):
    d, h = wide
    ox, oy, oz, pdf, w = v.vndf_sample_reflection(*(d[k] for k in KEYS), u1=d["u1"], u2=d["u2"], f0=0.04)
    got = np.stack(_np(ox, oy, oz))
    pg, wg = _np(pdf, w)
    assert np.isfinite(got).all() and np.isfinite(pg).all() and np.isfinite(wg).all()
    wi = np.stack([h["wi_x"], h["wi_y"], h["wi_z"]])
    ax, ay = h["alpha_x"], h["alpha_y"]
    with np.errstate(all="ignore"):
        wb, pr, wr = microfacet.sample_reflection(h["u1"], h["u2"], wi, ax, ay, 0.04)
    ok = ovndf.in_domain(wi, ax, ay)
    assert np.all(got[:, ~ok] == np.array([[0.0], [0.0], [1.0]])) and np.all(pg[~ok] == 0) and np.all(wg[~ok] == 0)
    # inside the accuracy contract the sample's bounds, doubled by the reflection for the direction
    cont = ok & (np.minimum(ax, ay) >= 1e-3) & (wi[2] / np.sqrt(ovndf.dot(wi, wi)) >= 1e-4)
    ang = parity.angle_between(got[:, cont], wb[:, cont])
    assert ang.max() <= 2 * parity.ANGLE_TOL
    assert np.abs(pg[cont] / pr[cont] - 1.0).max() <= parity.PDF_TOL
    print(f"wide reflection: {int(cont.sum())} samples in the contract, wo max {ang.max():.2e} rad")


@pytest.mark.parametrize("ext", [False, True])
def test_adjoint_on_wide_inputs(v, wide, ext):
    """The generic adjoint on the stress inputs: finite everywhere, zero outside the domain, and inside the
    contract (and where FP64 is not weak) the complex-step products to p99.9 1e-3 of the largest component."""
    from oracle import grad
    d, h = wide
    n = d["wi_x"].numel()
    g = torch.Generator(device=DEV).manual_seed(3)
    gw = [torch.randn(n, generator=g, device=DEV) for _ in range(3)]
    out = v.vndf_sample(*(d[k] for k in KEYS), u1=d["u1"], u2=d["u2"], method="cap_extended" if ext else "cap")
    gp = (1.0 / torch.clamp(out[3], min=1e-30)).contiguous()  # d log pdf
    gr = v.vndf_sample_backward(*(d[k] for k in KEYS), u1=d["u1"], u2=d["u2"], g_wm_x=gw[0], g_wm_y=gw[1],
                                g_wm_z=gw[2], g_pdf=gp, extended=ext)
    got = np.stack(_np(*gr))
    assert np.isfinite(got).all()
    wi = np.stack([h["wi_x"], h["wi_y"], h["wi_z"]])
    ax, ay = h["alpha_x"], h["alpha_y"]
    ok = ovndf.in_domain(wi, ax, ay, ext)
    assert np.all(got[:, ~ok] == 0.0)
    cont = ok & (np.minimum(ax, ay) >= 1e-3)
    if not ext:
        cont &= wi[2] / np.sqrt(ovndf.dot(wi, wi)) >= 1e-4
    else:
        cont &= ~parity.fp64_weak(h["u2"], wi, ax, ay)
    idx = np.flatnonzero(cont)[:20000]
    gwn = np.stack(_np(*gw))[:, idx]
    rwi, rax, ray = grad.vjp(h["u1"][idx], h["u2"][idx], wi[:, idx], ax[idx], ay[idx], gwn, _np(gp)[0][idx],
                             extended=ext)
    ref = np.concatenate([rwi, rax[None], ray[None]])
    err = np.abs(got[:, idx] - ref).max(axis=0) / np.maximum(np.abs(ref).max(axis=0), 1e-30)
    print(f"wide adjoint ext={ext}: {idx.size} samples, median {np.median(err):.1e} p99.9 {np.quantile(err, 0.999):.1e}"
          f" max {err.max():.1e}")
    assert np.quantile(err, 0.999) < 1e-3
