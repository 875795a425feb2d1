"""GPU parity of vndf_sample_reflection against the oracle's App. A composition.

Reflection doubles angular errors (wo = 2 (wi.wm) wm - wi), so wo is held to
twice the normal's 4e-6 rad and the pdf to 1e-5 relative.  The weight
F G2 / G1 is a steep function of the normal when wi or wo is grazing; it is
held to 1e-5 relative + 1e-7, plus its sensitivity to the sampled normal (a
tangent-plane central difference of the oracle's weight) times the normal's
4e-6 rad bound.
"""
import numpy as np
import pytest
import torch

import parity
import workloads
from oracle import microfacet, philox

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


def _weight_sensitivity(u1, u2, wi, ax, ay, f0, eps=1e-7):
    """|d weight / d wm| (per radian) by central differences along two tangents of the FP64 normal."""
    from oracle import vndf
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
    wa = wi / np.sqrt(vndf.dot(wi, wi))
    helper = np.where(np.abs(wm[0]) < 0.9, 1.0, 0.0)
    t1 = np.cross(wm.T, np.stack([helper, 1 - helper, np.zeros_like(helper)]).T).T
    t1 /= np.sqrt(vndf.dot(t1, t1))
    t2 = np.cross(wm.T, t1.T).T
    g = np.zeros(wm.shape[1])
    for t in (t1, t2):
        wp = wm + eps * t
        wq = wm - eps * t
        wp /= np.sqrt(vndf.dot(wp, wp))
        wq /= np.sqrt(vndf.dot(wq, wq))
        dp = microfacet.estimator_weight(wp, wa, ax, ay, f0) - microfacet.estimator_weight(wq, wa, ax, ay, f0)
        g = np.maximum(g, np.abs(dp) / (2 * eps))
    return g


def _check(v, d, n, seed, base, iso, f0=0.04):
    ay = None if iso else d["alpha_y"]
    ox, oy, oz, pdf, w = v.vndf_sample_reflection(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], ay, seed=seed,
                                                  counter_base=base, f0=f0)
    u1, u2 = philox.sample_uniforms(seed, base, 0, n)
    wi = np.stack([d[k].cpu().numpy().astype(np.float64) for k in ("wi_x", "wi_y", "wi_z")])
    axn = d["alpha_x"].cpu().numpy().astype(np.float64)
    ayn = axn if iso else d["alpha_y"].cpu().numpy().astype(np.float64)
    wb, pr, wr = microfacet.sample_reflection(u1, u2, wi, axn, ayn, f0)
    got = np.stack([t.cpu().numpy().astype(np.float64) for t in (ox, oy, oz)])
    ang = parity.angle_between(got, wb)
    rel = np.abs(pdf.cpu().numpy() / pr - 1)
    werr = np.abs(w.cpu().numpy() - wr)
    sens = _weight_sensitivity(u1, u2, wi, axn, ayn, f0)
    bound = 1e-5 * np.abs(wr) + 1e-7 + sens * parity.ANGLE_TOL
    worst = int(np.argmax(werr / bound))
    print(f"reflection iso={iso}: wo max {ang.max():.2e} rad, pdf max rel {rel.max():.2e}, "
          f"weight max err {werr.max():.2e} (worst/bound {werr[worst] / bound[worst]:.2f}: wi.z {wi[2, worst]:.2e}, "
          f"w {wr[worst]:.3e}, sensitivity {sens[worst]:.2e})")
    assert ang.max() <= 2 * parity.ANGLE_TOL
    assert rel.max() <= parity.PDF_TOL
    assert np.all(werr <= bound)
    return got, pdf, w


@pytest.mark.parametrize("n,base,iso", [((1 << 20) + 3, 0, False), ((1 << 18) + 1, 5, True)])
def test_reflection_matches_oracle(v, n, base, iso):
    d = workloads.anisotropic_stream(n=n, seed=12, device=DEV)
    _check(v, d, n, 2, base, iso)


def test_reflection_shares_the_sampled_normal(v):
    """wo is the reflection of vndf_sample's wm: the half vector of wi and wo is that normal."""
    n = 65537
    d = workloads.anisotropic_stream(n=n, seed=51, device=DEV)
    wm = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=9, with_pdf=False)
    wo = v.vndf_sample_reflection(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=9,
                                  with_pdf=False, with_weight=False)
    wi = torch.stack([d["wi_x"], d["wi_y"], d["wi_z"]]).double()
    wi = wi / wi.norm(dim=0)
    h = wi + torch.stack(wo[:3]).double()
    hn = h.norm(dim=0)
    # |wi + wo| = 2 wi.wm; below 0.05 the float32 rounding of wo dominates the rebuilt half vector
    keep = hn >= 0.05
    assert float(keep.double().mean()) > 0.99
    h = (h[:, keep] / hn[keep]).cpu().numpy()
    m = torch.stack(wm[:3]).double()[:, keep].cpu().numpy()
    ang = parity.angle_between(h, m)  # atan2 form: acos of a float32 dot product is not accurate here
    assert float(ang.max()) < 1e-5


def test_reflection_domain_fallback(v):
    t = lambda x: torch.tensor(x, dtype=torch.float32, device=DEV)  # noqa: E731
    ox, oy, oz, pdf, w = v.vndf_sample_reflection(t([0.1, 0.2]), t([0.0, 0.1]), t([-0.3, 0.9]), t([0.5, -1.0]),
                                                  None, seed=1)
    assert torch.equal(oz, t([1.0, 1.0])) and torch.equal(pdf, t([0.0, 0.0])) and torch.equal(w, t([0.0, 0.0]))
