"""GGX microfacet BRDF pieces and the directional-albedo estimator: FP64 oracle.

Test infrastructure only (imported by tests, the smoke entry point and the
bench's CPU-baseline leg); shares no code with the CUDA path.

Paper sections followed:
* ``smith_g2``        App. A, height-correlated G2 = Gi Go / (Gi + Go - Gi Go)
* ``brdf``            App. A, Eq. microfacet (Cook-Torrance): F G2 D / (4 cos_i cos_o)
* ``reflect``         Eq. reflect (Sec. 3.2) and App. A step (2)
* ``bsdf_pdf``        App. A: PDF(wb, wa) = G1(wm, wa) D(wm) / (4 cos_a)
* ``estimator_weight`` App. A, Eq. rendering_mc with L = 1: f_r |cos_b| / PDF
* ``sample_reflection`` App. A steps (1)-(2): reflected direction, its PDF and weight
* ``albedo_estimate``  the Monte Carlo estimator over Philox streams
* ``albedo_quadrature`` the same integral by a midpoint rule over (u1, u2)

Readings (the paper is silent on them):
* Fresnel: Schlick's approximation F = F0 + (1 - F0)(1 - cos)^5 at cos = wm.wa
  (Schlick 1994); the paper only names "the Fresnel term".
* The BRDF is zero when the reflected direction is below the surface (wb.z <= 0).
* Philox streams for query q use stream id = stream_base + q and sample j uses
  global index counter_base + j.
"""
import numpy as np

from . import philox
from .vndf import dot, ndf, sample_vndf, smith_g1, _stack


def schlick_fresnel(cos_theta, f0):
    """Schlick 1994: F0 + (1 - F0) (1 - cos)^5."""
    return f0 + (1.0 - f0) * (1.0 - cos_theta) ** 5


def smith_g2(wm, wi, wo, ax, ay):
    """App. A: height-correlated masking-shadowing Gi Go / (Gi + Go - Gi Go)."""
    gi = smith_g1(wm, wi, ax, ay)
    go = smith_g1(wm, wo, ax, ay)
    return gi * go / (gi + go - gi * go)


def reflect(wm, wa):
    """Eq. reflect: wb = 2 (wm.wa) wm - wa."""
    d = dot(wm, wa)
    return _stack(2.0 * d * wm[0] - wa[0], 2.0 * d * wm[1] - wa[1], 2.0 * d * wm[2] - wa[2])


def brdf(wi, wo, ax, ay, f0):
    """Eq. microfacet: F(wh.wo) G2(wh, wi, wo) D(wh) / (4 cos_i cos_o), zero below the surface."""
    h = _stack(wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2])
    wh = h / np.sqrt(dot(h, h))
    f = schlick_fresnel(dot(wh, wo), f0)
    val = f * smith_g2(wh, wi, wo, ax, ay) * ndf(wh, ax, ay) / (4.0 * wi[2] * wo[2])
    return np.where((wo[2] > 0.0) & (wi[2] > 0.0), val, 0.0)


def bsdf_pdf(wm, wa, ax, ay):
    """App. A: density of the reflected direction, G1(wm, wa) D(wm) / (4 cos_a)."""
    return smith_g1(wm, wa, ax, ay) * ndf(wm, ax, ay) / (4.0 * wa[2])


def estimator_weight(wm, wa, ax, ay, f0):
    """One term of Eq. rendering_mc with L = 1: f_r(wb, wa) |cos_b| / PDF(wb, wa).

    wb is wa reflected about the sampled normal wm.  Terms with wb below the
    surface contribute zero.
    """
    wb = reflect(wm, wa)
    below = wb[2] <= 0.0
    wb_safe = np.where(below, np.array([0.0, 0.0, 1.0]).reshape(3, *([1] * (wb.ndim - 1))), wb)
    f = brdf(wa, wb_safe, ax, ay, f0)
    w = f * np.abs(wb_safe[2]) / bsdf_pdf(wm, wa, ax, ay)
    return np.where(below, 0.0, w)


def sample_reflection(u1, u2, wa, ax, ay, f0):
    """App. A steps (1)-(2) per sample: (wb (3, N), PDF(wb) (N,), weight (N,)).

    wm is drawn with the cap sampler, wb = reflect(wm, wa) (Eq. reflect), PDF is the
    BSDF sampling density of App. A and weight the term of Eq. rendering_mc with L = 1.
    Out-of-domain samples give wb = (0, 0, 1), PDF = 0, weight = 0.
    """
    from .vndf import in_domain
    wa = np.asarray(wa, dtype=np.float64)
    ax = np.asarray(ax, dtype=np.float64)
    ay = np.asarray(ay, dtype=np.float64)
    ok = in_domain(wa, ax, ay)
    wa_u = wa / np.sqrt(dot(wa, wa))
    wm = sample_vndf(u1, u2, wa, ax, ay, "cap")
    wb = reflect(wm, wa_u)
    pdf = bsdf_pdf(wm, wa_u, ax, ay)
    w = estimator_weight(wm, wa_u, ax, ay, f0)
    fallback = np.array([0.0, 0.0, 1.0]).reshape(3, *([1] * (wb.ndim - 1)))
    return np.where(ok, wb, fallback), np.where(ok, pdf, 0.0), np.where(ok, w, 0.0)


def albedo_samples(wi, ax, ay, n, f0, seed, counter_base, stream_id):
    """Per-sample estimator terms for one query (FP64; u from the shared Philox layout)."""
    u1, u2 = philox.sample_uniforms(seed, counter_base, stream_id, n)
    wi = np.asarray(wi, dtype=np.float64).reshape(3, 1)
    wa = wi / np.sqrt(dot(wi, wi))
    wa = np.broadcast_to(wa, (3, n))
    wm = sample_vndf(u1, u2, wa, np.full(n, ax), np.full(n, ay), "cap")
    return estimator_weight(wm, wa, ax, ay, f0)


def albedo_estimate(wi, ax, ay, n_samples, f0, seed, counter_base=0, stream_base=0):
    """Directional albedo E[q] = (1/N_q) sum_j weight_j for a batch of queries.

    wi: array (3, Q); ax, ay: arrays (Q,); n_samples: ints (Q,).  Query q draws
    from Philox stream stream_base + q.
    """
    wi = np.asarray(wi, dtype=np.float64)
    out = np.empty(wi.shape[1])
    for q in range(wi.shape[1]):
        w = albedo_samples(wi[:, q], float(ax[q]), float(ay[q]), int(n_samples[q]), f0,
                           seed, counter_base, (int(stream_base) + q) & 0xFFFFFFFF)
        out[q] = w.mean() if w.size else 0.0
    return out


def albedo_quadrature(wi, ax, ay, f0, m=1024):
    """E = integral over (u1, u2) in [0,1)^2 of the weight, by an m x m midpoint rule.

    The sampler maps the unit square onto visible normals with density D_vis, so
    the expectation of the weight is this plain integral over u.
    """
    wi = np.asarray(wi, dtype=np.float64).reshape(3, 1)
    wa = wi / np.sqrt(dot(wi, wi))
    g = (np.arange(m) + 0.5) / m
    u1, u2 = np.meshgrid(g, g, indexing="ij")
    u1 = u1.reshape(-1)
    u2 = u2.reshape(-1)
    n = u1.size
    wa_b = np.broadcast_to(wa, (3, n))
    wm = sample_vndf(u1, u2, wa_b, np.full(n, ax), np.full(n, ay), "cap")
    return estimator_weight(wm, wa_b, ax, ay, f0).mean()
