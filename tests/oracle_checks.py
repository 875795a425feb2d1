"""Checks that pin the FP64 oracle to what the paper and the mathematics fix.

Each function returns a number (an error or a p-value) so the same checks can
be asserted by the pin tests and re-run on deliberately broken copies of the
oracle (the mutation test).  None of them re-derives the oracle's formulas:
they use closed forms, invariants, exact symmetries, quadrature of the
definitions, brute-force ray casting and an independent Philox implementation.
"""
import math

import numpy as np
from scipy import stats

from oracle import brute, grad, microfacet, philox, vndf

# (theta_i [deg], phi_i [deg], alpha_x, alpha_y) cases used by several pins
CASES = [
    (30.0, 40.0, 0.3, 0.3),
    (75.0, 120.0, 0.5, 0.1),
    (85.0, -60.0, 0.05, 0.2),
    (0.0, 0.0, 0.7, 0.7),
    (60.0, 10.0, 1.0, 1.0),
]


def direction(theta_deg, phi_deg):
    t = math.radians(theta_deg)
    p = math.radians(phi_deg)
    return np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])


def random_batch(n, seed, alpha_lo=1e-2, cos_lo=1e-3):
    rng = np.random.default_rng(seed)
    ct = rng.uniform(cos_lo, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    st = np.sqrt(1.0 - ct * ct)
    wi = np.stack([st * np.cos(ph), st * np.sin(ph), ct])
    ax = np.exp(rng.uniform(np.log(alpha_lo), 0.0, n))
    ay = np.exp(rng.uniform(np.log(alpha_lo), 0.0, n))
    u1 = rng.random(n)
    u2 = rng.random(n)
    return u1, u2, wi, ax, ay


def _bcast(wi, n):
    return np.broadcast_to(np.asarray(wi, np.float64).reshape(3, 1), (3, n)).copy()


# ---------------------------------------------------------------- P1 invariants
def invariants_error(n=20000, seed=1):
    """max(| |wm| - 1 |), and the minima of wm.wi and wm.z (must be > 0)."""
    u1, u2, wi, ax, ay = random_batch(n, seed)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
    return (np.abs(np.sqrt(vndf.dot(wm, wm)) - 1.0).max(),
            vndf.dot(wm, wi).min(), wm[2].min())


# ---------------------------------------------------------------- P2 mirror cap
def mirror_cap_error(n=20000, seed=2):
    """Reflecting wi' about the returned half vector must give back the cap point c (Sec. 3.2)."""
    u1, u2, wi, ax, ay = random_batch(n, seed)
    wi_std = vndf.warp_to_hemisphere(wi, ax, ay)
    h, c = vndf.sample_cap(u1, u2, wi_std)
    hn = h / np.sqrt(vndf.dot(h, h))
    d = vndf.dot(hn, wi_std)
    refl = 2.0 * d * hn - wi_std
    return np.abs(refl - c).max()


def cap_uniformity_pvalues(n=200000, seed=3, zi=0.4):
    """c.z must be uniform on [-zi, 1] and its azimuth uniform on [0, 2 pi) (Sec. 3.2, Eq. phase_function_cap)."""
    rng = np.random.default_rng(seed)
    u1 = rng.random(n)
    u2 = rng.random(n)
    wi_std = _bcast([math.sqrt(1 - zi * zi), 0.0, zi], n)
    _, c = vndf.sample_cap(u1, u2, wi_std)
    p_z = stats.kstest((c[2] + zi) / (1.0 + zi), "uniform").pvalue
    p_phi = stats.kstest(np.mod(np.arctan2(c[1], c[0]), 2 * np.pi) / (2 * np.pi), "uniform").pvalue
    return p_z, p_phi


# ---------------------------------------------------------------- P3 change of variables
def change_of_variables_error(n=5000, seed=4):
    """pdf(wm(u)) * |d wm/du1 x d wm/du2| = 1 for every sample (the sampler realises Eq. 1)."""
    u1, u2, wi, ax, ay = random_batch(n, seed)
    # keep away from the measure-zero rim where the Jacobian is singular
    u2 = np.clip(u2, 1e-6, 1 - 1e-6)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
    pdf = vndf.vndf_pdf(wm, wi, ax, ay)
    d1, d2 = grad.u_jacobian_complex_step(u1, u2, wi, ax, ay)
    cr = np.cross(d1.T, d2.T).T
    return np.abs(pdf * np.sqrt(vndf.dot(cr, cr)) - 1.0).max()


# ---------------------------------------------------------------- P4 quadrature
def hemisphere_quadrature(ax, ay, m_tau=2000, m_phi=1920):
    """Midpoint rule on the upper hemisphere with theta = atan(beta tan tau), beta = sqrt(ax ay).

    Returns (wm (3, M), weights (M,), tau (M,), phi (M,)).  The substitution
    concentrates nodes where a narrow lobe lives; the weights are the solid
    angle sin(theta) dtheta dphi of each cell.
    """
    beta = math.sqrt(ax * ay)
    tau = (np.arange(m_tau) + 0.5) * (0.5 * np.pi / m_tau)
    phi = (np.arange(m_phi) + 0.5) * (2.0 * np.pi / m_phi)
    tt = np.tan(tau)
    theta = np.arctan(beta * tt)
    dtheta = beta * (1.0 + tt * tt) / (1.0 + beta * beta * tt * tt)
    w_tau = np.sin(theta) * dtheta * (0.5 * np.pi / m_tau)
    th, ph = np.meshgrid(theta, phi, indexing="ij")
    wt, _ = np.meshgrid(w_tau, phi, indexing="ij")
    ta, _ = np.meshgrid(tau, phi, indexing="ij")
    wm = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]).reshape(3, -1)
    return wm, (wt * (2.0 * np.pi / m_phi)).reshape(-1), ta.reshape(-1), ph.reshape(-1)


def normalisation_errors(theta_deg, phi_deg, ax, ay):
    """|int pdf - 1|, |int D cos - 1| and the G1 definition (Eq. g1) by quadrature."""
    wi = direction(theta_deg, phi_deg)
    wm, w, _, _ = hemisphere_quadrature(ax, ay)
    n = wm.shape[1]
    wib = _bcast(wi, n)
    axb = np.full(n, ax)
    ayb = np.full(n, ay)
    pdf = vndf.vndf_pdf(wm, wib, axb, ayb)
    d = vndf.ndf(wm, axb, ayb)
    e_pdf = abs((pdf * w).sum() - 1.0)
    e_ndf = abs((d * wm[2] * w).sum() - 1.0)
    proj = (np.maximum(vndf.dot(wm, wib), 0.0) * d * w).sum()
    g1 = vndf.smith_g1(wi.reshape(3, 1), wi.reshape(3, 1), ax, ay)[0]
    e_g1 = abs(g1 - wi[2] / proj)
    return e_pdf, e_ndf, e_g1


# ---------------------------------------------------------------- P5 alpha = 1
def alpha_one_errors(n=20000, seed=5):
    """At alpha = 1 the stretch is the identity (Eqs. 2-4 directly).

    Returns (max rel. error of pdf vs 2 max(0, wi.wm) / (pi (1 + wz)),
             max |mz^2 - (1 - u2)| at normal incidence: the half vector of the
             pole and a uniform sphere point is cosine distributed).
    """
    u1, u2, wi, _, _ = random_batch(n, seed)
    one = np.ones(n)
    wm = vndf.sample_vndf(u1, u2, wi, one, one)
    pdf = vndf.vndf_pdf(wm, wi, one, one)
    ref = 2.0 * np.maximum(vndf.dot(wi, wm), 0.0) / (np.pi * (1.0 + wi[2]))
    e_pdf = np.abs(pdf / ref - 1.0).max()
    wz = _bcast([0.0, 0.0, 1.0], n)
    wm0 = vndf.sample_vndf(u1, u2, wz, one, one)
    e_pole = np.abs(wm0[2] ** 2 - (1.0 - u2)).max()
    return e_pdf, e_pole


def small_alpha_spread(alpha=1e-6, n=20000, seed=6):
    """Max angle between wm and the pole in units of alpha (alpha -> 0 limit)."""
    u1, u2, wi, _, _ = random_batch(n, seed, cos_lo=0.05)
    a = np.full(n, alpha)
    wm = vndf.sample_vndf(u1, u2, wi, a, a)
    ang = np.arctan2(np.hypot(wm[0], wm[1]), wm[2])
    return ang.max() / alpha


# ---------------------------------------------------------------- P10 symmetries
def symmetry_errors(n=20000, seed=7):
    """Exact symmetries of the construction (returns the max deviation of each)."""
    u1, u2, wi, ax, ay = random_batch(n, seed)
    base = vndf.sample_vndf(u1, u2, wi, ax, ay)
    # rotate wi by pi about z, shift the azimuth by half a turn
    r = vndf.sample_vndf(np.mod(u1 + 0.5, 1.0), u2, np.stack([-wi[0], -wi[1], wi[2]]), ax, ay)
    e_rot = max(np.abs(r[0] + base[0]).max(), np.abs(r[1] + base[1]).max(), np.abs(r[2] - base[2]).max())
    # mirror y, reverse the azimuth
    m = vndf.sample_vndf(np.mod(1.0 - u1, 1.0), u2, np.stack([wi[0], -wi[1], wi[2]]), ax, ay)
    e_mir = max(np.abs(m[0] - base[0]).max(), np.abs(m[1] + base[1]).max(), np.abs(m[2] - base[2]).max())
    # swap the x and y axes together with the roughnesses: azimuth phi -> pi/2 - phi
    s = vndf.sample_vndf(np.mod(0.25 - u1, 1.0), u2, np.stack([wi[1], wi[0], wi[2]]), ay, ax)
    e_swp = max(np.abs(s[0] - base[1]).max(), np.abs(s[1] - base[0]).max(), np.abs(s[2] - base[2]).max())
    return e_rot, e_mir, e_swp


# ---------------------------------------------------------------- histogram tests (P7, P8, P9)
N_TAU_BINS = 20
N_PHI_BINS = 24


def bin_index(wm, ax, ay):
    """Histogram bin of each normal in (tau, phi) cells matching ``hemisphere_quadrature``."""
    beta = math.sqrt(ax * ay)
    theta = np.arctan2(np.hypot(wm[0], wm[1]), wm[2])
    tau = np.arctan(np.tan(theta) / beta)
    phi = np.mod(np.arctan2(wm[1], wm[0]), 2 * np.pi)
    it = np.clip((tau / (0.5 * np.pi) * N_TAU_BINS).astype(int), 0, N_TAU_BINS - 1)
    ip = np.clip((phi / (2 * np.pi) * N_PHI_BINS).astype(int), 0, N_PHI_BINS - 1)
    return it * N_PHI_BINS + ip


def counts(wm, ax, ay):
    return np.bincount(bin_index(wm, ax, ay), minlength=N_TAU_BINS * N_PHI_BINS).astype(np.float64)


def two_sample_chi2_pvalue(a, b, min_count=10):
    """Two-sample chi-square homogeneity test on histogram counts a, b."""
    keep = (a + b) >= min_count
    ra, rb = a.sum(), b.sum()
    k1 = math.sqrt(rb / ra)
    k2 = math.sqrt(ra / rb)
    aa = np.append(a[keep], a[~keep].sum())
    bb = np.append(b[keep], b[~keep].sum())
    m = (aa + bb) > 0
    aa, bb = aa[m], bb[m]
    chi2 = (((k1 * aa - k2 * bb) ** 2) / (aa + bb)).sum()
    return stats.chi2.sf(chi2, aa.size - 1)


def expected_bin_probabilities(wi, ax, ay):
    """Integral of the pdf over each histogram bin (quadrature of Eq. 1)."""
    wm, w, tau, phi = hemisphere_quadrature(ax, ay)
    n = wm.shape[1]
    pdf = vndf.vndf_pdf(wm, _bcast(wi, n), np.full(n, ax), np.full(n, ay))
    it = np.clip((tau / (0.5 * np.pi) * N_TAU_BINS).astype(int), 0, N_TAU_BINS - 1)
    ip = np.clip((phi / (2 * np.pi) * N_PHI_BINS).astype(int), 0, N_PHI_BINS - 1)
    return np.bincount(it * N_PHI_BINS + ip, weights=pdf * w, minlength=N_TAU_BINS * N_PHI_BINS)


def sample_case(theta_deg, phi_deg, ax, ay, n, seed, method="cap"):
    rng = np.random.default_rng(seed)
    wi = direction(theta_deg, phi_deg)
    u1 = rng.random(n)
    u2 = rng.random(n)
    return vndf.sample_vndf(u1, u2, _bcast(wi, n), np.full(n, ax), np.full(n, ay), method)


def chi2_vs_pdf_pvalue(theta_deg, phi_deg, ax, ay, n=1_000_000, seed=8):
    """P8: sampled histogram against expected counts from the pdf."""
    wm = sample_case(theta_deg, phi_deg, ax, ay, n, seed)
    return chi2_samples_vs_pdf_pvalue(wm, direction(theta_deg, phi_deg), ax, ay)


def chi2_samples_vs_pdf_pvalue(wm, wi, ax, ay):
    """Chi-square p-value of the normals wm (3, n), drawn for one (wi, ax, ay), against the expected
    counts from the quadrature of Eq. 1 over each histogram bin (bins with fewer than 5 pooled)."""
    n = wm.shape[1]
    obs = counts(wm, ax, ay)
    exp = n * expected_bin_probabilities(wi, ax, ay)
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    m = e > 0
    chi2 = (((o - e) ** 2) / e)[m].sum()
    return stats.chi2.sf(chi2, m.sum() - 1)


def brute_force_pvalue(theta_deg, phi_deg, ax, ay, n=1_000_000, seed=9):
    """P9: cap sampler against ray casting on the truncated ellipsoid (definition, Sec. 2)."""
    rng = np.random.default_rng(seed)
    ref = brute.visible_normals(direction(theta_deg, phi_deg), ax, ay, n, rng)
    wm = sample_case(theta_deg, phi_deg, ax, ay, n, seed + 1)
    return two_sample_chi2_pvalue(counts(wm, ax, ay), counts(ref, ax, ay))


def prior_agreement_pvalue(theta_deg, phi_deg, ax, ay, n=1_000_000, seed=10):
    """P7: cap sampler against the prior polar-disk sampler (same distribution claimed)."""
    a = sample_case(theta_deg, phi_deg, ax, ay, n, seed, "cap")
    b = sample_case(theta_deg, phi_deg, ax, ay, n, seed + 1, "polar")
    return two_sample_chi2_pvalue(counts(a, ax, ay), counts(b, ax, ay))


# ---------------------------------------------------------------- gradients (P11)
def gradient_errors(n=400, seed=11):
    """(complex step vs central differences, relative), and max |g_wi . wi| (degree-0 homogeneity)."""
    u1, u2, wi, ax, ay = random_batch(n, seed, alpha_lo=0.05, cos_lo=0.05)
    u2 = np.clip(u2, 1e-3, 1 - 1e-3)
    jc = grad.jacobian_complex_step(u1, u2, wi, ax, ay)
    jf = grad.jacobian_central_difference(u1, u2, wi, ax, ay)
    scale = np.abs(jc).max(axis=0, keepdims=True) + 1e-12
    e_fd = (np.abs(jc - jf) / scale).max()
    e_hom = np.abs((jc[:3] * wi[:, None, :]).sum(axis=0)).max() / np.abs(jc).max()
    return e_fd, e_hom


# ---------------------------------------------------------------- albedo (P12)
def smith_lambda_textbook(w, ax, ay):
    """GGX Smith Lambda (Heitz 2014, JCGT 3(2)): (-1 + sqrt(1 + (ax^2 x^2 + ay^2 y^2) / z^2)) / 2."""
    return 0.5 * (-1.0 + np.sqrt(1.0 + (ax * ax * w[0] ** 2 + ay * ay * w[1] ** 2) / w[2] ** 2))


def g1_g2_textbook_errors(n=5000, seed=12):
    """G1 = 1/(1 + Lambda) and height-correlated G2 = 1/(1 + Lambda_i + Lambda_o)."""
    u1, u2, wi, ax, ay = random_batch(n, seed, cos_lo=0.05)
    _, _, wo, _, _ = random_batch(n, seed + 1, cos_lo=0.05)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
    vis = (vndf.dot(wm, wo) > 0)
    li = smith_lambda_textbook(wi, ax, ay)
    lo = smith_lambda_textbook(wo, ax, ay)
    e1 = np.abs(vndf.smith_g1(wm, wi, ax, ay) - 1.0 / (1.0 + li)).max()
    g2 = microfacet.smith_g2(wm, wi, wo, ax, ay)
    e2 = np.abs(g2[vis] - 1.0 / (1.0 + li[vis] + lo[vis])).max()
    return e1, e2


def brdf_albedo_quadrature(wi, ax, ay, f0, m_theta=1500, m_phi=1500):
    """E = integral over the upper hemisphere of f_r(wi, wo) cos(theta_o) (Eq. rendering, L = 1)."""
    th = (np.arange(m_theta) + 0.5) * (0.5 * np.pi / m_theta)
    ph = (np.arange(m_phi) + 0.5) * (2 * np.pi / m_phi)
    t, p = np.meshgrid(th, ph, indexing="ij")
    wo = np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)]).reshape(3, -1)
    dw = (np.sin(t) * (0.5 * np.pi / m_theta) * (2 * np.pi / m_phi)).reshape(-1)
    n = wo.shape[1]
    f = microfacet.brdf(_bcast(wi, n), wo, ax, ay, f0)
    return (f * wo[2] * dw).sum()


def albedo_consistency_error(theta_deg, ax, ay, f0=0.04):
    """Importance-sampled albedo (quadrature over u) vs direct BRDF integration over wo."""
    wi = direction(theta_deg, 0.0)
    e_u = microfacet.albedo_quadrature(wi, ax, ay, f0, m=1024)
    e_w = brdf_albedo_quadrature(wi, ax, ay, f0)
    return abs(e_u - e_w)


def reflection_errors(n=5000, seed=13):
    """Eq. halfvector inverts Eq. reflect: normalize(wa + wb) = wm and |wb| = 1."""
    u1, u2, wi, ax, ay = random_batch(n, seed, cos_lo=0.05)
    wa = wi
    wm = vndf.sample_vndf(u1, u2, wa, ax, ay)
    wb = microfacet.reflect(wm, wa)
    h = wa + wb
    hn = h / np.sqrt(vndf.dot(h, h))
    return np.abs(hn - wm).max(), np.abs(np.sqrt(vndf.dot(wb, wb)) - 1.0).max()


def reflected_change_of_variables_error(n=2000, seed=14):
    """PDF(wb) |d wb/du1 x d wb/du2| = 1: the BSDF pdf of App. A (with Eq. jacobian) is
    the density of the reflected direction, checked pointwise through the sampler."""
    u1, u2, wa, ax, ay = random_batch(n, seed, alpha_lo=0.05, cos_lo=0.05)
    u2 = np.clip(u2, 1e-4, 1 - 1e-4)
    wm = vndf.sample_vndf(u1, u2, wa, ax, ay)
    pdf = microfacet.bsdf_pdf(wm, wa, ax, ay)

    def wb_of(v1, v2):
        return microfacet.reflect(vndf.sample_vndf(v1, v2, wa.astype(np.complex128), ax, ay), wa)

    d1 = np.imag(wb_of(u1 + 1j * grad.H_CS, u2.astype(np.complex128))) / grad.H_CS
    d2 = np.imag(wb_of(u1.astype(np.complex128), u2 + 1j * grad.H_CS)) / grad.H_CS
    cr = np.cross(d1.T, d2.T).T
    return np.abs(pdf * np.sqrt(vndf.dot(cr, cr)) - 1.0).max()


# ---------------------------------------------------------------- the extended domain (wi below the horizon)
EXT_CASES = [
    (100.0, 40.0, 0.5, 0.3),
    (120.0, -60.0, 0.8, 0.6),
    (95.0, 10.0, 0.2, 0.25),
    (90.0, 30.0, 0.4, 0.7),
    (150.0, 0.0, 1.0, 1.0),
]


def random_batch_extended(n, seed, alpha_lo=1e-2, cos_lo=-0.95):
    """Directions with cos(theta_i) uniform in [cos_lo, 1] (most below the horizon when cos_lo ~ -1)."""
    return random_batch(n, seed, alpha_lo=alpha_lo, cos_lo=cos_lo)


def extended_mirror_cap_error(n=20000, seed=21):
    """Sec. 3.2's mirror property below the horizon: reflecting wi' about h/|h| gives c back.

    Rounding in h/|h| grows like eps/|h|, and below the horizon the whole cap can be small
    (|h|^2 <= 2 (1 + z_i')), so the error is returned scaled by min(1, |h|)."""
    u1, u2, wi, ax, ay = random_batch_extended(n, seed)
    wi_std = vndf.warp_to_hemisphere(wi, ax, ay)
    h, c = vndf.sample_cap(u1, u2, wi_std)
    hl = np.sqrt(vndf.dot(h, h))
    hn = h / hl
    refl = 2.0 * vndf.dot(hn, wi_std) * hn - wi_std
    return (np.abs(refl - c).max(axis=0) * np.minimum(hl, 1.0)).max()


def extended_cap_uniformity_pvalues(n=200000, seed=22, zi=-0.6):
    return cap_uniformity_pvalues(n=n, seed=seed, zi=zi)


def extended_change_of_variables_error(n=5000, seed=23):
    """pdf(wm(u)) |d wm/du1 x d wm/du2| = 1 pointwise for incident directions below the horizon."""
    u1, u2, wi, ax, ay = random_batch_extended(n, seed, cos_lo=-0.9)
    u2 = np.clip(u2, 1e-6, 1 - 1e-6)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay, extended=True)
    pdf = vndf.vndf_pdf(wm, wi, ax, ay, extended=True)
    d1, d2 = grad.u_jacobian_complex_step(u1, u2, wi, ax, ay, extended=True)
    cr = np.cross(d1.T, d2.T).T
    return np.abs(pdf * np.sqrt(vndf.dot(cr, cr)) - 1.0).max()


def extended_normalisation_errors(theta_deg, phi_deg, ax, ay):
    """|int pdf - 1| and |int max(0, wi.wm) D - (|M^-1 wi| + wi.z)/2| by quadrature, any theta_i."""
    wi = direction(theta_deg, phi_deg)
    wm, w, _, _ = hemisphere_quadrature(ax, ay)
    n = wm.shape[1]
    wib = _bcast(wi, n)
    axb = np.full(n, ax)
    ayb = np.full(n, ay)
    pdf = vndf.vndf_pdf(wm, wib, axb, ayb, extended=True)
    proj = (np.maximum(vndf.dot(wm, wib), 0.0) * vndf.ndf(wm, axb, ayb) * w).sum()
    closed = 0.5 * (math.sqrt((ax * wi[0]) ** 2 + (ay * wi[1]) ** 2 + wi[2] ** 2) + wi[2])
    return abs((pdf * w).sum() - 1.0), abs(proj - closed) / closed


def extended_alpha_one_errors(n=20000, seed=24):
    """alpha = 1: wm = normalize(c + wi) and pdf = 2 max(0, wi.wm) / (pi (1 + wi.z)) for any wi.z > -1."""
    u1, u2, wi, _, _ = random_batch_extended(n, seed)
    one = np.ones(n)
    wm = vndf.sample_vndf(u1, u2, wi, one, one, extended=True)
    _, c = vndf.sample_cap(u1, u2, wi)
    ref = (c + wi) / np.sqrt(vndf.dot(c + wi, c + wi))
    pdf = vndf.vndf_pdf(wm, wi, one, one, extended=True)
    closed = 2.0 * np.maximum(vndf.dot(wi, wm), 0.0) / (np.pi * (1.0 + wi[2]))
    return np.abs(wm - ref).max(), np.abs(pdf / closed - 1.0).max()


def horizon_continuity_error(n=5000, seed=25, eps=1e-9):
    """The extended sampler is one construction across the horizon: wi.z = +eps and -eps give the
    same normals and densities up to O(eps)."""
    rng = np.random.default_rng(seed)
    u1, u2 = rng.random(n), rng.random(n)
    ph = rng.uniform(0, 2 * np.pi, n)
    ax = np.exp(rng.uniform(np.log(0.05), 0.0, n))
    ay = np.exp(rng.uniform(np.log(0.05), 0.0, n))
    out = []
    for z in (eps, -eps):
        wi = np.stack([np.cos(ph), np.sin(ph), np.full(n, z)])
        out.append(vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, extended=True))
    (wa, pa), (wb, pb) = out
    return np.abs(wa - wb).max(), np.abs(pa / pb - 1.0).max()


def extended_expected_bin_probabilities(wi, ax, ay):
    wm, w, tau, phi = hemisphere_quadrature(ax, ay)
    n = wm.shape[1]
    pdf = vndf.vndf_pdf(wm, _bcast(wi, n), np.full(n, ax), np.full(n, ay), extended=True)
    it = np.clip((tau / (0.5 * np.pi) * N_TAU_BINS).astype(int), 0, N_TAU_BINS - 1)
    ip = np.clip((phi / (2 * np.pi) * N_PHI_BINS).astype(int), 0, N_PHI_BINS - 1)
    return np.bincount(it * N_PHI_BINS + ip, weights=pdf * w, minlength=N_TAU_BINS * N_PHI_BINS)


def _extended_case(theta_deg, phi_deg, ax, ay, n, seed):
    rng = np.random.default_rng(seed)
    u1, u2 = rng.random(n), rng.random(n)
    return vndf.sample_vndf(u1, u2, _bcast(direction(theta_deg, phi_deg), n), np.full(n, ax), np.full(n, ay),
                            extended=True)


def extended_chi2_vs_pdf_pvalue(theta_deg, phi_deg, ax, ay, n=1_000_000, seed=26):
    wm = _extended_case(theta_deg, phi_deg, ax, ay, n, seed)
    return extended_chi2_samples_vs_pdf_pvalue(wm, direction(theta_deg, phi_deg), ax, ay)


def extended_chi2_samples_vs_pdf_pvalue(wm, wi, ax, ay):
    """Chi-square p-value of normals wm (3, n) drawn for one wi (below the horizon allowed) against
    the quadrature of the extended density over each histogram bin."""
    n = wm.shape[1]
    obs = counts(wm, ax, ay)
    exp = n * extended_expected_bin_probabilities(wi, ax, ay)
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    m = e > 0
    chi2 = (((o - e) ** 2) / e)[m].sum()
    return stats.chi2.sf(chi2, m.sum() - 1)


def extended_brute_force_pvalue(theta_deg, phi_deg, ax, ay, n=1_000_000, seed=27):
    """Ray casting from below the horizon: first hits on the ellipsoid with z >= 0 (Sec. 2's definition)."""
    rng = np.random.default_rng(seed)
    ref = brute.visible_normals(direction(theta_deg, phi_deg), ax, ay, n, rng)
    wm = _extended_case(theta_deg, phi_deg, ax, ay, n, seed + 1)
    return two_sample_chi2_pvalue(counts(wm, ax, ay), counts(ref, ax, ay))


def hemisphere_sampler_errors(n=20000, seed=28):
    """The stand-alone hemisphere sampler against the GGX sampler at alpha = 1 (where D = 1/pi, the
    hemisphere configuration itself) and its density against Eq. 2 evaluated at the sample."""
    u1, u2, wi, _, _ = random_batch_extended(n, seed)
    scale = np.exp(np.random.default_rng(seed + 1).uniform(-3, 3, n))  # any length
    wm, pdf = vndf.sample_hemisphere(u1, u2, wi * scale)
    one = np.ones(n)
    ref, ref_pdf = vndf.sample_vndf_with_pdf(u1, u2, wi, one, one, extended=True)
    unit = np.abs(np.sqrt(vndf.dot(wm, wm)) - 1.0).max()
    return np.abs(wm - ref).max(), np.abs(pdf / ref_pdf - 1.0).max(), unit


def extended_gradient_errors(n=400, seed=32):
    """Below the horizon: complex step vs central differences (relative to the largest entry) and the
    degree-0 homogeneity g_wi . wi = 0 of every output."""
    u1, u2, wi, ax, ay = random_batch_extended(n, seed, alpha_lo=0.1, cos_lo=-0.7)
    u2 = np.clip(u2, 1e-3, 1 - 1e-3)
    jc = grad.jacobian_complex_step(u1, u2, wi, ax, ay, extended=True)
    jf = grad.jacobian_central_difference(u1, u2, wi, ax, ay, extended=True)
    scale = np.abs(jc).max(axis=0, keepdims=True) + 1e-12
    e_fd = (np.abs(jc - jf) / scale).max()
    e_hom = np.abs((jc[:3] * wi[:, None, :]).sum(axis=0)).max() / np.abs(jc).max()
    below = (wi[2] < 0).mean()
    return e_fd, e_hom, below


# ----------------------------------------------------------------------------
# Stored 50-digit samples (tests/golden/cap_samples_mp50.txt)
# ----------------------------------------------------------------------------

def golden_rows():
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    if here not in sys.path:
        sys.path.insert(0, here)
    import make_golden
    return make_golden.load()


def golden_jacobians():
    """{row index: 5 x 4 stored 50-digit Jacobian [input][output]} (tests/golden/cap_jacobians_mp50.txt)."""
    golden_rows()  # puts tests/golden on the path
    import make_golden
    return make_golden.load_jacobians()


def golden_reflection():
    """{row index: (wo (3,), pdf, weight)} stored at 50 digits (tests/golden/reflection_mp50.txt)."""
    golden_rows()
    import make_golden
    return make_golden.load_reflection()


def golden_oracle_sample(r):
    """The FP64 oracle's (wm, pdf) for one stored row.

    For the GGX rows the density is the oracle's Eq. 1 at its own hemisphere
    sample (vndf_pdf_at_cap_sample), which does not cancel; the definition form
    through wi.wm does cancel next to the visibility boundary (the cap's rim as
    u2 -> 1) and is pinned at the stored normal by a test of its own."""
    wi = r["wi"].reshape(3, 1)
    ax, ay = np.array([r["alpha_x"]]), np.array([r["alpha_y"]])
    u1, u2 = np.array([r["u1"]]), np.array([r["u2"]])
    if r["kind"] == "hemisphere":
        wm, pdf = vndf.sample_hemisphere(u1, u2, wi)
    else:
        ext = r["kind"] == "cap_extended"
        wm = vndf.sample_vndf(u1, u2, wi, ax, ay, "cap", ext)
        ok = vndf.in_domain(wi, ax, ay, ext)
        pdf = np.where(ok, vndf.vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay, ext), 0.0) if ok.all() else np.zeros(1)
    return wm[:, 0], float(pdf[0])


def golden_row_error(r):
    """(angle, pdf relative error, bound) of the FP64 oracle against one stored row.

    The bound is FP64 rounding amplified by 1 / (1 + z_i') where the cap bottom
    -z_i' is subtracted (Sec. 3.3), and by 1 / sin(theta) where sqrt(1 - z^2) is
    formed from z as the paper writes it (1 - z = u2 (1 + z_i'), so
    1 - z^2 = u2 a (2 - u2 a) with a = 1 + z_i').  The pdf is held to 4x the bound.
    Out-of-domain rows give (0, 0, 1) exactly or an infinite error.
    """
    wm, pdf = golden_oracle_sample(r)
    a = r["one_plus_zi"]
    if math.isnan(a):
        exact = tuple(wm) == (0.0, 0.0, 1.0) and pdf == 0.0
        return (0.0, 0.0, 1.0) if exact else (math.inf, math.inf, 1.0)
    eps = 2.0 ** -52
    s = r["u2"] * a * (2.0 - r["u2"] * a)
    tol = 64 * eps * max(1.0, 1.0 / a) + 8 * eps / max(math.sqrt(s), 2.0 ** -26)
    cr = np.cross(wm, r["wm"])
    ang = math.atan2(float(np.linalg.norm(cr)), float(wm @ r["wm"]))
    return ang, abs(pdf / r["pdf"] - 1.0), tol


def golden_excess():
    """Largest error / bound over the stored rows (<= 1 when the oracle agrees)."""
    worst = 0.0
    for r in golden_rows():
        ang, rel, tol = golden_row_error(r)
        worst = max(worst, ang / tol, rel / (4 * tol))
    return worst
