"""Pins for the oracle's sampler and pdf: invariants, closed forms, exact symmetries.

P1  per-sample invariants of the sampled normal (unit length, visible, upper hemisphere)
P2  mirror-cap theorem of Sec. 3.2: reflecting wi about the half vector gives the cap point,
    and the cap points are uniform in height and azimuth (Eq. phase_function_cap)
P3  change of variables: pdf(wm(u)) |d wm/du1 x d wm/du2| = 1 (the sampler realises Eq. 1)
P5  alpha = 1: Eqs. 2-4 without a stretch; normal incidence gives a cosine-weighted normal
P6  alpha -> 0: normals collapse onto the pole at a rate O(alpha)
P10 exact symmetries (rotation by pi, mirror in y, x/y swap with the roughnesses)
    which catch swapped axes and sign errors
"""
import numpy as np

import oracle_checks as oc
from oracle import vndf


def test_p1_invariants():
    norm_err, min_dot, min_z = oc.invariants_error()
    assert norm_err < 1e-14
    assert min_dot > 0.0
    assert min_z > 0.0


def test_p2_mirror_cap_reflection():
    assert oc.mirror_cap_error() < 1e-13


def test_p2_cap_is_uniform():
    p_z, p_phi = oc.cap_uniformity_pvalues()
    assert p_z > 1e-3 and p_phi > 1e-3


def test_p3_change_of_variables():
    assert oc.change_of_variables_error() < 1e-9


def test_p5_alpha_one_closed_form():
    e_pdf, e_pole = oc.alpha_one_errors()
    assert e_pdf < 1e-13
    assert e_pole < 1e-14


def test_p6_small_alpha_collapses_to_pole():
    assert oc.small_alpha_spread(alpha=1e-6) < 1e3


def test_p10_symmetries():
    for e in oc.symmetry_errors():
        assert e < 1e-13


def test_eq1_equals_app_a_form():
    """Eq. 1 (transformed hemisphere VNDF) and G1 max(0, wi.wm) D / wz (App. A) agree."""
    u1, u2, wi, ax, ay = oc.random_batch(20000, 13, alpha_lo=1e-3)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
    p1 = vndf.vndf_pdf(wm, wi, ax, ay)
    p2 = vndf.vndf_pdf_eq1(wm, wi, ax, ay)
    assert np.abs(p1 / p2 - 1.0).max() < 1e-12


def test_sigma_std_is_projected_area():
    """Eq. 4: integral of max(wm.wi, 0) D_std over the sphere is (1 + zi)/2."""
    wm, w, _, _ = oc.hemisphere_quadrature(1.0, 1.0, 1000, 960)
    for th in (0.0, 40.0, 89.0):
        wi = oc.direction(th, 25.0)
        val = (np.maximum(vndf.dot(wm, wi.reshape(3, 1)), 0.0) * vndf.ndf_std(wm) * w).sum()
        assert abs(val - vndf.sigma_std(wi[2])) < 1e-6


def test_domain_fallback():
    wi = np.array([[0.1, 0.1, 0.0, 0.2], [0.0, 0.0, 0.3, 0.1], [-0.5, 0.0, 0.9, 0.9]])
    ax = np.array([0.5, 0.5, 0.0, np.nan])
    ay = np.array([0.5, 0.5, 0.5, 0.5])
    u = np.full(4, 0.3)
    wm, pdf = vndf.sample_vndf_with_pdf(u, u, wi, ax, ay)
    np.testing.assert_array_equal(wm, np.tile(np.array([[0.0], [0.0], [1.0]]), (1, 4)))
    np.testing.assert_array_equal(pdf, np.zeros(4))


def test_scale_invariance_in_wi():
    u1, u2, wi, ax, ay = oc.random_batch(1000, 14)
    a, pa = vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay)
    b, pb = vndf.sample_vndf_with_pdf(u1, u2, 3.7 * wi, ax, ay)
    assert np.abs(a - b).max() < 1e-14
    assert np.abs(pa / pb - 1).max() < 1e-13


def test_prior_sampler_invariants_and_pole_case():
    u1, u2, wi, ax, ay = oc.random_batch(20000, 15)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay, "polar")
    assert np.abs(np.sqrt(vndf.dot(wm, wm)) - 1).max() < 1e-14
    assert vndf.dot(wm, wi).min() > 0.0
    # normal incidence takes the special-case basis; alpha = 1 gives mz^2 = 1 - u2 there too
    n = u1.size
    one = np.ones(n)
    pole = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, n))
    wp = vndf.sample_vndf(u1, u2, pole, one, one, "polar")
    assert np.abs(wp[2] ** 2 - (1 - u2)).max() < 1e-13


def test_pdf_at_cap_sample_equals_definition():
    """The hemisphere-sample form of Eq. 1 agrees with G1 max(0, wi.wm) D / wz where the latter is
    well conditioned (away from the visibility boundary)."""
    u1, u2, wi, ax, ay = oc.random_batch(20000, 16, alpha_lo=1e-3)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
    p_def = vndf.vndf_pdf(wm, wi, ax, ay)
    p_cap = vndf.vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay)
    good = vndf.dot(wm, wi) / np.sqrt(vndf.dot(wi, wi)) > 1e-3
    assert good.mean() > 0.99
    assert np.abs(p_cap[good] / p_def[good] - 1).max() < 1e-10
