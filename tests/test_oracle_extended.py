"""Pins of the oracle's extended domain (incident directions below the horizon) and of the
stand-alone hemisphere sampler (Sec. 3.3 with its normalisation).

The paper states the cap construction for the upper hemisphere only; nothing in
Sec. 3.2-3.3 or Eq. 4 uses wi.z > 0.  These checks fix the extension by what the
mathematics fixes: the mirror property of the cap, the change of variables per
sample, normalisation and the projected area by quadrature, the alpha = 1
closed form, continuity across the horizon, a histogram against the density,
and ray casting on the ellipsoid from below the horizon.
"""
import numpy as np
import pytest

import oracle_checks as oc
from oracle import vndf


def test_mirror_cap_below_horizon():
    assert oc.extended_mirror_cap_error() < 1e-13


def test_cap_uniform_below_horizon():
    p_z, p_phi = oc.extended_cap_uniformity_pvalues()
    assert p_z > 1e-3 and p_phi > 1e-3


def test_change_of_variables_below_horizon():
    assert oc.extended_change_of_variables_error() < 1e-8


@pytest.mark.parametrize("case", oc.EXT_CASES)
def test_normalisation_and_projected_area(case):
    e_pdf, e_sigma = oc.extended_normalisation_errors(*case)
    assert e_pdf < 1e-6, e_pdf
    assert e_sigma < 1e-6, e_sigma


def test_alpha_one_closed_form_below_horizon():
    e_wm, e_pdf = oc.extended_alpha_one_errors()
    assert e_wm < 1e-13 and e_pdf < 1e-12


def test_continuous_across_horizon():
    e_wm, e_pdf = oc.horizon_continuity_error()
    assert e_wm < 1e-7 and e_pdf < 1e-6


@pytest.mark.parametrize("case", oc.EXT_CASES[:3])
def test_histogram_matches_pdf_below_horizon(case):
    assert oc.extended_chi2_vs_pdf_pvalue(*case, n=400_000) > 1e-3


@pytest.mark.parametrize("case", [(110.0, 30.0, 0.6, 0.4), (135.0, -45.0, 1.0, 0.5)])
def test_matches_ray_casting_below_horizon(case):
    assert oc.extended_brute_force_pvalue(*case, n=400_000) > 1e-3


def test_extended_equals_upper_domain_above_horizon():
    u1, u2, wi, ax, ay = oc.random_batch(5000, 29)
    a = vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay)
    b = vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, extended=True)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_allclose(b[1], a[1], rtol=1e-13)
    np.testing.assert_allclose(vndf.vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay, extended=True),
                               vndf.vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay), rtol=0)


def test_pdf_forms_agree_below_horizon():
    """The projected-area form, Eq. 1 written literally and the at-sample form are one density."""
    u1, u2, wi, ax, ay = oc.random_batch_extended(5000, 30, cos_lo=-0.9)
    wm = vndf.sample_vndf(u1, u2, wi, ax, ay, extended=True)
    p = vndf.vndf_pdf(wm, wi, ax, ay, extended=True)
    np.testing.assert_allclose(vndf.vndf_pdf_eq1(wm, wi, ax, ay), p, rtol=1e-9)
    np.testing.assert_allclose(vndf.vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay, extended=True), p, rtol=1e-9)


def test_hemisphere_sampler():
    e_wm, e_pdf, e_unit = oc.hemisphere_sampler_errors()
    # wi is rescaled before normalising, so the two differ by rounding amplified near small |h|
    assert e_wm < 1e-12 and e_pdf < 1e-10 and e_unit < 1e-15


def test_extended_domain_edges():
    one = np.ones(6)
    wi = np.array([[0.0, 1e-5, 1e-7, 0.0, 0.6, np.nan],
                   [0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                   [-1.0, -1.0, -1.0, 0.0, -0.8, 0.5]])
    u = np.full(6, 0.3)
    wm, pdf = vndf.sample_vndf_with_pdf(u, u, wi, one, one, extended=True)
    # straight down, (1 + z_i') = 5e-15 < 2^-40 (outside), the zero vector, NaN: fallback
    for k in (0, 2, 3, 5):
        assert wm[2, k] == 1.0 and pdf[k] == 0.0
    # (1 + z_i') = 5e-11 and an ordinary below-horizon direction: inside
    assert pdf[1] > 0 and pdf[4] > 0 and wm[2, 1] > 0 and wm[2, 4] > 0
    # the prior sampler has no extended domain
    with pytest.raises(ValueError):
        vndf.sample_vndf(u, u, wi, one, one, "polar", extended=True)
    # the upper-domain oracle keeps its fallback for wi.z <= 0
    assert np.all(vndf.vndf_pdf(wm, wi, one, one)[[1, 4]] == 0.0)


def test_mp_reference_agrees_with_fp64_where_fp64_is_accurate():
    """The 50-digit restatement against the FP64 oracle on well-conditioned samples, and against
    the alpha = 1 closed form (Eqs. 2-4 with D = 1/pi) for directions below the horizon."""
    mp = pytest.importorskip("oracle.vndf_mp")
    u1, u2, wi, ax, ay = oc.random_batch_extended(200, 31, alpha_lo=0.1, cos_lo=-0.5)
    wm, pdf = vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, extended=True)
    for k in range(200):
        m, p = mp.sample_with_pdf(u1[k], u2[k], wi[:, k], ax[k], ay[k])
        assert np.abs(np.array(m) - wm[:, k]).max() < 1e-12
        assert abs(p / pdf[k] - 1) < 1e-10
    for k in range(50):
        m, p = mp.sample_with_pdf(u1[k], u2[k], wi[:, k], 1.0, 1.0)
        closed = 2 * max(0.0, float(np.dot(wi[:, k], m))) / (np.pi * (1 + wi[2, k]))
        assert abs(p / closed - 1) < 1e-13


def test_fp64_oracle_loses_digits_at_tiny_one_plus_zi():
    """Why the 50-digit reference exists: at 1 + z_i' ~ 1e-11 the FP64 oracle's pdf is off by far more
    than its accuracy elsewhere, while the 50-digit value keeps the alpha = 1 closed form."""
    mp = pytest.importorskip("oracle.vndf_mp")
    wi = np.array([4.5e-6, 0.0, -1.0])
    m, p = mp.sample_with_pdf(0.3, 0.7, wi, 1.0, 1.0)
    a = mp.one_plus_zi(wi, 1.0, 1.0)
    assert 1e-11 < a < 1e-10
    closed = 2 * max(0.0, float(np.dot(wi / np.linalg.norm(wi), m))) / (np.pi * a)
    assert abs(p / closed - 1) < 1e-6
    wm, pd = vndf.sample_vndf_with_pdf(np.array([0.3]), np.array([0.7]), wi.reshape(3, 1), np.ones(1), np.ones(1),
                                       extended=True)
    assert abs(pd[0] / p - 1) > 1e-7 and np.abs(wm[:, 0] - m).max() > 1e-7  # FP64: ~1e-6 off here


def test_gradients_below_horizon():
    """The complex-step derivative of the extended sampler and density against central differences, and
    the degree-0 homogeneity in wi that every output has."""
    e_fd, e_hom, below = oc.extended_gradient_errors()
    assert below > 0.3
    assert e_fd < 1e-6, e_fd
    assert e_hom < 1e-12, e_hom
