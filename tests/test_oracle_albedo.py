"""P12 and App. A pins for the albedo estimator pieces.

* G1 and the height-correlated G2 match the textbook GGX Smith Lambda form
  (Heitz 2014, JCGT 3(2)): G1 = 1/(1 + Lambda), G2 = 1/(1 + Lambda_i + Lambda_o).
* The importance-sampled albedo (VNDF samples, reflection, weight f cos / PDF)
  equals the albedo obtained by integrating the Cook-Torrance BRDF directly over
  outgoing directions: this ties the sampler, the reflection Jacobian (Eq. jacobian)
  and the BSDF pdf of App. A together.
* 0 <= E <= 1; alpha -> 0 gives a mirror, E -> F(cos theta_i).
* The Philox Monte Carlo estimate agrees with the quadrature within 4 sigma.
"""
import numpy as np
import pytest

import oracle_checks as oc
from oracle import microfacet


def test_g1_g2_textbook_forms():
    e1, e2 = oc.g1_g2_textbook_errors()
    assert e1 < 1e-13 and e2 < 1e-13


@pytest.mark.parametrize("theta,alpha", [(30.0, 0.3), (70.0, 0.6), (10.0, 1.0), (80.0, 0.25)])
def test_importance_sampled_albedo_equals_brdf_integral(theta, alpha):
    assert oc.albedo_consistency_error(theta, alpha, alpha) < 1e-5


def test_schlick_endpoints():
    assert microfacet.schlick_fresnel(1.0, 0.04) == 0.04
    assert microfacet.schlick_fresnel(0.0, 0.04) == 1.0


def test_albedo_bounds_and_mirror_limit():
    for th in (5.0, 45.0, 80.0):
        wi = oc.direction(th, 0.0)
        for a in (1e-3, 0.1, 0.5, 1.0):
            e = microfacet.albedo_quadrature(wi, a, a, 0.04, m=256)
            assert 0.0 <= e <= 1.0
        e0 = microfacet.albedo_quadrature(wi, 1e-5, 1e-5, 0.04, m=256)
        assert abs(e0 - microfacet.schlick_fresnel(wi[2], 0.04)) < 1e-3


def test_monte_carlo_estimate_within_4_sigma():
    wi = oc.direction(50.0, 0.0)
    w = microfacet.albedo_samples(wi, 0.4, 0.4, 1 << 16, 0.04, seed=3, counter_base=0, stream_id=17)
    e_q = microfacet.albedo_quadrature(wi, 0.4, 0.4, 0.04, m=1024)
    sigma = w.std() / np.sqrt(w.size)
    assert abs(w.mean() - e_q) < 4 * sigma


def test_reflection_recovers_half_vector():
    e_h, e_n = oc.reflection_errors()
    assert e_h < 1e-12 and e_n < 1e-13


def test_reflected_direction_density():
    assert oc.reflected_change_of_variables_error() < 1e-8


def test_sample_reflection_composition():
    """The per-sample reflection oracle is the composition of the pinned App. A pieces: its weights
    average to the albedo quadrature, and its pdf integrates the reflected directions correctly."""
    rng = np.random.default_rng(11)
    n = 1 << 16
    u1, u2 = rng.random(n), rng.random(n)
    wi = oc.direction(40.0, 30.0)
    wa = np.tile(wi.reshape(3, 1), (1, n))
    wb, pdf, w = microfacet.sample_reflection(u1, u2, wa, np.full(n, 0.3), np.full(n, 0.3), 0.04)
    assert np.abs(np.sqrt((wb * wb).sum(0)) - 1).max() < 1e-13
    e_q = microfacet.albedo_quadrature(wi, 0.3, 0.3, 0.04, m=512)
    assert abs(w.mean() - e_q) < 4 * w.std() / np.sqrt(n)
    assert np.all(pdf > 0)
