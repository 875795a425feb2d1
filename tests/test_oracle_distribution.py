"""Distribution-level pins for the oracle (fixed seeds, p-value threshold 1e-3 each).

P4  normalisation by quadrature on the sphere: the pdf integrates to 1 (Eq. 1),
    the NDF satisfies int D cos = 1 (App. A), and G1 equals its definition
    (Eq. g1, projected area) -- all to 1e-6
P7  the cap sampler and the prior polar-disk sampler draw the same distribution
P8  sampled histograms match bin integrals of the pdf
P9  sampled histograms match ray casting on the truncated ellipsoid (the VNDF's
    definition, Sec. 2), which uses none of the paper's formulas
"""
import pytest

import oracle_checks as oc


@pytest.mark.parametrize("case", oc.CASES)
def test_p4_normalisation(case):
    e_pdf, e_ndf, e_g1 = oc.normalisation_errors(*case)
    assert e_pdf < 1e-6
    assert e_ndf < 1e-6
    assert e_g1 < 1e-6


@pytest.mark.parametrize("case", oc.CASES[:3])
def test_p7_cap_matches_prior_sampler(case):
    assert oc.prior_agreement_pvalue(*case) > 1e-3


@pytest.mark.parametrize("case", oc.CASES[:3])
def test_p8_histogram_matches_pdf(case):
    assert oc.chi2_vs_pdf_pvalue(*case) > 1e-3


@pytest.mark.parametrize("case", oc.CASES)
def test_p9_matches_ray_casting(case):
    assert oc.brute_force_pvalue(*case) > 1e-3
