"""The stored 50-digit cap samples (tests/golden/cap_samples_mp50.txt) against the FP64 oracle.

The fixture is written by tests/golden/make_golden.py from oracle/ only.  These
checks pin the FP64 oracle's sampler (Sec. 2 steps (1)-(3), Sec. 3.3) and its
definition-based density (Eq. 1 through D and G1 of App. A) to an evaluation
in 50 digits, on inputs at the edges of the domain:
* where 1 + z_i' is not tiny, FP64 agrees to within its rounding bound,
* where it is, FP64 loses digits in proportion to 1 / (1 + z_i') (Sec. 3.3
  subtracts z_i' from the cap bottom), and the error stays inside that bound,
* the density written out from its definition (D, G1, wi.wm) at the stored
  normal equals the stored density, which the sampler's fused form produced,
* the closed forms the paper's own reasoning gives: wm = (0, 0, 1) and
  pdf = 1/pi at alpha = 1, normal incidence, u2 = 0; the hemisphere rows obey
  Eq. 2 with D_std = 1/pi and sigma_std = (1 + z_i)/2 (Eqs. 3-4).
"""
import math

import numpy as np
import pytest

import oracle_checks as oc
from oracle import vndf

ROWS = oc.golden_rows()
import make_golden  # noqa: E402  (on the path once golden_rows has run)


def test_fixture_shape():
    kinds = {r["kind"] for r in ROWS}
    assert kinds == {"cap", "cap_extended", "hemisphere"}
    assert len(ROWS) == len(make_golden.CASES)
    for r in ROWS:
        for t in (*r["wi"], r["alpha_x"], r["alpha_y"], r["u1"], r["u2"]):
            assert float(np.float32(t)) == t  # inputs are exact float32 values
        assert 0.0 <= r["u1"] < 1.0 and 0.0 <= r["u2"] < 1.0
        if math.isnan(r["one_plus_zi"]):
            assert tuple(r["wm"]) == (0.0, 0.0, 1.0) and r["pdf"] == 0.0
        else:
            assert abs(np.linalg.norm(r["wm"]) - 1.0) < 1e-15 and r["pdf"] > 0.0


def test_fixture_is_what_the_script_writes():
    pytest.importorskip("mpmath")
    with open(make_golden.OUT) as fh:
        assert fh.read() == make_golden.render(make_golden.rows())


@pytest.mark.parametrize("k", range(len(ROWS)))
def test_fp64_oracle_matches_50_digits(k):
    ang, rel, tol = oc.golden_row_error(ROWS[k])
    assert ang <= tol, (ROWS[k]["note"], ang, tol)
    assert rel <= 4 * tol, (ROWS[k]["note"], rel, tol)


@pytest.mark.parametrize("k", [k for k, r in enumerate(ROWS) if r["kind"] != "hemisphere"
                               and not math.isnan(r["one_plus_zi"])])
def test_density_definition_at_stored_normal(k):
    """Eq. 1 through D and G1 (App. A) at the stored wm reproduces the stored fused density."""
    r = ROWS[k]
    wi = r["wi"].reshape(3, 1)
    ax, ay = np.array([r["alpha_x"]]), np.array([r["alpha_y"]])
    p = float(vndf.vndf_pdf(r["wm"].reshape(3, 1), wi, ax, ay, r["kind"] == "cap_extended")[0])
    # the density's sensitivity to wm: D varies on the angular scale of alpha, and wi.wm
    # cancels near the visibility boundary; both are resolved by the 17-digit normal except
    # at the smallest roughness
    wu = wi[:, 0] / np.linalg.norm(wi)
    cos_iv = float(wu @ r["wm"])
    tol = 1e-12 / min(r["alpha_x"], r["alpha_y"]) ** 2 + 1e-14 / max(abs(cos_iv), 1e-300)
    assert abs(p / r["pdf"] - 1.0) <= max(tol, 1e-12), (r["note"], p, r["pdf"])


def test_closed_form_at_normal_incidence():
    r = ROWS[0]
    assert r["u2"] == 0.0 and r["alpha_x"] == r["alpha_y"] == 1.0
    assert tuple(r["wm"]) == (0.0, 0.0, 1.0)
    assert abs(r["pdf"] * math.pi - 1.0) < 1e-15


def test_extended_rows_above_horizon_equal_cap_rows():
    ext = [r for r in ROWS if r["kind"] == "cap_extended" and r["wi"][2] > 0]
    assert ext
    for r in ext:
        same = [c for c in ROWS if c["kind"] == "cap" and np.array_equal(c["wi"], r["wi"])
                and c["alpha_x"] == r["alpha_x"] and c["u1"] == r["u1"] and c["u2"] == r["u2"]]
        assert same and np.array_equal(same[0]["wm"], r["wm"]) and same[0]["pdf"] == r["pdf"]


def test_hemisphere_rows_follow_eq2():
    """Hemisphere rows: pdf = max(0, wi.wm) / (pi (1 + z_i) / 2) with z_i the unit wi's height (Eqs. 2-4)."""
    for r in ROWS:
        if r["kind"] != "hemisphere" or math.isnan(r["one_plus_zi"]):
            continue
        wu = r["wi"] / np.linalg.norm(r["wi"])
        a = r["one_plus_zi"]
        expect = max(0.0, float(wu @ r["wm"])) / (math.pi * a / 2.0)
        # wi.wm carries the 17-digit rounding of wm, relative to its own size
        tol = 1e-15 * (np.abs(wu) @ np.abs(r["wm"])) / max(float(wu @ r["wm"]), 1e-300)
        assert abs(expect / r["pdf"] - 1.0) <= max(tol, 1e-14), (r["note"], expect, r["pdf"])
        assert r["wm"][2] > 0.0


def _kd(r, wm):
    wu = r["wi"] / np.linalg.norm(r["wi"])
    return float(np.abs(wu * wm).sum() / abs(wu @ wm))


@pytest.mark.parametrize("k", [k for k, r in enumerate(ROWS) if not math.isnan(r["one_plus_zi"])])
def test_density_of_normal_forms_agree_at_50_digits(k):
    """The 50-digit density of the float32-rounded normal (max(0, wi.wm) D / sigma, App. A and
    Eq. 4) against the 50-digit fused density at the exact sample (Sec. 3.3 and Eq. 1): two
    different formulas, apart only by the density's change over the float32 rounding of wm
    (relative 2^-24 times 4 / alpha for D, plus wi.wm's amplification of the rounding)."""
    r = ROWS[k]
    amin = min(r["alpha_x"], r["alpha_y"], 1.0)
    wm32 = r["wm"].astype(np.float32).astype(np.float64)
    bound = 8 * 2.0 ** -24 * (4.0 / amin + _kd(r, wm32))
    assert abs(r["pdf_wm32"] / r["pdf"] - 1.0) <= bound, (r["note"], r["pdf_wm32"], r["pdf"])


@pytest.mark.parametrize("k", [k for k, r in enumerate(ROWS) if not math.isnan(r["one_plus_zi"])])
def test_fp64_density_of_normal_matches_50_digits(k):
    """The FP64 oracle's vndf_pdf at the float32 normal against the stored 50-digit value; its
    G1 / sigma forms 1 + z_i' by cancellation, so the bound grows like 1 / (1 + z_i')."""
    r = ROWS[k]
    wm32 = r["wm"].astype(np.float32).astype(np.float64)
    ext = r["kind"] != "cap"
    p = float(vndf.vndf_pdf(wm32.reshape(3, 1), r["wi"].reshape(3, 1), np.array([r["alpha_x"]]),
                            np.array([r["alpha_y"]]), ext)[0])
    bound = 64 * 2.0 ** -52 * max(1.0, 1.0 / r["one_plus_zi"]) * _kd(r, wm32)
    assert abs(p / r["pdf_wm32"] - 1.0) <= bound, (r["note"], p, r["pdf_wm32"])


JACS = make_golden.load_jacobians()


def _jacobian_amplification(r):
    """FP64 rounding amplification of the oracle's derivatives at one row: 1 / (1 + z_i') (the cap
    bottom -z_i' subtracted), 1 / (1 - u2) and 1 / sqrt(u2 a) (the cap height and sin(theta) formed
    as the paper writes them), |wi| / |wi.z| (grazing incidence)."""
    a, u2 = r["one_plus_zi"], r["u2"]
    amp = max(1.0, 1.0 / a) * max(1.0, 1.0 / (1.0 - u2), 1.0 / math.sqrt(u2 * a) if u2 > 0 else 1.0)
    return amp * max(1.0, float(np.linalg.norm(r["wi"])) / abs(r["wi"][2]))


def test_jacobian_fixture_is_what_the_script_writes():
    pytest.importorskip("mpmath")
    with open(make_golden.OUT_JAC) as fh:
        assert fh.read() == make_golden.render_jacobians(make_golden.rows())


def test_jacobian_fixture_covers_every_ggx_row():
    want = {k for k, r in enumerate(ROWS) if r["kind"] != "hemisphere" and not math.isnan(r["one_plus_zi"])}
    assert set(JACS) == want


def test_jacobian_closed_forms_at_normal_incidence():
    """alpha = 1, wi = z, u2 = 0 (cap top): h = i + z, so wm = normalize(wx, wy, 1 + wz) and
    d wm_x / d wi_x = d wm_y / d wi_y = 1/2; the density there is D = 1 / (pi ax ay), so
    d pdf / d alpha_x = d pdf / d alpha_y = -1 / pi."""
    J = JACS[0]
    assert abs(J[0, 0] - 0.5) < 1e-15 and abs(J[1, 1] - 0.5) < 1e-15
    assert abs(J[3, 3] + 1 / math.pi) < 1e-15 and abs(J[4, 3] + 1 / math.pi) < 1e-15


def test_jacobian_scale_invariance_in_wi():
    """The sampler and its density are invariant to the length of wi (Sec. 2 normalises it):
    J^T wi = 0 for every output."""
    for k, J in JACS.items():
        wi = ROWS[k]["wi"]
        for j in range(4):
            col = J[:3, j]
            assert abs(col @ wi) <= 1e-9 * max(np.abs(col).max() * np.linalg.norm(wi), 1e-300), (k, j)


@pytest.mark.parametrize("k", [k for k in sorted(JACS)
                               if 64 * 2.0 ** -52 * _jacobian_amplification(ROWS[k]) <= 1e-3])
def test_fp64_complex_step_matches_50_digit_jacobian(k):
    """The FP64 oracle's complex-step derivatives (oracle/grad.py) against the stored 50-digit ones,
    column by column, within 64 ulp times the row's rounding amplification.  Rows where that bound
    exceeds 1e-3 (1 + z_i' near 1e-12) are beyond FP64 and left out; there the stored values are
    the reference."""
    from oracle import grad
    r = ROWS[k]
    tol = 64 * 2.0 ** -52 * _jacobian_amplification(r)
    Jc = grad.jacobian_complex_step(np.array([r["u1"]]), np.array([r["u2"]]), r["wi"].reshape(3, 1),
                                    np.array([r["alpha_x"]]), np.array([r["alpha_y"]]), "cap",
                                    r["kind"] == "cap_extended")[:, :, 0]
    J = JACS[k]
    for j in range(4):
        err = np.linalg.norm(Jc[:, j] - J[:, j])
        assert err <= tol * max(np.linalg.norm(J[:, j]), 1e-300), (r["note"], j, err)


REFL = make_golden.load_reflection()


def test_reflection_fixture_is_what_the_script_writes():
    pytest.importorskip("mpmath")
    with open(make_golden.OUT_REFL) as fh:
        assert fh.read() == make_golden.render_reflection(make_golden.rows())


def test_reflection_closed_form_at_normal_incidence():
    """alpha = 1, wi = z, wm = z: wo = z, its density pdf(wm) / 4 = 1 / (4 pi), and the weight is
    F(1) G2 / G1 = f0 (G1 = G2 = 1 at normal incidence and exit)."""
    wo, p, w = REFL[0]
    assert tuple(wo) == (0.0, 0.0, 1.0)
    assert abs(p * 4 * math.pi - 1.0) < 1e-15 and abs(w - make_golden.REFL_F0) < 1e-17


def test_reflection_rows_are_consistent():
    """|wo| = 1, wo.z <= 0 exactly where the weight is 0, and 0 <= weight <= 1 (energy)."""
    for k, (wo, p, w) in REFL.items():
        if math.isnan(ROWS[k]["one_plus_zi"]):
            continue
        assert abs(np.linalg.norm(wo) - 1.0) < 1e-15
        assert (wo[2] <= 0) == (w == 0.0)
        assert 0.0 <= w <= 1.0 and p > 0.0


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # out-of-domain lanes divide by zero before the select
@pytest.mark.parametrize("k", sorted(REFL))
def test_fp64_reflection_matches_50_digits(k):
    """The FP64 oracle's sample_reflection (oracle/microfacet.py: reflect, bsdf_pdf through G1 and D,
    estimator_weight through the BRDF of Eq. microfacet) against the stored 50-digit values, which
    take the density as pdf(wm) / (4 wi.wm) and the weight as F G2 / G1: different routes.  The
    oracle's weight divides D at the recomputed half vector normalize(wi + wo) by D at wm; D varies
    on the angular scale of alpha, so that ratio carries the rounding times 1 / alpha."""
    from oracle import microfacet
    r = ROWS[k]
    wo_ref, p_ref, w_ref = REFL[k]
    wo, p, w = microfacet.sample_reflection(np.array([r["u1"]]), np.array([r["u2"]]), r["wi"].reshape(3, 1),
                                            np.array([r["alpha_x"]]), np.array([r["alpha_y"]]), make_golden.REFL_F0)
    wo, p, w = wo[:, 0], float(p[0]), float(w[0])
    if math.isnan(r["one_plus_zi"]):
        assert tuple(wo) == (0.0, 0.0, 1.0) and p == 0.0 and w == 0.0
        return
    tol = 64 * 2.0 ** -52 * _jacobian_amplification(r)
    ang = math.atan2(float(np.linalg.norm(np.cross(wo, wo_ref))), float(wo @ wo_ref))
    assert ang <= 2 * tol, (r["note"], ang)
    assert abs(p / p_ref - 1.0) <= 4 * tol, (r["note"], p, p_ref)
    wtol = 4 * tol * max(1.0, 1.0 / min(r["alpha_x"], r["alpha_y"]))
    assert abs(w - w_ref) <= wtol * max(w_ref, 1e-300) or (w == 0.0 and w_ref == 0.0), (r["note"], w, w_ref)
