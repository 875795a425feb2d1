"""Plant plausible mistakes in the oracle and check that the pins catch each one.

Every mutant below is a one-line slip someone could make while restating the
paper (a dropped term, a wrong sign, a transposed operand, a wrong exponent, a
swapped random number).  The test patches it into the oracle in-process, runs a
fast version of the pin checks and requires at least one of them to fail.
Nothing here touches the CUDA library.
"""
import numpy as np
import pytest

# planted mistakes produce NaNs and divisions by zero; that is what the detectors catch
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

import oracle_checks as oc
from oracle import microfacet, philox, vndf

PI = np.pi
_stack = vndf._stack


def _cap_no_wi(u1, u2, wi_std):
    zi = wi_std[2]
    phi = 2 * PI * u1
    z = (1 - u2) * (1 + zi) - zi
    st = np.sqrt(vndf._clamp01(1 - z * z))
    c = _stack(st * np.cos(phi), st * np.sin(phi), z)
    return c, c


def _cap_sign(u1, u2, wi_std):
    zi = wi_std[2]
    phi = 2 * PI * u1
    z = (1 - u2) * (1 + zi) + zi
    st = np.sqrt(vndf._clamp01(1 - z * z))
    c = _stack(st * np.cos(phi), st * np.sin(phi), z)
    return c + wi_std, c


def _cap_swap_u(u1, u2, wi_std):
    return _CAP(u2, u1, wi_std)


def _cap_half_turn(u1, u2, wi_std):
    return _CAP(0.5 * u1, u2, wi_std)


def _warp_inverse(wi, ax, ay):
    return vndf.normalize(_stack(wi[0] / ax, wi[1] / ay, wi[2]))


def _warp_transposed(wi, ax, ay):
    return vndf.normalize(_stack(ay * wi[0], ax * wi[1], wi[2]))


def _unwarp_inverse(h, ax, ay):
    return vndf.normalize(_stack(h[0] / ax, h[1] / ay, h[2]))


def _sigma_no_half(zi):
    return 1.0 + zi


def _ndf_cubed(wm, ax, ay):
    t = vndf._mt(wm, ax, ay)
    n = np.sqrt(vndf.dot(t, t))
    return vndf.ndf_std(t / n) * (1.0 / (ax * ay)) / n ** 3


def _eq1_fourth(wm, wi, ax, ay):
    return _EQ1(wm, wi, ax, ay) / np.sqrt(vndf.dot(vndf._mt(wm, ax, ay), vndf._mt(wm, ax, ay)))


def _g1_unwarped(wm, wk, ax, ay):
    wk_n = vndf.normalize(wk)
    return wk_n[2] / vndf.sigma_std(wk_n[2])


def _polar_impl(u1, u2, wi_std):
    # the prior sampler with the disk warp factor s = (1 - z)/2 instead of (1 + z)/2
    wx, wy, wz = wi_std
    rho2 = wx * wx + wy * wy
    inv = 1.0 / np.sqrt(np.where(rho2 > 0, rho2, 1.0))
    w1 = _stack(np.where(rho2 > 0, -wy * inv, 1.0), np.where(rho2 > 0, wx * inv, 0.0), 0 * wx)
    w2 = _stack(wy * w1[2] - wz * w1[1], wz * w1[0] - wx * w1[2], wx * w1[1] - wy * w1[0])
    phi = 2 * PI * u1
    r = np.sqrt(u2)
    t1 = r * np.cos(phi)
    t2 = r * np.sin(phi)
    s = 0.5 * (1.0 - wz)
    t2 = (1 - s) * np.sqrt(1 - t1 * t1) + s * t2
    ti = np.sqrt(np.maximum(1 - t1 * t1 - t2 * t2, 0))
    return _stack(t1 * w1[0] + t2 * w2[0] + ti * wx, t1 * w1[1] + t2 * w2[1] + ti * wy,
                  t1 * w1[2] + t2 * w2[2] + ti * wz)


def _reflect_sign(wm, wa):
    d = vndf.dot(wm, wa)
    return _stack(wa[0] - 2 * d * wm[0], wa[1] - 2 * d * wm[1], 2 * d * wm[2] - wa[2])


def _bsdf_pdf_no4(wm, wa, ax, ay):
    return _BSDF(wm, wa, ax, ay) * 4.0


def _g2_separable(wm, wi, wo, ax, ay):
    return vndf.smith_g1(wm, wi, ax, ay) * vndf.smith_g1(wm, wo, ax, ay)


def _philox_swapped(counter, key):
    c = np.asarray(counter)
    return _PHILOX(np.stack([c[2], c[1], c[0], c[3]]), key)


def _words_same_pair(seed, counter_base, stream_id, n):
    g = np.uint64(counter_base) + np.arange(n, dtype=np.uint64)
    out = philox.philox4x32_10(philox.block_counters(g >> np.uint64(1), stream_id), philox.seed_key(seed))
    return out[0], out[1]


def _projected_area_abs(wi_unit, ax, ay):
    s = _stack(ax * wi_unit[0], ay * wi_unit[1], wi_unit[2])
    return 0.5 * (np.sqrt(vndf.dot(s, s)) + np.abs(wi_unit[2]))


def _cap_abs_height(u1, u2, wi_std):
    # the cap height range built from |z_i|: identical above the horizon, wrong below it
    w = _stack(wi_std[0], wi_std[1], np.abs(wi_std[2]))
    h, c = _CAP(u1, u2, w)
    return c + wi_std, c


_CAP = vndf.sample_cap
_EQ1 = vndf.vndf_pdf_eq1
_BSDF = microfacet.bsdf_pdf
_PHILOX = philox.philox4x32_10

MUTANTS = {
    "cap_drops_wi": [(vndf, "sample_cap", _cap_no_wi)],
    "cap_height_sign": [(vndf, "sample_cap", _cap_sign)],
    "cap_swaps_u1_u2": [(vndf, "sample_cap", _cap_swap_u)],
    "cap_half_azimuth": [(vndf, "sample_cap", _cap_half_turn)],
    "stretch_uses_M": [(vndf, "warp_to_hemisphere", _warp_inverse)],
    "stretch_transposed": [(vndf, "warp_to_hemisphere", _warp_transposed)],
    "unstretch_uses_M": [(vndf, "warp_to_ellipsoid", _unwarp_inverse)],
    "sigma_std_no_half": [(vndf, "sigma_std", _sigma_no_half)],
    "ndf_cubed": [(vndf, "ndf", _ndf_cubed), (microfacet, "ndf", _ndf_cubed)],
    "eq1_jacobian_fourth": [(vndf, "vndf_pdf_eq1", _eq1_fourth)],
    "g1_without_stretch": [(vndf, "smith_g1", _g1_unwarped), (microfacet, "smith_g1", _g1_unwarped)],
    "prior_disk_warp": [(vndf, "sample_polar_disk", _polar_impl)],
    "reflect_sign": [(microfacet, "reflect", _reflect_sign)],
    "bsdf_pdf_no_4": [(microfacet, "bsdf_pdf", _bsdf_pdf_no4)],
    "g2_separable": [(microfacet, "smith_g2", _g2_separable)],
    "philox_operands_swapped": [(philox, "philox4x32_10", _philox_swapped)],
    "philox_pair_words": [(philox, "sample_words", _words_same_pair)],
    "projected_area_abs_wz": [(vndf, "projected_area", _projected_area_abs)],
    "cap_height_abs_zi": [(vndf, "sample_cap", _cap_abs_height)],
}


def _fails(fn):
    try:
        return bool(fn())
    except Exception:
        return True


def _detectors():
    import test_oracle_philox as tp

    def philox_vs_curand():
        lib = tp._curand()
        if lib is None:
            # fall back to a property that any correct Philox layout keeps
            w1, w2 = philox.sample_words(1, 0, 0, 1024)
            return np.any(w1[0::2] == w1[1::2])
        ref = tp._curand_words(lib, 0x1234, 0, 64)
        k = np.arange(64, dtype=np.uint64)
        blk = k // np.uint64(4)
        ctr = np.stack([np.zeros(64, np.uint32), np.zeros(64, np.uint32),
                        blk.astype(np.uint32), np.zeros(64, np.uint32)])
        out = philox.philox4x32_10(ctr, philox.seed_key(0x1234))
        return np.any(out[(k % np.uint64(4)).astype(np.int64), np.arange(64)] != ref)

    def pair_words():
        w1, w2 = philox.sample_words(1, 0, 0, 1024)
        return np.any(w1[0::2] == w1[1::2])

    def invariants():
        e, d, z = oc.invariants_error(n=2000)
        return e > 1e-14 or d <= 0 or z <= 0

    def mirror():
        return oc.mirror_cap_error(n=2000) > 1e-13

    def cov():
        return oc.change_of_variables_error(n=500) > 1e-9

    def alpha_one():
        a, b = oc.alpha_one_errors(n=2000)
        return a > 1e-13 or b > 1e-14

    def symmetry():
        return max(oc.symmetry_errors(n=2000)) > 1e-13

    def normalisation():
        return max(oc.normalisation_errors(75.0, 120.0, 0.5, 0.1)) > 1e-6

    def eq1():
        u1, u2, wi, ax, ay = oc.random_batch(500, 13)
        wm = vndf.sample_vndf(u1, u2, wi, ax, ay)
        return np.abs(vndf.vndf_pdf(wm, wi, ax, ay) / vndf.vndf_pdf_eq1(wm, wi, ax, ay) - 1).max() > 1e-12

    def brute_force():
        return oc.brute_force_pvalue(75.0, 120.0, 0.5, 0.1, n=200_000) < 1e-3

    def prior():
        return oc.prior_agreement_pvalue(75.0, 120.0, 0.5, 0.1, n=200_000) < 1e-3

    def g_textbook():
        return max(oc.g1_g2_textbook_errors(n=500)) > 1e-13

    def albedo():
        wi = oc.direction(60.0, 0.0)
        return abs(microfacet.albedo_quadrature(wi, 0.5, 0.5, 0.04, m=256)
                   - oc.brdf_albedo_quadrature(wi, 0.5, 0.5, 0.04, 600, 600)) > 1e-3

    def reflection():
        e_h, e_n = oc.reflection_errors(n=500)
        return e_h > 1e-12 or e_n > 1e-13

    def reflected_density():
        return oc.reflected_change_of_variables_error(n=200) > 1e-8

    def extended_normalisation():
        return max(oc.extended_normalisation_errors(120.0, -60.0, 0.8, 0.6)) > 1e-6

    def extended_cov():
        return oc.extended_change_of_variables_error(n=500) > 1e-8

    def extended_alpha_one():
        a, b = oc.extended_alpha_one_errors(n=2000)
        return a > 1e-13 or b > 1e-12

    def golden_mp50():
        return oc.golden_excess() > 1.0

    return dict(golden_mp50=golden_mp50, extended_normalisation=extended_normalisation, extended_cov=extended_cov,
                extended_alpha_one=extended_alpha_one, reflection=reflection, reflected_density=reflected_density, philox_vs_curand=philox_vs_curand, pair_words=pair_words, invariants=invariants,
                mirror=mirror, cov=cov, alpha_one=alpha_one, symmetry=symmetry,
                normalisation=normalisation, eq1=eq1, brute_force=brute_force, prior=prior,
                g_textbook=g_textbook, albedo=albedo)


def test_unmutated_oracle_passes_fast_detectors():
    failed = [k for k, f in _detectors().items() if _fails(f)]
    assert failed == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    for module, attr, repl in MUTANTS[name]:
        monkeypatch.setattr(module, attr, repl)
    caught = [k for k, f in _detectors().items() if _fails(f)]
    assert caught, f"mutant {name} passed every pin"
