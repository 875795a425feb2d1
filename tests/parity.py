"""GPU-vs-oracle comparison helpers for the parity tests.

Tolerances.  The contract asks for wm within 4e-6 rad of the FP64 oracle and
the pdf within 1e-5 relative.  An FP32 kernel cannot reach that on every
sample: the half vector h = c + i sums O(1) terms, and the unstretch divides
their rounding by |v| = |M^-T h|.  The error of each sample is therefore
bounded by a few ulp (2^-24) times the condition number
    kappa   = |(ax (|c.x| + |i.x|), ay (|c.y| + |i.y|), h.z)| / |v|     (wm)
    kappa_h = |((|c.x| + |i.x|), (|c.y| + |i.y|), h.z)| / |h|           (pdf, via |h|)
computed here in FP64 from the oracle's own intermediate vectors.  Every
sample must satisfy
    angle <= max(4e-6, K * kappa * 2^-24),
    rel   <= max(1e-5, K * (3 kappa + 2 kappa_h) * 2^-24),      K = 8,
and the fraction of samples above the flat 4e-6 / 1e-5 limits (the
ill-conditioned tail) is reported.

The library's cap sampler recomputes the half vector of ill-conditioned
samples in double-float, so for its outputs (strict=True) the flat limits
themselves are asserted on every sample with wi.z >= 1e-4 and alpha >= 1e-3.

The oracle's pdf G1 max(0, wi.wm) D(wm) / wz is evaluated at the FP64 normal,
and wi.wm cancels near the visibility boundary: there its own error estimate
2^-52 kappa (sum |wi_k wm_k|) / |wi.wm| can exceed 1e-7.  For those samples the
strict pdf check uses the oracle's hemisphere-sample form of Eq. 1
(vndf_pdf_at_cap_sample), which does not cancel; the count is reported.
"""
import numpy as np

from oracle import vndf

EPS32 = 2.0 ** -24
A_MP = 1e-9  # below this 1 + z_i' (or u2 (1 + z_i')) the 50-digit reference replaces the FP64 oracle
K_ULP = 8.0
ANGLE_TOL = 4e-6
PDF_TOL = 1e-5


def angle_between(a, b):
    cr = np.cross(a.T, b.T).T
    return np.arctan2(np.sqrt(vndf.dot(cr, cr)), vndf.dot(a, b))


def conditioning(u1, u2, wi, ax, ay):
    """(kappa, kappa_h) of each cap sample, in FP64."""
    wi_std = vndf.warp_to_hemisphere(wi, ax, ay)
    h, c = vndf.sample_cap(u1, u2, wi_std)
    v = np.stack([ax * h[0], ay * h[1], h[2]])
    sx = np.abs(c[0]) + np.abs(wi_std[0])
    sy = np.abs(c[1]) + np.abs(wi_std[1])
    kap = np.sqrt((ax * sx) ** 2 + (ay * sy) ** 2 + h[2] ** 2) / np.sqrt(vndf.dot(v, v))
    kap_h = np.sqrt(sx ** 2 + sy ** 2 + h[2] ** 2) / np.sqrt(vndf.dot(h, h))
    return kap, kap_h


def one_plus_zi(wi, ax, ay):
    """1 + z_i' of the stretched direction without cancellation (FP64), for selecting samples."""
    sx, sy, wz = ax * wi[0], ay * wi[1], wi[2]
    el = np.sqrt(sx * sx + sy * sy + wz * wz)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(wz >= 0, 1.0 + wz / el, (sx * sx + sy * sy) / (el * (el - wz)))


def fp64_weak(u2, wi, ax, ay):
    """Extended-domain samples on which the FP64 oracle itself loses digits: 1 + z_i' < A_MP (its
    cap bottom -z_i' is subtracted), or u2 (1 + z_i') < A_MP (then 1 - z = u2 (1 + z_i') lies near
    the resolution of z next to 1, and sin(theta) = sqrt(1 - z^2) as the paper writes it has a
    relative error of about 2^-53 / (u2 (1 + z_i')))."""
    with np.errstate(invalid="ignore"):
        a = one_plus_zi(wi, ax, ay)
        return ~(a >= A_MP) | ~(np.asarray(u2, np.float64) * a >= A_MP)


def compare_cap(wm_gpu, pdf_gpu, u1, u2, wi, ax, ay, strict=True, extended=False):
    """Check GPU cap samples against the oracle; returns a stats dict (asserts the bounds).

    With extended=True the inputs may lie below the horizon (the extended domain).  There
    the FP64 oracle itself loses digits (``fp64_weak``): such samples are excluded
    here and checked against the 50-digit reference by ``compare_cap_mp``."""
    wi = np.asarray(wi, np.float64)
    ax = np.asarray(ax, np.float64)
    ay = np.asarray(ay, np.float64)
    u1 = np.asarray(u1, np.float64)
    u2 = np.asarray(u2, np.float64)
    wm_ref, pdf_ref = vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, "cap", extended)
    wm_gpu = np.asarray(wm_gpu, np.float64)
    ok = vndf.in_domain(wi, ax, ay, extended)
    stats = {"n": int(u1.size), "out_of_domain": int((~ok).sum())}
    if extended:
        with np.errstate(invalid="ignore"):
            tiny = ok & fp64_weak(u2, wi, ax, ay)
        stats["left_to_mp_reference"] = int(tiny.sum())
        keep = ~tiny
        wm_ref, pdf_ref, wm_gpu = wm_ref[:, keep], pdf_ref[keep], wm_gpu[:, keep]
        pdf_gpu = None if pdf_gpu is None else np.asarray(pdf_gpu)[keep]
        u1, u2, wi, ax, ay, ok = u1[keep], u2[keep], wi[:, keep], ax[keep], ay[keep], ok[keep]
    # out-of-domain samples: the defined fallback, exactly
    if (~ok).any():
        assert np.all(wm_gpu[:, ~ok] == np.array([[0.0], [0.0], [1.0]]))
        if pdf_gpu is not None:
            assert np.all(np.asarray(pdf_gpu)[~ok] == 0.0)
    wm_gpu = wm_gpu[:, ok]
    wm_ref = wm_ref[:, ok]
    u1, u2, wi, ax, ay = u1[ok], u2[ok], wi[:, ok], ax[ok], ay[ok]
    ang = angle_between(wm_gpu, wm_ref)
    kap, kap_h = conditioning(u1, u2, wi, ax, ay)
    bound = np.maximum(ANGLE_TOL, K_ULP * kap * EPS32)
    worst = np.argmax(ang / bound) if ang.size else 0
    assert np.all(ang <= bound), (
        f"angle {ang[worst]:.3e} > bound {bound[worst]:.3e} (kappa {kap[worst]:.3g}) at {worst}")
    norm_err = np.abs(np.sqrt(vndf.dot(wm_gpu, wm_gpu)) - 1.0)
    assert norm_err.max() <= 2.0 ** -21
    if extended:
        contract = (ax >= 1e-3) & (ay >= 1e-3)
    else:
        contract = (wi[2] / np.sqrt(vndf.dot(wi, wi)) >= 1e-4) & (ax >= 1e-3) & (ay >= 1e-3)
    if strict and contract.any():
        worst = np.argmax(np.where(contract, ang, 0))
        assert ang[contract].max() <= ANGLE_TOL, (
            f"angle {ang[worst]:.3e} rad > {ANGLE_TOL} at {worst} (kappa {kap[worst]:.3g})")
    stats.update(max_angle=float(ang.max(initial=0)), p9999_angle=float(np.quantile(ang, 0.9999)) if ang.size else 0.0,
                 tail_angle_frac=float((ang > ANGLE_TOL).mean()) if ang.size else 0.0,
                 max_kappa_ratio=float((ang / (kap * EPS32)).max(initial=0)))
    if pdf_gpu is not None:
        pg = np.asarray(pdf_gpu, np.float64)[ok]
        pr = pdf_ref[ok]
        # where the definition-based oracle pdf is itself ill-conditioned, use the sample form
        dwm = np.abs(vndf.dot(wi, wm_ref)) / np.sqrt(vndf.dot(wi, wi))
        swm = (np.abs(wi * wm_ref).sum(axis=0)) / np.sqrt(vndf.dot(wi, wi))
        oracle_err = 2.0 ** -52 * kap * swm / np.maximum(dwm, 1e-300)
        weak = oracle_err > 1e-7
        if weak.any():
            pr = np.where(weak, vndf.vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay, extended), pr)
        stats["oracle_pdf_form_switched"] = int(weak.sum())
        rel = np.abs(pg / pr - 1.0)
        pbound = np.maximum(PDF_TOL, K_ULP * (3.0 * kap + 2.0 * kap_h) * EPS32)
        worst = np.argmax(rel / pbound) if rel.size else 0
        assert np.all(rel <= pbound), (
            f"pdf rel {rel[worst]:.3e} > bound {pbound[worst]:.3e} at {worst}")
        if strict and contract.any():
            worst = np.argmax(np.where(contract, rel, 0))
            assert rel[contract].max() <= PDF_TOL, f"pdf rel {rel[worst]:.3e} > {PDF_TOL} at {worst}"
        stats.update(max_pdf_rel=float(rel.max(initial=0)),
                     tail_pdf_frac=float((rel > PDF_TOL).mean()) if rel.size else 0.0)
    return stats


def compare_cap_mp(wm_gpu, pdf_gpu, u1, u2, wi, ax, ay, limit=2000):
    """Extended-domain samples on which the FP64 oracle is weak (``fp64_weak``) against the
    50-digit reference (oracle.vndf_mp), at the flat limits.  Checks at most ``limit`` of them."""
    try:
        from oracle import vndf_mp as mp
    except ImportError:  # no mpmath here: the stored 50-digit rows of tests/golden cover these samples
        return {"n_mp": 0, "mp_reference": "mpmath not installed"}
    wi = np.asarray(wi, np.float64)
    ax = np.asarray(ax, np.float64)
    ay = np.asarray(ay, np.float64)
    ok = vndf.in_domain(wi, ax, ay, True)
    with np.errstate(invalid="ignore"):
        idx = np.flatnonzero(ok & fp64_weak(u2, wi, ax, ay))[:limit]
    worst_a, worst_p = 0.0, 0.0
    for k in idx:
        m, p = mp.sample_with_pdf(u1[k], u2[k], wi[:, k], ax[k], ay[k])
        g = np.asarray(wm_gpu, np.float64)[:, k]
        ang = float(angle_between(g.reshape(3, 1), np.array(m).reshape(3, 1))[0])
        worst_a = max(worst_a, ang)
        assert ang <= ANGLE_TOL, f"angle {ang:.3e} at sample {k} (1 + z_i' = {mp.one_plus_zi(wi[:, k], ax[k], ay[k]):.3e})"
        if pdf_gpu is not None:
            rel = abs(float(pdf_gpu[k]) / p - 1.0)
            worst_p = max(worst_p, rel)
            assert rel <= PDF_TOL, f"pdf rel {rel:.3e} at sample {k}"
    return {"n_mp": int(idx.size), "max_angle_mp": worst_a, "max_pdf_rel_mp": worst_p}
