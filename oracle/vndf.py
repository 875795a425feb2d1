"""GGX visible-normal sampling and its pdf: FP64 CPU oracle (test infrastructure).

This module is the plain, slow, obviously-correct restatement that the CUDA
path is checked against.  It is test infrastructure: only ``tests/``, the
smoke entry point and the CPU-baseline leg of the bench import it, and it
shares no code with the CUDA library.  Everything is numpy in FP64; FP32
inputs are promoted exactly.  Vectors are stacked as arrays of shape (3, N).

Paper: Dupuy & Benyoub, "Sampling Visible GGX Normals with Spherical Caps",
HPG 2023 (arXiv 2306.05044).  Functions cite the section / equation they
follow:

* ``warp_to_hemisphere``   Sec. 2, "Importance Sampling", step (1)
* ``sample_cap``           Sec. 3.3 (spherical-cap sampler, steps 1-2)
* ``sample_polar_disk``    Sec. 2, step (2): the prior sampler of Heitz 2018
* ``warp_to_ellipsoid``    Sec. 2, step (3): normals transform by M^-T
* ``sample_vndf``          Sec. 2 steps (1)-(3) with either hemisphere sampler
* ``ndf_std, sigma_std``   Eqs. 3 and 4
* ``vndf_std``             Eq. 2
* ``ndf``                  App. A, GGX NDF as a transformed hemisphere NDF
* ``smith_g1``             App. A, Eq. g1 and its hemisphere form
* ``vndf_pdf``             D_vis = G1(wi) max(0, wi.wm) D(wm) / wi.z (App. A + Eq. 2)
* ``vndf_pdf_eq1``         Eq. 1 written out literally (transformed hemisphere VNDF)
* ``vndf_pdf_at_cap_sample`` Eq. 1 at the cap sampler's own hemisphere sample (Sec. 3.2-3.3),
                           the form that stays accurate near the visibility boundary
* ``projected_area``       Eq. 4 carried through M (App. A): sigma(wi) = |M^-1 wi| sigma_std(z_i')
* ``sample_hemisphere``    Sec. 3.3 used stand-alone: the cap sample normalised, with its Eq. 2 density

Readings where the paper is silent (domain, extended domain, scale of wi, which uniform drives which angle):
* Domain: wi.z > 0, alpha_x > 0, alpha_y > 0, all inputs finite.  Outside it a
  sample returns the defined fallback wm = (0, 0, 1) with pdf = 0.
* Extended domain (``extended=True``): the construction of Sec. 3.2-3.3 never
  uses wi.z > 0.  The cap z in (-z_i', 1] and sigma_std = (1 + z_i')/2 (Eq. 4)
  stay valid for every z_i' > -1, i.e. for incident directions below the
  horizon, and sample the normals with wm.z > 0 that face wi.  The paper is
  silent on it; the extended domain requires 1 + z_i' >= MIN_CAP_A (the
  stretched direction at least about 1.4e-6 rad from straight down), finite
  inputs and positive roughness.
* wi need not be unit length: every step normalises or is scale free.
* u1 drives the azimuth and u2 the cap height, as in both printed samplers.

Complex inputs are accepted so that gradients can be taken by the complex-step
method (``oracle.grad``).  For complex arrays the clamp of Sec. 3.3 and the
max(0, .) of Eq. 2 are the identity; callers only use complex inputs at
points where the real part lies strictly inside those ranges, so the
derivative is the derivative of the interior expression.
"""
import numpy as np

PI = np.pi

# Smallest 1 + z_i' of the extended domain (a reading: below it the cap has
# shrunk to a point and FP32 results would be meaningless).
MIN_CAP_A = 2.0 ** -40


# ----------------------------------------------------------------------------
# small vector helpers (plain definitions)
# ----------------------------------------------------------------------------

def _stack(x, y, z):
    return np.stack(np.broadcast_arrays(x, y, z))


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def normalize(v):
    # sqrt of the sum of squares (not abs()) so that complex steps stay analytic
    return v / np.sqrt(dot(v, v))


def _clamp01(x):
    if np.iscomplexobj(x):
        return x
    return np.clip(x, 0.0, 1.0)


def _pos(x):
    if np.iscomplexobj(x):
        return x
    return np.maximum(x, 0.0)


def _as_f64(x):
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return x.astype(np.complex128)
    return x.astype(np.float64)


# ----------------------------------------------------------------------------
# Sec. 2: stretch / unstretch (matrices M = diag(1/ax, 1/ay, 1), M^-1 = diag(ax, ay, 1))
# ----------------------------------------------------------------------------

def warp_to_hemisphere(wi, ax, ay):
    """Step (1): wi -> M^-1 wi / |M^-1 wi| (hemisphere configuration)."""
    return normalize(_stack(ax * wi[0], ay * wi[1], wi[2]))


def warp_to_ellipsoid(wm_std, ax, ay):
    """Step (3): a hemisphere normal back to the ellipsoid: normalize(M^-T wm_std)."""
    return normalize(_stack(ax * wm_std[0], ay * wm_std[1], wm_std[2]))


# ----------------------------------------------------------------------------
# Sec. 3.3: the spherical-cap hemisphere sampler (the paper's contribution)
# ----------------------------------------------------------------------------

def sample_cap(u1, u2, wi_std):
    """Draw c uniformly on the spherical cap z in (-wi.z, 1] and return (h, c).

    Sec. 3.2 proves that a mirror hemisphere reflects the parallel rays from wi
    uniformly into that cap; Sec. 3.3 then returns the half vector h = c + wi
    between wi and the cap direction as a visible normal.  h is left
    unnormalised (the caller normalises after unstretching, Sec. 3.3).
    """
    zi = wi_std[2]
    phi = 2.0 * PI * u1                      # azimuth, uniform in [0, 2 pi)
    z = (1.0 - u2) * (1.0 + zi) - zi         # height, uniform in (-zi, 1]
    sin_theta = np.sqrt(_clamp01(1.0 - z * z))
    c = _stack(sin_theta * np.cos(phi), sin_theta * np.sin(phi), z)
    h = c + wi_std
    return h, c


# ----------------------------------------------------------------------------
# Sec. 2 step (2): the prior sampler of Heitz 2018 (cross-section / polar disk)
# ----------------------------------------------------------------------------

def sample_polar_disk(u1, u2, wi_std):
    """Heitz 2018 as described in Sec. 2: sample the projected cross section.

    A point (t1, t2) is drawn uniformly on the unit disk (polar coordinates),
    the half of the disk facing away from wi is compressed by the factor s =
    (1 + wi.z) / 2 (the normaliser of Eq. 4), and the point is lifted back
    onto the hemisphere along wi in the basis (w1, w2, wi).
    """
    wx, wy, wz = wi_std[0], wi_std[1], wi_std[2]
    rho2 = wx * wx + wy * wy
    degenerate = np.real(rho2) <= 0.0
    safe = np.where(degenerate, 1.0, rho2)
    inv = 1.0 / np.sqrt(safe)
    # w1 orthogonal to wi in the xy plane; fixed axis when wi is the pole
    w1 = _stack(np.where(degenerate, 1.0, -wy * inv),
                np.where(degenerate, 0.0, wx * inv),
                np.zeros_like(wx))
    # w2 = wi x w1
    w2 = _stack(wy * w1[2] - wz * w1[1],
                wz * w1[0] - wx * w1[2],
                wx * w1[1] - wy * w1[0])
    phi = 2.0 * PI * u1
    r = np.sqrt(u2)
    t1 = r * np.cos(phi)
    t2 = r * np.sin(phi)
    s = 0.5 * (1.0 + wz)
    t2 = (1.0 - s) * np.sqrt(1.0 - t1 * t1) + s * t2
    ti = np.sqrt(_pos(1.0 - t1 * t1 - t2 * t2))
    return _stack(t1 * w1[0] + t2 * w2[0] + ti * wx,
                  t1 * w1[1] + t2 * w2[1] + ti * wy,
                  t1 * w1[2] + t2 * w2[2] + ti * wz)


# ----------------------------------------------------------------------------
# Sec. 2: the full GGX VNDF sampler
# ----------------------------------------------------------------------------

def in_domain(wi, ax, ay, extended=False):
    """Inputs on which the sampler is defined (a reading; see module docstring).

    extended=False: wi.z > 0.  extended=True: 1 + z_i' >= MIN_CAP_A, where
    z_i' is the height of the stretched direction M^-1 wi / |M^-1 wi|.
    """
    wi = [np.real(_as_f64(w)) for w in wi]
    ax = np.real(_as_f64(ax))
    ay = np.real(_as_f64(ay))
    ok = (ax > 0) & (ay > 0)
    for q in (wi[0], wi[1], wi[2], ax, ay):
        ok &= np.isfinite(q)
    if not extended:
        return ok & (wi[2] > 0)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        sx, sy = ax * wi[0], ay * wi[1]
        zi = wi[2] / np.sqrt(sx * sx + sy * sy + wi[2] * wi[2])
        return ok & (1.0 + zi >= MIN_CAP_A)


def _fallback_inputs(ok, wi, ax, ay):
    """Finite stand-in inputs on lanes outside the domain (their results are replaced)."""
    wi = np.where(ok, wi, np.array([0.0, 0.0, 1.0]).reshape(3, *([1] * (wi.ndim - 1))))
    return wi, np.where(ok, ax, 1.0), np.where(ok, ay, 1.0)


def sample_vndf(u1, u2, wi, ax, ay, method="cap", extended=False):
    """Steps (1)-(3) of Sec. 2: wm for each (u1, u2, wi, ax, ay).

    method = "cap" uses the spherical-cap sampler (Sec. 3.3), "polar" the prior
    sampler (Heitz 2018).  extended=True (cap only) accepts the extended domain
    (incident directions below the horizon).  Out-of-domain samples return (0, 0, 1).
    """
    if extended and method != "cap":
        raise ValueError("the extended domain is defined for the cap sampler only")
    wi = _stack(*[_as_f64(w) for w in wi])
    ax = _as_f64(ax)
    ay = _as_f64(ay)
    u1 = _as_f64(u1)
    u2 = _as_f64(u2)
    ok = in_domain(wi, ax, ay, extended)
    # keep the arithmetic finite on fallback lanes
    wi, ax, ay = _fallback_inputs(ok, wi, ax, ay)
    wi_std = warp_to_hemisphere(wi, ax, ay)
    if method == "cap":
        h, _ = sample_cap(u1, u2, wi_std)
    elif method == "polar":
        h = sample_polar_disk(u1, u2, wi_std)
    else:
        raise ValueError(method)
    wm = warp_to_ellipsoid(h, ax, ay)
    fallback = np.array([0.0, 0.0, 1.0]).reshape(3, *([1] * (wm.ndim - 1)))
    return np.where(ok, wm, fallback)


# ----------------------------------------------------------------------------
# Eqs. 2-4: the hemisphere VNDF
# ----------------------------------------------------------------------------

def ndf_std(wm_std):
    """Eq. 3: D_std = 1/pi on the upper hemisphere, 0 below."""
    return np.where(np.real(wm_std[2]) > 0.0, 1.0 / PI, 0.0)


def sigma_std(zi):
    """Eq. 4: projected area of the unit hemisphere seen from direction with height zi."""
    return 0.5 * (1.0 + zi)


def vndf_std(wm_std, wi_std):
    """Eq. 2: max(wm.wi, 0) D_std(wm) / sigma_std(wi)."""
    return _pos(dot(wm_std, wi_std)) * ndf_std(wm_std) / sigma_std(wi_std[2])


# ----------------------------------------------------------------------------
# App. A: GGX NDF and Smith G1 through the same linear transformation
# ----------------------------------------------------------------------------

def _mt(wm, ax, ay):
    """M^T wm with M = diag(1/ax, 1/ay, 1)."""
    return _stack(wm[0] / ax, wm[1] / ay, wm[2])


def ndf(wm, ax, ay):
    """App. A: D(wm) = D_std(M^T wm / |M^T wm|) |det M^T| / |M^T wm|^4 (wm unit)."""
    t = _mt(wm, ax, ay)
    n = np.sqrt(dot(t, t))
    return ndf_std(t / n) * (1.0 / (ax * ay)) / n ** 4


def smith_g1(wm, wk, ax, ay):
    """App. A: G1(wm, wk) = G1_std(M^T wm/|.|, M^-1 wk/|.|) = chi+(wk.wm) zk'/sigma_std(zk')."""
    wk_std = warp_to_hemisphere(wk, ax, ay)
    if np.iscomplexobj(wk_std) or np.iscomplexobj(wm):
        chi = 1.0
    else:
        chi = (dot(wm, wk) > 0.0).astype(np.float64)
    return chi * wk_std[2] / sigma_std(wk_std[2])


def projected_area(wi_unit, ax, ay):
    """sigma(wi) = integral of max(0, wi.wm) D(wm) over wm, for unit wi.

    Eq. 4 gives it for the hemisphere configuration; M maps projected areas by
    |M^-1 wi| (App. A's derivation of G1 through the same transformation), so
    sigma(wi) = |M^-1 wi| (1 + z_i') / 2 = (|M^-1 wi| + wi.z) / 2.
    """
    s = _stack(ax * wi_unit[0], ay * wi_unit[1], wi_unit[2])
    return np.sqrt(dot(s, s)) * sigma_std(warp_to_hemisphere(wi_unit, ax, ay)[2])


def vndf_pdf(wm, wi, ax, ay, extended=False):
    """GGX VNDF density of wm given wi: G1(wi) max(0, wi.wm) D(wm) / wi.z (wi normalised).

    This is Eq. 2's definition of a visible-normal density (Heitz & d'Eon 2014)
    with the GGX D and G1 of App. A; it equals Eq. 1.  On the extended domain
    (wi.z may be <= 0, where G1 / wi.z is 0/0 at the horizon) it is written as
    max(0, wi.wm) D(wm) / sigma(wi) with the projected area sigma, the same
    quantity since G1(wi) / wi.z = 1 / sigma(wi).  Out-of-domain inputs give 0.
    """
    wm = _stack(*[_as_f64(w) for w in wm])
    wi = _stack(*[_as_f64(w) for w in wi])
    ax = _as_f64(ax)
    ay = _as_f64(ay)
    ok = in_domain(wi, ax, ay, extended)
    wi, ax, ay = _fallback_inputs(ok, wi, ax, ay)
    wi_unit = normalize(wi)
    if extended:
        p = _pos(dot(wi_unit, wm)) * ndf(wm, ax, ay) / projected_area(wi_unit, ax, ay)
    else:
        p = smith_g1(wm, wi_unit, ax, ay) * _pos(dot(wi_unit, wm)) * ndf(wm, ax, ay) / wi_unit[2]
    return np.where(ok, p, 0.0)


def vndf_pdf_eq1(wm, wi, ax, ay):
    """Eq. 1 literally: D_vis_std(M^T wm/|M^T wm|, M^-1 wi/|M^-1 wi|) |det M^T| / |M^T wm|^3."""
    wm = _stack(*[_as_f64(w) for w in wm])
    wi = _stack(*[_as_f64(w) for w in wi])
    t = _mt(wm, ax, ay)
    n = np.sqrt(dot(t, t))
    wm_std = t / n
    wi_std = warp_to_hemisphere(wi, ax, ay)
    return vndf_std(wm_std, wi_std) * (1.0 / (ax * ay)) / n ** 3


def vndf_pdf_at_cap_sample(u1, u2, wi, ax, ay, extended=False):
    """Eq. 1 evaluated at the cap sampler's own hemisphere sample (Sec. 3.3).

    For the sample wm = normalize(M^-T h) with h = c + wi' (wi' = M^-1 wi / |.|,
    c the cap point), the hemisphere normal of Eq. 1 is M^T wm / |M^T wm| = h / |h|
    and |M^T wm| = |h| / |v| with v = M^-T h.  Since c and wi' are unit vectors,
    |h|^2 = 2 (1 + c.wi') and h.wi' = |h|^2 / 2, so Eqs. 1-4 give
        D_vis = (|h| / 2) / (pi (1 + z_i') / 2) * |det M^T| * |v|^3 / |h|^3
              = |v|^3 / (pi ax ay (1 + z_i') |h|^2).
    This avoids forming wi . wm, which cancels near the visibility boundary;
    it is the better-conditioned of the two forms there and equals vndf_pdf
    elsewhere (a pinned test checks the two against each other).
    """
    wi = _stack(*[_as_f64(w) for w in wi])
    ax = _as_f64(ax)
    ay = _as_f64(ay)
    ok = in_domain(wi, ax, ay, extended)
    wi, ax, ay = _fallback_inputs(ok, wi, ax, ay)
    wi_std = warp_to_hemisphere(wi, ax, ay)
    h, _ = sample_cap(_as_f64(u1), _as_f64(u2), wi_std)
    v = _stack(ax * h[0], ay * h[1], h[2])
    vv = dot(v, v)
    p = vv * np.sqrt(vv) / (PI * ax * ay * (1.0 + wi_std[2]) * dot(h, h))
    return np.where(ok, p, 0.0)


def sample_vndf_with_pdf(u1, u2, wi, ax, ay, method="cap", extended=False):
    """(wm, pdf) per sample: the sampled normal and the VNDF density at it."""
    wm = sample_vndf(u1, u2, wi, ax, ay, method, extended)
    return wm, vndf_pdf(wm, wi, ax, ay, extended)


# ----------------------------------------------------------------------------
# Sec. 3.3 used on its own: the hemisphere sampler with its normalisation
# ----------------------------------------------------------------------------

def sample_hemisphere(u1, u2, wi_std):
    """Visible normal of the hemisphere configuration for direction wi_std, and its density.

    Sec. 3.3 leaves the half vector h = c + wi_std unnormalised because the
    GGX sampler normalises after unstretching; used on its own the sample is
    h / |h| (the normalisation the paper says a stand-alone use needs).  The
    density is Eq. 2, max(wm.wi, 0) D_std(wm) / sigma_std(z_i) with D_std and
    sigma_std of Eqs. 3-4.  wi_std need not be unit length.  Its domain is the
    extended one: finite, non-zero, 1 + z_i >= MIN_CAP_A.  Returns (wm (3, N),
    pdf (N,)); out-of-domain lanes give ((0, 0, 1), 0).
    """
    w = _stack(*[_as_f64(x) for x in wi_std])
    one = np.ones_like(np.real(w[0]))
    ok = in_domain(w, one, one, extended=True)
    w, _, _ = _fallback_inputs(ok, w, one, one)
    w = normalize(w)
    h, _ = sample_cap(_as_f64(u1), _as_f64(u2), w)
    wm = normalize(h)
    pdf = vndf_std(wm, w)
    fallback = np.array([0.0, 0.0, 1.0]).reshape(3, *([1] * (wm.ndim - 1)))
    return np.where(ok, wm, fallback), np.where(ok, pdf, 0.0)
