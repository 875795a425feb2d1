"""The cap sampler and its density in 50-digit arithmetic (mpmath): test infrastructure.

Below the horizon at small roughness, 1 + z_i' (z_i' the height of the
stretched incident direction) can be as small as 1e-10, and the FP64 oracle
(``oracle.vndf``) then loses digits to cancellation in 1 + z_i', in the cap
height and in 1 - z^2.  This module evaluates the same steps at 50 significant
digits, one sample at a time, as the reference for those samples.  Only tests
import it; it shares no code with the CUDA library.

Steps (Dupuy & Benyoub, HPG 2023):
* Sec. 2 step (1): i = M^-1 wi / |M^-1 wi|, M^-1 = diag(ax, ay, 1)
* Sec. 3.3: phi = 2 pi u1, z = (1 - u2)(1 + i.z) - i.z, c = (sqrt(1 - z^2) cos phi,
  sqrt(1 - z^2) sin phi, z), h = c + i
* Sec. 2 step (3): v = (ax hx, ay hy, hz), wm = v / |v|
* Eqs. 1-4 at the sample: pdf = |v|^3 / (pi ax ay (1 + i.z) |h|^2)
* derivatives of (wm, pdf) with respect to (wi, ax, ay) at fixed u (``jacobian``): central
  differences of the same steps at 50 digits with step 1e-20, written with the exact identities
  1 - z = u2 (1 + i.z) (so 1 - z^2 = u2 a (2 - u2 a), a = 1 + i.z) and h.z = (1 - u2) a, so that no
  rounding at 1e-50 is divided by the step
* reflection sampling (``reflection``, App. A): wo = 2 (wi.wm) wm - wi (Eq. reflect) for unit wi,
  the density of wo, pdf(wm) / (4 wi.wm), and the estimator weight F(wi.wm) G2 / G1(wi) with
  Schlick's F = f0 + (1 - f0)(1 - wi.wm)^5 and the height-correlated G2 = Gi Go / (Gi + Go - Gi Go),
  G1(w) = 2 w.z / (w.z + |M^-1 w|) (unit w above the surface); weight 0 when wo.z <= 0
* the density of a given normal (``pdf_of_normal``): max(0, wi.wm) D(wm) / sigma(wi)
  with the GGX D of App. A and the projected area sigma(wi) = (|M^-1 wi| + wi.z) / 2
  of unit wi (Eq. 4 carried through the stretch; G1(wi) / wi.z = 1 / sigma(wi))
"""
import mpmath

DIGITS = 50


def sample_with_pdf(u1, u2, wi, ax, ay):
    """(wm (3 floats), pdf float) for one sample; inputs are exact binary floats."""
    with mpmath.workdps(DIGITS):
        u1, u2, ax, ay = (mpmath.mpf(float(t)) for t in (u1, u2, ax, ay))
        wx, wy, wz = (mpmath.mpf(float(t)) for t in wi)
        sx, sy = ax * wx, ay * wy
        el = mpmath.sqrt(sx * sx + sy * sy + wz * wz)
        ix, iy, iz = sx / el, sy / el, wz / el
        phi = 2 * mpmath.pi * u1
        z = (1 - u2) * (1 + iz) - iz
        st = mpmath.sqrt(max(1 - z * z, mpmath.mpf(0)))
        hx = st * mpmath.cos(phi) + ix
        hy = st * mpmath.sin(phi) + iy
        hz = z + iz
        vx, vy, vz = ax * hx, ay * hy, hz
        vn = mpmath.sqrt(vx * vx + vy * vy + vz * vz)
        hh = hx * hx + hy * hy + hz * hz
        pdf = vn ** 3 / (mpmath.pi * ax * ay * (1 + iz) * hh)
        return (float(vx / vn), float(vy / vn), float(vz / vn)), float(pdf)


def one_plus_zi(wi, ax, ay):
    """1 + z_i' of the stretched direction, in 50 digits (for selecting and reporting samples)."""
    with mpmath.workdps(DIGITS):
        sx, sy = mpmath.mpf(float(ax)) * mpmath.mpf(float(wi[0])), mpmath.mpf(float(ay)) * mpmath.mpf(float(wi[1]))
        wz = mpmath.mpf(float(wi[2]))
        return float(1 + wz / mpmath.sqrt(sx * sx + sy * sy + wz * wz))


def pdf_of_normal(wm, wi, ax, ay):
    """Density of the given normal wm (3 floats) for direction wi (any length), 50 digits."""
    with mpmath.workdps(DIGITS):
        ax, ay = mpmath.mpf(float(ax)), mpmath.mpf(float(ay))
        wx, wy, wz = (mpmath.mpf(float(t)) for t in wi)
        n = mpmath.sqrt(wx * wx + wy * wy + wz * wz)
        wx, wy, wz = wx / n, wy / n, wz / n
        mx, my, mz = (mpmath.mpf(float(t)) for t in wm)
        if mz <= 0:
            return 0.0
        s = mpmath.sqrt((ax * wx) ** 2 + (ay * wy) ** 2 + wz * wz)
        sigma = (s + wz) / 2
        q = (mx / ax) ** 2 + (my / ay) ** 2 + mz * mz
        d = max(wx * mx + wy * my + wz * mz, mpmath.mpf(0))
        return float(d / (mpmath.pi * ax * ay * q * q * sigma))


def _forward(u1, u2, wx, wy, wz, ax, ay):
    """(wm_x, wm_y, wm_z, pdf) as mpf from mpf inputs: the steps of sample_with_pdf."""
    sx, sy = ax * wx, ay * wy
    el = mpmath.sqrt(sx * sx + sy * sy + wz * wz)
    ix, iy, iz = sx / el, sy / el, wz / el
    a = 1 + iz
    phi = 2 * mpmath.pi * u1
    st = mpmath.sqrt(u2 * a * (2 - u2 * a))
    hx = st * mpmath.cos(phi) + ix
    hy = st * mpmath.sin(phi) + iy
    hz = (1 - u2) * a
    vx, vy, vz = ax * hx, ay * hy, hz
    vn = mpmath.sqrt(vx * vx + vy * vy + vz * vz)
    hh = hx * hx + hy * hy + hz * hz
    return vx / vn, vy / vn, vz / vn, vn ** 3 / (mpmath.pi * ax * ay * a * hh)


def jacobian(u1, u2, wi, ax, ay):
    """d(wm_x, wm_y, wm_z, pdf)/d(wi_x, wi_y, wi_z, alpha_x, alpha_y) at fixed u: a 5 x 4 list of
    floats [input][output], by central differences at 50 digits (truncation ~ 1e-40, rounding
    ~ 1e-30 relative)."""
    with mpmath.workdps(DIGITS):
        u1, u2 = mpmath.mpf(float(u1)), mpmath.mpf(float(u2))
        x = [mpmath.mpf(float(t)) for t in (*wi, ax, ay)]
        out = []
        for k in range(5):
            step = mpmath.mpf("1e-20") * max(1, abs(x[k]))
            xp, xm = list(x), list(x)
            xp[k] += step
            xm[k] -= step
            fp = _forward(u1, u2, *xp)
            fm = _forward(u1, u2, *xm)
            out.append([float((p - m) / (2 * step)) for p, m in zip(fp, fm)])
        return out


def reflection(u1, u2, wi, ax, ay, f0):
    """(wo (3 floats), pdf of wo, weight) for one upper-domain sample, at 50 digits."""
    with mpmath.workdps(DIGITS):
        u1, u2, ax, ay, f0 = (mpmath.mpf(float(t)) for t in (u1, u2, ax, ay, f0))
        w = [mpmath.mpf(float(t)) for t in wi]
        mx, my, mz, pdf_m = _forward(u1, u2, *w, ax, ay)
        n = mpmath.sqrt(w[0] ** 2 + w[1] ** 2 + w[2] ** 2)
        ux, uy, uz = w[0] / n, w[1] / n, w[2] / n
        d = ux * mx + uy * my + uz * mz
        ox, oy, oz = 2 * d * mx - ux, 2 * d * my - uy, 2 * d * mz - uz
        pdf_o = pdf_m / (4 * d)

        def g1(x, y, z):
            return 2 * z / (z + mpmath.sqrt((ax * x) ** 2 + (ay * y) ** 2 + z * z))

        if oz <= 0:
            weight = mpmath.mpf(0)
        else:
            gi, go = g1(ux, uy, uz), g1(ox, oy, oz)
            fr = f0 + (1 - f0) * (1 - d) ** 5
            weight = fr * go / (gi + go - gi * go)
        return (float(ox), float(oy), float(oz)), float(pdf_o), float(weight)
