"""Writes cap_samples_mp50.txt, cap_jacobians_mp50.txt and reflection_mp50.txt: stored
expected samples of the spherical-cap sampler, their derivatives, and reflection sampling
through them.

Every expected value comes from the oracle alone: the 50-digit evaluation of
Sec. 2 steps (1)-(3) with the Sec. 3.3 cap sampler and the density of Eq. 1
(``oracle.vndf_mp.sample_with_pdf``), and, for inputs outside the sampler's
domain, the fallback the oracle defines (``oracle.vndf.in_domain``; normal
(0, 0, 1), density 0); the derivatives of each in-domain sample with respect to
(wi, alpha) at fixed u come from ``oracle.vndf_mp.jacobian``, the reflected
directions, their densities and estimator weights from ``oracle.vndf_mp.reflection``.  Nothing here calls
the CUDA library.

The inputs are fixed float32 values chosen to reach the places where a
plausible mistake shows: normal incidence, grazing and below-horizon incident
directions, roughness from 1e-7 to 1.5, strong anisotropy, unnormalised wi,
and uniforms at the ends of [0, 1) (the cap's top at u2 = 0, its rim as
u2 -> 1, phi -> 2 pi as u1 -> 1).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import vndf  # noqa: E402  (oracle.vndf_mp, which needs mpmath, is imported where it is used)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cap_samples_mp50.txt")
OUT_JAC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cap_jacobians_mp50.txt")
OUT_REFL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reflection_mp50.txt")
REFL_F0 = 0.04
JAC_INPUTS = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
JAC_OUTPUTS = ("wm_x", "wm_y", "wm_z", "pdf")
ONE_M = 1.0 - 2.0 ** -24  # largest float32 uniform below 1
TINY_U = 2.0 ** -24

# kind, wi (x, y, z), alpha (x, y), u (1, 2), what the row exercises
CASES = [
    ("cap", (0.0, 0.0, 1.0), (1.0, 1.0), (0.0, 0.0), "alpha = 1 at normal incidence, cap top: wm = (0, 0, 1), pdf = 1/pi"),
    ("cap", (0.0, 0.0, 1.0), (0.5, 0.5), (0.25, 0.5), "normal incidence, isotropic"),
    ("cap", (0.6, 0.0, 0.8), (0.3, 0.3), (0.125, 0.75), "oblique, isotropic"),
    ("cap", (0.3, -0.4, 0.8660254), (0.05, 0.8), (0.7, 0.2), "anisotropic"),
    ("cap", (1.0, 0.0, 1e-3), (0.2, 0.2), (0.5, 0.5), "grazing wi.z = 1e-3"),
    ("cap", (0.6, 0.8, 1e-5), (0.5, 0.05), (0.9, 0.99), "grazing wi.z = 1e-5, anisotropic, near the rim"),
    ("cap", (0.5, 0.5, 0.70710678), (1e-4, 1e-4), (0.9, 0.1), "alpha = 1e-4"),
    ("cap", (0.8, 0.0, 0.6), (1.0, 1.0), (0.3, ONE_M), "alpha = 1, u2 at its largest (the rim)"),
    ("cap", (0.0, 0.99, 0.1), (1e-3, 1.0), (0.6, 0.4), "alpha_x / alpha_y = 1e-3"),
    ("cap", (-0.2, 0.5, 0.8), (1.5, 0.7), (0.05, 0.95), "alpha above 1"),
    ("cap", (3.0, -4.0, 12.0), (0.4, 0.4), (0.33, 0.66), "unnormalised wi, length 13"),
    ("cap", (0.1, 0.2, 0.97), (0.6, 0.3), (ONE_M, TINY_U), "u1 at its largest, u2 at its smallest non-zero"),
    ("cap", (-0.7, -0.1, 0.3), (0.02, 0.02), (0.37, 0.81), "small alpha, wi in the third quadrant"),
    ("cap", (0.3, 0.4, 0.8660254), (1e-7, 1e-7), (0.2, 0.6), "alpha = 1e-7"),
    ("cap", (0.5, 0.5, 0.0), (0.5, 0.5), (0.5, 0.5), "outside the domain: wi.z = 0"),
    ("cap", (0.6, 0.0, -0.8), (0.3, 0.3), (0.4, 0.6), "outside the domain: below the horizon"),
    ("cap", (0.0, 0.0, 1.0), (0.0, 0.5), (0.5, 0.5), "outside the domain: alpha_x = 0"),
    ("cap_extended", (0.6, 0.0, -0.8), (0.3, 0.3), (0.4, 0.6), "below the horizon, 1 + z_i' = 0.024"),
    ("cap_extended", (0.0, 0.8, -0.6), (0.01, 0.01), (0.2, 0.3), "below the horizon, 1 + z_i' = 9e-5"),
    ("cap_extended", (1.0, 0.0, -0.1), (1e-3, 1e-3), (0.75, 0.5), "below the horizon, 1 + z_i' = 5e-5"),
    ("cap_extended", (0.8660254, 0.0, -0.5), (1e-6, 1e-6), (0.1, 0.9), "below the horizon, 1 + z_i' = 1.5e-12"),
    ("cap_extended", (0.8660254, 0.0, -0.5), (1e-6, 1e-6), (0.3, ONE_M), "below the horizon, 1 + z_i' = 1.5e-12, the rim"),
    ("cap_extended", (1.0, 0.0, -0.05), (1e-7, 1e-7), (0.7, 0.3), "below the horizon, alpha = 1e-7, 1 + z_i' = 2e-12"),
    ("cap_extended", (0.5, 0.5, -0.5), (1.0, 1.0), (0.5, 0.25), "below the horizon, alpha = 1"),
    ("cap_extended", (0.3, 0.9, -0.3), (0.02, 0.5), (0.8, 0.05), "below the horizon, anisotropic"),
    ("cap_extended", (0.6, 0.0, 0.8), (0.3, 0.3), (0.125, 0.75), "above the horizon: same as the cap row"),
    ("cap_extended", (0.0, 0.0, -1.0), (0.5, 0.5), (0.5, 0.5), "outside the domain: straight down (1 + z_i' = 0)"),
    ("hemisphere", (0.0, 0.0, 1.0), (1.0, 1.0), (0.25, 0.5), "normal incidence"),
    ("hemisphere", (0.6, 0.0, 0.8), (1.0, 1.0), (0.5, 0.5), "oblique"),
    ("hemisphere", (0.8, 0.0, -0.6), (1.0, 1.0), (0.3, 0.7), "below the horizon"),
    ("hemisphere", (1e-5, 0.0, -1.0), (1.0, 1.0), (0.6, 0.4), "nearly straight down, 1 + z_i = 5e-11"),
    ("hemisphere", (0.0, 0.0, -1.0), (1.0, 1.0), (0.5, 0.5), "outside the domain: straight down"),
]


def f32(x):
    return float(np.float32(x))


def rows():
    from oracle import vndf_mp
    out = []
    for kind, wi, al, u, note in CASES:
        wi = tuple(f32(t) for t in wi)
        ax, ay = f32(al[0]), f32(al[1])
        u1, u2 = f32(u[0]), f32(u[1])
        w = np.array(wi, np.float64).reshape(3, 1)
        ok = bool(vndf.in_domain(w, np.array([ax]), np.array([ay]), kind != "cap")[0])
        if ok:
            wm, pdf = vndf_mp.sample_with_pdf(u1, u2, wi, ax, ay)
            a = vndf_mp.one_plus_zi(wi, ax, ay)
            p32 = vndf_mp.pdf_of_normal(tuple(f32(t) for t in wm), wi, ax, ay)
        else:
            wm, pdf, a, p32 = (0.0, 0.0, 1.0), 0.0, float("nan"), 0.0
        out.append((kind, wi, ax, ay, u1, u2, wm, pdf, a, p32, note))
    return out


def render(rs):
    lines = [
        "# Spherical-cap VNDF samples at 50 significant digits (Dupuy & Benyoub, HPG 2023).",
        "# Sec. 2 steps (1)-(3) with the Sec. 3.3 cap sampler; pdf = Eq. 1 at the sample.",
        "# kind = cap (upper domain, wi.z > 0), cap_extended (1 + z_i' >= 2^-40), or hemisphere",
        "# (Sec. 3.3 on its own: wm = h / |h|, the GGX sampler at alpha = 1).  Outside the domain",
        "# the expected output is wm = (0, 0, 1), pdf = 0.",
        "# Inputs are float32 values written as exact hexadecimal floats; outputs are the",
        "# 50-digit results rounded to float64.  one_plus_zi = 1 + z_i' (nan outside the domain).",
        "# pdf_wm32 = the density of the normal wm rounded to float32 (Eq. 1 through the App. A",
        "# forms of D and G1, G1(wi)/wi.z = 1/sigma(wi)), for checking density-of-a-normal entries.",
        "# Written by tests/golden/make_golden.py from oracle/ only.",
        "# kind wi_x wi_y wi_z alpha_x alpha_y u1 u2 | wm_x wm_y wm_z pdf one_plus_zi pdf_wm32 | note",
    ]
    for kind, wi, ax, ay, u1, u2, wm, pdf, a, p32, note in rs:
        ins = " ".join(float.hex(t) for t in (*wi, ax, ay, u1, u2))
        outs = " ".join(repr(float(t)) for t in (*wm, pdf, a, p32))
        lines.append(f"{kind} {ins} | {outs} | {note}")
    return "\n".join(lines) + "\n"


def load(path=OUT):
    """Parsed rows: dicts with kind, wi (3,), alpha_x, alpha_y, u1, u2, wm (3,), pdf, one_plus_zi,
    pdf_wm32, note."""
    res = []
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            ins, outs, note = (s.strip() for s in line.split("|", 2))
            f = ins.split()
            x = [float.fromhex(t) for t in f[1:]]
            y = [float(t) for t in outs.split()]
            res.append({"kind": f[0], "wi": np.array(x[0:3]), "alpha_x": x[3], "alpha_y": x[4],
                        "u1": x[5], "u2": x[6], "wm": np.array(y[0:3]), "pdf": y[3],
                        "one_plus_zi": y[4], "pdf_wm32": y[5], "note": note})
    return res


def jacobian_rows(rs):
    """(row index, 5 x 4 Jacobian) for every in-domain GGX row (cap and cap_extended)."""
    from oracle import vndf_mp
    out = []
    for k, (kind, wi, ax, ay, u1, u2, wm, pdf, a, p32, note) in enumerate(rs):
        if kind == "hemisphere" or a != a:
            continue
        out.append((k, vndf_mp.jacobian(u1, u2, wi, ax, ay)))
    return out


def render_jacobians(rs):
    lines = [
        "# Derivatives of the spherical-cap sample (wm) and its density (pdf) with respect to the inputs",
        "# (wi, alpha_x, alpha_y), with the uniforms held fixed: the reparameterised gradients that an",
        "# adjoint of Sec. 2 steps (1)-(3), Sec. 3.3 and Eq. 1 computes.  50-digit central differences",
        "# (oracle/vndf_mp.py: jacobian), rounded to float64.",
        "# row = index of the sample's row in cap_samples_mp50.txt (its non-comment lines, from 0).",
        "# The 20 numbers are J[input][output], inputs " + " ".join(JAC_INPUTS) + ",",
        "# outputs " + " ".join(JAC_OUTPUTS) + " (input-major).",
        "# Written by tests/golden/make_golden.py from oracle/ only.",
    ]
    for k, jac in jacobian_rows(rs):
        lines.append(f"{k} | " + " ".join(repr(float(v)) for row in jac for v in row))
    return "\n".join(lines) + "\n"


def reflection_rows(rs):
    """(row index, wo, pdf, weight) for every upper-domain cap row; out-of-domain rows give the
    fallback (0, 0, 1), 0, 0."""
    from oracle import vndf_mp
    out = []
    for k, (kind, wi, ax, ay, u1, u2, wm, pdf, a, p32, note) in enumerate(rs):
        if kind != "cap":
            continue
        if a != a:
            out.append((k, (0.0, 0.0, 1.0), 0.0, 0.0))
        else:
            out.append((k, *vndf_mp.reflection(u1, u2, wi, ax, ay, REFL_F0)))
    return out


def render_reflection(rs):
    lines = [
        "# Reflection sampling through the spherical-cap sampler (App. A), 50 digits, rounded to float64:",
        "# for each upper-domain row of cap_samples_mp50.txt (its sample wm), wo = 2 (wi.wm) wm - wi with",
        "# unit wi (Eq. reflect), the density of wo, pdf(wm) / (4 wi.wm), and the estimator weight",
        "# F(wi.wm) G2 / G1(wi) (Schlick's F with f0 = %r, height-correlated G2; 0 when wo.z <= 0)." % REFL_F0,
        "# Outside the domain: wo = (0, 0, 1), pdf = 0, weight = 0.",
        "# row | wo_x wo_y wo_z pdf weight",
        "# Written by tests/golden/make_golden.py from oracle/ only.",
    ]
    for k, wo, p, w in reflection_rows(rs):
        lines.append(f"{k} | " + " ".join(repr(float(t)) for t in (*wo, p, w)))
    return "\n".join(lines) + "\n"


def load_reflection(path=OUT_REFL):
    """{row index: (wo (3,), pdf, weight)}."""
    res = {}
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            k, vals = line.split("|", 1)
            v = [float(t) for t in vals.split()]
            res[int(k)] = (np.array(v[:3]), v[3], v[4])
    return res


def load_jacobians(path=OUT_JAC):
    """{row index: 5 x 4 array [input][output]}."""
    res = {}
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            k, vals = line.split("|", 1)
            res[int(k)] = np.array([float(t) for t in vals.split()]).reshape(5, 4)
    return res


if __name__ == "__main__":
    rs = rows()
    with open(OUT, "w") as fh:
        fh.write(render(rs))
    with open(OUT_JAC, "w") as fh:
        fh.write(render_jacobians(rs))
    with open(OUT_REFL, "w") as fh:
        fh.write(render_reflection(rs))
    print(f"wrote {OUT}, {OUT_JAC} and {OUT_REFL}")
