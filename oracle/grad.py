"""Derivatives of the sampled normal and its pdf: FP64 oracle (test infrastructure).

The paper defines no gradient; reparameterised gradients of (wm, pdf) with the
uniforms u held fixed are what inverse rendering needs from the sampler.  This
module differentiates the oracle's own forward map (``oracle.vndf``: Sec. 2
steps (1)-(3) with the cap sampler of Sec. 3.3 and the pdf of Eq. 1 / App. A)
by the complex-step method (Squire & Trapp 1998; Martins, Sturdza & Alonso
2003): for an analytic f, f'(x) = Im f(x + i h) / h with no subtractive
cancellation, so h = 1e-30 gives the derivative to FP64 rounding.  Central
finite differences are kept as an independent second referee.

Only tests, the smoke entry point and the bench's CPU-baseline leg import this.
"""
import numpy as np

from .vndf import sample_vndf, vndf_pdf

H_CS = 1e-30
INPUT_NAMES = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")


def _forward(u1, u2, wi, ax, ay, method="cap", extended=False):
    wm = sample_vndf(u1, u2, wi, ax, ay, method, extended)
    pdf = vndf_pdf(wm, wi, ax, ay, extended)
    return np.concatenate([wm, pdf[None]], axis=0)  # (4, N): wm_x, wm_y, wm_z, pdf


def jacobian_complex_step(u1, u2, wi, ax, ay, method="cap", extended=False):
    """d(wm_x, wm_y, wm_z, pdf)/d(input) for each input in INPUT_NAMES.

    Returns an array of shape (5, 4, N): [input, output, sample].  extended=True differentiates
    the sampler and density on the extended domain (incident directions below the horizon).
    """
    base = [np.asarray(wi[0], np.float64), np.asarray(wi[1], np.float64),
            np.asarray(wi[2], np.float64), np.asarray(ax, np.float64), np.asarray(ay, np.float64)]
    out = []
    for k in range(5):
        args = [b.astype(np.complex128) for b in base]
        args[k] = args[k] + 1j * H_CS
        f = _forward(u1, u2, args[:3], args[3], args[4], method, extended)
        out.append(np.imag(f) / H_CS)
    return np.stack(out)


def jacobian_central_difference(u1, u2, wi, ax, ay, rel_step=1e-6, method="cap", extended=False):
    """Same Jacobian by central differences, step rel_step * max(1, |x|)."""
    base = [np.asarray(wi[0], np.float64), np.asarray(wi[1], np.float64),
            np.asarray(wi[2], np.float64), np.asarray(ax, np.float64), np.asarray(ay, np.float64)]
    out = []
    for k in range(5):
        step = rel_step * np.maximum(1.0, np.abs(base[k]))
        plus = [b.copy() for b in base]
        minus = [b.copy() for b in base]
        plus[k] = plus[k] + step
        minus[k] = minus[k] - step
        fp = _forward(u1, u2, plus[:3], plus[3], plus[4], method, extended)
        fm = _forward(u1, u2, minus[:3], minus[3], minus[4], method, extended)
        out.append((fp - fm) / (2.0 * step))
    return np.stack(out)


def u_jacobian_complex_step(u1, u2, wi, ax, ay, extended=False):
    """d wm / d u1 and d wm / d u2 (each (3, N)) for the cap sampler."""
    u1 = np.asarray(u1, np.float64)
    u2 = np.asarray(u2, np.float64)
    d1 = np.imag(sample_vndf(u1 + 1j * H_CS, u2.astype(np.complex128), wi, ax, ay, "cap", extended)) / H_CS
    d2 = np.imag(sample_vndf(u1.astype(np.complex128), u2 + 1j * H_CS, wi, ax, ay, "cap", extended)) / H_CS
    return d1, d2


def vjp(u1, u2, wi, ax, ay, g_wm=None, g_pdf=None, isotropic=False, extended=False):
    """Vector-Jacobian product: (g_wi (3, N), g_alpha_x (N,), g_alpha_y (N,) or None).

    g_wm: (3, N) adjoint of wm (None = zero); g_pdf: (N,) adjoint of pdf (None = zero).
    With isotropic=True, alpha_y is alpha_x and the single alpha gradient is
    returned as g_alpha_x (g_alpha_y is None).  extended=True: on the extended domain.
    """
    n = np.asarray(u1).shape[0]
    g = np.zeros((4, n))
    if g_wm is not None:
        g[:3] = np.asarray(g_wm, np.float64)
    if g_pdf is not None:
        g[3] = np.asarray(g_pdf, np.float64)
    jac = jacobian_complex_step(u1, u2, wi, ax, ay, extended=extended)
    grads = (jac * g[None]).sum(axis=1)  # (5, N)
    if isotropic:
        return grads[:3], grads[3] + grads[4], None
    return grads[:3], grads[3], grads[4]
