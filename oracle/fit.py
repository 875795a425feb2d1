"""Roughness-map fitting step: FP64 oracle (test infrastructure).

The paper gives the sampler, not an optimiser; this restates the fitting step
the library runs so the GPU can be checked against it.  Per texel t, with the
incident direction wi_t and roughness (ax_t, ay_t):

* draw S reparameterised samples wm_tj with the spherical-cap sampler
  (Sec. 2 steps (1)-(3), Sec. 3.3); uniforms from Philox stream stream_base + t,
  global index counter_base + (step - 1) S + j, so every step draws fresh samples;
* lobe mean m_t = (1/S) sum_j wm_tj;
* loss L = (1 / 3T) sum_t |m_t - target_t|^2 (mean squared error over all
  3T components);
* gradient dL/d(ax_t, ay_t) = (2 / 3T)(m_t - target_t) . (1/S) sum_j d wm_tj / d(ax_t, ay_t),
  the per-sample derivative taken by the complex-step method (oracle.grad);
* Adam (Kingma & Ba, ICLR 2015, Algorithm 1) with bias correction at the
  1-based step number, then projection of alpha onto [alpha_min, alpha_max].

Only tests, the smoke entry point and the bench's CPU legs import this.
"""
import numpy as np

from . import philox
from .grad import H_CS
from .vndf import sample_vndf


def texel_uniforms(n_texels, samples, step, seed, counter_base=0, stream_base=0):
    """(u1, u2), each (T, S): the uniforms of every texel's samples at a 1-based step."""
    u1 = np.empty((n_texels, samples))
    u2 = np.empty((n_texels, samples))
    base = (int(counter_base) + (int(step) - 1) * samples) & 0xFFFFFFFFFFFFFFFF
    for t in range(n_texels):
        u1[t], u2[t] = philox.sample_uniforms(seed, base, (int(stream_base) + t) & 0xFFFFFFFF, samples)
    return u1, u2


def lobe_means(u1, u2, wi, ax, ay):
    """m_t = mean over samples of wm (wi: (3, T), alphas: (T,), u: (T, S)) -> (3, T)."""
    t, s = u1.shape
    wib = np.repeat(np.asarray(wi)[:, :, None], s, axis=2).reshape(3, -1)
    wm = sample_vndf(u1.reshape(-1), u2.reshape(-1), wib, np.repeat(ax, s), np.repeat(ay, s))
    return wm.reshape(3, t, s).mean(axis=2)


def loss_and_grad(u1, u2, wi, ax, ay, target, n_total=None):
    """(L, dL/dax (T,), dL/day (T,), m (3, T)) at fixed uniforms.

    n_total: number of texels of the whole map when these T texels are a subset
    of it (the MSE divides by 3 n_total); defaults to T.
    """
    t, s = u1.shape
    nt = t if n_total is None else int(n_total)
    m = lobe_means(u1, u2, wi, ax, ay)
    diff = m - target
    loss = (diff ** 2).sum() / (3.0 * nt)
    wib = np.repeat(np.asarray(wi)[:, :, None], s, axis=2).reshape(3, -1).astype(np.complex128)
    g = []
    for which in (0, 1):
        axc = np.repeat(ax, s).astype(np.complex128)
        ayc = np.repeat(ay, s).astype(np.complex128)
        if which == 0:
            axc = axc + 1j * H_CS
        else:
            ayc = ayc + 1j * H_CS
        dwm = np.imag(sample_vndf(u1.reshape(-1), u2.reshape(-1), wib, axc, ayc)) / H_CS
        dm = dwm.reshape(3, t, s).mean(axis=2)
        g.append((2.0 / (3.0 * nt)) * (diff * dm).sum(axis=0))
    return loss, g[0], g[1], m


def adam(param, grad, m, v, step, lr, beta1, beta2, eps):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); step is 1-based."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return param - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def fit_step(state, wi, target, samples, step, seed, counter_base=0, stream_base=0, lr=1e-2, beta1=0.9,
             beta2=0.999, eps=1e-8, alpha_min=1e-3, alpha_max=1.0, n_total=None):
    """One fitting step.  state: dict with ax, ay, mx, my, vx, vy (each (T,)).

    Returns (new state, loss, (dL/dax, dL/day)).  With n_total, the T texels are a
    subset of a map of n_total texels that starts at stream stream_base.
    """
    t = wi.shape[1]
    u1, u2 = texel_uniforms(t, samples, step, seed, counter_base, stream_base)
    loss, gx, gy, _ = loss_and_grad(u1, u2, wi, state["ax"], state["ay"], target, n_total)
    ax, mx, vx = adam(state["ax"], gx, state["mx"], state["vx"], step, lr, beta1, beta2, eps)
    ay, my, vy = adam(state["ay"], gy, state["my"], state["vy"], step, lr, beta1, beta2, eps)
    new = {"ax": np.clip(ax, alpha_min, alpha_max), "ay": np.clip(ay, alpha_min, alpha_max),
           "mx": mx, "my": my, "vx": vx, "vy": vy}
    return new, loss, (gx, gy)
