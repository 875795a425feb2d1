"""Pins for the roughness-map fitting oracle (oracle.fit).

* the loss gradient equals central finite differences of the loss itself at
  fixed uniforms (chain rule through the lobe mean and the sampler);
* Adam's first step moves every parameter by lr * sign(g) (m_hat = g,
  v_hat = g^2 after bias correction: Kingma & Ba 2015, Algorithm 1);
* the projection keeps alpha inside [alpha_min, alpha_max];
* fitting a target produced by a known roughness map lowers the loss and
  moves alpha toward that map.
"""
import numpy as np

from oracle import fit


def _setup(t=16, seed=0):
    rng = np.random.default_rng(seed)
    ct = rng.uniform(0.1, 1.0, t)
    ph = rng.uniform(0, 2 * np.pi, t)
    st = np.sqrt(1 - ct * ct)
    wi = np.stack([st * np.cos(ph), st * np.sin(ph), ct])
    ax = rng.uniform(0.05, 0.8, t)
    ay = rng.uniform(0.05, 0.8, t)
    return wi, ax, ay, rng


def test_gradient_matches_finite_differences():
    wi, ax, ay, rng = _setup()
    target = rng.normal(0, 0.1, (3, 16)) + np.array([[0.0], [0.0], [0.9]])
    u1, u2 = fit.texel_uniforms(16, 64, 1, seed=5)
    loss, gx, gy, _ = fit.loss_and_grad(u1, u2, wi, ax, ay, target)
    h = 1e-6
    for t in (0, 7, 15):
        for which, g in ((0, gx), (1, gy)):
            p = [ax.copy(), ay.copy()]
            q = [ax.copy(), ay.copy()]
            p[which][t] += h
            q[which][t] -= h
            lp = fit.loss_and_grad(u1, u2, wi, p[0], p[1], target)[0]
            lq = fit.loss_and_grad(u1, u2, wi, q[0], q[1], target)[0]
            assert abs((lp - lq) / (2 * h) - g[t]) <= 1e-6 * max(abs(g[t]), 1e-3)


def test_first_adam_step_is_signed_lr():
    g = np.array([3e-4, -2.0, 1e-2, -5e-6])
    p = np.array([0.5, 0.5, 0.5, 0.5])
    new, m, v = fit.adam(p, g, np.zeros(4), np.zeros(4), 1, 1e-2, 0.9, 0.999, 1e-8)
    np.testing.assert_allclose(new - p, -1e-2 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_projection_bounds_and_recovery():
    wi, _, _, rng = _setup(8, seed=1)
    true_ax = np.linspace(0.1, 0.7, 8)
    true_ay = np.linspace(0.6, 0.15, 8)
    u1, u2 = fit.texel_uniforms(8, 4096, 1, seed=99, stream_base=1000)
    target = fit.lobe_means(u1, u2, wi, true_ax, true_ay)
    state = {"ax": np.full(8, 0.4), "ay": np.full(8, 0.4), "mx": np.zeros(8), "my": np.zeros(8),
             "vx": np.zeros(8), "vy": np.zeros(8)}
    first = None
    for step in range(1, 61):
        state, loss, _ = fit.fit_step(state, wi, target, 256, step, seed=7, lr=2e-2, alpha_min=0.05,
                                      alpha_max=0.9)
        first = loss if first is None else first
        assert state["ax"].min() >= 0.05 and state["ax"].max() <= 0.9
        assert state["ay"].min() >= 0.05 and state["ay"].max() <= 0.9
    assert loss < 0.2 * first
    err0 = np.abs(0.4 - true_ax).mean() + np.abs(0.4 - true_ay).mean()
    err1 = np.abs(state["ax"] - true_ax).mean() + np.abs(state["ay"] - true_ay).mean()
    assert err1 < 0.5 * err0
