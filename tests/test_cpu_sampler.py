"""The host-CPU sampler (vndf_cpu_sample) against the FP64 oracle; runs without a GPU.

It carries no double-float path, so it is held to the condition-scaled bound
of tests/parity.py (non-strict), like the GPU kernels were before their rescue;
the prior sampler is checked in bulk.
"""
import numpy as np
import pytest

import parity
import workloads
from oracle import philox, vndf as ovndf


@pytest.fixture(scope="module")
def v():
    from paper_2306_05044_gb300 import _build
    _build.build()
    import paper_2306_05044_gb300 as lib
    lib.load()
    return lib


def _inputs(n, seed=12):
    d = workloads.anisotropic_stream(n=n, seed=seed)
    return {k: t.numpy() for k, t in d.items()}


def test_cpu_cap_matches_oracle(v):
    n = (1 << 18) + 3
    d = _inputs(n)
    u1, u2 = philox.sample_uniforms(2, 0, 0, n)
    wx, wy, wz, pdf = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2)
    wi = np.stack([d["wi_x"], d["wi_y"], d["wi_z"]])
    st = parity.compare_cap(np.stack([wx, wy, wz]), pdf, u1, u2, wi, d["alpha_x"], d["alpha_y"], strict=False)
    print("cpu cap", st)
    assert st["tail_angle_frac"] < 1e-4


def test_cpu_cap_extended_matches_oracle(v):
    n = (1 << 17) + 5
    d = {k: t.numpy() for k, t in workloads.sphere_stream(n=n, seed=15).items()}
    u1, u2 = philox.sample_uniforms(5, 0, 0, n)
    wx, wy, wz, pdf = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2,
                                        method="cap_extended")
    wi = np.stack([d["wi_x"], d["wi_y"], d["wi_z"]])
    wm = np.stack([wx, wy, wz])
    st = parity.compare_cap(wm, pdf, u1, u2, wi, d["alpha_x"], d["alpha_y"], strict=False, extended=True)
    print("cpu cap extended", st)
    assert st["tail_angle_frac"] < 1e-3
    assert (wz > 0).all()
    # above the horizon the extended method is the upper-domain method, bit for bit
    up = wi[2] > 0
    ref = v.vndf_cpu_sample(*(d[k][up] for k in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")), u1[up], u2[up])
    for a, b in zip((wx, wy, wz, pdf), ref):
        assert np.array_equal(a[up], b)


def test_cpu_prior_matches_oracle(v):
    n = 1 << 16
    d = _inputs(n, seed=13)
    u1, u2 = philox.sample_uniforms(3, 0, 0, n)
    wx, wy, wz, pdf = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2,
                                        method="polar")
    wi = np.stack([d["wi_x"], d["wi_y"], d["wi_z"]]).astype(np.float64)
    ref = ovndf.sample_vndf(u1, u2, wi, d["alpha_x"], d["alpha_y"], "polar")
    pr = ovndf.vndf_pdf(ref, wi, d["alpha_x"], d["alpha_y"])
    ang = parity.angle_between(np.stack([wx, wy, wz]).astype(np.float64), ref)
    rel = np.abs(pdf / pr - 1)
    assert np.median(ang) < 1e-7 and (ang > 4e-6).mean() < 1e-3
    assert np.median(rel) < 1e-6 and (rel > 1e-5).mean() < 1e-3


def test_cpu_results_independent_of_threads_and_isotropy(v):
    n = 50001
    d = _inputs(n, seed=14)
    u1, u2 = philox.sample_uniforms(4, 0, 0, n)
    one = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2, threads=1)
    many = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2, threads=7)
    for a, b in zip(one, many):
        np.testing.assert_array_equal(a, b)
    iso = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], None, u1, u2, threads=3)
    same = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_x"], u1, u2, threads=3)
    for a, b in zip(iso, same):
        np.testing.assert_array_equal(a, b)


def test_cpu_domain_fallback_and_errors(v):
    x = np.array([0.3, 0.3, np.nan], np.float32)
    z = np.array([-0.1, 0.9, 0.9], np.float32)
    a = np.array([0.5, 0.0, 0.5], np.float32)
    u = np.full(3, 0.4, np.float32)
    wx, wy, wz, pdf = v.vndf_cpu_sample(x, x, z, a, a, u, u)
    np.testing.assert_array_equal(wz, np.ones(3, np.float32))
    np.testing.assert_array_equal(pdf, np.zeros(3, np.float32))
    with pytest.raises(v.VndfError):
        v.vndf_cpu_sample(x, x, z, a, a, u, u, method=5)


@pytest.mark.parametrize("kind", ["cap", "cap_extended"])
def test_cpu_sampler_on_stored_samples(v, kind):
    """The host sampler on the stored 50-digit rows (tests/golden), held to the
    condition-scaled bound (it has no double-float path); exact fallback outside the domain."""
    import oracle_checks as oc
    rows = [r for r in oc.golden_rows() if r["kind"] == kind]
    wi = np.stack([r["wi"] for r in rows], axis=1).astype(np.float32)
    col = {k: np.array([r[k] for r in rows], np.float32) for k in ("alpha_x", "alpha_y", "u1", "u2")}
    wx, wy, wz, pdf = v.vndf_cpu_sample(wi[0], wi[1], wi[2], col["alpha_x"], col["alpha_y"], col["u1"], col["u2"],
                                        method=kind)
    for k, r in enumerate(rows):
        g = np.array([wx[k], wy[k], wz[k]], np.float64)
        if np.isnan(r["one_plus_zi"]):
            assert tuple(g) == (0.0, 0.0, 1.0) and pdf[k] == 0.0
            continue
        kap, kap_h = parity.conditioning(np.array([r["u1"]]), np.array([r["u2"]]), r["wi"].reshape(3, 1),
                                         np.array([r["alpha_x"]]), np.array([r["alpha_y"]]))
        ang = float(parity.angle_between(g.reshape(3, 1), r["wm"].reshape(3, 1))[0])
        assert ang <= max(parity.ANGLE_TOL, parity.K_ULP * float(kap[0]) * parity.EPS32), (r["note"], ang)
        rel = abs(float(pdf[k]) / r["pdf"] - 1.0)
        assert rel <= max(parity.PDF_TOL, parity.K_ULP * float(3 * kap[0] + 2 * kap_h[0]) * parity.EPS32), \
            (r["note"], rel)


@pytest.mark.parametrize("kind", ["cap", "cap_extended"])
def test_cpu_precise_meets_the_flat_bounds(v, kind):
    """With precise=1 the host sampler recomputes ill-conditioned samples in double precision and meets
    4e-6 rad / 1e-5 relative on every sample inside the contract, as vndf_sample does; the other
    samples are those of the plain path, bit for bit."""
    n = (1 << 17) + 3
    if kind == "cap":
        d = _inputs(n, seed=16)
    else:
        d = {k: t.numpy() for k, t in workloads.sphere_stream(n=n, seed=17).items()}
    u1, u2 = philox.sample_uniforms(6, 0, 0, n)
    args = (d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2)
    strict = v.vndf_cpu_sample(*args, method=kind, precise=True)
    plain = v.vndf_cpu_sample(*args, method=kind)
    wi = np.stack([d["wi_x"], d["wi_y"], d["wi_z"]])
    st = parity.compare_cap(np.stack(strict[:3]), strict[3], u1, u2, wi, d["alpha_x"], d["alpha_y"], strict=True,
                            extended=kind == "cap_extended")
    print("cpu precise", kind, st)
    changed = np.zeros(n, bool)
    for a, b in zip(strict, plain):
        changed |= a != b
    assert 0 < changed.mean() < 1e-2  # only the flagged samples differ


def test_cpu_precise_on_stored_samples(v):
    """The stored 50-digit rows (tests/golden) inside the contract, at the flat bounds."""
    import oracle_checks as oc
    for kind in ("cap", "cap_extended"):
        rows = [r for r in oc.golden_rows() if r["kind"] == kind and not np.isnan(r["one_plus_zi"])
                and min(r["alpha_x"], r["alpha_y"]) >= 1e-3
                and (kind == "cap_extended" or r["wi"][2] / np.linalg.norm(r["wi"]) >= 1e-4)]
        wi = np.stack([r["wi"] for r in rows], axis=1).astype(np.float32)
        col = {k: np.array([r[k] for r in rows], np.float32) for k in ("alpha_x", "alpha_y", "u1", "u2")}
        wx, wy, wz, pdf = v.vndf_cpu_sample(wi[0], wi[1], wi[2], col["alpha_x"], col["alpha_y"], col["u1"],
                                            col["u2"], method=kind, precise=True)
        for k, r in enumerate(rows):
            g = np.array([wx[k], wy[k], wz[k]], np.float64).reshape(3, 1)
            assert float(parity.angle_between(g, r["wm"].reshape(3, 1))[0]) <= parity.ANGLE_TOL, r["note"]
            assert abs(float(pdf[k]) / r["pdf"] - 1.0) <= parity.PDF_TOL, r["note"]


@pytest.mark.parametrize("kind", ["cap", "cap_extended"])
def test_cpu_precise_on_wide_inputs(v, kind):
    """Stress inputs (wi on the whole sphere with lengths 1e-3 to 1e3, roughness 1e-5 to 10, uniforms at
    the ends of [0, 1)): every output finite, the flat bounds inside the contract, the condition-scaled
    bound outside it, the exact fallback outside the domain; extended-domain samples on which FP64 is
    weak are checked against the 50-digit reference."""
    d = {k: t.numpy() for k, t in workloads.wide_stream(n=1 << 15, seed=18).items()}
    u1, u2 = d["u1"].astype(np.float64), d["u2"].astype(np.float64)
    out = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], d["u1"], d["u2"],
                            method=kind, precise=True)
    assert all(np.isfinite(t).all() for t in out)
    wi = np.stack([d["wi_x"], d["wi_y"], d["wi_z"]])
    ext = kind == "cap_extended"
    st = parity.compare_cap(np.stack(out[:3]), out[3], u1, u2, wi, d["alpha_x"], d["alpha_y"], strict=True,
                            extended=ext)
    if ext:
        st.update(parity.compare_cap_mp(np.stack(out[:3]), out[3], u1, u2, wi, d["alpha_x"], d["alpha_y"], limit=150))
    print("cpu wide", kind, st)


_FORK_INPUTS = {}


def _child_samples(q):
    # only the library runs in the child (torch's own thread pools are not fork-safe)
    import paper_2306_05044_gb300 as lib
    d, u = _FORK_INPUTS["d"], _FORK_INPUTS["u"]
    out = lib.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u, u, threads=4)
    q.put(float(np.sum(out[3], dtype=np.float64)))


def test_cpu_worker_pool_after_fork(v):
    """The host worker threads live in the process that made them; a forked child starts its own on first use
    (it must not wait on workers that fork did not copy) and gets the parent's results."""
    import multiprocessing as mp
    d = _inputs(1 << 16, seed=21)
    u = np.full(1 << 16, 0.25, np.float32)
    ref = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u, u, threads=4)
    _FORK_INPUTS.update(d=d, u=u)
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_child_samples, args=(q,))
    p.start()
    p.join(60)
    if p.is_alive():
        p.kill()
        pytest.fail("the forked child did not finish")
    assert p.exitcode == 0
    assert q.get(timeout=10) == float(np.sum(ref[3], dtype=np.float64))


def test_cpu_concurrent_callers(v):
    """Calls from several host threads at once are served one after the other, each with its own results."""
    import threading
    inputs = [_inputs(50000, seed=30 + k) for k in range(4)]
    u = np.linspace(0, 1 - 2.0 ** -24, 50000).astype(np.float32)
    want = [v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u, u[::-1].copy(),
                              threads=3) for d in inputs]
    got = [None] * 4

    def call(k):
        d = inputs[k]
        got[k] = v.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u, u[::-1].copy(),
                                   threads=3)
    ts = [threading.Thread(target=call, args=(k,)) for k in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for a, b in zip(got, want):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
