"""GPU parity of the sampling path against the FP64 oracle (through the C ABI).

Sizes span many CTAs and a ragged tail; the full 2^28-sample anisotropic
workload is checked on sampled outputs in the launch configuration the bench
times.  Tolerances are explained in tests/parity.py.
"""
import numpy as np
import pytest
import torch

import parity
import workloads
from oracle import philox, vndf as ovndf

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


def _np(*ts):
    return [t.detach().cpu().numpy() for t in ts]


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=DEV)


@pytest.mark.parametrize("n,seed,base,sid", [
    (1 << 20, 1, 0, 0),
    ((1 << 20) + 3, 2, 7, 1),
    (4097, 0xFFFFFFFFFFFFFFFF, (1 << 64) - 6, 0xFFFFFFFF),
    (33, 5, (1 << 32) - 3, 12),
])
def test_philox_bit_exact(v, n, seed, base, sid):
    u1, u2 = v.vndf_rng_uniform(n, seed, base, sid, device=DEV)
    r1, r2 = philox.sample_uniforms(seed, base, sid, n)
    g1, g2 = _np(u1, u2)
    np.testing.assert_array_equal(g1.astype(np.float64), r1)
    np.testing.assert_array_equal(g2.astype(np.float64), r2)


def test_philox_unaligned_output(v):
    buf1 = torch.empty(1030, device=DEV)
    buf2 = torch.empty(1030, device=DEV)
    v.vndf_rng_uniform(1027, 9, 4, 2, u1=buf1[1:1028], u2=buf2[3:1030])
    r1, r2 = philox.sample_uniforms(9, 4, 2, 1027)
    np.testing.assert_array_equal(buf1[1:1028].cpu().numpy().astype(np.float64), r1)
    np.testing.assert_array_equal(buf2[3:1030].cpu().numpy().astype(np.float64), r2)


def test_cap_isotropic_2e20_explicit_u(v):
    """2^20 samples, isotropic alpha ~ U[0.01, 1], wi uniform on the hemisphere, u from Philox(1)."""
    n = 1 << 20
    d = workloads.isotropic_2e20(n=n, device=DEV)
    u1, u2 = philox.sample_uniforms(1, 0, 0, n)
    wx, wy, wz, pdf = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], None, _dev(u1), _dev(u2))
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"]))
    a = d["alpha_x"].cpu().numpy()
    st = parity.compare_cap(np.stack(_np(wx, wy, wz)), pdf.cpu().numpy(), u1, u2, wi, a, a)
    print("isotropic_2e20", st)


@pytest.mark.parametrize("n,base", [((1 << 20) + 5, 0), ((1 << 20) + 2, 3)])
def test_cap_anisotropic_philox(v, n, base):
    """Anisotropic workload distribution (log-uniform alphas in [1e-3, 1]), in-kernel Philox(2)."""
    d = workloads.anisotropic_stream(n=n, device=DEV)
    wx, wy, wz, pdf = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"],
                                    seed=2, counter_base=base)
    u1, u2 = philox.sample_uniforms(2, base, 0, n)
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"]))
    st = parity.compare_cap(np.stack(_np(wx, wy, wz)), pdf.cpu().numpy(), u1, u2, wi,
                            d["alpha_x"].cpu().numpy(), d["alpha_y"].cpu().numpy())
    print("anisotropic", n, base, st)


def test_philox_mode_equals_explicit_uniforms(v):
    n = 100003
    d = workloads.anisotropic_stream(n=n, seed=31, device=DEV)
    a = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=77, counter_base=11,
                      stream_id=4)
    u1, u2 = v.vndf_rng_uniform(n, 77, 11, 4, device=DEV)
    b = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_results_independent_of_path_and_split(v):
    """Vector path, scalar path (unaligned views) and split calls give identical bits."""
    n = 50001
    d = workloads.anisotropic_stream(n=n + 1, seed=32, device=DEV)
    full = v.vndf_sample(d["wi_x"][:n], d["wi_y"][:n], d["wi_z"][:n], d["alpha_x"][:n], d["alpha_y"][:n],
                         seed=5, counter_base=100)
    # shift every input by one element: misaligned, so the scalar path runs
    shifted = {k: torch.cat([d[k][:1], d[k][:n]]) for k in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")}
    s = v.vndf_sample(shifted["wi_x"][1:], shifted["wi_y"][1:], shifted["wi_z"][1:], shifted["alpha_x"][1:],
                      shifted["alpha_y"][1:], seed=5, counter_base=100, n=n)
    for x, y in zip(full, s):
        assert torch.equal(x, y)
    # two calls over [0, k) and [k, n) with the counter base advanced by k
    for k in (4, 9, 25000, 33333):
        p1 = v.vndf_sample(*(d[q][:k] for q in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")),
                           seed=5, counter_base=100)
        p2 = v.vndf_sample(*(d[q][k:n].contiguous() for q in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")),
                           seed=5, counter_base=100 + k)
        for x, a, b in zip(full, p1, p2):
            assert torch.equal(x, torch.cat([a, b]))


def test_without_pdf_same_normals(v):
    n = 4099
    d = workloads.anisotropic_stream(n=n, seed=33, device=DEV)
    a = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=1)
    b = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=1, with_pdf=False)
    assert b[3] is None
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 7, 8, 9])
def test_tiny_sizes(v, n):
    d = workloads.anisotropic_stream(n=max(n, 1), seed=34, device=DEV)
    sl = {k: t[:n] for k, t in d.items()}
    wx, wy, wz, pdf = v.vndf_sample(sl["wi_x"], sl["wi_y"], sl["wi_z"], sl["alpha_x"], sl["alpha_y"], seed=3)
    if n == 0:
        return
    u1, u2 = philox.sample_uniforms(3, 0, 0, n)
    wi = np.stack(_np(sl["wi_x"], sl["wi_y"], sl["wi_z"]))
    parity.compare_cap(np.stack(_np(wx, wy, wz)), pdf.cpu().numpy(), u1, u2, wi,
                       sl["alpha_x"].cpu().numpy(), sl["alpha_y"].cpu().numpy())


def test_domain_edges_and_extremes(v):
    """Fallback on invalid inputs; the extremes of the parity domain (alpha = 1e-3, wi.z = 1e-4,
    u2 = 0 and u2 = 1 - 2^-24, u1 = 0)."""
    nan = float("nan")
    inf = float("inf")
    wx = [0.3, 0.3, 0.3, 0.3, nan, 0.3, inf, 1.0, 0.99999, 0.0, 0.6, 0.6, 0.6, 0.6]
    wy = [0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1, 0.0, 0.0, 0.0, 0.8, 0.8, -0.8, 0.8]
    wz = [0.0, -0.5, 0.9, 0.9, 0.9, 0.9, 0.9, 1e-4, 1e-4, 1.0, 0.05, 0.05, 0.05, 0.05]
    ax = [0.5, 0.5, 0.0, -1.0, 0.5, nan, 0.5, 1e-3, 1.0, 1e-3, 1e-3, 1.0, 1e-3, 0.3]
    ay = [0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 1e-3, 1e-3, 1e-3, 1.0, 1e-3, 1e-3, 0.7]
    u1 = [0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.25, 0.0, 0.5, 0.75, 0.1, 0.9, 0.3, 0.0]
    u2 = [0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.0, 1 - 2 ** -24, 1 - 2 ** -24, 0.999, 0.5, 1 - 2 ** -24, 0.0]
    t = [_dev(x) for x in (wx, wy, wz, ax, ay, u1, u2)]
    wmx, wmy, wmz, pdf = v.vndf_sample(*t[:5], t[5], t[6])
    wi = np.array([wx, wy, wz], dtype=np.float32)
    st = parity.compare_cap(np.stack(_np(wmx, wmy, wmz)), pdf.cpu().numpy(),
                            np.array(u1, np.float32), np.array(u2, np.float32), wi,
                            np.array(ax, np.float32), np.array(ay, np.float32))
    assert st["out_of_domain"] == 7


def test_prior_sampler_parity(v):
    """The prior (polar-disk) sampler against its own FP64 oracle (the paper's prior sampler, Sec. 2
    step (2)), same I/O as the cap sampler."""
    n = (1 << 20) + 1
    d = workloads.anisotropic_stream(n=n, device=DEV)
    wx, wy, wz, pdf = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=2,
                                    method="polar")
    u1, u2 = philox.sample_uniforms(2, 0, 0, n)
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"])).astype(np.float64)
    ax, ay = (t.cpu().numpy().astype(np.float64) for t in (d["alpha_x"], d["alpha_y"]))
    ref = ovndf.sample_vndf(u1, u2, wi, ax, ay, "polar")
    pref = ovndf.vndf_pdf(ref, wi, ax, ay)
    ang = parity.angle_between(np.stack(_np(wx, wy, wz)).astype(np.float64), ref)
    rel = np.abs(pdf.cpu().numpy() / pref - 1.0)
    print(f"prior: max angle {ang.max():.3e} p99.99 {np.quantile(ang, 0.9999):.3e} "
          f"tail>4e-6 {(ang > 4e-6).mean():.2e}; pdf max rel {rel.max():.3e} tail>1e-5 {(rel > 1e-5).mean():.2e}")
    # the prior kernel gets the same cancellation-free rewrites as the cap sampler, so it must
    # meet the same accuracy: "faster at equal accuracy" compares like with like
    assert (ang > 4e-6).mean() < 1e-4 and ang.max() < 1e-3
    assert (rel > 1e-5).mean() < 1e-4


def test_pdf_entry_at_given_normals(v):
    """vndf_pdf against the oracle's density at the same float32 normals."""
    n = (1 << 18) + 3
    d = workloads.anisotropic_stream(n=n, seed=35, device=DEV)
    wx, wy, wz, _ = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=8,
                                  with_pdf=False)
    p = v.vndf_pdf(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], wx, wy, wz)
    wi = np.stack(_np(d["wi_x"], d["wi_y"], d["wi_z"])).astype(np.float64)
    wm = np.stack(_np(wx, wy, wz)).astype(np.float64)
    ax, ay = (t.cpu().numpy().astype(np.float64) for t in (d["alpha_x"], d["alpha_y"]))
    ref = ovndf.vndf_pdf(wm, wi, ax, ay)
    rel = np.abs(p.cpu().numpy() / ref - 1.0)
    # the dot product wi.wm cancels for normals near the visibility boundary
    kd = (np.abs(wi * wm).sum(0) / np.abs(ovndf.dot(wi, wm))) / np.sqrt(ovndf.dot(wi, wi))
    bound = np.maximum(1e-5, parity.K_ULP * (kd + 8.0) * parity.EPS32)
    assert np.all(rel <= bound), rel.max()
    # isotropic form
    pi = v.vndf_pdf(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], None, wx, wy, wz)
    refi = ovndf.vndf_pdf(wm, wi, ax, ax)
    assert np.all(np.abs(pi.cpu().numpy() / refi - 1.0) <= bound)


@pytest.mark.slow
def test_full_size_anisotropic_stream_sampled(v):
    """2^28 samples in one call (the bench's launch), checked on 2^16 sampled outputs + both ends."""
    n = 1 << 28
    d = workloads.anisotropic_stream(n=n, device=DEV)
    out = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=2)
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([np.arange(1024), n - 1 - np.arange(1024), rng.integers(0, n, 1 << 16)]))
    ti = torch.as_tensor(idx, device=DEV)
    wi = np.stack([d[k].index_select(0, ti).cpu().numpy() for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = (d[k].index_select(0, ti).cpu().numpy() for k in ("alpha_x", "alpha_y"))
    wm = np.stack([o.index_select(0, ti).cpu().numpy() for o in out[:3]])
    pdf = out[3].index_select(0, ti).cpu().numpy()
    u1, u2 = philox.uniforms_at(2, 0, 0, idx)
    st = parity.compare_cap(wm, pdf, u1, u2, wi, ax, ay)
    print("full size sampled", st)
    del d, out
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_indices_beyond_int32(v):
    """2^31 + 4101 samples in one call (77 GB of inputs and outputs): element indices past 2^31 and
    Philox counters past 2^31 must be formed in 64 bits, and the n % 4 = 1 tail must run.  The
    inputs tile a 2^20 + 3 block of the anisotropic workload (an odd period, so every residue mod 4
    meets every input); outputs are checked at the int32 boundaries, the end and random windows
    against the oracle with the same uniforms; vndf_pdf is run over the same normals, and reflection
    sampling and the hemisphere sampler over the same inputs.
    Only this library's kernels touch the full arrays: they are filled and read back through
    slices, each a separate copy of at most 2^20 + 3 elements (torch's gather kernel asserts on
    tensors of more than 2^31 elements)."""
    n = (1 << 31) + 4101  # n % 4 = 1
    free, _ = torch.cuda.mem_get_info()
    if free < 100 * (1 << 30):
        pytest.skip(f"needs about 86 GB of free device memory, {free / 2**30:.0f} GB free")
    period = (1 << 20) + 3
    blk = workloads.anisotropic_stream(n=period, seed=41, device=DEV)
    d = {}
    for k, t in blk.items():
        x = torch.empty(n, dtype=torch.float32, device=DEV)
        for s0 in range(0, n, period):
            m = min(period, n - s0)
            x[s0:s0 + m].copy_(t[:m])
        d[k] = x
    out = v.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=9, counter_base=3)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    L = 64
    starts = np.unique(np.concatenate([[0, (1 << 30) - L // 2, (1 << 31) - L // 2, n - L],
                                       rng.integers(0, n - L, 60)]))
    idx = np.concatenate([s0 + np.arange(L) for s0 in starts])

    assert starts.max() + L <= n

    def gather(t):
        return np.concatenate([t[int(s0):int(s0) + L].cpu().numpy() for s0 in starts])

    blk_np = {k: t.cpu().numpy() for k, t in blk.items()}
    wi = np.stack([blk_np[k][idx % period] for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = blk_np["alpha_x"][idx % period], blk_np["alpha_y"][idx % period]
    for k in ("wi_x", "alpha_y"):  # the tiled inputs themselves, at the same windows
        assert np.array_equal(gather(d[k]), blk_np[k][idx % period])
    wm = np.stack([gather(o) for o in out[:3]])
    pdf = gather(out[3])
    u1, u2 = philox.uniforms_at(9, 3, 0, idx)
    st = parity.compare_cap(wm, pdf, u1, u2, wi, ax, ay)
    print("beyond int32", st)
    # the density entry over the same normals
    p2 = v.vndf_pdf(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], out[0], out[1], out[2])
    torch.cuda.synchronize()
    p2s = gather(p2).astype(np.float64)
    wi64, wm64 = wi.astype(np.float64), wm.astype(np.float64)
    ref = ovndf.vndf_pdf(wm64, wi64, ax.astype(np.float64), ay.astype(np.float64))
    kd = (np.abs(wi64 * wm64).sum(0) / np.abs(ovndf.dot(wi64, wm64))) / np.sqrt(ovndf.dot(wi64, wi64))
    assert np.all(np.abs(p2s / ref - 1.0) <= np.maximum(1e-5, parity.K_ULP * (kd + 8.0) * parity.EPS32))
    del out, p2
    torch.cuda.empty_cache()
    # reflection sampling over the same inputs, with the bounds of test_gpu_reflection.py
    from oracle import microfacet
    from test_gpu_reflection import _weight_sensitivity
    ax64, ay64 = ax.astype(np.float64), ay.astype(np.float64)
    refl = v.vndf_sample_reflection(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=9,
                                    counter_base=3, f0=0.04)
    torch.cuda.synchronize()
    got = np.stack([gather(t) for t in refl[:3]]).astype(np.float64)
    pg, wg = (gather(t).astype(np.float64) for t in refl[3:])
    wb, pr, wr = microfacet.sample_reflection(u1, u2, wi64, ax64, ay64, 0.04)
    assert parity.angle_between(got, wb).max() <= 2 * parity.ANGLE_TOL
    assert np.abs(pg / pr - 1.0).max() <= parity.PDF_TOL
    sens = _weight_sensitivity(u1, u2, wi64, ax64, ay64, 0.04)
    assert np.all(np.abs(wg - wr) <= 1e-5 * np.abs(wr) + 1e-7 + sens * parity.ANGLE_TOL)
    del refl
    torch.cuda.empty_cache()
    # the hemisphere sampler over the same directions
    hemi = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], seed=9, counter_base=3)
    torch.cuda.synchronize()
    hm = np.stack([gather(t) for t in hemi[:3]]).astype(np.float64)
    hp = gather(hemi[3]).astype(np.float64)
    href, hpref = ovndf.sample_hemisphere(u1, u2, wi64)
    assert parity.angle_between(hm, href).max() <= parity.ANGLE_TOL
    assert np.quantile(np.abs(hp / hpref - 1.0), 0.999) <= parity.PDF_TOL
    del d, hemi
    torch.cuda.empty_cache()
