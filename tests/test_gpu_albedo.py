"""GPU parity of the batched albedo estimator against the FP64 oracle.

The oracle (oracle.microfacet.albedo_estimate) evaluates the App. A estimator
term by term (BRDF, reflection pdf, |cos|) on the same Philox streams, in
FP64; it is pinned on the CPU against direct BRDF integration and quadrature.
"""
import numpy as np
import pytest
import torch

import workloads
from oracle import microfacet

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


@pytest.fixture(scope="module")
def grid():
    return workloads.albedo_grid(device=DEV)


def _oracle(d, idx, f0=0.04, seed=3, base=0, sid=0):
    wi = np.stack([d[k].cpu().numpy().astype(np.float64)[idx] for k in ("wi_x", "wi_y", "wi_z")])
    a = d["alpha_x"].cpu().numpy().astype(np.float64)[idx]
    ay = d["alpha_y"].cpu().numpy().astype(np.float64)[idx] if "alpha_y" in d else a
    ns = d["n_samples"].cpu().numpy()[idx]
    out = np.empty(len(idx))
    for i, q in enumerate(idx):
        w = microfacet.albedo_samples(wi[:, i], a[i], ay[i], int(ns[i]), f0, seed, base, (sid + int(q)) & 0xFFFFFFFF)
        out[i] = w.mean() if w.size else 0.0
    return out


def test_albedo_grid_matches_oracle(v, grid):
    E = v.vndf_albedo_batched(grid["wi_x"], grid["wi_y"], grid["wi_z"], grid["alpha_x"], None, grid["n_samples"])
    e = E.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(e)) and e.min() >= 0.0 and e.max() <= 1.0
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, 63, 64 * 63, 4095], rng.choice(4096, 60, replace=False)]))
    ref = _oracle(grid, idx)
    rel = np.abs(e[idx] / ref - 1.0)
    print(f"albedo: max rel {rel.max():.2e} over {len(idx)} queries")
    assert rel.max() < 1e-5


def test_albedo_small_alpha_is_fresnel(v, grid):
    """alpha = 1e-3 (grid column 0): a near-mirror reflects E ~ F(cos theta_i) once alpha tan(theta_i)
    is small (Smith's Lambda ~ (alpha tan theta)^2 / 4 otherwise still shadows grazing directions)."""
    E = v.vndf_albedo_batched(grid["wi_x"], grid["wi_y"], grid["wi_z"], grid["alpha_x"], None,
                              grid["n_samples"]).cpu().numpy().reshape(64, 64)
    cos_t = grid["wi_z"].cpu().numpy().reshape(64, 64)[:, 0].astype(np.float64)
    f = microfacet.schlick_fresnel(cos_t, 0.04)
    tan_t = np.sqrt(1 - cos_t ** 2) / cos_t
    rows = 1e-3 * tan_t <= 5e-3
    assert rows.sum() > 50
    assert np.abs(E[rows, 0] - f[rows]).max() < 2e-4


def test_albedo_bit_identical_across_configs_splits_and_graphs(v, grid):
    args = (grid["wi_x"], grid["wi_y"], grid["wi_z"], grid["alpha_x"], None, grid["n_samples"])
    ref = v.vndf_albedo_batched(*args, seed=11, counter_base=5)
    for cfg in [(1, 1, 1), (4, 1, 2), (8, 4, 4), (16, 8, 4), (20, 2, 1), (2, 256, 32)]:
        assert torch.equal(v.vndf_albedo_batched(*args, seed=11, counter_base=5, config=cfg), ref)
    # split the queries into two calls with the stream id advanced by the split point
    k = 1500
    part = [v.vndf_albedo_batched(*(t[s] if t is not None else None for t in args), seed=11, counter_base=5,
                                  stream_id=s.start or 0) for s in (slice(0, k), slice(k, 4096))]
    assert torch.equal(torch.cat(part), ref)
    # CUDA graph capture and replay
    E = torch.empty(4096, device=DEV)
    ws = torch.empty(v.vndf_albedo_workspace_bytes(4096, 65536), dtype=torch.uint8, device=DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        v.vndf_albedo_batched(*args, seed=11, counter_base=5, E=E, workspace=ws)  # warm-up on the side stream
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        v.vndf_albedo_batched(*args, seed=11, counter_base=5, E=E, workspace=ws)
    for _ in range(3):
        E.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(E, ref)


def test_albedo_autotune_keeps_results(v, grid):
    args = (grid["wi_x"], grid["wi_y"], grid["wi_z"], grid["alpha_x"], None, grid["n_samples"])
    ref = v.vndf_albedo_batched(*args, config=(8, 2, 4))
    best, ms = v.vndf_albedo_autotune(*args)
    print("albedo autotune:", best, f"{ms:.4f} ms")
    assert ms > 0.0
    assert torch.equal(v.vndf_albedo_batched(*args), ref)


def test_albedo_autotune_cache_sets_the_stored_configuration(v, grid, tmp_path):
    """A configuration tuned once is stored on disk and, in a later run, set without timing; E does not depend
    on it."""
    args = (grid["wi_x"], grid["wi_y"], grid["wi_z"], grid["alpha_x"], None, grid["n_samples"])
    cache = str(tmp_path / "albedo_tune.json")
    ref = v.vndf_albedo_batched(*args, config=(8, 1, 8))
    try:
        tuned, ms = v.vndf_albedo_autotune(*args, cache=cache)
        assert v.vndf_albedo_get_config() == (tuned, True)
        v.vndf_albedo_set_config(None)  # as in a fresh process
        assert v.vndf_albedo_get_config() == ((20, 2, 1), False)
        hit = v.vndf_albedo_autotune(*args, cache=cache)
        assert hit == (tuned, ms)
        assert v.vndf_albedo_get_config() == (tuned, True)
        assert torch.equal(v.vndf_albedo_batched(*args), ref)
        v.vndf_albedo_set_config((4, 4, 16))
        assert v.vndf_albedo_get_config() == ((4, 4, 16), True)
        assert torch.equal(v.vndf_albedo_batched(*args), ref)
        with pytest.raises(v.VndfError):
            v.vndf_albedo_set_config((0, 1, 1))
    finally:
        v.vndf_albedo_set_config(None)


def test_albedo_edge_counts(v):
    """Counts 0, 1, 255, 257, above the bound and negative; anisotropic alphas; odd counter base."""
    counts = [0, 1, 255, 257, 3000, 70000, -4, 65536]
    nq = len(counts)
    rng = np.random.default_rng(3)
    ct = rng.uniform(0.05, 1.0, nq)
    ph = rng.uniform(0, 2 * np.pi, nq)
    st = np.sqrt(1 - ct * ct)
    d = {"wi_x": st * np.cos(ph), "wi_y": st * np.sin(ph), "wi_z": ct,
         "alpha_x": rng.uniform(0.05, 1, nq), "alpha_y": rng.uniform(0.05, 1, nq)}
    t = {k: torch.as_tensor(x.astype(np.float32), device=DEV) for k, x in d.items()}
    t["n_samples"] = torch.as_tensor(np.array(counts, np.int32), device=DEV)
    E = v.vndf_albedo_batched(t["wi_x"], t["wi_y"], t["wi_z"], t["alpha_x"], t["alpha_y"], t["n_samples"],
                              max_samples_per_query=65536, seed=7, counter_base=3, stream_id=100).cpu().numpy()
    assert E[0] == 0.0
    assert np.isnan(E[5]) and np.isnan(E[6])
    ok = [1, 2, 3, 4, 7]
    tn = {k: x.cpu() for k, x in t.items()}
    ref = _oracle(tn, ok, seed=7, base=3, sid=100)
    err = np.abs(E[ok] - ref)
    assert np.all(err <= 1e-5 * np.abs(ref) + 1e-7), (E[ok], ref)


def test_albedo_on_wide_queries(v):
    """Stress queries: roughness 1e-5 to 10 per axis (anisotropic), wi of any length on the upper
    hemisphere down to grazing 1e-4, counts 0 to 3000 (ragged, many below one group), plus queries
    outside the domain (wi.z <= 0, alpha = 0): E = NaN outside the domain, 0 for a count of 0, and
    elsewhere finite, in [0, 1] and equal to the oracle's same-u estimate."""
    g = torch.Generator().manual_seed(23)
    q = 512
    ct = torch.exp(torch.empty(q, dtype=torch.float64).uniform_(np.log(1e-4), 0.0, generator=g))
    phi = torch.empty(q, dtype=torch.float64).uniform_(0.0, 2 * np.pi, generator=g)
    r = torch.exp(torch.empty(q, dtype=torch.float64).uniform_(np.log(1e-2), np.log(1e2), generator=g))
    st = torch.sqrt(1 - ct * ct)
    wx, wy, wz = st * torch.cos(phi) * r, st * torch.sin(phi) * r, ct * r
    ax = torch.exp(torch.empty(q, dtype=torch.float64).uniform_(np.log(1e-5), np.log(10.0), generator=g))
    ay = torch.exp(torch.empty(q, dtype=torch.float64).uniform_(np.log(1e-5), np.log(10.0), generator=g))
    ns = torch.randint(0, 3001, (q,), generator=g, dtype=torch.int32)
    wz[:8] = -wz[:8]  # below the horizon: outside the domain
    ax[8:12] = 0.0    # alpha = 0: outside the domain
    ns[12:16] = 0
    d = {k: t.to(torch.float32).to(DEV) for k, t in (("wi_x", wx), ("wi_y", wy), ("wi_z", wz), ("alpha_x", ax),
                                                        ("alpha_y", ay))}
    d["n_samples"] = ns.to(DEV)
    E = v.vndf_albedo_batched(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], d["n_samples"],
                              max_samples_per_query=3000)
    e = E.cpu().numpy().astype(np.float64)
    assert np.all(np.isnan(e[:12])) and np.all(e[12:16] == 0.0)
    assert np.all(np.isfinite(e[12:])) and e[12:].min() >= 0.0 and e[12:].max() <= 1.0
    idx = np.arange(16, q)
    with np.errstate(all="ignore"):
        ref = _oracle(d, idx)
    err = np.abs(e[idx] - ref)
    print(f"wide albedo: max abs err {err.max():.2e} over {idx.size} queries")
    assert np.all(err <= 1e-5 * np.abs(ref) + 2e-7)
