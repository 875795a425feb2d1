"""GPU parity of the roughness-map fitting step against the FP64 oracle (oracle.fit),
plus CUDA-graph replay and checkpoint/resume determinism."""
import numpy as np
import pytest
import torch

import workloads
from oracle import fit as ofit

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


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _inputs(res):
    d = workloads.roughness_map(res=res, device=DEV)
    wi = [d["wi_x"], d["wi_y"], d["wi_z"]]
    tg = [d["target_x"], d["target_y"], d["target_z"]]
    return d, wi, tg


def test_fit_steps_match_oracle(v):
    d, wi, tg = _inputs(16)  # 256 texels
    st = v.fit_state(d["alpha_x"], d["alpha_y"])
    loss = torch.empty(1, device=DEV)
    ref = {"ax": _np(d["alpha_x"]), "ay": _np(d["alpha_y"]), "mx": np.zeros(256), "my": np.zeros(256),
           "vx": np.zeros(256), "vy": np.zeros(256)}
    wi_n = np.stack([_np(t) for t in wi])
    tg_n = np.stack([_np(t) for t in tg])
    for step in range(1, 4):
        v.vndf_fit_step(st, *wi, *tg, seed=5, loss=loss)
        ref, rloss, _ = ofit.fit_step(ref, wi_n, tg_n, 1024, step, seed=5)
        got = float(loss.item())
        print(f"step {step}: loss gpu {got:.8e} oracle {rloss:.8e}")
        assert abs(got / rloss - 1) < 1e-5
        for k, r in (("alpha_x", "ax"), ("alpha_y", "ay"), ("m_x", "mx"), ("m_y", "my")):
            np.testing.assert_allclose(_np(st[k]), ref[r], rtol=1e-4, atol=1e-7)
        for k, r in (("v_x", "vx"), ("v_y", "vy")):
            np.testing.assert_allclose(_np(st[k]), ref[r], rtol=1e-3, atol=1e-14)
    assert int(st["step"].item()) == 3


def test_fit_graph_replay_and_resume_are_bit_identical(v):
    d, wi, tg = _inputs(16)
    # eager: 6 steps
    a = v.fit_state(d["alpha_x"], d["alpha_y"])
    la = torch.empty(1, device=DEV)
    losses_a = []
    for _ in range(6):
        v.vndf_fit_step(a, *wi, *tg, seed=9, loss=la)
        losses_a.append(la.clone())
    # graph: capture one step, replay 6 times
    b = v.fit_state(d["alpha_x"], d["alpha_y"])
    lb = torch.empty(1, device=DEV)
    ws = torch.empty(v.vndf_fit_workspace_bytes(256), dtype=torch.uint8, device=DEV)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        v.vndf_fit_step(b, *wi, *tg, seed=9, loss=lb, workspace=ws)
    # capture does not execute: state still at step 0
    assert int(b["step"].item()) == 0
    for k in range(6):
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(lb, losses_a[k])
    for key in a:
        assert torch.equal(a[key], b[key]), key
    # checkpoint after 3 steps, restore into fresh tensors, 3 more steps
    c = v.fit_state(d["alpha_x"], d["alpha_y"])
    for _ in range(3):
        v.vndf_fit_step(c, *wi, *tg, seed=9)
    saved = {k: t.cpu().clone() for k, t in c.items()}
    del c
    restored = {k: t.to(DEV) for k, t in saved.items()}
    for _ in range(3):
        v.vndf_fit_step(restored, *wi, *tg, seed=9)
    for key in a:
        assert torch.equal(a[key], restored[key]), key


@pytest.mark.slow
def test_full_map_step_sampled_texels(v):
    """256 x 256 texels x 1024 samples (the full map): one step, checked on sampled texels."""
    d, wi, tg = _inputs(256)
    nt = 256 * 256
    st = v.fit_state(d["alpha_x"], d["alpha_y"])
    loss = torch.empty(1, device=DEV)
    v.vndf_fit_step(st, *wi, *tg, seed=5, loss=loss)
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(nt, 48, replace=False))
    for q in idx[:48]:
        sub = slice(int(q), int(q) + 1)
        ref = {"ax": _np(d["alpha_x"][sub]), "ay": _np(d["alpha_y"][sub]), "mx": np.zeros(1), "my": np.zeros(1),
               "vx": np.zeros(1), "vy": np.zeros(1)}
        wi_n = np.stack([_np(t[sub]) for t in wi])
        tg_n = np.stack([_np(t[sub]) for t in tg])
        new, _, (gx, gy) = ofit.fit_step(ref, wi_n, tg_n, 1024, 1, seed=5, stream_base=int(q), n_total=nt)
        np.testing.assert_allclose(_np(st["m_x"][sub]), new["mx"], rtol=1e-4, atol=1e-12)
        np.testing.assert_allclose(_np(st["m_y"][sub]), new["my"], rtol=1e-4, atol=1e-12)
        if min(abs(gx[0]), abs(gy[0])) > 1e-9:
            np.testing.assert_allclose(_np(st["alpha_x"][sub]), new["ax"], rtol=1e-5, atol=1e-7)
            np.testing.assert_allclose(_np(st["alpha_y"][sub]), new["ay"], rtol=1e-5, atol=1e-7)
    assert np.isfinite(loss.item())


def test_fit_split_map_equals_one_call(v):
    """One map fitted as two parts (texels [0, T0) and [T0, T), each call with stream_id = its first
    texel and n_texels_total = T) gives the same alpha and moments, bit for bit, as one call over the
    map, and the parts' losses add up to its loss; the parts may run on different GPUs."""
    d, wi, tg = _inputs(16)  # 256 texels
    t_all, t0 = 256, 100
    full = v.fit_state(d["alpha_x"], d["alpha_y"])
    lf = torch.empty(1, device=DEV)
    parts = [v.fit_state(d["alpha_x"][:t0].contiguous(), d["alpha_y"][:t0].contiguous()),
             v.fit_state(d["alpha_x"][t0:].contiguous(), d["alpha_y"][t0:].contiguous())]
    lp = [torch.empty(1, device=DEV), torch.empty(1, device=DEV)]
    sl = [slice(0, t0), slice(t0, t_all)]
    for step in range(3):
        v.vndf_fit_step(full, *wi, *tg, seed=7, loss=lf)
        for k in range(2):
            v.vndf_fit_step(parts[k], *(x[sl[k]].contiguous() for x in wi), *(x[sl[k]].contiguous() for x in tg),
                            seed=7, stream_id=sl[k].start, loss=lp[k], n_texels_total=t_all)
        torch.cuda.synchronize()
        assert abs((lp[0].item() + lp[1].item()) / lf.item() - 1.0) < 1e-6
    for key in ("alpha_x", "alpha_y", "m_x", "m_y", "v_x", "v_y"):
        assert torch.equal(torch.cat([parts[0][key], parts[1][key]]), full[key]), key
    assert int(parts[0]["step"].item()) == int(parts[1]["step"].item()) == 3
