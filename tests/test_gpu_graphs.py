"""Every streaming and adjoint entry point inside one captured CUDA graph.

The calls are asynchronous on the caller's stream and allocate nothing, so a CUDA graph can capture
them.  The replayed graph must give, bit for bit, what the same calls give eagerly, and must follow
in-place changes of its inputs (it keeps pointers, not values).  Albedo and the fitting step have
their own graph tests, next to their parity tests.
"""
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N = (1 << 16) + 3   # full staged chunks and a ragged tail


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


def _run_all(v, d, a, u1, u2, ws):
    """One call of each entry point; returns every output tensor in a fixed order."""
    wi = (d["wi_x"], d["wi_y"], d["wi_z"])
    out = list(v.vndf_rng_uniform(N, 7, 3, 1, device=DEV))
    for method in ("cap", "polar", "cap_extended"):
        out += v.vndf_sample(*wi, d["alpha_x"], d["alpha_y"], method=method, seed=2, counter_base=9)
        out += v.vndf_sample(*wi, d["alpha_x"], None, u1=u1, u2=u2, method=method)
    wm = out[-4:-1]
    out.append(v.vndf_pdf(*wi, d["alpha_x"], d["alpha_y"], *wm))
    out.append(v.vndf_pdf_extended(*wi, d["alpha_x"], d["alpha_y"], *wm))
    out += [t for t in v.vndf_sample_reflection(*wi, d["alpha_x"], d["alpha_y"], seed=4)]
    out += [t for t in v.vndf_sample_hemisphere(*wi, seed=5)]
    adj = (a["wi_x"], a["wi_y"], a["wi_z"], a["alpha_x"], a["alpha_y"])
    for ext in (False, True):
        out += v.vndf_sample_backward(*adj, seed=6, g_wm_x=a["c_x"], g_wm_y=a["c_y"], g_wm_z=a["c_z"],
                                      g_pdf=a["c_x"], extended=ext)
    out += v.vndf_sample_loss_backward(*adj, a["c_x"], a["c_y"], a["c_z"], seed=8, workspace=ws)
    out.append(v.vndf_microbench(4099, samples_per_lane=8, device=DEV))
    return [t for t in out if t is not None]


def _same(xs, ys):
    assert len(xs) == len(ys)
    for k, (x, y) in enumerate(zip(xs, ys)):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32)), f"output {k} differs"


def test_entry_points_replay_in_a_cuda_graph(v):
    d = workloads.anisotropic_stream(n=N, seed=12, device=DEV)
    a = workloads.adjoint_2e24(n=N, seed=4, device=DEV)
    u1, u2 = v.vndf_rng_uniform(N, 1, 0, 0, device=DEV)
    ws = torch.empty(max(v.vndf_loss_workspace_bytes(N), 4), dtype=torch.uint8, device=DEV)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _run_all(v, d, a, u1, u2, ws)  # warm-up: one-time kernel attributes are set outside the capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        captured = _run_all(v, d, a, u1, u2, ws)
    for t in captured:
        t.view(torch.int32).fill_(0x7FA5A5A5)
    g.replay()
    torch.cuda.synchronize()
    _same(captured, _run_all(v, d, a, u1, u2, ws))
    # the graph reads its inputs at replay time
    d["alpha_x"].mul_(0.5)
    a["alpha_y"].mul_(0.75)
    u2.mul_(0.5)
    g.replay()
    torch.cuda.synchronize()
    _same(captured, _run_all(v, d, a, u1, u2, ws))
