"""Host-side fault injection through the Python binding, on the GPU host.

With VNDF_FAULT set, every GPU entry point returns the injected status after
its argument checks and before it enqueues any work, so no kernel runs and no
GPU is made to fail.  Each binding must turn that status into VndfError with
the same code: a failed launch (VNDF_ERR_CUDA) and, for the entry points that
take a workspace, a workspace error.  The C-level behaviour is also checked on
the CPU host (tests/test_abi.py).
"""
import pytest
import torch

import workloads

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


def _bindings(v):
    """name -> (call, takes a workspace); small real inputs on the device."""
    n = 1027
    d = workloads.anisotropic_stream(n=n, seed=12, device=DEV)
    a = workloads.adjoint_2e24(n=n, seed=4, device=DEV)
    wi = (d["wi_x"], d["wi_y"], d["wi_z"])
    al = (d["alpha_x"], d["alpha_y"])
    g = workloads.albedo_grid(device=DEV)
    q = (g["wi_x"][:64].contiguous(), g["wi_y"][:64].contiguous(), g["wi_z"][:64].contiguous(),
         g["alpha_x"][:64].contiguous(), None, g["n_samples"][:64].contiguous())
    m = workloads.roughness_map(device=DEV)
    st = v.fit_state(m["alpha_x"], m["alpha_y"])
    fit_in = (m["wi_x"], m["wi_y"], m["wi_z"], m["target_x"], m["target_y"], m["target_z"])
    wm = [torch.rand(n, device=DEV) for _ in range(3)]
    return {
        "vndf_rng_uniform": (lambda: v.vndf_rng_uniform(n, 1, device=DEV), False),
        "vndf_sample": (lambda: v.vndf_sample(*wi, *al, seed=1), False),
        "vndf_pdf": (lambda: v.vndf_pdf(*wi, *al, *wm), False),
        "vndf_pdf_extended": (lambda: v.vndf_pdf_extended(*wi, *al, *wm), False),
        "vndf_sample_reflection": (lambda: v.vndf_sample_reflection(*wi, *al, seed=1), False),
        "vndf_sample_hemisphere": (lambda: v.vndf_sample_hemisphere(*wi, seed=1), False),
        "vndf_sample_backward": (lambda: v.vndf_sample_backward(*wi, *al, seed=1, g_pdf=d["alpha_x"]), False),
        "vndf_sample_backward_extended": (lambda: v.vndf_sample_backward_extended(*wi, *al, seed=1,
                                                                                  g_pdf=d["alpha_x"]), False),
        "vndf_sample_loss_backward": (lambda: v.vndf_sample_loss_backward(
            a["wi_x"], a["wi_y"], a["wi_z"], a["alpha_x"], a["alpha_y"], a["c_x"], a["c_y"], a["c_z"], seed=1),
            True),
        "vndf_albedo_batched": (lambda: v.vndf_albedo_batched(*q, max_samples_per_query=65536), True),
        "vndf_albedo_autotune": (lambda: v.vndf_albedo_autotune(*q, max_samples_per_query=65536), True),
        "vndf_fit_step": (lambda: v.vndf_fit_step(st, *fit_in, loss=torch.empty(1, device=DEV)), True),
        "vndf_microbench": (lambda: v.vndf_microbench(1024, 8, device=DEV), False),
        "vndf_rescue_count": (lambda: v.vndf_rescue_count(*wi, *al, seed=1), False),
        "vndf_albedo_set_config": (lambda: v.vndf_albedo_set_config(None), False),
    }


def test_every_binding_raises_the_injected_status(v, monkeypatch):
    calls = _bindings(v)
    torch.cuda.synchronize()
    for kind, status in (("launch", -6), ("workspace", -5)):
        monkeypatch.setenv("VNDF_FAULT", kind)
        for name, (call, takes_ws) in calls.items():
            if kind == "workspace" and not takes_ws:
                continue
            with pytest.raises(v.VndfError) as err:
                call()
            assert err.value.status == status, (kind, name)
            assert name in str(err.value)
    # only the named entry point fails; the others run normally
    monkeypatch.setenv("VNDF_FAULT", "launch@vndf_pdf")
    with pytest.raises(v.VndfError):
        calls["vndf_pdf"][0]()
    out = calls["vndf_sample"][0]()
    monkeypatch.delenv("VNDF_FAULT")
    torch.cuda.synchronize()
    assert torch.isfinite(out[3]).all()
    # and the context is untouched: every entry point runs again once the variable is cleared
    for name, (call, _) in calls.items():
        if name != "vndf_albedo_autotune":
            call()
    torch.cuda.synchronize()


def test_in_place_calls_are_rejected_before_any_work(v):
    """An output aliasing an input would let the batched double-float recomputation reread overwritten inputs;
    every entry point refuses such a call with VNDF_ERR_ARG and leaves the buffers untouched."""
    n = (1 << 16) + 3
    d = workloads.sphere_stream(n=n, seed=15, device=DEV)  # below-horizon inputs: many flagged samples
    wi = [d["wi_x"], d["wi_y"], d["wi_z"]]
    al = [d["alpha_x"], d["alpha_y"]]
    keep = [t.clone() for t in wi + al]
    calls = [
        lambda: v.vndf_sample(*wi, *al, seed=1, method="cap_extended", wm_x=wi[0]),
        lambda: v.vndf_sample(*wi, *al, seed=1, pdf=al[1]),
        lambda: v.vndf_sample_reflection(*wi, *al, seed=1, wo_z=wi[2]),
        lambda: v.vndf_sample_hemisphere(*wi, seed=1, wm_y=wi[1]),
        lambda: v.vndf_pdf(*wi, *al, wi[0], wi[1], wi[2], pdf=wi[2]),
        lambda: v.vndf_sample_backward(*wi, *al, seed=1, g_pdf=al[0], outputs=(None, None, None, al[0], None)),
    ]
    for call in calls:
        with pytest.raises(v.VndfError) as err:
            call()
        assert err.value.status == -7
    torch.cuda.synchronize()
    for a, b in zip(wi + al, keep):
        assert torch.equal(a, b)
