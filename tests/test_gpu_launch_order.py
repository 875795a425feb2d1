"""Back-to-back calls on one stream see each other's results (programmatic dependent launches).

Outside graph capture the streaming and adjoint kernels are launched so that
their CTAs may become resident while the kernel ahead of them drains; each
waits in hardware for that kernel's completion before it reads or writes
memory.  These tests chain producers and consumers with no synchronisation in
between, a library kernel after a torch kernel and the other way round, and
a kernel that overwrites a buffer the kernel ahead of it still reads, and
compare every result with the same calls made one at a time with a full
synchronisation after each.
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


def _chain(v, d, u1, u2, wm, pdf, pdf2, seed, sync):
    s = torch.cuda.synchronize if sync else (lambda: None)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
    v.vndf_rng_uniform(u1.numel(), seed, 0, 0, u1=u1, u2=u2)                     # writes u
    s()
    v.vndf_sample(*(d[k] for k in keys), u1, u2, wm_x=wm[0], wm_y=wm[1], wm_z=wm[2], pdf=pdf)  # reads u
    s()
    v.vndf_pdf(*(d[k] for k in keys), wm[0], wm[1], wm[2], pdf=pdf2)              # reads wm
    s()
    u1.mul_(0.5)                                                                  # torch kernel rewrites u
    s()
    v.vndf_sample(*(d[k] for k in keys), u1, u2, wm_x=wm[0], wm_y=wm[1], wm_z=wm[2])  # overwrites wm
    s()
    out = [t.clone() for t in (*wm, pdf, pdf2, u1)]
    torch.cuda.synchronize()
    return out


def test_chained_calls_equal_synchronised_calls(v):
    n = (1 << 22) + 3
    d = workloads.anisotropic_stream(n=n, seed=12, device=DEV)
    bufs = lambda: ([torch.empty(n, device=DEV) for _ in range(2)], [torch.empty(n, device=DEV) for _ in range(3)],  # noqa: E731
                    torch.empty(n, device=DEV), torch.empty(n, device=DEV))
    for seed in (3, 4, 5):
        (u1, u2), wm, pdf, pdf2 = bufs()
        ref = _chain(v, d, u1, u2, wm, pdf, pdf2, seed, sync=True)
        (u1, u2), wm, pdf, pdf2 = bufs()
        got = _chain(v, d, u1, u2, wm, pdf, pdf2, seed, sync=False)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)


def test_adjoint_after_forward_without_synchronisation(v):
    n = (1 << 22) + 1
    d = workloads.adjoint_2e24(n=n, seed=4, device=DEV)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")

    def run(sync):
        s = torch.cuda.synchronize if sync else (lambda: None)
        wm = v.vndf_sample(*(d[k] for k in keys), seed=9)
        s()
        g = v.vndf_sample_backward(*(d[k] for k in keys), seed=9, g_wm_x=wm[0], g_wm_y=wm[1], g_wm_z=wm[2],
                                   g_pdf=wm[3])
        s()
        loss = v.vndf_sample_loss_backward(*(d[k] for k in keys), g[0], g[1], g[2], seed=9)
        torch.cuda.synchronize()
        return [t for t in (*wm, *g, *loss) if t is not None]

    ref = run(True)
    got = run(False)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_hemisphere_then_reflection_without_synchronisation(v):
    """The stand-alone hemisphere sampler's normals feed reflection sampling as incident directions."""
    n = (1 << 21) + 7
    h = workloads.hemisphere_stream(n=n, seed=14, device=DEV)
    a = torch.full((n,), 0.3, device=DEV)

    def run(sync):
        s = torch.cuda.synchronize if sync else (lambda: None)
        wm = v.vndf_sample_hemisphere(h["wi_x"], h["wi_y"], h["wi_z"], seed=6)
        s()
        out = v.vndf_sample_reflection(wm[0], wm[1], wm[2], a, None, seed=7)
        s()
        rng = v.vndf_rng_uniform(n, 8, 0, 0, device=DEV)
        s()
        dens = v.vndf_pdf(out[0], out[1], out[2], a, None, wm[0], wm[1], wm[2])
        torch.cuda.synchronize()
        return [*wm, *out, *rng, dens]

    ref = run(True)
    got = run(False)
    for x, y in zip(got, ref):
        assert torch.equal(x, y)
