"""Guard bands around every buffer of every GPU entry point.

Each input, output and workspace is a slice of a larger buffer whose elements before and after the
slice hold a canary bit pattern (a quiet NaN with a payload no kernel writes).  After each call the
guards must still hold the canary bit for bit (no write outside the caller's elements, none into an
input), and the results must equal, bit for bit, those of the same call on fresh 16-byte-aligned
buffers: the vector, staged and scalar paths give the same bits.  Sizes: empty, 1, 3, 5, a few
thousand with a ragged tail, and enough for full staged chunks plus a tail; starts: 16-byte aligned
and 4, 8 and 12 bytes past a boundary.  This checks the library's index arithmetic without any
instrumentation of the kernels.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CANARY32 = 0x7FA5A5A5               # bits of a quiet NaN with a payload
CANARY64 = 0x7FA5A5A57FA5A5A5
CANARY8 = 0xA5
PAD = 64                            # guard elements per side: 256 bytes of 32-bit elements
SIZES = (0, 1, 3, 5, 1027, 4097, (1 << 16) + 3)
OFFSETS = (0, 1, 2, 3)              # elements past a 16-byte boundary


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


class Guards:
    """Guarded slices; check() compares every guard (and every input buffer) with what it held."""

    def __init__(self):
        self.items = []

    @staticmethod
    def _raw(count, dtype):
        if dtype == torch.uint8:
            return torch.full((count,), CANARY8, dtype=torch.uint8, device=DEV)
        if dtype == torch.int64:
            return torch.full((count,), CANARY64, dtype=torch.int64, device=DEV)
        return torch.full((count,), CANARY32, dtype=torch.int32, device=DEV)

    def make(self, n, off=0, src=None, dtype=torch.float32, pad=PAD, inout=False):
        """n elements `off` past a 16-byte boundary, filled from src when given; an input unless
        `inout` (state updated in place) or no src (an output): those get only their guards checked."""
        raw = self._raw(pad + off + n + pad, dtype)
        view = raw.view(torch.float32) if dtype == torch.float32 else raw
        t = view[pad + off:pad + off + n]
        if src is not None:
            t.copy_(src.reshape(-1)[:n])
        read_only = src is not None and not inout
        self.items.append((raw, pad + off, n, raw.clone() if read_only else None, dtype))
        return t

    def check(self):
        torch.cuda.synchronize()
        for raw, lo, n, snap, dtype in self.items:
            if snap is not None:
                assert torch.equal(raw, snap), "an input buffer or its guards changed"
            else:
                ref = self._raw(raw.numel(), dtype)
                assert torch.equal(raw[:lo], ref[:lo]), "write before the start of an output"
                assert torch.equal(raw[lo + n:], ref[lo + n:]), "write past the end of an output"


def _bits(t):
    return t.contiguous().view(torch.int32) if t.dtype == torch.float32 else t


def _same(a, b):
    if a is None or b is None:
        assert a is None and b is None
        return
    assert torch.equal(_bits(a), _bits(b)), "a guarded, offset call differs from the aligned call"


def _fresh(t):
    return t.clone()  # a new, aligned allocation with the same contents


@pytest.mark.parametrize("off", OFFSETS)
@pytest.mark.parametrize("n", SIZES)
def test_streaming_entry_points(v, n, off):
    G = Guards()
    d = workloads.sphere_stream(n=max(n, 1), seed=17, device=DEV)
    wi = [G.make(n, off, d[k]) for k in ("wi_x", "wi_y", "wi_z")]
    ax, ay = G.make(n, off, d["alpha_x"]), G.make(n, off, d["alpha_y"])
    fwi, fax, fay = [_fresh(t) for t in wi], _fresh(ax), _fresh(ay)
    # the uniforms of the in-kernel generator, written into guarded outputs
    u1, u2 = G.make(n, off), G.make(n, off)
    v.vndf_rng_uniform(n, 7, 3, 1, u1=u1, u2=u2, device=DEV)
    r1, r2 = v.vndf_rng_uniform(n, 7, 3, 1, device=DEV)
    _same(u1, r1)
    _same(u2, r2)
    ui = [G.make(n, off, u1), G.make(n, off, u2)]
    fu = [_fresh(t) for t in ui]
    wm_cap = None
    for method in ("cap", "polar", "cap_extended"):
        for explicit in (False, True):
            for iso in (False, True):
                outs = [G.make(n, off) for _ in range(4)]
                kw = dict(u1=ui[0], u2=ui[1]) if explicit else dict(seed=11, counter_base=5, stream_id=2)
                got = v.vndf_sample(*wi, ax, None if iso else ay, method=method, wm_x=outs[0], wm_y=outs[1],
                                    wm_z=outs[2], pdf=outs[3], **kw)
                fk = dict(u1=fu[0], u2=fu[1]) if explicit else kw
                ref = v.vndf_sample(*fwi, fax, None if iso else fay, method=method, **fk)
                for a, b in zip(got, ref):
                    _same(a, b)
                if method == "cap_extended" and not explicit and not iso:
                    wm_cap = [G.make(n, off, t) for t in got[:3]]
    # the density of given normals
    for ext in (False, True):
        p = G.make(n, off)
        v.vndf_pdf(*wi, ax, ay, *wm_cap, pdf=p, extended=ext)
        _same(p, v.vndf_pdf(*fwi, fax, fay, *[_fresh(t) for t in wm_cap], extended=ext))
    # reflection and the stand-alone hemisphere sampler
    for explicit in (False, True):
        kw = dict(u1=ui[0], u2=ui[1]) if explicit else dict(seed=12)
        fk = dict(u1=fu[0], u2=fu[1]) if explicit else kw
        outs = [G.make(n, off) for _ in range(5)]
        got = v.vndf_sample_reflection(*wi, ax, ay, f0=0.04, wo_x=outs[0], wo_y=outs[1], wo_z=outs[2], pdf=outs[3],
                                       weight=outs[4], **kw)
        for a, b in zip(got, v.vndf_sample_reflection(*fwi, fax, fay, f0=0.04, **fk)):
            _same(a, b)
        outs = [G.make(n, off) for _ in range(4)]
        got = v.vndf_sample_hemisphere(*wi, wm_x=outs[0], wm_y=outs[1], wm_z=outs[2], pdf=outs[3], **kw)
        for a, b in zip(got, v.vndf_sample_hemisphere(*fwi, **fk)):
            _same(a, b)
    G.check()


@pytest.mark.parametrize("off", OFFSETS)
@pytest.mark.parametrize("n", SIZES)
def test_adjoint_entry_points(v, n, off):
    G = Guards()
    d = workloads.adjoint_2e24(n=max(n, 1), seed=23, device=DEV)
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y", "c_x", "c_y", "c_z")
    g = {k: G.make(n, off, d[k]) for k in keys}
    f = {k: _fresh(t) for k, t in g.items()}
    gp = G.make(n, off, torch.linspace(-1.0, 1.0, max(n, 1), device=DEV))
    fgp = _fresh(gp)
    for ext in (False, True):
        for iso in (False, True):
            outs = [G.make(n, off) for _ in range(5)]
            got = v.vndf_sample_backward(g["wi_x"], g["wi_y"], g["wi_z"], g["alpha_x"], None if iso else g["alpha_y"],
                                         seed=4, counter_base=1, g_wm_x=g["c_x"], g_wm_y=g["c_y"], g_wm_z=g["c_z"],
                                         g_pdf=gp, extended=ext, outputs=outs)
            ref = v.vndf_sample_backward(f["wi_x"], f["wi_y"], f["wi_z"], f["alpha_x"], None if iso else f["alpha_y"],
                                         seed=4, counter_base=1, g_wm_x=f["c_x"], g_wm_y=f["c_y"], g_wm_z=f["c_z"],
                                         g_pdf=fgp, extended=ext)
            for a, b in zip(got, ref):
                _same(a, b)
    # fused loss: the partial sums depend only on n, so the loss matches bit for bit too
    ws = G.make(max(v.vndf_loss_workspace_bytes(n), 4), 0, dtype=torch.uint8, pad=256)
    outs = (G.make(1), *[G.make(n, off) for _ in range(5)])
    got = v.vndf_sample_loss_backward(*(g[k] for k in keys), seed=6, workspace=ws, outputs=outs)
    ref = v.vndf_sample_loss_backward(*(f[k] for k in keys), seed=6)
    for a, b in zip(got, ref):
        _same(a, b)
    G.check()


@pytest.mark.parametrize("off", OFFSETS)
@pytest.mark.parametrize("n", SIZES)
def test_batched_entry_points(v, n, off):
    G = Guards()
    # albedo: up to 1027 queries on the whole sphere (out-of-domain queries get NaN), ragged counts with zeros
    nq = min(n, 1027)
    d = workloads.sphere_stream(n=max(nq, 1), seed=29, device=DEV)
    counts = torch.as_tensor(np.random.default_rng(n + off).integers(0, 601, max(nq, 1)), dtype=torch.int32,
                             device=DEV)
    q = [G.make(nq, off, d[k]) for k in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")]
    cnt = G.make(nq, off, counts, dtype=torch.int32)
    E = G.make(nq, off)
    ws = G.make(max(v.vndf_albedo_workspace_bytes(nq, 600), 256), 0, dtype=torch.uint8, pad=256)
    v.vndf_albedo_batched(*q, cnt, max_samples_per_query=600, E=E, workspace=ws)
    _same(E, v.vndf_albedo_batched(*[_fresh(t) for t in q], _fresh(cnt), max_samples_per_query=600))
    # fitting: up to 1027 texels of a roughness map, two steps, state updated in place
    nt = min(n, 1027)
    m = workloads.roughness_map(res=33, seed=31, device=DEV)
    tex = [G.make(nt, off, m[k]) for k in ("wi_x", "wi_y", "wi_z", "target_x", "target_y", "target_z")]
    st = {k: G.make(nt, off, m[k], inout=True) for k in ("alpha_x", "alpha_y")}
    st.update({k: G.make(nt, off, torch.zeros(max(nt, 1), device=DEV), inout=True)
               for k in ("m_x", "m_y", "v_x", "v_y")})
    st["step"] = G.make(1, 0, torch.zeros(1, dtype=torch.int64, device=DEV), dtype=torch.int64, inout=True)
    ref_st = v.fit_state(m["alpha_x"][:nt].clone(), m["alpha_y"][:nt].clone())
    ftex = [_fresh(t) for t in tex]
    ws = G.make(max(v.vndf_fit_workspace_bytes(nt), 4), 0, dtype=torch.uint8, pad=256)
    # (with no texels the step writes nothing, so both losses start from the canary)
    loss, ref_loss = G.make(1), Guards._raw(1, torch.float32).view(torch.float32)
    for _ in range(2):
        v.vndf_fit_step(st, *tex, samples_per_texel=64, seed=5, loss=loss, workspace=ws)
        v.vndf_fit_step(ref_st, *ftex, samples_per_texel=64, seed=5, loss=ref_loss)
    _same(loss, ref_loss)
    for k in ("alpha_x", "alpha_y", "m_x", "m_y", "v_x", "v_y", "step"):
        _same(st[k], ref_st[k])
    # the paper-protocol kernel: one float4 per lane (16-byte aligned by contract)
    sums = G.make(4 * n, 0).view(n, 4)
    v.vndf_microbench(n, samples_per_lane=8, sums=sums, device=DEV)
    _same(sums, v.vndf_microbench(n, samples_per_lane=8, device=DEV))
    G.check()
