"""The paper's 64-samples-per-lane protocol kernel against the FP64 oracle.

The lane inputs are drawn in the kernel from Philox (see vndf_microbench in
include/vndf.h); this test re-derives them from the oracle's Philox words in
FP64.  The kernel rounds them to FP32 first, so sums are compared at 1e-4.
"""
import numpy as np
import pytest
import torch

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


def _lane_inputs(seed, lanes):
    ctr = np.stack([lanes.astype(np.uint32), (lanes >> 32).astype(np.uint32),
                    np.full(lanes.size, 0xFFFFFFFF, np.uint32), np.zeros(lanes.size, np.uint32)])
    w = philox.philox4x32_10(ctr, philox.seed_key(seed))
    v0, v1, v2, v3 = (philox.word_to_unit(w[k]) for k in range(4))
    ct = 1e-4 + (1 - 1e-4) * v0
    st = np.sqrt(1 - ct * ct)
    wi = np.stack([st * np.cos(2 * np.pi * v1), st * np.sin(2 * np.pi * v1), ct])
    return wi, 1e-3 ** (1 - v2), 1e-3 ** (1 - v3)


@pytest.mark.parametrize("method,precise", [("cap", True), ("cap", False), ("polar", False)])
def test_microbench_sums_match_oracle(v, method, precise):
    lanes, spl, seed = 4096, 64, 17
    sums = v.vndf_microbench(lanes, spl, method, seed, precise=precise).cpu().numpy().astype(np.float64)
    check = np.arange(0, lanes, 37, dtype=np.int64)
    wi, ax, ay = _lane_inputs(seed, check)
    g = (check[:, None] * spl + np.arange(spl)[None, :]).reshape(-1)
    u1, u2 = philox.uniforms_at(seed, 0, 0, g)
    rep = lambda x: np.repeat(x, spl, axis=-1)  # noqa: E731
    wm, pdf = ovndf.sample_vndf_with_pdf(u1, u2, rep(wi), rep(ax), rep(ay), method)
    ref = np.concatenate([wm, pdf[None]]).reshape(4, check.size, spl).sum(axis=2).T
    got = sums[check]
    np.testing.assert_allclose(got[:, :3], ref[:, :3], rtol=1e-4, atol=1e-3)
    rel = np.abs(got[:, 3] / ref[:, 3] - 1)
    print(method, "pdf-sum rel: median", np.median(rel), "max", rel.max())
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.95) < 1e-4
