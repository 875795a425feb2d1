"""vndf_rescue_count: the number of samples vndf_sample recomputes in double-float.

The count comes from the same per-sample function and condition test as the
sampler, so it must agree with the condition numbers the FP64 oracle gives for
the same samples (up to the few samples whose FP32 and FP64 condition numbers
fall on opposite sides of the threshold), be the same with Philox and with the
same uniforms given explicitly, be independent of the batch split, and be 0 for
the prior sampler and for empty batches.
"""
import numpy as np
import pytest
import torch

import parity
import workloads
from oracle import philox

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KAPPA = 24.0  # the threshold of the library's condition test


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


def _count(v, d, method="cap", **kw):
    c = v.vndf_rescue_count(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d.get("alpha_y"), method=method, **kw)
    torch.cuda.synchronize()
    return int(c.item())


def test_rescue_count_matches_the_oracle_condition_numbers(v):
    n = (1 << 20) + 3
    d = workloads.anisotropic_stream(n=n, seed=12, device=DEV)
    got = _count(v, d, seed=2, counter_base=5)
    u1, u2 = philox.sample_uniforms(2, 5, 0, n)
    wi = np.stack([d[k].cpu().numpy().astype(np.float64) for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = (d[k].cpu().numpy().astype(np.float64) for k in ("alpha_x", "alpha_y"))
    kap, kap_h = parity.conditioning(u1, u2, wi, ax, ay)
    want = int(np.sum((kap > KAPPA) | (kap_h > KAPPA)))
    near = int(np.sum((np.abs(kap / KAPPA - 1) < 1e-3) | (np.abs(kap_h / KAPPA - 1) < 1e-3)))
    print(f"flagged {got} of {n} (FP64 condition numbers: {want}; {near} within 0.1 % of the threshold)")
    assert want > 100
    assert abs(got - want) <= near + 2


def test_rescue_count_is_the_same_for_philox_explicit_u_and_splits(v):
    n = (1 << 20) + 5
    d = workloads.sphere_stream(n=n, seed=15, device=DEV)
    whole = _count(v, d, method="cap_extended", seed=3, counter_base=11)
    u1, u2 = v.vndf_rng_uniform(n, 3, 11, 0, device=DEV)
    explicit = _count(v, dict(d), method="cap_extended", u1=u1, u2=u2)
    m = 300001
    first = {k: t[:m].contiguous() for k, t in d.items()}
    rest = {k: t[m:].contiguous() for k, t in d.items()}
    split = _count(v, first, method="cap_extended", seed=3, counter_base=11) + \
        _count(v, rest, method="cap_extended", seed=3, counter_base=11 + m)
    print(f"extended, sphere workload: {whole} of {n} flagged ({whole / n:.2e})")
    assert whole == explicit == split
    assert whole > 0
    up = _count(v, d, method="cap", seed=3, counter_base=11)
    assert 0 < up < whole  # below the horizon the upper-domain method takes the fallback: nothing to flag


def test_rescue_count_edge_cases(v):
    d = workloads.anisotropic_stream(n=4096, seed=12, device=DEV)
    assert _count(v, d, method="polar", seed=1) == 0
    c = torch.full((1,), 12345, dtype=torch.int64, device=DEV)
    v.vndf_rescue_count(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], count=c, n=0)
    torch.cuda.synchronize()
    assert int(c.item()) == 0
    with pytest.raises(v.VndfError) as err:
        v.vndf_rescue_count(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], method=7)
    assert err.value.status == -4
