"""The packed-pair path against the one-sample path, bit for bit, at scale.

The streaming kernels compute a thread's four samples as two packed FP32x2
pairs (fma / mul / add / sub on a float2 in one instruction); the one-sample
kernels, which serve ragged tails and arrays that do not start on a 16-byte
boundary, evaluate the same formulas one lane per instruction.  Each lane of a
packed instruction rounds as the scalar instruction does and nothing is left
for the compiler to contract, so both must give the same bits.  A call whose
arrays start 4 bytes past a 16-byte boundary runs entirely on the one-sample
kernel; the same call on aligned arrays runs on the pair kernel.  The inputs
are the stress workload (wi anywhere on the sphere with lengths 1e-3 to 1e3,
roughness 1e-5 to 10 per axis, uniforms at the ends of [0, 1)) and the sphere
workload, so that both rounding-sensitive regimes and the double-float
recomputation are crossed.
"""
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KEYS = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
N = (1 << 18) + 3


@pytest.fixture(scope="module")
def v():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as lib
    return lib


def _offset(t):
    """The same values in an array that starts 4 bytes past a 16-byte boundary."""
    raw = torch.empty(t.numel() + 4, dtype=t.dtype, device=t.device)
    raw[1:1 + t.numel()] = t
    return raw[1:1 + t.numel()]


def _same_bits(a, b, what):
    assert a.dtype == b.dtype
    diff = (a.view(torch.int32) != b.view(torch.int32)).nonzero().flatten()
    assert diff.numel() == 0, f"{what}: {diff.numel()} samples differ, first at {int(diff[0])}"


@pytest.fixture(scope="module", params=["wide", "sphere"])
def inputs(request):
    if request.param == "wide":
        d = workloads.wide_stream(n=N, seed=29, device=DEV)
    else:
        d = workloads.sphere_stream(n=N, seed=31, device=DEV)
        u1, u2 = torch.rand(2, N, generator=torch.Generator(device=DEV).manual_seed(7), device=DEV)
        d["u1"], d["u2"] = (torch.floor(u1 * 2 ** 24) * 2.0 ** -24), (torch.floor(u2 * 2 ** 24) * 2.0 ** -24)
    return request.param, d


@pytest.mark.parametrize("method", ["cap", "polar", "cap_extended"])
@pytest.mark.parametrize("explicit", [False, True])
def test_sampler_pairs_equal_single_samples(v, inputs, method, explicit):
    name, d = inputs
    kw = dict(u1=d["u1"], u2=d["u2"]) if explicit else dict(seed=3, counter_base=11, stream_id=5)
    okw = dict(u1=_offset(d["u1"]), u2=_offset(d["u2"])) if explicit else kw
    a = v.vndf_sample(*(d[k] for k in KEYS), method=method, **kw)
    b = v.vndf_sample(*(_offset(d[k]) for k in KEYS), method=method, **okw)
    for x, y, what in zip(a, b, ("wm_x", "wm_y", "wm_z", "pdf")):
        _same_bits(x, y, f"{name} {method} {what}")


@pytest.mark.parametrize("explicit", [False, True])
def test_reflection_and_hemisphere_pairs_equal_single_samples(v, inputs, explicit):
    name, d = inputs
    kw = dict(u1=d["u1"], u2=d["u2"]) if explicit else dict(seed=8)
    okw = dict(u1=_offset(d["u1"]), u2=_offset(d["u2"])) if explicit else kw
    a = v.vndf_sample_reflection(*(d[k] for k in KEYS), f0=0.04, **kw)
    b = v.vndf_sample_reflection(*(_offset(d[k]) for k in KEYS), f0=0.04, **okw)
    for x, y, what in zip(a, b, ("wo_x", "wo_y", "wo_z", "pdf", "weight")):
        _same_bits(x, y, f"{name} reflection {what}")
    a = v.vndf_sample_hemisphere(d["wi_x"], d["wi_y"], d["wi_z"], **kw)
    b = v.vndf_sample_hemisphere(*(_offset(d[k]) for k in ("wi_x", "wi_y", "wi_z")), **okw)
    for x, y, what in zip(a, b, ("wm_x", "wm_y", "wm_z", "pdf")):
        _same_bits(x, y, f"{name} hemisphere {what}")


def test_rescue_is_crossed(v, inputs):
    """The inputs reach the double-float recomputation, so its interplay with the pairs is exercised."""
    name, d = inputs
    count = v.vndf_rescue_count(*(d[k] for k in KEYS), seed=3, counter_base=11, stream_id=5, method="cap_extended")
    assert int(count.item()) > 0, name
