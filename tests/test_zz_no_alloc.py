"""The albedo entry point that allocates nothing, checked against the workspace one.

vndf_albedo_batched_noalloc serves callers that cannot allocate device memory
or hand over a workspace (a frame loop that must not stall on cudaMalloc, a
plugin that only receives pointers).  It keeps its scratch in a fixed device
array inside the library.  This file is named so that pytest collects it last.
It calls the entry point through the C ABI twice in a row (the second call
reuses the array the first one left behind) and compares each result with
vndf_albedo_batched bit for bit: both run the same kernels, and the albedo sums
run in an order fixed by the data, so any difference (a control word or
partial left over from the previous call) is a fault, however small.
"""
import ctypes

import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
VNDF_ERR_SIZE = -2


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2306_05044_gb300 as v
    return v


def _call_noalloc(v, g, nq, max_n, seed, E):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return v.load().vndf_albedo_batched_noalloc(
        nq, g["wi_x"].data_ptr(), g["wi_y"].data_ptr(), g["wi_z"].data_ptr(), g["alpha_x"].data_ptr(), None,
        g["n_samples"].data_ptr(), max_n, 0.04, seed, 0, 0, E.data_ptr(), None, stream)


def test_noalloc_matches_workspace_entry_point_twice(lib):
    g = workloads.albedo_grid(device=DEV)
    nq = g["wi_x"].numel()
    for seed in (3, 17):  # two calls in a row, with different streams of samples
        ref = lib.vndf_albedo_batched(g["wi_x"], g["wi_y"], g["wi_z"], g["alpha_x"], None, g["n_samples"],
                                      max_samples_per_query=65536, seed=seed)
        E = torch.full((nq,), float("nan"), device=DEV)  # a query never finished stays NaN
        assert _call_noalloc(lib, g, nq, 65536, seed, E) == 0
        torch.cuda.synchronize()
        assert torch.isfinite(ref).all()
        assert torch.equal(E, ref)


def test_noalloc_rejects_batches_larger_than_its_scratch(lib):
    g = workloads.albedo_grid(device=DEV)
    E = torch.empty(g["wi_x"].numel(), device=DEV)
    # 4096 queries of up to 2^20 samples need 64 MiB of scratch, more than the fixed 8 MiB
    assert _call_noalloc(lib, g, g["wi_x"].numel(), 1 << 20, 3, E) == VNDF_ERR_SIZE
