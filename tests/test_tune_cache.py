"""The albedo autotune cache of the Python binding (host logic, no GPU) and the C entry points that set and read
the tuned configuration (argument checks only)."""
import ctypes
import json

import pytest

import paper_2306_05044_gb300 as v


def test_cache_key_groups_batches_by_device_and_size_class():
    k = v.tune_cache_key("NVIDIA GB300", 152, 4096, 65536)
    assert k == "NVIDIA GB300|sm152|nq4096|max65536"
    assert v.tune_cache_key("NVIDIA GB300", 152, 3000, 65536) == k  # same power-of-two class
    assert v.tune_cache_key("NVIDIA GB300", 152, 4097, 65536) != k
    assert v.tune_cache_key("NVIDIA GB300", 148, 4096, 65536) != k
    assert v.tune_cache_key("NVIDIA GB300", 152, 4096, 1 << 20) != k
    assert v.tune_cache_key("x", 1, 1, 1) == v.tune_cache_key("x", 1, 0, 1)


def test_cache_store_and_lookup(tmp_path):
    path = str(tmp_path / "sub" / "albedo_tune.json")
    assert v.tune_cache_lookup(path, "a") is None  # no file yet
    v.tune_cache_store(path, "a", (16, 2, 4), 0.2041)
    v.tune_cache_store(path, "b", (8, 1, 8), 0.31)
    assert v.tune_cache_lookup(path, "a") == ((16, 2, 4), 0.2041)
    assert v.tune_cache_lookup(path, "b") == ((8, 1, 8), 0.31)
    assert v.tune_cache_lookup(path, "c") is None
    v.tune_cache_store(path, "a", (4, 4, 16), 0.25)  # replaced, the other key kept
    assert v.tune_cache_lookup(path, "a") == ((4, 4, 16), 0.25)
    assert json.load(open(path))["b"]["config"] == [8, 1, 8]


def test_cache_survives_a_damaged_file(tmp_path):
    path = tmp_path / "albedo_tune.json"
    path.write_text("{not json")
    assert v.tune_cache_lookup(str(path), "a") is None
    v.tune_cache_store(str(path), "a", (8, 2, 8), 0.2)
    assert v.tune_cache_lookup(str(path), "a") == ((8, 2, 8), 0.2)
    path.write_text("[1, 2]")
    assert v.tune_cache_lookup(str(path), "a") is None


@pytest.fixture(scope="module")
def lib():
    from paper_2306_05044_gb300 import _build
    _build.build()
    return v.load()


def test_config_entry_points_check_their_arguments(lib):
    for bad in ((0, 1, 8), (21, 1, 8), (8, 0, 8), (8, 257, 8), (8, 1, 0), (8, 1, 33)):
        assert lib.vndf_albedo_set_config((ctypes.c_int32 * 3)(*bad)) == -7
    assert lib.vndf_albedo_get_config(None) == -1


@pytest.mark.skipif(__import__("torch").cuda.is_available(), reason="checks the behaviour without a device")
def test_config_entry_points_without_a_device(lib):
    assert lib.vndf_albedo_set_config((ctypes.c_int32 * 3)(8, 1, 8)) == -6
    assert lib.vndf_albedo_set_config(None) == -6
    assert lib.vndf_albedo_get_config((ctypes.c_int32 * 3)()) == -6
