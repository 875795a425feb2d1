"""Host logic of bench.py that needs no GPU: the clock-record rule, the gating of profile
values on the kernels' source hashes, and the roofline denominators."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_rule():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clock_rejected(None)
    assert not bench.clock_rejected(ok)
    # a power cap during a long streaming step is normal and kept
    assert not bench.clock_rejected(dict(ok, sm_mhz=1900.0, reasons=["sw_power_cap"]))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clock_rejected(dict(ok, reasons=[r]))
    # clocks well below the maximum with no reason: a leftover lock
    assert bench.clock_rejected(dict(ok, sm_mhz=1400.0))
    assert not bench.clock_rejected(dict(ok, sm_mhz=1950.0))


def test_profile_values_follow_the_source_hash(tmp_path):
    kernel = "stream"
    h = bench.kernel_source_hash(kernel)
    good = tmp_path / "good.md"
    good.write_text(f"- dram_bytes_per_sample: 35.5\n- kernel_source_sha.{kernel}: `{h}`\n")
    stale = tmp_path / "stale.md"
    stale.write_text(f"- dram_bytes_per_sample: 35.5\n- kernel_source_sha.{kernel}: `0000000000000000`\n")
    assert bench._profile_values(str(good), kernel)["dram_bytes_per_sample"] == "35.5"
    assert bench._profile_values(str(stale), kernel) == {}
    assert bench._profile_values(str(tmp_path / "missing.md"), kernel) == {}


def test_hash_covers_every_listed_file():
    for kernel, files in bench.KERNEL_FILES.items():
        assert files, kernel
        for f in files:
            assert os.path.exists(os.path.join(ROOT, "paper_2306_05044_gb300", "csrc", f)), (kernel, f)


def test_roofline_denominators(monkeypatch, tmp_path):
    """The HBM peak and the maximum SM clock come from MEASURED_PEAKS.json, else the stated fallbacks."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
    assert bench.max_sm_clock_mhz() == 2070.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6787.6, "sm_max_mhz": 2032}')
    assert bench.hbm_peak() == (6787.6, "measured")
    assert bench.max_sm_clock_mhz() == 2032.0
