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


def _full_record():
    """A record with every leg bench.py times, with full-precision floats, shaped as run_ours builds it."""
    x = 1.0 / 3.0
    clock = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 28, "source": "nvml 5 ms"}
    issue = {"bound": "alu", "achieved": 28.4 + x, "peak": 40.27 + x, "frac": 0.7 + x / 10}
    leg = lambda **kw: dict({"value": 100 + x, "ms_per_step": 1 + x, "roofline_frac": 0.9 + x / 10,  # noqa: E731
                             "issue": issue, "clock": clock}, **kw)
    fb = lambda: dict(leg(), hbm={"frac": 0.89 + x / 100}, steps=500)  # noqa: E731
    r = {k: v for k, v in zip(("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                               "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "gpu_launches"),
                              (bench.METRIC, 185.7 + x, "Gsamples/s", 1, 20, 5, 1.44 + x, True, "weak", None, "f32",
                               "synthetic", 20))}
    r["roofline"] = {"bound": "hbm", "achieved": 6688 + x, "peak": 6792.1, "unit": "GB/s", "frac": 0.98 + x / 100,
                     "traffic": 9532143042.56, "peak_kind": "measured copy bandwidth", "algorithmic_bytes": 1}
    r["config"] = {"workload": bench.WORKLOAD, "samples_per_gpu": 1 << 28, "method": "spherical_cap",
                   "rng": "philox4x32-10 in-kernel", "alpha": "log-uniform [1e-3, 1] x, y independent",
                   "cos_theta_i": "uniform [1e-4, 1]",
                   "l2": "inputs > L2 (9.66 GB per step), no flush",
                   "parallelism": "index-range shards x1"}
    r["clocks"] = clock
    r["fwd_bwd"] = {"2e24": fb(), "2e26": fb()}
    r["backward_generic"] = fb()
    r["albedo"] = dict(leg(), config={"warps_per_cta": 16, "groups_per_item": 2, "ctas_per_sm": 4})
    r["prior_sampler"] = dict(leg(), cap_over_prior=1.06 + x)
    r["extended"] = {"sphere": dict(leg(), rescued_frac=4.5e-3 + x / 1e4), "hemisphere": leg()}
    r["rescued_frac"] = 7e-4 + x / 1e5
    r["device"] = "NVIDIA GB300, 152 SMs"
    for k in ("reflection", "pdf", "isotropic", "fit"):
        r[k] = leg()
    r["paper_protocol"] = {"cap": leg(), "cap_strict": leg(), "polar": leg(), "cap_over_prior": 1.33 + x}
    row = {"cap": {"value": 0.2 + x}, "cap_strict": {"value": 0.2 + x}, "polar": {"value": 0.14 + x},
           "cap_over_prior": 1.5 + x}
    r["cpu_protocol"] = {"threads_1": row, "threads_16": row, "paper_reference": "p"}
    e = {"value": 9.3 + x, "unit": "Gsamples/s", "h2d_bytes_per_step": 20 << 28, "d2h_bytes_per_step": 16 << 28,
         "ms_per_step": 28.9 + x, "pipeline": "zero copy"}
    r["e2e"] = dict(e, alternatives={"copy_pipeline": dict(e, value=7.4 + x), "zero_copy": e},
                    host_link={"h2d_gbs": 210.9 + x, "d2h_gbs": 193.2 + x, "both_gbs": 339.3 + x,
                               "how": "copy engines", "achieved_gbs": 332.3 + x, "frac": 0.979 + x / 100})
    r["cpu_baseline"] = {"value": 0.0497 + x / 1000, "unit": "Gsamples/s", "cores": 16, "kind": "oracle",
                         "sample": "x" * 300, "sample_short": "1424x2^20 samples, FP64 numpy oracle, 16 processes"}
    return r


def test_printed_line_is_short_and_complete():
    """The printed line must fit in the few KB of stdout a driver keeps: every leg in short form (value,
    fractions, own clock), the long records only on stderr."""
    import json
    line = bench.compact_line(_full_record())
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < 2700, len(text)
    keys = list(line)
    assert keys[:13] == ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                         "scaling", "vs_baseline", "dtype", "data", "gpu_launches"]
    for k in ("roofline", "fwd_bwd", "albedo", "prior_sampler", "extended", "config", "clocks", "e2e",
              "cpu_baseline"):
        assert k in line, k
    assert set(line["fwd_bwd"]) == {"2e24", "2e26"}
    assert set(line["e2e"]["host_link"]) == {"achieved_gbs", "both_gbs", "frac"}
    for leg in (line["fwd_bwd"]["2e24"], line["albedo"], line["extended"]["sphere"]):
        assert leg["issue"] is not None and leg["mhz"] == 2070.0
    assert line["fwd_bwd"]["2e26"]["hbm"] is not None
    assert line["rescued"] > 0 and line["extended"]["sphere"]["rescued"] > 0
    assert line["e2e"]["how"] == "zero_copy" and line["e2e"]["h2d_bytes_per_step"] == 20 << 28
    assert line["cpu_baseline"]["sample"].startswith("1424x2^20")


def test_config_option_keeps_only_that_workloads_legs(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--config", "4"])
    a = bench.parse_args()
    assert not a.no_fwd_bwd
    assert a.no_albedo and a.no_fit and a.no_prior and a.no_e2e and a.no_cpu_baseline and a.no_extended
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse_args()
    assert not (a.no_fwd_bwd or a.no_albedo or a.no_fit or a.no_prior or a.no_e2e or a.no_cpu_baseline)


def test_committed_profiles_match_the_current_sources():
    """Every kernel the bench quotes ncu figures for has a summary taken from its current sources: a source
    change without a new capture would silently drop `roofline.traffic` and the issue fractions."""
    assert bench.measured_traffic_per_sample() is not None
    for kernel in bench.KERNEL_FILES:
        if kernel == "stream":
            continue
        vals = {}
        for path in bench.ISSUE_FILES:
            vals.update(bench._profile_values(path, kernel))
        assert f"tinst_per_sample.{kernel}" in vals, kernel
