#!/usr/bin/env python3
"""Throughput of spherical-cap GGX VNDF sampling on GB300 (one JSON line on rank 0).

Workload (the anisotropic streaming case): 2^28 samples per GPU per step,
float32 structure-of-arrays, alpha_x and alpha_y independently log-uniform in
[1e-3, 1], cos(theta_i) uniform in [1e-4, 1], phi_i uniform, uniforms drawn in
the kernel from Philox4x32-10 (seed 2).  A step is one vndf_sample call over
the whole batch (stretch, cap sample, half vector, unstretch, fused pdf,
store): 20 B read + 16 B written per sample, 9.66 GB per step, far larger than
L2, so no flush is needed between steps.  The same step is timed with the prior
polar-disk sampler for comparison.

Arms:
  default            the CUDA library (this repository)
  --impl reference   the FP64 CPU oracle timed on bounded samples of the same
                     workload (no GPU work)

Multi-GPU (torchrun): every rank samples its own 2^28 slice of one global index
range (weak scaling, no collective on the data path); the barrier and
max-over-ranks timing are the only communication.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VNDF Gsamples/s (fwd, fwd+bwd) vs prior-sampler kernel; % HBM/SFU roofline"
UNIT = "Gsamples/s"
WORKLOAD = "anisotropic_stream_2e28"
BYTES_PER_SAMPLE = 36  # in: wi xyz + alpha xy (20 B); out: wm xyz + pdf (16 B)
FALLBACK_HBM_GBS = 6800.0
CSRC = os.path.join(ROOT, "paper_2306_05044_gb300", "csrc")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "vndf_sample_cap_anisotropic_stream.md")
ISSUE_FILES = (os.path.join(ROOT, "profiles", "compute_kernels_issue.md"),
               os.path.join(ROOT, "profiles", "vndf_sample_extended_sphere_and_hemisphere_stream.md"))
LANES_PER_SM = 4 * 32  # 4 schedulers x 32 lanes issue one instruction each per clock


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--log2n", type=int, default=28, help="samples per GPU per step = 2^log2n")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-prior", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--no-fwd-bwd", action="store_true")
    p.add_argument("--no-albedo", action="store_true")
    p.add_argument("--no-fit", action="store_true")
    p.add_argument("--no-microbench", action="store_true")
    p.add_argument("--no-reflection", action="store_true")
    p.add_argument("--no-cpu-protocol", action="store_true")
    p.add_argument("--no-extended", action="store_true")
    p.add_argument("--no-isotropic", action="store_true")
    p.add_argument("--no-pdf", action="store_true")
    p.add_argument("--log2n-adjoint", type=int, nargs="+", default=[24, 26],
                   help="sizes of the fused forward+adjoint leg (2^k samples; the first is the workload's)")
    p.add_argument("--detail-out", default=None,
                   help="also write the full record (every leg with every field) to this file")
    p.add_argument("--config", type=int, choices=(1, 2, 3, 4, 5), default=None,
                   help="time the headline and only the legs of one workload: 1 isotropic 2^20, 2 anisotropic "
                        "stream (prior sampler, reflection, density, end to end), 3 albedo grid, 4 forward+adjoint, "
                        "5 roughness-map fitting")
    args = p.parse_args()
    if args.config is not None:
        keep = {1: {"isotropic"}, 2: {"prior", "reflection", "pdf", "e2e"}, 3: {"albedo"}, 4: {"fwd_bwd"},
                5: {"fit"}}[args.config]
        for leg in ("prior", "reflection", "pdf", "e2e", "isotropic", "albedo", "fwd_bwd", "fit", "extended",
                    "microbench", "cpu_protocol", "cpu_baseline"):
            if leg not in keep:
                setattr(args, "no_" + leg, True)
    return args


# ----------------------------------------------------------------------------- helpers
KERNEL_FILES = {
    "stream": ("sample.cu", "rescue.cuh", "staging.cuh", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
    "microbench_cap": ("microbench.cu", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
    "microbench_cap_strict": ("microbench.cu", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
    "microbench_polar": ("microbench.cu", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
    "loss_backward": ("backward.cu", "staging.cuh", "vndf_adjoint.cuh", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh",
                      "common.cuh"),
    "albedo": ("albedo.cu", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
    "fit": ("fit.cu", "vndf_adjoint.cuh", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
    "reflection": ("reflect.cu", "rescue.cuh", "staging.cuh", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh",
                   "common.cuh"),
    "hemisphere": ("hemisphere.cu", "rescue.cuh", "staging.cuh", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh",
                   "common.cuh"),
    "extended": ("sample.cu", "rescue.cuh", "staging.cuh", "vndf_math.cuh", "pair.cuh", "precise.cuh", "philox.cuh", "common.cuh"),
}


def kernel_source_hash(kernel):
    """Hash of the CUDA sources a kernel is built from: its profile figures are quoted only while it matches."""
    h = hashlib.sha256()
    for f in KERNEL_FILES[kernel]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_values(path, kernel):
    """`key: value` lines of a committed ncu summary for one kernel, or {} when its sources changed."""
    try:
        text = open(path).read()
    except OSError:
        return {}
    vals = {}
    for line in text.splitlines():
        line = line.strip().strip("-* ")
        if ":" in line:
            k, _, v = line.partition(":")
            vals[k.strip().strip("`")] = v.strip().strip("`")
    return vals if vals.get(f"kernel_source_sha.{kernel}") == kernel_source_hash(kernel) else {}


def measured_traffic_per_sample():
    """DRAM bytes per sample from the committed ncu summary, if it matches the current kernels."""
    try:
        return float(_profile_values(TRAFFIC_FILE, "stream")["dram_bytes_per_sample"])
    except (KeyError, ValueError):
        return None


def issue_roofline(kernel, samples, ms, clock):
    """ALU issue roofline of a compute-bound kernel: thread instructions per second against
    SMs x 4 schedulers x 32 lanes x SM clock, the clock being the median sampled during this
    kernel's own timed region (`clock`, the leg's clock record; the maximum clock when none was
    taken).  Instructions per sample come from the committed ncu summary (null when the kernel
    sources changed since)."""
    import torch
    clock_mhz = (clock or {}).get("sm_mhz")
    basis = "sampled" if clock_mhz else "maximum"
    clock_mhz = clock_mhz or max_sm_clock_mhz()
    try:
        vals = {}
        for path in ISSUE_FILES:
            vals.update(_profile_values(path, kernel))
        per = float(vals[f"tinst_per_sample.{kernel}"])
    except (KeyError, ValueError):
        return {"bound": "alu", "achieved": None, "peak": None, "frac": None, "unit": "Tinst/s",
                "note": "instruction count not measured for the current kernel sources"}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * LANES_PER_SM * clock_mhz * 1e6 / 1e12
    achieved = per * samples / (ms * 1e-3) / 1e12
    max_mhz = max_sm_clock_mhz()
    peak_max = sms * LANES_PER_SM * max_mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
            "thread_inst_per_sample": per, "peak_basis": f"{sms} SMs x 128 lanes x {clock_mhz:.0f} MHz ({basis})",
            "clock_mhz": clock_mhz, "reasons": (clock or {}).get("reasons"),
            "peak_at_max_clock": peak_max, "frac_at_max_clock": achieved / peak_max}


def max_sm_clock_mhz():
    """Maximum SM clock: the measured figure in MEASURED_PEAKS.json, else the GB300 nominal 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh).get("sm_max_mhz") or 2070.0)
    except (OSError, ValueError):
        return 2070.0


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """SM clock and clock-event reasons sampled every 5 ms during the timed region.

    Reads NVML through ctypes (libnvidia-ml ships with the driver); falls back to
    `nvidia-smi -lms 200` when NVML cannot be loaded.  Read-only: it changes no
    GPU setting.
    """
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import threading
        self.dev = torch_device
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self._smi = None
        self._nvml = self._open_nvml()

    def _open_nvml(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            handle = ctypes.c_void_p()
            bus = None
            try:
                import torch
                props = torch.cuda.get_device_properties(self.dev)
                bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
            except Exception:
                bus = None
            ok = bus is not None and lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(handle)) == 0
            if not ok and lib.nvmlDeviceGetHandleByIndex_v2(self.dev.index or 0, ctypes.byref(handle)) != 0:
                return None
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(handle, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            return lib, handle
        except OSError:
            return None

    def _poll(self):
        import ctypes
        lib, handle = self._nvml
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(handle, 1, ctypes.byref(clk)) == 0:
                r = rs.value if get_reasons(handle, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(clk.value), int(r)))
            self._stop.wait(0.005)

    def start(self):
        import threading
        if self._nvml is not None:
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
            return
        import tempfile
        fd, self._path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self._smi = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev.index or 0}", "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self._path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self._smi = None

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()
            if not self.samples:
                return None
            reasons = sorted({name for _, r in self.samples for bit, name in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.samples), "source": "nvml 5 ms"}
        if self._smi is None:
            return None
        self._smi.terminate()
        self._smi.wait(timeout=5)
        rows = [[x.strip() for x in line.split(",")] for line in open(self._path)]
        os.unlink(self._path)
        rows = [r for r in rows if len(r) >= 6 and r[0].replace(".", "").isdigit()]
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        return {"sm_mhz": statistics.median(float(r[0]) for r in rows),
                "sm_max_mhz": max(float(r[1]) for r in rows),
                "reasons": sorted({n for r in rows for n, v in zip(names, r[2:6]) if v.lower() == "active"}),
                "samples": len(rows), "source": "nvidia-smi 200 ms"}


def clock_rejected(clock):
    """True when the clock record of a timed region disqualifies it: a hardware or thermal slowdown was
    active, or the SM clock sat well below its maximum with no reason given (a leftover clock lock)."""
    if not clock:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    reasons = set(clock.get("reasons") or [])
    if reasons & bad:
        return True
    mhz, top = clock.get("sm_mhz"), clock.get("sm_max_mhz")
    return bool(mhz and top and mhz < 0.9 * top and not reasons)


def time_oracle_sample(n, seed=2, chunk=1 << 22):
    """Oracle (FP64 numpy) over the first n samples of the workload, timed in chunks; returns seconds."""
    import numpy as np
    import torch

    import workloads
    from oracle import philox, vndf
    torch.set_num_threads(1)
    d = workloads.anisotropic_stream(n=n, device="cpu")
    cols = {k: d[k].numpy() for k in ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")}
    del d
    total = 0.0
    for off in range(0, n, chunk):
        m = min(chunk, n - off)
        wi = np.stack([cols[k][off:off + m] for k in ("wi_x", "wi_y", "wi_z")])
        ax, ay = cols["alpha_x"][off:off + m], cols["alpha_y"][off:off + m]
        t0 = time.perf_counter()
        u1, u2 = philox.sample_uniforms(seed, off, 0, m)
        vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, "cap")
        total += time.perf_counter() - t0
    return total


def _oracle_chunk(job):
    """Pool worker: the oracle (Philox + cap sampler + pdf, FP64) over m samples of the workload recipe drawn
    with its own seed; returns (m, seconds spent in the oracle, worker pid)."""
    m, seed = job
    import numpy as np
    import torch

    import workloads
    from oracle import philox, vndf
    torch.set_num_threads(1)
    d = workloads.anisotropic_stream(n=m, seed=seed, device="cpu")
    wi = np.stack([d[k].numpy() for k in ("wi_x", "wi_y", "wi_z")])
    ax, ay = d["alpha_x"].numpy(), d["alpha_y"].numpy()
    t0 = time.perf_counter()
    u1, u2 = philox.sample_uniforms(2, 0, 0, m)
    vndf.sample_vndf_with_pdf(u1, u2, wi, ax, ay, "cap")
    return m, time.perf_counter() - t0, os.getpid()


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """A spawn-context process pool over all host cores for the oracle (never forked after CUDA starts).
    The pool is warmed before timing, so worker start-up is not counted."""

    def __init__(self, cores=None):
        import multiprocessing
        self.cores = cores or _host_cores()
        self.pool = multiprocessing.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_chunk, [(256, 1000 + k) for k in range(self.cores)])

    def run(self, m, chunks, seed0):
        """Seconds the pool spends in the oracle for `chunks` jobs of m samples: the largest per-process
        sum of oracle time (input generation, done in the workers before each timed region, excluded)."""
        per_pid = {}
        for _, secs, pid in self.pool.map(_oracle_chunk, [(m, seed0 + k) for k in range(chunks)], chunksize=1):
            per_pid[pid] = per_pid.get(pid, 0.0) + secs
        return max(per_pid.values())

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(budget_s=15.0):
    """The oracle on all host cores over a bounded sample of the workload recipe (about budget_s seconds)."""
    probe = 1 << 16
    t1 = time_oracle_sample(probe)  # one core, sizes the sample
    pool = OraclePool()
    try:
        m = 1 << 20
        chunks = max(pool.cores, int(budget_s * pool.cores * probe / max(t1, 1e-6) / m))
        chunks = (chunks + pool.cores - 1) // pool.cores * pool.cores
        wall = pool.run(m, chunks, 100)
    finally:
        pool.close()
    n = m * chunks
    return {"value": n / wall / 1e9, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{chunks} chunks of {m} samples of the anisotropic workload recipe (one seed per chunk), "
                      f"FP64 numpy oracle (Philox + cap sampler + pdf), one process per core, {wall:.1f} s of "
                      f"oracle time on the busiest core",
            "sample_short": f"{chunks}x2^20 workload samples, FP64 numpy oracle, {pool.cores} "
                            f"processes, {wall:.0f} s"}


def emit(obj):
    print(json.dumps(obj, separators=(",", ":")), flush=True)


def _sig(x, digits=4):
    """Floats rounded to `digits` significant digits, recursively (keeps the printed line short)."""
    if isinstance(x, bool) or x is None:
        return x
    if isinstance(x, float):
        return float(f"{x:.{digits}g}") if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: _sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_sig(v, digits) for v in x]
    return x


def _leg(d, hbm_key=None):
    """One leg in short form: Gsamples/s, ms per step, HBM and issue fractions, the leg's own median SM
    clock (MHz) and any clock-event reasons seen during its timed region."""
    if d is None:
        return None
    out = {"value": d.get("value"), "ms": d.get("ms_per_step", d.get("ms_per_launch"))}
    hbm = d.get(hbm_key) if hbm_key else d.get("roofline_frac", d.get("hbm_frac"))
    if isinstance(hbm, dict):
        hbm = hbm.get("frac")
    if hbm is not None:
        out["hbm"] = hbm
    issue = (d.get("issue") or {}).get("frac")
    if issue is not None:
        out["issue"] = issue
    clock = d.get("clock") or {}
    if clock.get("sm_mhz"):
        out["mhz"] = clock["sm_mhz"]
    if clock.get("reasons"):
        out["reasons"] = clock["reasons"]
    return out


def compact_line(r):
    """The printed JSON line: the contract's keys first, then every leg in short form (value, fractions,
    own clock), then the longer records.  The full record of every leg goes to stderr (and --detail-out)."""
    line = {k: r[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "gpu_launches")}
    rf = r["roofline"]
    line["roofline"] = {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    line["roofline"]["kernel"] = "sample_pipe_kernel<cap,philox,aniso,pdf>"
    if r.get("device"):
        line["device"] = r["device"]
    if r.get("rescued_frac") is not None:
        line["rescued"] = r["rescued_frac"]
    if "fwd_bwd" in r:
        line["fwd_bwd"] = {k: _leg(v, "hbm") for k, v in r["fwd_bwd"].items()}
    if "albedo" in r:
        line["albedo"] = dict(_leg(r["albedo"]), cfg=list(r["albedo"]["config"].values()))
    if "prior_sampler" in r:
        line["prior_sampler"] = dict(_leg(r["prior_sampler"]), cap_over_prior=r["prior_sampler"]["cap_over_prior"])
    if "extended" in r:
        line["extended"] = {k: _leg(v) for k, v in r["extended"].items()}
        if "rescued_frac" in r["extended"].get("sphere", {}):
            line["extended"]["sphere"]["rescued"] = r["extended"]["sphere"]["rescued_frac"]
    for k in ("reflection", "pdf", "isotropic", "fit"):
        if k in r:
            line[k] = _leg(r[k])
    if "backward_generic" in r:
        line["backward_generic"] = _leg(r["backward_generic"], "hbm")
    if "paper_protocol" in r:
        pp = r["paper_protocol"]
        line["paper_protocol"] = {k: _leg(pp[k]) for k in ("cap", "cap_strict", "polar")}
        line["paper_protocol"]["cap_over_prior"] = pp["cap_over_prior"]
    if "cpu_protocol" in r:
        cp = r["cpu_protocol"]
        line["cpu_protocol"] = {t: {"cap": cp[t]["cap"]["value"], "polar": cp[t]["polar"]["value"],
                                    "cap_over_prior": cp[t]["cap_over_prior"]}
                                for t in cp if t.startswith("threads_")}
    line["config"] = r["config"]
    line["clocks"] = {k: v for k, v in (r.get("clocks") or {}).items() if k != "remeasured_after"} or None
    if r.get("clocks") and r["clocks"].get("remeasured_after"):
        line["clocks"]["remeasured"] = True
    if "e2e" in r:
        e = r["e2e"]
        line["e2e"] = {k: e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "ms_per_step")}
        line["e2e"]["how"] = "zero_copy" if e.get("alternatives", {}).get("zero_copy") is not None and \
            e["value"] == e["alternatives"]["zero_copy"]["value"] else "copy_pipeline"
        line["e2e"]["alternatives"] = {k: (v or {}).get("value") for k, v in e.get("alternatives", {}).items()}
        if e.get("host_link"):
            hl = e["host_link"]
            line["e2e"]["host_link"] = {"achieved_gbs": hl["achieved_gbs"], "both_gbs": hl["both_gbs"],
                                        "frac": hl["frac"]}
    if "cpu_baseline" in r:
        cb = r["cpu_baseline"]
        line["cpu_baseline"] = dict(cb, sample=cb.get("sample_short", cb["sample"]))
        line["cpu_baseline"].pop("sample_short", None)
    line["detail"] = "stderr"
    return _sig(line)


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return
    steps, warm = max(args.steps, 1), max(args.warmup, 0)
    probe = 1 << 14
    t = time_oracle_sample(probe)
    pool = OraclePool()
    try:
        # each step: one chunk per core, sized so that the whole run takes about two minutes
        m = int(min(1 << 22, max(1 << 12, probe * (120.0 / (steps + warm)) / max(t, 1e-6))))
        m = 1 << int(math.log2(m))
        for w in range(warm):
            pool.run(m, pool.cores, 10_000 + w * pool.cores)
        times = [pool.run(m, pool.cores, 20_000 + k * pool.cores) for k in range(steps)]
    finally:
        pool.close()
    per_step = m * pool.cores
    total = sum(times)
    value = per_step * steps / total / 1e9
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
          "steps": steps, "warmup": warm, "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": WORKLOAD, "samples_per_step": per_step, "seed": 2,
                     "note": "bounded sample of the 2^28-sample workload per step"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                           "sample": f"{per_step} samples per step ({pool.cores} chunks of {m}, one seed each), "
                                     f"FP64 numpy oracle, one process per core"},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ----------------------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch

    import paper_2306_05044_gb300 as vndf
    import workloads
    from paper_2306_05044_gb300 import _build, sharding

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    vndf.load()
    base, n = sharding.sample_shard(rank, world, 1 << args.log2n)
    d = workloads.anisotropic_stream(n=n, device=dev)
    outs = [torch.empty(n, device=dev) for _ in range(4)]
    refl_w = None if args.no_reflection else torch.empty(n, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(method="cap"):
        vndf.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=2,
                         counter_base=base, method=method, wm_x=outs[0], wm_y=outs[1], wm_z=outs[2],
                         pdf=outs[3])

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    def timed(fn, steps, warmup, clocks=True, per_step=False):
        """Device time of `steps` calls of fn after `warmup` untimed ones: CUDA events before the first and
        after the last call, on the launching stream.  With per_step, an event after every call too (the
        per-step times); those events sit between the launches and cost a short step a few microseconds (the
        next launch no longer overlaps the one before), so the timed legs go without them."""
        for _ in range(warmup):
            fn()
        barrier()
        sampler = ClockSampler(dev) if clocks and not args.no_clocks else None
        if sampler:
            sampler.start()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1 if per_step else 2)]
        evs[0].record(stream)
        for k in range(steps):
            fn()
            if per_step:
                evs[k + 1].record(stream)
        if not per_step:
            evs[-1].record(stream)
        barrier()
        clock = sampler.stop() if sampler else None
        per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)] if per_step else []
        total = sharding.max_over_ranks(evs[0].elapsed_time(evs[-1]), dev)
        return total, per, clock

    steps, warm = max(args.steps, 1), max(args.warmup, 3)
    total, per, clock = timed(step, steps, warm)
    first_clock = None
    if clock_rejected(clock):  # throttled or clock-locked during the timed region: measure once more
        first_clock = clock
        total, per, clock = timed(step, steps, warm, clocks=True)
        if clock is not None:
            clock = dict(clock, remeasured_after=first_clock)
    value = world * n * steps / (total * 1e-3) / 1e9
    avg_ms = total / steps
    # share of the samples recomputed in double-float (untimed diagnostic, same arguments as the step)
    rescued = vndf.vndf_rescue_count(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=2,
                                     counter_base=base)
    rescued_frac = float(rescued.item()) / n

    peak, peak_kind = hbm_peak()
    achieved = BYTES_PER_SAMPLE * n / (avg_ms * 1e-3) / 1e9
    tps = measured_traffic_per_sample()
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "samples_per_gpu": n, "method": "spherical_cap", "rng": "philox4x32-10 in-kernel",
                   "alpha": "log-uniform [1e-3, 1] x, y independent", "cos_theta_i": "uniform [1e-4, 1]",
                   "l2": "inputs > L2 (9.66 GB per step), no flush",
                   "parallelism": f"index-range shards x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "traffic": (tps * n) if tps is not None else None,
                     "algorithmic_bytes": BYTES_PER_SAMPLE * n, "kernel": "sample_pipe_kernel<cap, philox, aniso, pdf>"},
        "gpu_launches": steps,
        "device": f"{torch.cuda.get_device_name(dev)}, "
                  f"{torch.cuda.get_device_properties(dev).multi_processor_count} SMs",
        "rescued_frac": rescued_frac,
        "clocks": clock,
    }
    # per-step spread from a separate pass with an event after every step (not part of the timed value)
    _, per, _ = timed(step, min(steps, 20), 1, clocks=False, per_step=True)
    result["per_step_ms"] = {"min": min(per), "median": statistics.median(per), "max": max(per),
                             "note": "separate pass with an event after every step"}

    if not args.no_prior:
        ptotal, pper, pclock = timed(lambda: step("polar"), steps, warm)
        pv = world * n * steps / (ptotal * 1e-3) / 1e9
        result["prior_sampler"] = {
            "value": pv, "unit": UNIT, "ms_per_step": ptotal / steps,
            "roofline_frac": BYTES_PER_SAMPLE * n / (ptotal / steps * 1e-3) / 1e9 / peak,
            "cap_over_prior": value / pv, "clock": pclock}
        result["gpu_launches_prior"] = steps

    if not args.no_reflection:
        rt, _, rclock = timed(lambda: vndf.vndf_sample_reflection(
            d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=2, counter_base=base, wo_x=outs[0],
            wo_y=outs[1], wo_z=outs[2], pdf=outs[3], weight=refl_w), steps, warm)
        rv = world * n * steps / (rt * 1e-3) / 1e9
        result["reflection"] = {"value": rv, "unit": UNIT, "ms_per_step": rt / steps,
                                "roofline_frac": 40 * n / (rt / steps * 1e-3) / 1e9 / peak,
                                "bytes_per_sample": 40, "note": "wo, pdf and F G2/G1 weight per sample (App. A)",
                                "issue": issue_roofline("reflection", n, rt / steps, rclock),
                                "clock": rclock}
        result["gpu_launches_reflection"] = steps

    if not args.no_extended:
        result["extended"] = extended_legs(vndf, dev, base, n, outs, timed, steps, warm, world, peak)
        result["gpu_launches_extended"] = 2 * steps

    if not args.no_pdf:
        pt, _, pdclock = timed(lambda: vndf.vndf_pdf(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"],
                                                     outs[0], outs[1], outs[2], pdf=outs[3]), steps, warm)
        result["pdf"] = {"value": world * n * steps / (pt * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": pt / steps,
                         "bytes_per_sample": 36, "roofline_frac": 36 * n / (pt / steps * 1e-3) / 1e9 / peak,
                         "note": "vndf_pdf at the headline's sampled normals (wi, alpha, wm in; pdf out)",
                         "clock": pdclock}
        result["gpu_launches_pdf"] = steps

    if not args.no_isotropic:
        result["isotropic"] = isotropic_leg(vndf, dev, rank, world, timed, peak)
        result["gpu_launches_isotropic"] = result["isotropic"]["launches"]

    if not args.no_fwd_bwd:
        result["fwd_bwd"] = {}
        for k in args.log2n_adjoint:
            leg = fwd_bwd(vndf, dev, rank, world, timed, peak, k)
            leg["issue"] = issue_roofline("loss_backward", 1 << k, leg["ms_per_step"], leg["clock"])
            result["fwd_bwd"][f"2e{k}"] = leg
            result[f"gpu_launches_fwd_bwd_2e{k}"] = 2 * leg["steps"]
        result["backward_generic"] = backward_generic(vndf, dev, rank, world, timed, peak, args.log2n_adjoint[0])
        result["gpu_launches_backward_generic"] = result["backward_generic"]["steps"]

    if not args.no_albedo:
        result["albedo"] = albedo(vndf, dev, rank, world, timed)
        result["albedo"]["issue"] = issue_roofline("albedo", result["albedo"]["samples"],
                                                   result["albedo"]["ms_per_step"], result["albedo"]["clock"])
        result["gpu_launches_albedo"] = 2 * result["albedo"]["steps"]

    if not args.no_microbench:
        result["paper_protocol"] = microbench(vndf, dev, world, timed)
        for m, k in (("cap", "microbench_cap"), ("cap_strict", "microbench_cap_strict"), ("polar", "microbench_polar")):
            leg = result["paper_protocol"][m]
            leg["issue"] = issue_roofline(k, result["paper_protocol"]["samples_per_step"], leg["ms_per_step"],
                                          leg["clock"])

    if not args.no_fit:
        result["fit"] = fit_leg(vndf, dev, rank, world, timed)
        result["fit"]["issue"] = issue_roofline("fit", result["fit"]["samples_per_step"],
                                                result["fit"]["ms_per_step"], result["fit"]["clock"])
        result["gpu_launches_fit"] = 2 * result["fit"]["steps"]

    if not args.no_e2e:
        piped = e2e(vndf, d, n, base, dev, stream, steps, warm, barrier, world)
        direct = e2e_zero_copy(vndf, d, n, base, dev, stream, steps, warm, barrier, world)
        best = max((x for x in (piped, direct) if x is not None), key=lambda x: x["value"])
        result["e2e"] = dict(best, alternatives={"copy_pipeline": piped, "zero_copy": direct})
        link = host_link(dev)
        moved = (best["h2d_bytes_per_step"] + best["d2h_bytes_per_step"]) / (best["ms_per_step"] * 1e-3) / 1e9
        result["e2e"]["host_link"] = dict(link, achieved_gbs=moved, frac=moved / link["both_gbs"])

    if rank == 0 and not args.no_cpu_protocol:
        result["cpu_protocol"] = cpu_protocol(vndf)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        detail = json.dumps(result)
        print(detail, file=sys.stderr, flush=True)
        if args.detail_out:
            with open(args.detail_out, "w") as fh:
                fh.write(detail + "\n")
        emit(compact_line(result))


def fwd_bwd(vndf, dev, rank, world, timed, peak, log2n):
    """Fused forward + loss + adjoint on the 2^24-sample adjoint workload (52 B/sample)."""
    import torch

    import workloads
    n = 1 << log2n
    d = workloads.adjoint_2e24(n=n, device=dev)
    outs = (torch.empty(1, device=dev), *(torch.empty(n, device=dev) for _ in range(5)))
    ws = torch.empty(max(vndf.vndf_loss_workspace_bytes(n), 4), dtype=torch.uint8, device=dev)

    def step():
        vndf.vndf_sample_loss_backward(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], d["c_x"],
                                       d["c_y"], d["c_z"], seed=4, counter_base=rank * n, workspace=ws,
                                       outputs=outs)

    steps = max(20, (500 << 24) >> log2n)  # about 70 ms of timed work, so the clock record has samples
    total, per, clock = timed(step, steps, 5)
    ms = total / steps
    del d
    return {"workload": f"adjoint_2e{log2n}", "value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "clock": clock,
            "hbm": {"algorithmic_bytes": 52 * n, "achieved_gbs": 52 * n / (ms * 1e-3) / 1e9,
                    "frac": 52 * n / (ms * 1e-3) / 1e9 / peak},
            "kernels": "loss_backward_pipe_kernel (+ loss_backward_kernel for a ragged last chunk) + sum_partials_kernel (programmatic dependent launch)"}


def backward_generic(vndf, dev, rank, world, timed, peak, log2n):
    """Generic adjoint (vndf_sample_backward) on the 2^24-sample adjoint workload: g_wm = c and a uniform
    g_pdf given, gradients of wi and both alphas returned (56 B/sample)."""
    import torch

    import workloads
    n = 1 << log2n
    d = workloads.adjoint_2e24(n=n, device=dev)
    gp = torch.rand(n, device=dev, generator=torch.Generator(device=dev).manual_seed(9))
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")

    def step():
        vndf.vndf_sample_backward(*(d[k] for k in keys), seed=4, counter_base=rank * n, g_wm_x=d["c_x"],
                                  g_wm_y=d["c_y"], g_wm_z=d["c_z"], g_pdf=gp)

    steps = max(20, (500 << 24) >> log2n)
    total, _, clock = timed(step, steps, 5)
    ms = total / steps
    del d
    return {"workload": f"adjoint_2e{log2n}", "value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "bytes_per_sample": 56, "clock": clock,
            "hbm": {"algorithmic_bytes": 56 * n, "achieved_gbs": 56 * n / (ms * 1e-3) / 1e9,
                    "frac": 56 * n / (ms * 1e-3) / 1e9 / peak},
            "kernels": "backward_pipe_kernel (vector path), backward_scalar_kernel for a ragged tail"}


def albedo(vndf, dev, rank, world, timed):
    """Batched directional albedo: 4096 ragged queries, one captured CUDA graph (prologue + persistent kernel)."""
    import torch

    import workloads
    g = workloads.albedo_grid(device=dev)
    nq = g["wi_x"].numel()
    total = int(g["n_samples"].sum().item())
    E = torch.empty(nq, device=dev)
    ws = torch.empty(vndf.vndf_albedo_workspace_bytes(nq, 65536), dtype=torch.uint8, device=dev)
    args = (g["wi_x"], g["wi_y"], g["wi_z"], g["alpha_x"], None, g["n_samples"])
    best, tuned_ms = vndf.vndf_albedo_autotune(*args, stream_id=rank * nq, E=E, workspace=ws)
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        vndf.vndf_albedo_batched(*args, stream_id=rank * nq, E=E, workspace=ws)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        vndf.vndf_albedo_batched(*args, stream_id=rank * nq, E=E, workspace=ws)
    steps = 500
    tot, per, clock = timed(graph.replay, steps, 5)
    ms = tot / steps
    return {"workload": "albedo_grid_4096", "queries": nq, "samples": total,
            "value": world * total / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "clock": clock,
            "config": {"warps_per_cta": best[0], "groups_per_item": best[1], "ctas_per_sm": best[2]},
            "captured": "cuda graph (prologue + persistent kernel)",
            "E_range": [float(E.min().item()), float(E.max().item())]}


def isotropic_leg(vndf, dev, rank, world, timed, peak):
    """2^20 isotropic samples with precomputed uniforms (Philox seed 1): 40 B/sample, 42 MB in all, so the
    working set stays in L2 and a single launch is short; timed as replays of a graph of 100 launches."""
    import torch

    import workloads
    n, reps, steps = 1 << 20, 100, 20
    d = workloads.isotropic_2e20(n=n, device=dev)
    u1, u2 = vndf.vndf_rng_uniform(n, 1, rank * n, 0, device=dev)
    outs = [torch.empty(n, device=dev) for _ in range(4)]

    def call():
        vndf.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], None, u1, u2, wm_x=outs[0], wm_y=outs[1],
                         wm_z=outs[2], pdf=outs[3])
    side = torch.cuda.Stream(dev)
    with torch.cuda.stream(side):
        call()
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        for _ in range(reps):
            call()
    tot, _, clock = timed(graph.replay, steps, 3)
    ms = tot / (steps * reps)
    return {"workload": "isotropic_2e20", "samples": n, "value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
            "ms_per_launch": ms, "launches": steps * reps, "bytes_per_sample": 40,
            "achieved_gbs": 40 * n / (ms * 1e-3) / 1e9, "hbm_frac": 40 * n / (ms * 1e-3) / 1e9 / peak,
            "note": "L2-resident (42 MB < 129 MB L2): the HBM fraction can exceed 1; launch-bound at this size",
            "captured": f"cuda graph of {reps} launches", "clock": clock}


def microbench(vndf, dev, world, timed):
    """The paper's GPU protocol: 64 samples per lane from register inputs, only sums written (ALU-bound)."""
    import torch
    lanes, spl = 1 << 22, 64
    sums = torch.empty(lanes, 4, device=dev)
    out = {"protocol": "64 samples per lane, inputs in registers, 16 B written per lane", "lanes": lanes,
           "samples_per_step": lanes * spl}
    for key, method, precise in (("cap", "cap", False), ("cap_strict", "cap", True), ("polar", "polar", False)):
        # the paper's protocol: median (and best) of 100 invocations, each timed on its own
        tot, per, clock = timed(lambda: vndf.vndf_microbench(lanes, spl, method, 1, sums=sums, precise=precise),
                                100, 3, per_step=True)
        ms = statistics.median(per)
        out[key] = {"value": world * lanes * spl / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
                    "ms_best": min(per), "ms_mean": tot / 100, "timing": "median of 100 invocations",
                    "clock": clock}
    out["cap"]["note"] = "plain FP32 cap sampler: the prior sampler's accuracy class (tails above 4e-6 rad ~1e-5)"
    out["cap_strict"]["note"] = "as vndf_sample: ill-conditioned samples redone in double-float, all within 4e-6 rad"
    out["cap_over_prior"] = out["cap"]["value"] / out["polar"]["value"]
    out["cap_strict_over_prior"] = out["cap_strict"]["value"] / out["polar"]["value"]
    out["paper_reference"] = "paper: cap faster by 52.96 % (Arc A770) and 39.25 % (RTX 2080), DX12 compute"
    return out


def extended_legs(vndf, dev, base, n, outs, timed, steps, warm, world, peak):
    """The extended domain (2^28 sphere workload, half below the horizon) and the stand-alone
    hemisphere sampler (2^28 directions of mixed length), HBM-resident, Philox in-kernel."""
    import torch

    import workloads
    res = {}
    d = workloads.sphere_stream(n=n, device=dev)
    t, _, clock = timed(lambda: vndf.vndf_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"],
                                                 seed=2, counter_base=base, method="cap_extended", wm_x=outs[0],
                                                 wm_y=outs[1], wm_z=outs[2], pdf=outs[3]), steps, warm)
    ms = t / steps
    rescued = vndf.vndf_rescue_count(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], seed=2,
                                     counter_base=base, method="cap_extended")
    res["sphere"] = {"workload": "sphere_stream_2e28", "value": world * n / (ms * 1e-3) / 1e9, "unit": UNIT,
                     "rescued_frac": float(rescued.item()) / n,
                     "ms_per_step": ms, "bytes_per_sample": BYTES_PER_SAMPLE,
                     "roofline_frac": BYTES_PER_SAMPLE * n / (ms * 1e-3) / 1e9 / peak,
                     "method": "spherical_cap_extended", "issue": issue_roofline("extended", n, ms, clock),
                     "clock": clock}
    del d
    h = workloads.hemisphere_stream(n=n, device=dev)
    t, _, clock = timed(lambda: vndf.vndf_sample_hemisphere(h["wi_x"], h["wi_y"], h["wi_z"], seed=2,
                                                            counter_base=base, wm_x=outs[0], wm_y=outs[1],
                                                            wm_z=outs[2], pdf=outs[3]), steps, warm)
    ms = t / steps
    res["hemisphere"] = {"workload": "hemisphere_stream_2e28", "value": world * n / (ms * 1e-3) / 1e9,
                         "unit": UNIT, "ms_per_step": ms, "bytes_per_sample": 28,
                         "roofline_frac": 28 * n / (ms * 1e-3) / 1e9 / peak,
                         "issue": issue_roofline("hemisphere", n, ms, clock), "clock": clock}
    del h
    torch.cuda.empty_cache()
    return res


def cpu_protocol(vndf, n=1 << 20, runs=100):
    """The paper's CPU protocol (Sec. 4): the sampler in a loop, median time of 100 invocations.

    Runs the library's host entry point (vndf_cpu_sample) over the first n samples of
    the anisotropic workload, normals only (as the paper's benchmark), on one thread
    and on all host threads, for both samplers, and for the cap sampler also with its
    double-precision recomputation of ill-conditioned samples (precise=1)."""
    import numpy as np
    import torch

    import workloads
    d = {k: t.numpy() for k, t in workloads.anisotropic_stream(n=n).items()}
    g = torch.Generator().manual_seed(7)
    u1, u2 = (t.numpy() for t in torch.rand(2, n, generator=g).unbind(0))
    outs = [np.empty(n, np.float32) for _ in range(3)]
    cores = os.cpu_count() or 1
    res = {"protocol": f"median of {runs} invocations over {n} samples, wm only, inputs in host memory",
           "samples": n}
    for threads in (1, cores):
        row = {}
        for label, method, precise in (("cap", "cap", False), ("cap_strict", "cap", True), ("polar", "polar", False)):
            def call():
                vndf.vndf_cpu_sample(d["wi_x"], d["wi_y"], d["wi_z"], d["alpha_x"], d["alpha_y"], u1, u2,
                                     method=method, with_pdf=False, threads=threads, out=outs, precise=precise)
            for _ in range(3):
                call()
            ts = []
            for _ in range(runs):
                t0 = time.perf_counter()
                call()
                ts.append(time.perf_counter() - t0)
            med = statistics.median(ts)
            row[label] = {"ms_median": 1e3 * med, "value": n / med / 1e9, "unit": UNIT}
        row["cap_over_prior"] = row["polar"]["ms_median"] / row["cap"]["ms_median"]
        row["cap_strict_over_prior"] = row["polar"]["ms_median"] / row["cap_strict"]["ms_median"]
        res[f"threads_{threads}"] = row
    res["paper_reference"] = "paper: cap faster by 37.67 % on an i7-13700K (C++ loop)"
    return res


def fit_leg(vndf, dev, rank, world, timed):
    """Roughness-map fitting: 256 x 256 texels x 1024 samples, forward + adjoint + Adam as one captured graph."""
    import torch

    import workloads
    d = workloads.roughness_map(device=dev)
    nt = d["alpha_x"].numel()
    st = vndf.fit_state(d["alpha_x"], d["alpha_y"])
    loss = torch.empty(1, device=dev)
    ws = torch.empty(vndf.vndf_fit_workspace_bytes(nt), dtype=torch.uint8, device=dev)
    args = (d["wi_x"], d["wi_y"], d["wi_z"], d["target_x"], d["target_y"], d["target_z"])
    side = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        vndf.vndf_fit_step(st, *args, seed=5, stream_id=rank * nt, loss=loss, workspace=ws)
    graph.replay()
    torch.cuda.synchronize(dev)
    first = float(loss.item())
    steps = 100
    tot, per, clock = timed(graph.replay, steps, 2)
    ms = tot / steps
    samples = nt * 1024
    return {"workload": "roughness_map_256x256", "texels": nt, "samples_per_step": samples,
            "value": world * samples / (ms * 1e-3) / 1e9, "unit": "Gsamples/s (fwd + adjoint per sample)",
            "ms_per_step": ms, "steps": steps, "captured": "cuda graph (fit kernel + loss/step kernel)",
            "loss_first": first, "loss_last": float(loss.item()), "steps_done": int(st["step"].item()),
            "clock": clock}


def e2e(vndf, d, n, base, dev, stream, steps, warm, barrier, world):
    """Same step through the public API with host buffers: H2D inputs, sample, D2H outputs.

    Chunks of 2^24 samples are pipelined over three streams so copies in both
    directions overlap the kernels; the timed region covers all of it.
    """
    import torch
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
    host_in = {k: d[k].cpu().pin_memory() for k in keys}
    host_out = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(4)]
    chunk = min(n, 1 << 24)
    nstreams = 3
    streams = [torch.cuda.Stream(dev) for _ in range(nstreams)]
    dev_in = [{k: torch.empty(chunk, device=dev) for k in keys} for _ in range(nstreams)]
    dev_out = [[torch.empty(chunk, device=dev) for _ in range(4)] for _ in range(nstreams)]
    start_ev = torch.cuda.Event()

    def one_step():
        start_ev.record(stream)
        done = []
        for c, off in enumerate(range(0, n, chunk)):
            m = min(chunk, n - off)
            s = streams[c % nstreams]
            s.wait_event(start_ev)
            with torch.cuda.stream(s):
                di, do = dev_in[c % nstreams], dev_out[c % nstreams]
                for k in keys:
                    di[k][:m].copy_(host_in[k][off:off + m], non_blocking=True)
                vndf.vndf_sample(di["wi_x"], di["wi_y"], di["wi_z"], di["alpha_x"], di["alpha_y"], seed=2,
                                 counter_base=base + off, wm_x=do[0], wm_y=do[1], wm_z=do[2], pdf=do[3], n=m,
                                 stream=s)
                for j in range(4):
                    host_out[j][off:off + m].copy_(do[j][:m], non_blocking=True)
        for s in streams:
            ev = torch.cuda.Event()
            ev.record(s)
            stream.wait_event(ev)

    for _ in range(warm):
        one_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one_step()
    e1.record(stream)
    barrier()
    from paper_2306_05044_gb300 import sharding
    total = sharding.max_over_ranks(e0.elapsed_time(e1), dev)
    return {"value": world * n * steps / (total * 1e-3) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": 20 * n, "d2h_bytes_per_step": 16 * n,
            "ms_per_step": total / steps, "pipeline": f"{nstreams} streams, {chunk}-sample chunks, pinned host memory"}


def host_link(dev, nbytes=1 << 28, reps=5):
    """Ceiling of the end-to-end step: the copy engines' host<->device bandwidth over the host link (pinned
    host memory), host-to-device alone, device-to-host alone and both directions at once (GB/s)."""
    import torch
    hb = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
    db = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def rate(fn, moved):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return moved * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9

    def h2d():
        db[0].copy_(hb[0], non_blocking=True)

    def d2h():
        hb[1].copy_(db[1], non_blocking=True)

    def both():
        cur = torch.cuda.current_stream(dev)
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            h2d()
        with torch.cuda.stream(s2):
            d2h()
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    return {"h2d_gbs": rate(h2d, nbytes), "d2h_gbs": rate(d2h, nbytes), "both_gbs": rate(both, 2 * nbytes),
            "how": f"copy engines, {nbytes >> 20} MiB pinned buffers, {reps} copies each"}


def e2e_zero_copy(vndf, d, n, base, dev, stream, steps, warm, barrier, world):
    """Same step with the kernel reading its inputs from, and writing its outputs to, pinned host memory
    directly (NVLink-C2C); no staging copies.  None when the device cannot address pinned host memory."""
    import torch

    from paper_2306_05044_gb300 import sharding
    keys = ("wi_x", "wi_y", "wi_z", "alpha_x", "alpha_y")
    host_in = {k: d[k].cpu().pin_memory() for k in keys}
    host_out = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(4)]
    if not all(vndf.vndf_pointer_device_accessible(t) for t in (*host_in.values(), *host_out)):
        return None

    def one_step():
        vndf.vndf_sample(host_in["wi_x"], host_in["wi_y"], host_in["wi_z"], host_in["alpha_x"], host_in["alpha_y"],
                         seed=2, counter_base=base, wm_x=host_out[0], wm_y=host_out[1], wm_z=host_out[2],
                         pdf=host_out[3], stream=stream)

    for _ in range(warm):
        one_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one_step()
    e1.record(stream)
    barrier()
    total = sharding.max_over_ranks(e0.elapsed_time(e1), dev)
    return {"value": world * n * steps / (total * 1e-3) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": 20 * n, "d2h_bytes_per_step": 16 * n, "ms_per_step": total / steps,
            "pipeline": "kernel reads and writes pinned host memory directly over NVLink-C2C (no staging copies)"}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
