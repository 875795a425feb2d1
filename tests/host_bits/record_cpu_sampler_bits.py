"""Writes cpu_sampler_x86_64.txt: digests of vndf_cpu_sample's outputs on the fixed inputs of
tests/cpu_bits.py, from an x86-64 build of the library.

This is a record of one ISA's bits, not an expected value of the method: parity of the host
sampler is checked against the FP64 oracle (tests/test_cpu_sampler.py).  The record lets a run
on another ISA (the AArch64 host of the GPU) check that the same source gives the same bits.
Rewrite it whenever the host sampler's arithmetic changes.

Run from the repository root on an x86-64 host:  python tests/host_bits/record_cpu_sampler_bits.py
"""
import os
import platform
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)

import cpu_bits  # noqa: E402
from paper_2306_05044_gb300 import _build  # noqa: E402


def main():
    if platform.machine() not in ("x86_64", "AMD64"):
        raise SystemExit("the record holds the x86-64 build's bits: run this on an x86-64 host")
    _build.build()
    import paper_2306_05044_gb300 as vndf
    vndf.load()
    d = cpu_bits.current(vndf)
    with open(cpu_bits.RECORD, "w") as fh:
        fh.write("# sha256 of vndf_cpu_sample outputs (wm_x, wm_y, wm_z, pdf as little-endian float32) on the\n")
        fh.write(f"# inputs of tests/cpu_bits.py ({cpu_bits.N} samples), precise = 0, x86-64 build\n")
        for k, h in d.items():
            fh.write(f"{k} {h}\n")
    print(open(cpu_bits.RECORD).read())


if __name__ == "__main__":
    main()
