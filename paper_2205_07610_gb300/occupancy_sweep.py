"""Occupancy table of the inter-sequence kernel (maintenance tool).

    python -m paper_2205_07610_gb300.occupancy_sweep [--jobs N] [--max-spill BYTES]

Compiles every (cell type, mode, K) instantiation of ka_kernel for sm_103a at
each candidate __launch_bounds__ minimum-blocks value and prints, per
instantiation, the largest value at which ptxas allocates registers with at
most --max-spill bytes of spill stores (default 0), as the C++ initialisers of
KAMinBlocks in csrc/ga_inter.cuh.  The library takes the packed global and
semi-global rows from --max-spill 16 and every other row from the default
(which limit pays off was measured on GB300).  Run it after changing the
kernel; a CPU test checks the spill limits of the built library.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(HERE, "..", "include")
KS = [6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 24, 32]
MODES = {"local": "kModeLocal", "global": "kModeGlobal", "semi": "kModeSemi"}
CELLS = {"packed": "CellS16x2", "scalar": "CellS32"}
CANDIDATES = (1, 3, 4, 5, 6, 8)


def _compile(args):
    cell, mode, k, mb, nvcc = args
    d = tempfile.mkdtemp(prefix="occ_")
    try:
        for f in os.listdir(CSRC):
            if f.endswith((".cuh", ".h")):
                s = open(os.path.join(CSRC, f)).read()
                if f == "ga_inter.cuh":
                    s = s.replace("__launch_bounds__(128, KAMinBlocks<Cell, MODE, K>::value)",
                                  f"__launch_bounds__(128, {mb})")
                if f == "ga_common.cuh":
                    s = s.replace("../../include/gotoh_align.h",
                                  os.path.abspath(os.path.join(INCLUDE, "gotoh_align.h")))
                open(os.path.join(d, f), "w").write(s)
        src = os.path.join(d, "t.cu")
        open(src, "w").write(
            '#include "ga_launch.h"\nnamespace ga { void go(const KAParams &p) { '
            f"ka_kernel<{CELLS[cell]}, {MODES[mode]}, 16, {k}><<<1, 128>>>(p); }} }}\n")
        r = subprocess.run([nvcc, "-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                            "--expt-relaxed-constexpr", "-Xptxas", "-v", "-c", src, "-o",
                            os.path.join(d, "t.o")], capture_output=True, text=True)
        m = re.search(r"(\d+) bytes spill stores.*?Used (\d+) registers", r.stdout + r.stderr, re.S)
        return args[:4], (int(m.group(2)), int(m.group(1))) if m else None
    finally:
        shutil.rmtree(d, ignore_errors=True)


def sweep(jobs: int = 8, max_spill: int = 0) -> dict:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    work = [(c, m, k, mb, nvcc) for c in CELLS for m in MODES for k in KS for mb in CANDIDATES]
    res = {}
    with cf.ThreadPoolExecutor(jobs) as ex:
        for key, val in ex.map(_compile, work):
            res[key] = val
    table = {}
    for c in CELLS:
        for m in MODES:
            table[(c, m)] = [max([mb for mb in CANDIDATES
                                  if res[(c, m, k, mb)] and res[(c, m, k, mb)][1] <= max_spill] or [1])
                             for k in KS]
    return table


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 8)
    ap.add_argument("--max-spill", type=int, default=0, help="bytes of spill stores allowed")
    a = ap.parse_args()
    t = sweep(a.jobs, a.max_spill)
    for c in CELLS:
        rows = ",\n".join("{" + ", ".join(str(v) for v in t[(c, m)]) + "}" for m in MODES)
        print(f"k{c.capitalize()}[3][kKaNumBins] = {{{rows}}};")
