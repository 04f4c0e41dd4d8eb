"""Integer-issue roofline of the DP kernels on the current GPU.

    python -m paper_2205_07610_gb300.roofline [--iters N]

Runs every issue-rate probe (include/gotoh_probe.h) and prints one JSON line:
lane-ops per clock per SM for each operation of the cell update, measured at
the SM clock sampled by nvidia-smi during the run, and the packed-column
probe (prmt + 5 DPX/SIMD ops) converted to an upper bound in GCUPS.  The
bound follows the paper's theoretical-peak model (Sec. 4.2, Eq. TPP):
cells/s <= SMs x clock x lane-ops-per-clock-per-SM / ops-per-cell.
"""
from __future__ import annotations

import argparse
import json
import subprocess

from . import _binding as b


def sm_clock_mhz() -> float | None:
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=10).stdout.strip()
        return float(out.splitlines()[0])
    except Exception:
        return None


def measure(iters: int = 1024) -> dict:
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nsm = props.multi_processor_count
    res = {}
    for name in b.PROBES:
        ms, ops = b.probe_issue_rate(name, iters=iters)
        mhz = sm_clock_mhz() or 2070.0
        per_clk_sm = ops / (ms * 1e-3) / (mhz * 1e6) / nsm
        res[name] = {"ms": ms, "lane_ops_per_clk_per_sm": per_clk_sm, "sm_mhz": mhz}
    cell = res["cell"]
    # the probe counts 6 lane-ops per packed column = 2 cells
    cells_per_clk_sm = cell["lane_ops_per_clk_per_sm"] / 6.0 * 2.0
    return {"gpu": props.name, "sms": nsm, "probes": res,
            "cell_probe_gcups_bound": cells_per_clk_sm * nsm * cell["sm_mhz"] * 1e6 / 1e9}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=1024)
    print(json.dumps(measure(ap.parse_args().iters)))
