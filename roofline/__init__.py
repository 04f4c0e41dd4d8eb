"""Integer-issue roofline of the alignment kernels, measured on the current GPU.

The benchmark's measurement module (not part of the alignment library): it
builds ``roofline/_lib/libga_roofline.so`` from ``issue_rate.cu`` and runs
its probes.  The roofline follows the paper's theoretical-peak model
(Sec. 4.2, Eq. TPP, Table 2):

    cells/s <= SMs x clock x (lane-ops per clock per SM) / (ops per cell)

``measure()`` returns lane-ops per clock per SM for every single-operation
probe and for the two cell-update mixes (packed int16x2 and int32), each at
the SM clock nvidia-smi reports after the probe, and the peaks ``bench.py``
divides by:

* ``issue_peak_lane_ops``: the int16 issue peak of one SM, the measured
  rate of the packed add (FMA pipe) plus that of the packed max (ALU pipe):
  the paper's model counts every op of its 7 per cell against it;
* ``mix_ka_cells_per_clk_sm``: cells per clock per SM of the packed column
  update the inter-sequence kernel issues (6 ops, 2 cells).

    python -m roofline [--iters N]     prints one JSON line
"""
from __future__ import annotations

import ctypes
import json
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "issue_rate.cu")
HDR = os.path.join(HERE, "issue_rate.h")
LIB_PATH = os.path.join(HERE, "_lib", "libga_roofline.so")

PROBES = {"vadd2": 0, "vmaxs2": 1, "viaddmax_s16x2": 2, "vimax3_s16x2": 3,
          "viaddmax_s16x2_relu": 4, "prmt": 5, "iadd": 6, "imax": 7, "viaddmax_s32": 8,
          "vimax3_s32": 9, "imad": 10, "lop3": 11, "hadd2": 12, "hmax2": 13,
          "mix_ka": 14, "mix_s32": 15}
MIX_OPS = {"mix_ka": (6, 2), "mix_s32": (6, 1)}  # ops per column, cells per column

_lib = None


def build(force: bool = False) -> str:
    """nvcc the probes for sm_103a into the module's own shared library."""
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and \
            os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(SRC), os.path.getmtime(HDR)):
        return LIB_PATH
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", "-gencode", "arch=compute_103a,code=sm_103a",
           "-Xcompiler", "-fPIC", "-shared", "-cudart", "static", "-o", tmp, SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError(f"nvcc failed for issue_rate.cu:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.rl_issue_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_double)]
        lib.rl_issue_rate.restype = ctypes.c_int
        _lib = lib
    return _lib


def issue_rate(op: str, iters: int = 1024, blocks: int = 0, threads: int = 256):
    """(ms, lane_ops) of one timed launch of probe `op`."""
    if blocks <= 0:
        import torch
        blocks = 8 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    ms = ctypes.c_float(0)
    ops = ctypes.c_double(0)
    rc = load().rl_issue_rate(PROBES[op], int(iters), int(blocks), int(threads), ctypes.byref(ms),
                              ctypes.byref(ops))
    if rc:
        raise RuntimeError(f"rl_issue_rate({op}) failed: {rc}")
    return float(ms.value), float(ops.value)


def sm_clock_mhz() -> float | None:
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=10).stdout.strip()
        return float(out.splitlines()[0])
    except Exception:
        return None


def measure(iters: int = 1024, ops=None) -> dict:
    """Rates of the probes in `ops` (default: all) on the current device."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    nsm = props.multi_processor_count
    res = {}
    for name in (ops or PROBES):
        issue_rate(name, iters=max(1, iters // 8))  # clocks up before the timed launch
        ms, lane_ops = issue_rate(name, iters=iters)
        mhz = sm_clock_mhz() or 2070.0
        res[name] = {"ms": round(ms, 4), "sm_mhz": mhz,
                     "lane_ops_per_clk_per_sm": lane_ops / (ms * 1e-3) / (mhz * 1e6) / nsm}
    out = {"gpu": props.name, "sms": nsm, "probes": res}
    if "vadd2" in res and "vmaxs2" in res:
        out["issue_peak_lane_ops"] = (res["vadd2"]["lane_ops_per_clk_per_sm"] +
                                      res["vmaxs2"]["lane_ops_per_clk_per_sm"])
    for mix, (nops, cells) in MIX_OPS.items():
        if mix in res:
            out[f"{mix}_cells_per_clk_sm"] = res[mix]["lane_ops_per_clk_per_sm"] / nops * cells
    return out


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=1024)
    print(json.dumps(measure(ap.parse_args().iters)))
