#!/usr/bin/env python
"""Benchmark of the score-only Gotoh alignment hot path on GB300.

Workload (one "step"): 1M DNA pairs, |Q| ~ U{100..300}, S = Q with 5 %
substitutions and 1 % indels (geometric length, mean 2), scored in global AND
semi-global mode (+2/-3, gap open 5, extend 2) through ga_align_batch_modes.  The
metric is GCUPS: full-DP cells (sum of m*n, both modes) per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The line also carries "serve": p50/p99 latency and GCUPS of a Poisson stream
of 200k mixed requests through the alignment server (--no-serve skips it),
"band": the learned-band vs full-DP time to exact global
scores on 20k long DNA pairs (|Q| ~ U{1000..20000}, divergence 1-15 %), with
the band predictor trained first on its own seeded pairs (--no-band skips it),
"protein": GCUPS of 512 protein queries against a 200k-target database in
local mode with BLOSUM62 (--no-protein skips it), and "plan": preallocated
batch plans and their CUDA-graph replays against eager calls, on 1,000
150 x 150 pairs and on the 1M-pair step with autotuned bins (--no-plan).

Multi-GPU (torchrun, one process per GPU): every rank aligns its own seeded
batch of the same shape (weak scaling, no data-path collective); the step time
is the max over ranks and `value` counts the cells of all ranks.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# int16 operations per cell in the paper's count for global / semi-global
# affine alignment (Sec. 4.2: 4 max + 3 add/sub); local adds 2.
OPS_PER_CELL = 7
# ALU-pipe operations per packed column (two cells) that the kernels issue:
# ka_kernel prmt + vimax3 + 2 viaddmax; kp_kernel vimax3_relu + 2 viaddmax
# + half a vimax3 (running maximum).  The FMA-pipe adds run beside them.
KA_ALU_OPS_PER_COLUMN = 4.0
KP_ALU_OPS_PER_COLUMN = 3.5
# DRAM bytes (read + write) of one launch of the dominant DP kernel,
# ka_kernel<CellS16x2, semi, 16, 18> (pairs of 273..288 columns), on this
# batch: one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of
# the current kernel code and bins.
KA_TRAFFIC_BYTES = 48514304 + 5376
SIMD = 2                 # int16x2: two cells per lane-op
FALLBACK_SM_MHZ = 2070.0  # GB300 maximum SM clock, used only if no measured value is available
PROBE_OPS = ("vadd2", "vmaxs2", "vimax3_s16x2", "mix_ka")


def device_peak(dev, clocks=None):
    """(SM count, maximum SM clock in MHz, source) of the device: the SM count
    from the device properties, the clock from the nvidia-smi samples of the
    run, else MEASURED_PEAKS.json, else the GB300 figure."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz, src = None, None
    if clocks and clocks.get("sm_max_mhz"):
        mhz, src = float(clocks["sm_max_mhz"]), "nvidia-smi clocks.max.sm"
    if mhz is None:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        except (OSError, KeyError, ValueError):
            pass
    if mhz is None:
        mhz, src = FALLBACK_SM_MHZ, "GB300 nominal maximum"
    return n_sm, mhz, src


def measured_peaks(rates: dict, n_sm: int, mhz: float) -> dict:
    """Issue peaks of this GPU from the probes run at the start of the bench
    (roofline.measure: lane-ops per clock per SM), scaled to `mhz`.

    issue_ops   int16 lane-ops/s the SMs can issue: the packed add's rate (FMA
                pipe) plus the packed max's (ALU pipe), x2 for int16x2; the
                paper's model (Sec. 4.2) divides its 7 ops per cell by this;
    *_alu_gcups the ALU-pipe ceiling of a kernel's own op mix: the measured
                3-way max rate (ALU pipe) over the kernel's ALU ops per cell;
    ka_mix_gcups the measured rate of ka_kernel's whole packed column update
                (6 ops on two pipes, probe mix_ka), a cross-check.
    """
    clk = n_sm * mhz * 1e6
    r = {k: v["lane_ops_per_clk_per_sm"] for k, v in rates["probes"].items()}
    issue = r["vadd2"] + r["vmaxs2"]
    return {
        "issue_lane_ops_per_clk_sm": issue,
        "issue_ops": issue * clk * SIMD,
        "ka_alu_gcups": r["vimax3_s16x2"] * clk * 2 / KA_ALU_OPS_PER_COLUMN / 1e9,
        "kp_alu_gcups": r["vimax3_s16x2"] * clk * 2 / KP_ALU_OPS_PER_COLUMN / 1e9,
        "ka_mix_gcups": rates["mix_ka_cells_per_clk_sm"] * clk / 1e9,
        "basis": f"{n_sm} SM x {mhz:.0f} MHz x measured lane-ops/clk/SM: vadd2 {r['vadd2']:.1f} + "
                 f"vmaxs2 {r['vmaxs2']:.1f} (issue), vimax3 {r['vimax3_s16x2']:.1f} (ALU), "
                 f"ka column mix {rates['mix_ka_cells_per_clk_sm']:.1f} cells",
    }


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--npairs", type=int, default=1_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the bounded oracle sample")
    ap.add_argument("--no-band", action="store_true", help="skip the learned-band measurement")
    ap.add_argument("--band-pairs", type=int, default=20_000)
    ap.add_argument("--band-train", type=int, default=4_000)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-protein", action="store_true", help="skip the protein database search")
    ap.add_argument("--no-plan", action="store_true", help="skip the batch-plan / graph measurement")
    ap.add_argument("--protein-queries", type=int, default=512)
    ap.add_argument("--protein-targets", type=int, default=200_000)
    ap.add_argument("--protein-qmin", type=int, default=100, help="shortest protein query")
    ap.add_argument("--protein-qmax", type=int, default=1000, help="longest protein query")
    ap.add_argument("--serve-requests", type=int, default=200_000)
    ap.add_argument("--probe-iters", type=int, default=128,
                    help="outer iterations of each issue-rate probe (about 0.1 s each)")
    ap.add_argument("--detail", default=None,
                    help="also write every section's full record to this JSON file")
    return ap.parse_args()


def workload(npairs: int, rank: int):
    """Each rank aligns its own seeded batch of the same shape (weak scaling)."""
    return synth.mutated_dna_pairs(npairs=npairs, seed=shard_seed(rank))


def shard_seed(rank: int) -> int:
    return synth.SEED_BASE + 2 + 1000 * rank


def reduce_max(value: float, dist=None, device=None) -> float:
    """Max over ranks (a step lasts as long as its slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gcups(cells_per_rank_step: int, world: int, steps: int, max_ms: float) -> float:
    """Cells of all ranks over the slowest rank's time, in GCUPS."""
    return cells_per_rank_step * world * steps / (max_ms / 1e3) / 1e9


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.t0 = None
        self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        import datetime
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
                rows.append((ts, parts[1:]))
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        inside = [r for ts, r in rows
                  if ts is not None and self.t0 is not None and self.t0 - 0.25 <= ts <= self.t1 + 0.25]
        used = inside if inside else [r for _, r in rows]
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no-samples"], "samples": 0}
        sm = [float(r[1]) for r in used if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in used if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in used if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in used for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "power_w_max": max(pw) if pw else None,
                "samples": len(used), "samples_in_timed_region": len(inside)}


def cpu_baseline(b, seconds: float):
    """The oracle as it stands, on a bounded sample of the same workload."""
    import oracle
    nthreads = os.cpu_count() or 1
    probe = min(b.npairs, 2000)
    sub = b.subset(np.arange(probe))
    t0 = time.perf_counter()
    for mode in ("global", "semiglobal"):
        oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, sub.matrix, sub.alpha,
                     sub.beta, mode, nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-6)
    k = int(min(b.npairs, max(probe, probe * seconds / dt)))
    sub = b.subset(np.arange(k))
    t0 = time.perf_counter()
    for mode in ("global", "semiglobal"):
        oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, sub.matrix, sub.alpha,
                     sub.beta, mode, nthreads=nthreads)
    dt = time.perf_counter() - t0
    cells = 2 * sub.cells()
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": nthreads, "kind": "oracle",
            "sample": f"first {k} of {b.npairs} pairs, global+semiglobal, {dt:.1f} s"}


def band_section(ga, dev, stream, npairs: int, ntrain: int, reps: int = 3):
    """Learned-band vs full-DP time to exact global scores (20k long DNA pairs).

    The predictor is trained first, on its own seeded pairs of the same
    distribution (labels = minimal certified widths computed by the library),
    then four ways to the same exact scores are timed on the test pairs:
    full DP, band doubling from the default start (16), from the best
    constant start chosen on the training pairs, and from the learned start
    (prediction kernel included).
    """
    import torch
    from paper_2205_07610_gb300 import band
    mat = synth.dna_matrix(2, -3)
    t0 = time.perf_counter()
    te = synth.long_dna_pairs(npairs=npairs)
    tr = synth.long_dna_pairs(npairs=ntrain, seed=synth.SEED_BASE + 400)
    gen_s = time.perf_counter() - t0

    def to_dev(b):
        return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                     for a in (b.q_codes, b.q_off, b.t_codes, b.t_off))
    d_te, d_tr = to_dev(te), to_dev(tr)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    w_min, _ = band.labels(*d_tr, mat, 5, 2, stream=stream)
    torch.cuda.synchronize(dev)
    labels_s = time.perf_counter() - t0
    steps, batch = 1500, 256
    t0 = time.perf_counter()
    pred, info = band.train(*d_tr, mat, 5, 2, synth.mlp_init(synth.SEED_BASE + 401),
                            synth.minibatches(tr.npairs, batch, steps, synth.SEED_BASE + 402),
                            lr=2e-3, w_min=w_min, stream=stream)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    c_w0, _ = band.best_constant_w0(*d_tr, mat, 5, 2, stream=stream)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        out = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            out.append(e0.elapsed_time(e1))
        return float(np.median(out)), r

    full_ms, (full, st_full) = timed(lambda: ga.align_batch(*d_te, mat, 5, 2, "global",
                                                            stream=stream, stats=True))
    runs = {}
    for name, fn in (("default_w0_16", lambda: ga.align_banded(*d_te, mat, 5, 2, default_w0=16,
                                                               stream=stream, stats=True)),
                     (f"best_constant_w0_{c_w0}", lambda: ga.align_banded(
                         *d_te, mat, 5, 2, default_w0=c_w0, stream=stream, stats=True)),
                     ("learned", lambda: pred.align(*d_te, mat, 5, 2, stream=stream, stats=True))):
        ms, (sc, wu, st) = timed(fn)
        runs[name] = {"ms": ms, "exact": bool(torch.equal(sc, full)),
                      "banded_cells": st["banded_cells"], "band_retries": st["band_retries"],
                      "speedup_vs_full_dp": full_ms / ms}
    losses = info["losses"]
    return {
        "metric": "time to exact global scores (ms)", "higher_is_better": False,
        "workload": f"{npairs} DNA pairs L~U{{1000..20000}}, divergence U(1%,15%), "
                    "indel fraction U(10%,40%); global, +2/-3, gap open 5, extend 2",
        "full_dp_ms": full_ms, "full_dp_cells": st_full["cells"],
        "full_dp_gcups": st_full["cells"] / full_ms / 1e6, "runs": runs,
        "train": {"pairs": tr.npairs, "steps": steps, "batch": batch, "labels_s": labels_s,
                  "train_s": train_s, "gen_s": gen_s, "loss_first": float(losses[:10].mean()),
                  "loss_last": float(losses[-50:].mean()), "rmse_log2": info["rmse_log2"],
                  "margin": info["margin"], "best_constant_w0": c_w0,
                  "phase_s": info["seconds"]},
    }


def serve_section(ga, dev, nreq: int, load: float = 0.7, burst: int = 50_000):
    """Serving: a Poisson stream of mixed requests through the alignment server.

    Capacity is measured first with a burst (the first `burst` requests
    released at once); the stream's arrival times are then rescaled to
    `load` x that capacity and replayed (release times on the server clock).
    Latency = completion seen by the scheduler - release.  Every score is
    checked against ga_align_batch of the same pairs.
    """
    import torch
    t0 = time.perf_counter()
    s = synth.serving_stream(nreq=nreq)
    gen_s = time.perf_counter() - t0
    cells = np.diff(s.q_off) * np.diff(s.t_off)
    with ga.Server(arena_bytes=32 << 30, max_inflight=65536, max_tasks=1 << 22,
                   device=dev.index or 0) as srv:
        d = srv.add_scoring(*s.dna_scoring)
        p = srv.add_scoring(*s.protein_scoring)
        sid = np.where(s.protein, p, d).astype(np.int32)
        nb = min(burst, s.nreq)
        t0 = time.perf_counter()
        srv.submit(s.q_codes, s.q_off[:nb + 1], s.t_codes, s.t_off[:nb + 1], s.mode[:nb], sid[:nb])
        srv.drain(600_000)
        burst_s = time.perf_counter() - t0
        srv.poll(nb + 16)
        cap_req_s = nb / burst_s
        cap_gcups = float(cells[:nb].sum()) / burst_s / 1e9
        rate = load * cap_req_s
        arr = (s.arrival - s.arrival[0]) * (1.0e4 / rate)  # generator rate is 1e4/s
        st_burst = srv.stats()
        # the stream starts 2 s after submission begins: submitting copies the
        # whole stream (~0.8 GB), which must not eat into the first arrivals
        start = srv.clock_ns() + 2_000_000_000
        rel = (start + arr * 1e9).astype(np.int64)
        srv.submit(s.q_codes, s.q_off, s.t_codes, s.t_off, s.mode, sid, rel)
        srv.drain(600_000)
        res = srv.poll(s.nreq + 16)
        st = srv.stats()
    res = res[np.argsort(res["id"])]
    lat_ms = (res["done_ns"] - res["release_ns"]) / 1e6
    wait_ms = (res["admit_ns"] - res["release_ns"]) / 1e6   # host: memory / slot admission
    dev_ms = (res["done_ns"] - res["admit_ns"]) / 1e6       # device queue + strips
    span_s = (res["done_ns"].max() - res["release_ns"].min()) / 1e9
    # exactness: the same pairs through ga_align_batch, grouped by scoring and mode
    exact = True
    scores = res["score"].astype(np.int64)
    for prot in (False, True):
        for md in (0, 1):
            idx = np.nonzero((s.protein == prot) & (s.mode == md))[0]
            if not len(idx):
                continue
            mat, al, be = s.protein_scoring if prot else s.dna_scoring
            qc, qo = synth.pack_csr([s.q_codes[s.q_off[i]:s.q_off[i + 1]] for i in idx])
            tc, to = synth.pack_csr([s.t_codes[s.t_off[i]:s.t_off[i + 1]] for i in idx])
            ref = ga.align_batch(*(torch.from_numpy(a).to(dev) for a in (qc, qo, tc, to)), mat, al, be,
                                 "global" if md else "local")
            exact &= bool(np.array_equal(ref.cpu().numpy().astype(np.int64), scores[idx]))
    return {
        "metric": "serve latency p50 / p99 (ms) at the offered load", "higher_is_better": False,
        "workload": f"{s.nreq} requests, Poisson arrivals at {load:.0%} of measured capacity, "
                    "lengths LogNormal(median 1000, sigma 1.2) in [100, 50000], 60% DNA (+2/-3, 5/2) "
                    "/ 40% protein (BLOSUM62, 11/1), 50/50 local/global",
        "p50_ms": float(np.percentile(lat_ms, 50)), "p90_ms": float(np.percentile(lat_ms, 90)),
        "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
        "admit_wait_p50_ms": float(np.percentile(wait_ms, 50)),
        "admit_wait_p99_ms": float(np.percentile(wait_ms, 99)),
        "device_p50_ms": float(np.percentile(dev_ms, 50)), "device_p99_ms": float(np.percentile(dev_ms, 99)),
        "gcups": float(cells.sum()) / span_s / 1e9, "offered_req_s": rate,
        "capacity_req_s": cap_req_s, "capacity_gcups": cap_gcups, "span_s": span_s,
        "exact": exact, "status_errors": int((res["status"] != 0).sum()),
        "kernel_launches": st["kernel_launches"], "arena_high_water": st["arena_high_water"],
        "burst_scheduler_s": {k: st_burst[k] / 1e9 for k in ("admit_host_ns", "copy_ns", "complete_ns")},
        "burst_ticks": st_burst["scheduler_ticks"],
        "gen_s": gen_s,
    }


def protein_section(ga, dev, stream, nq: int, nt: int, qmin: int = 100, qmax: int = 1000, reps: int = 2,
                    check_targets: int = 512, peaks: dict | None = None):
    """Protein database search: every query against every target, local mode.

    512 queries |Q| ~ U{100..1000} against 200k targets |T| ~ LogNormal(ln 300,
    0.6) in [10, 5000], BLOSUM62 background residues, gap open 11, extend 1,
    through ga_align_cross (packed int16x2 query-profile kernel, flagged pairs
    rerun in int32).  GCUPS = sum over pairs of m*n / time.  The int16 scores
    of every query against a seeded sample of targets (the 64 longest
    included) are checked against the int32 warp-per-pair path of
    ga_align_batch on the same pairs.
    """
    import torch
    t0 = time.perf_counter()
    cr = synth.protein_database(nq=nq, nt=nt, qmin=qmin, qmax=qmax)
    gen_s = time.perf_counter() - t0
    d = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (cr.q_codes, cr.q_off, cr.t_codes, cr.t_off)]
    scores = torch.empty((cr.nq, cr.nt), dtype=torch.int32, device=dev)
    # warm-up on a few queries (kernel attributes, workspace pool)
    ga.align_cross(d[0], d[1][:9], d[2], d[3], cr.matrix, cr.alpha, cr.beta, "local", stream=stream)
    torch.cuda.synchronize(dev)
    times, st = [], None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = ga.align_cross(*d, cr.matrix, cr.alpha, cr.beta, "local", scores=scores, stream=stream,
                               stats=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    cells = cr.cells()
    # sampled int32 check: all queries x `check_targets` targets
    rng = np.random.default_rng(synth.SEED_BASE + 303)
    tl = np.diff(cr.t_off)
    longest = np.argsort(tl)[-64:]
    pick = np.unique(np.concatenate([longest, rng.choice(cr.nt, size=check_targets - 64, replace=False)]))
    qi = np.repeat(np.arange(cr.nq), len(pick))
    ti = np.tile(pick, cr.nq)
    qo = np.concatenate([[0], np.cumsum(np.diff(cr.q_off)[qi])]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(tl[ti])]).astype(np.int64)
    qstart = torch.from_numpy(cr.q_off[qi]).to(dev)
    tstart = torch.from_numpy(cr.t_off[ti]).to(dev)
    dqo, dto = torch.from_numpy(qo).to(dev), torch.from_numpy(to).to(dev)
    # gather the pairs' residues on the device (index arithmetic only)
    qidx = torch.repeat_interleave(qstart - dqo[:-1], dqo.diff()) + torch.arange(int(qo[-1]), device=dev)
    tidx = torch.repeat_interleave(tstart - dto[:-1], dto.diff()) + torch.arange(int(to[-1]), device=dev)
    ref = ga.align_batch(d[0][qidx], dqo, d[2][tidx], dto, cr.matrix, cr.alpha, cr.beta, "local", stream=stream)
    got = scores[torch.from_numpy(qi).to(dev), torch.from_numpy(ti).to(dev)]
    exact = bool(torch.equal(ref, got))
    return {
        "metric": "GCUPS", "higher_is_better": True,
        "workload": f"{cr.nq} protein queries L~U{{{qmin}..{qmax}}} x {cr.nt} targets L~LogNormal(ln 300, 0.6) "
                    "in [10, 5000]; local, BLOSUM62, gap open 11, extend 1",
        "ms": ms, "ms_runs": times, "cells": cells, "gcups": cells / ms / 1e6,
        "dp_ms": st["dp_ms"], "dp_gcups": cells / st["dp_ms"] / 1e6 if st["dp_ms"] > 0 else None,
        "pairs_int32_rerun": st["pairs_int32_rerun"], "status": st["status"],
        "exact_vs_int32_sample": exact, "checked_pairs": int(len(qi)), "gen_s": gen_s,
        "roofline": protein_roofline(cells, st["dp_ms"], peaks),
    }


def protein_roofline(cells: int, dp_ms: float, peaks: dict | None) -> dict | None:
    """kp_kernel against the paper's 9-op local model and its own ALU mix."""
    if not peaks or dp_ms <= 0:
        return None
    gcups = cells / dp_ms / 1e6
    ops = cells * 9 / (dp_ms / 1e3)
    return {"bound": "alu", "achieved": ops / 1e12, "peak": peaks["issue_ops"] / 1e12,
            "unit": "Tops/s (int16, 9 ops per local cell)", "frac": ops / peaks["issue_ops"],
            "alu_ceiling_gcups": peaks["kp_alu_gcups"], "frac_alu_mix": gcups / peaks["kp_alu_gcups"],
            "kernel": "kp_kernel"}


def plan_section(ga, dev, stream, big, d_big, reps: int = 200):
    """Batch plans: eager calls vs preallocated runs vs CUDA-graph replays.

    small: 1,000 pairs of 150 x 150 uniform DNA, local mode (+2/-3, 5/2), the
    launch-bound case; `reps` back-to-back calls per path, CUDA events around
    the loop.  large: the 1M-pair mutated-DNA step (global + semi-global)
    replayed from graphs of autotuned plans (tuned on a 100k-pair sample of
    another seed), against the eager ga_align_batch step.
    """
    import torch
    out = {}
    c1 = synth.uniform_dna_pairs()
    d1 = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (c1.q_codes, c1.q_off, c1.t_codes, c1.t_off)]
    s1 = torch.empty(c1.npairs, dtype=torch.int32, device=dev)

    def loop_ms(fn, n):
        fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    eager = loop_ms(lambda: ga.align_batch(*d1, c1.matrix, c1.alpha, c1.beta, "local", scores=s1, stream=stream),
                    reps)
    ref = s1.clone()
    with ga.Plan(c1.matrix, c1.alpha, c1.beta, "local", c1.npairs, max(c1.q_off[-1], c1.t_off[-1]), 160) as pl:
        run_untuned = loop_ms(lambda: pl.run(*d1, scores=s1, stream=stream), reps)
        tuning1, _ = pl.autotune(*d1, reps=20, stream=stream)
        run = loop_ms(lambda: pl.run(*d1, scores=s1, stream=stream), reps)
        pl.capture(*d1, s1)
        graph = loop_ms(lambda: pl.launch(stream), reps)
        exact = bool(torch.equal(s1, ref))
    cells = c1.cells()
    out["small"] = {"workload": "1000 DNA pairs 150 x 150, local", "cells": cells, "tuning": tuning1,
                    "eager_us": eager * 1e3, "plan_run_untuned_us": run_untuned * 1e3,
                    "plan_run_us": run * 1e3, "graph_us": graph * 1e3,
                    "eager_gcups": cells / eager / 1e6, "plan_run_gcups": cells / run / 1e6,
                    "graph_gcups": cells / graph / 1e6, "exact": exact}

    sample = synth.mutated_dna_pairs(npairs=100_000, seed=synth.SEED_BASE + 2 + 777)
    ds = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
          (sample.q_codes, sample.q_off, sample.t_codes, sample.t_off)]
    cap = int(max(big.q_off[-1], big.t_off[-1]))
    outs = {m: torch.empty(big.npairs, dtype=torch.int32, device=dev) for m in ("global", "semiglobal")}
    plans, tunings = {}, {}
    for m in ("global", "semiglobal"):
        plans[m] = ga.Plan(big.matrix, big.alpha, big.beta, m, big.npairs, cap, 512)
        tunings[m], _ = plans[m].autotune(*ds, reps=5, stream=stream)
        plans[m].capture(*d_big, outs[m])

    def graph_step():
        plans["global"].launch(stream)
        plans["semiglobal"].launch(stream)

    step_ms = loop_ms(graph_step, 10)
    tmp = torch.empty(big.npairs, dtype=torch.int32, device=dev)
    eager_big = loop_ms(lambda: [ga.align_batch(*d_big, big.matrix, big.alpha, big.beta, m, scores=tmp,
                                                stream=stream) for m in ("global", "semiglobal")], 5)
    ref_g = ga.align_batch(*d_big, big.matrix, big.alpha, big.beta, "global", stream=stream)
    ref_s = ga.align_batch(*d_big, big.matrix, big.alpha, big.beta, "semiglobal", stream=stream)
    graph_step()
    torch.cuda.synchronize(dev)
    exact_big = bool(torch.equal(ref_g, outs["global"]) and torch.equal(ref_s, outs["semiglobal"]))
    for p in plans.values():
        p.close()
    cells_big = 2 * big.cells()
    out["large"] = {"workload": f"{big.npairs} mutated DNA pairs, global + semi-global (one bench step)",
                    "tuning": tunings, "graph_step_ms": step_ms, "eager_step_ms": eager_big,
                    "graph_gcups": cells_big / step_ms / 1e6, "eager_gcups": cells_big / eager_big / 1e6,
                    "exact": exact_big}
    return out


def r4(x):
    """Round floats to 4 significant digits, recursively (keeps the line short)."""
    if isinstance(x, float):
        return float(f"{x:.4g}")
    if isinstance(x, dict):
        return {k: r4(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [r4(v) for v in x]
    return x


def compact_plan(p):
    if not p:
        return None
    return r4({"small_eager_us": p["small"]["eager_us"], "small_graph_us": p["small"]["graph_us"],
               "large_graph_ms": p["large"]["graph_step_ms"], "large_eager_ms": p["large"]["eager_step_ms"],
               "exact": p["small"]["exact"] and p["large"]["exact"]})


def compact_protein(p):
    if not p:
        return None
    rf = p["roofline"] or {}
    return r4({"gcups": p["gcups"], "frac": rf.get("frac"), "frac_alu_mix": rf.get("frac_alu_mix"),
               "rerun": p["pairs_int32_rerun"], "exact": p["exact_vs_int32_sample"]})


def compact_serve(v):
    if not v:
        return None
    return r4({k: v[k] for k in ("p50_ms", "p99_ms", "max_ms", "gcups", "capacity_gcups", "exact")})


def compact_band(v):
    if not v:
        return None
    runs = v["runs"]
    best = next(k for k in runs if k.startswith("best_constant"))
    lr = runs["learned"]
    return r4({"full_dp_ms": v["full_dp_ms"], "learned_ms": lr["ms"],
               "best_const_ms": runs[best]["ms"], "w0_16_ms": runs["default_w0_16"]["ms"],
               "speedup": v["full_dp_ms"] / lr["ms"],
               # cells of the block-rounded bands the learned run evaluated, per
               # second (full DP: every m x n cell; the two rates compare the
               # kernels' speed per evaluated cell)
               "learned_region_gcups": lr["banded_cells"] / (lr["ms"] / 1e3) / 1e9 if lr["ms"] else None,
               "full_dp_gcups": v.get("full_dp_gcups"),
               "exact": all(r["exact"] for r in runs.values())})


def run_reference(args, rank: int):
    if rank != 0:
        return
    b = workload(args.npairs, 0)
    import oracle
    nthreads = os.cpu_count() or 1
    # per step: a bounded sample sized so the whole run stays within minutes
    per_step = max(1, args.cpu_seconds / max(1, args.steps + args.warmup) * 2)
    probe = min(b.npairs, 1000)
    sub = b.subset(np.arange(probe))
    t0 = time.perf_counter()
    oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, sub.matrix, 5, 2, "global",
                 nthreads=nthreads)
    dt = max(time.perf_counter() - t0, 1e-6)
    k = int(min(b.npairs, max(probe, probe * per_step / (2 * dt))))
    sub = b.subset(np.arange(k))

    def step():
        for mode in ("global", "semiglobal"):
            oracle.batch(sub.q_codes, sub.q_off, sub.t_codes, sub.t_off, sub.matrix, sub.alpha,
                         sub.beta, mode, nthreads=nthreads)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    cells = 2 * sub.cells() * args.steps
    value = cells / dt / 1e9
    line = {
        "impl": "reference", "metric": "GCUPS", "value": value, "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": "dna-mutated-pairs L~U{100..300}, 5% sub, 1% indel; global+semiglobal",
                   "npairs": args.npairs, "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": nthreads, "kind": "oracle",
                         "sample": f"first {k} of {b.npairs} pairs per step"},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_2205_07610_gb300 as ga

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ga.build()
    ga.load()
    # issue-rate probes of this GPU (the roofline's denominators), before the
    # workload so that nothing else runs beside them
    import roofline as rl
    rates = rl.measure(iters=args.probe_iters, ops=PROBE_OPS)

    b = workload(args.npairs, rank)
    cells_mode = b.cells()
    step_cells = 2 * cells_mode
    q = torch.from_numpy(b.q_codes).to(dev)
    qo = torch.from_numpy(b.q_off).to(dev)
    t = torch.from_numpy(b.t_codes).to(dev)
    to = torch.from_numpy(b.t_off).to(dev)
    s_both = torch.empty((2, b.npairs), dtype=torch.int32, device=dev)
    s_glob, s_semi = s_both[0], s_both[1]
    stream = torch.cuda.current_stream(dev)

    def step(stats=False):  # both modes from one packing of the inputs
        r = ga.align_batch_modes(q, qo, t, to, b.matrix, b.alpha, b.beta, ("global", "semiglobal"),
                                 scores=s_both, stream=stream, stats=stats)
        return (r[1],) if stats else None

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- warm-up, then the timed region: K steps, events on the launching
    # stream; nvidia-smi samples clocks from before the warm-up on and only
    # the samples inside the timed window are reported.
    sts = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        # every call reads its bin populations back once, so a host pause
        # (a garbage-collector pass over the batch's arrays) would leave the
        # GPU idle: no Python collection inside the timed region
        gc.collect()
        gc.disable()
        clk.mark_start()
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
        ev0.record(stream)
        for k in range(args.steps):
            step_ev[k][0].record(stream)
            sts.append(step(stats=True))
            step_ev[k][1].record(stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        gc.enable()
        clk.mark_end()
        barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), dist, dev)
    # the paper's statistic (Sec. 4.1): the median of the runs, for 10 runs
    # the mean of the 5th and 6th decile; per-step CUDA events of this rank
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    step_ms_median = float(np.median(step_ms))
    clocks = clk.summary()
    ms_per_step = ms / args.steps
    value = whole_job_gcups(step_cells, world, args.steps, ms)

    status = [s["status"] for pair in sts for s in pair]
    dp_ms = sum(s["dp_ms"] for pair in sts for s in pair)
    dp_launches = sum(s["dp_launches"] for pair in sts for s in pair)
    launches = sum(s["launches"] for pair in sts for s in pair)
    int16_pairs = sum(s["pairs_int16"] for pair in sts for s in pair)

    # ---- roofline of the dominant kernel (packed int16x2 inter-sequence DP)
    n_sm, max_mhz, _ = device_peak(dev, clocks)
    sm_mhz = clocks.get("sm_mhz") or max_mhz   # median SM clock inside the timed region
    peaks = measured_peaks(rates, n_sm, sm_mhz)
    alg_ops = step_cells * args.steps * OPS_PER_CELL
    achieved_ops = alg_ops / (dp_ms / 1e3) if dp_ms > 0 else 0.0
    dp_gcups = step_cells * args.steps / (dp_ms / 1e3) / 1e9 if dp_ms > 0 else None
    roofline = {
        "bound": "alu", "achieved": r4(achieved_ops / 1e12), "peak": r4(peaks["issue_ops"] / 1e12),
        "unit": "Tops/s (int16, 7 ops per cell, Sec. 4.2)", "frac": r4(achieved_ops / peaks["issue_ops"]),
        "traffic": KA_TRAFFIC_BYTES, "kernel": "ka_kernel<CellS16x2> (all launches of the timed region)",
        "dp_gcups": r4(dp_gcups), "alu_ceiling_gcups": r4(peaks["ka_alu_gcups"]),
        "frac_alu_mix": r4(dp_gcups / peaks["ka_alu_gcups"]) if dp_gcups else None,
        "mix_probe_gcups": r4(peaks["ka_mix_gcups"]),
        "peak_basis": peaks["basis"],
    }
    # ---- end to end through the host entry point (pinned buffers) ---------
    e2e = None
    if not args.no_e2e:
        hq = torch.from_numpy(b.q_codes).pin_memory()
        hqo = torch.from_numpy(b.q_off).pin_memory()
        ht = torch.from_numpy(b.t_codes).pin_memory()
        hto = torch.from_numpy(b.t_off).pin_memory()
        hs = torch.empty((2, b.npairs), dtype=torch.int32).pin_memory()

        def hstep():  # both modes of the step from one host copy of the inputs
            ga.align_batch_host_modes(hq, hqo, ht, hto, b.matrix, b.alpha, b.beta, ("global", "semiglobal"),
                                      scores=hs, stream=stream)
        hstep()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        barrier()
        et = reduce_max(time.perf_counter() - t0, dist, dev)
        assert torch.equal(hs[0], s_glob.cpu()) and torch.equal(hs[1], s_semi.cpu())
        h2d = hq.numel() + ht.numel() + 8 * (hqo.numel() + hto.numel())
        e2e = {"value": step_cells * world * args.steps / et / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(2 * 4 * b.npairs)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(b, args.cpu_seconds)

    band_res = None
    if world == 1 and not args.no_band:
        band_res = band_section(ga, dev, stream, args.band_pairs, args.band_train)
    plan_res = None
    if world == 1 and not args.no_plan:
        plan_res = plan_section(ga, dev, stream, b, (q, qo, t, to))
    prot_res = None
    if world == 1 and not args.no_protein:
        prot_res = protein_section(ga, dev, stream, args.protein_queries, args.protein_targets,
                                   args.protein_qmin, args.protein_qmax, peaks=peaks)
    serve_res = None
    if world == 1 and not args.no_serve:
        serve_res = serve_section(ga, dev, args.serve_requests)

    if rank == 0:
        line = {
            "metric": "GCUPS", "value": r4(value), "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r4(ms_per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int16x2", "data": "synthetic",
            "config": {
                "workload": "dna-mutated-pairs L~U{100..300}, 5% sub, 1% indel; global+semiglobal",
                "npairs_per_gpu": b.npairs, "cells_per_step_per_gpu": step_cells,
                "scoring": "+2/-3, gap open 5, extend 2",
                "parallelism": f"pairs sharded, {world} independent rank(s)",
                "l2": "inputs larger than L2 (2 x 200 MB codes per step)",
            },
            "clocks": {k: clocks.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples_in_timed_region")},
            "roofline": roofline, "e2e": r4(e2e), "cpu_baseline": r4(cpu),
            "gpu_launches": launches, "dp_status": max(status) if status else 0,
            "step_ms_median": r4(step_ms_median),
            "plan": compact_plan(plan_res), "protein": compact_protein(prot_res),
            "serve": compact_serve(serve_res), "band": compact_band(band_res),
        }
        print(json.dumps(line, separators=(",", ":")), flush=True)
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump(r4({"line": line, "rates": rates, "peaks": peaks, "band": band_res,
                              "protein": prot_res, "plan": plan_res, "serve": serve_res,
                              "pairs_int16_per_step": int16_pairs / args.steps}), f, indent=1)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
