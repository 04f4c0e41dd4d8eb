"""The bench line's summaries of its side measurements (host logic, no GPU).

bench.py prints one JSON line; the band, protein, serving and plan sections
are folded into short summaries by compact_* helpers.  These tests feed them
section results of the shape bench.py's measurement functions return and
check the figures a reader takes from the line: times, speedups, rates and
the exactness flags.
"""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _band_section(exact=True):
    run = lambda ms, cells, retries: {"ms": ms, "exact": exact, "banded_cells": cells,
                                      "band_retries": retries, "speedup_vs_full_dp": 400.0 / ms}
    return {"metric": "time to exact global scores (ms)", "full_dp_ms": 400.0,
            "full_dp_cells": 2_800_000_000_000, "full_dp_gcups": 7000.0,
            "runs": {"default_w0_16": run(380.0, 1.2e12, 100), "best_constant_w0_1024": run(150.0, 9e11, 7),
                     "learned": run(100.0, 5e11, 2)},
            "train": {"pairs": 4000}}


def test_band_summary_figures(bench):
    out = bench.compact_band(_band_section())
    assert out["full_dp_ms"] == 400.0 and out["learned_ms"] == 100.0
    assert out["best_const_ms"] == 150.0 and out["w0_16_ms"] == 380.0
    assert out["speedup"] == 4.0
    # 5e11 evaluated band cells in 0.1 s
    assert out["learned_region_gcups"] == 5000.0
    assert out["full_dp_gcups"] == 7000.0
    assert out["exact"] is True
    json.dumps(out)  # one JSON line


def test_band_summary_flags_any_inexact_run(bench):
    sec = _band_section()
    sec["runs"]["best_constant_w0_1024"]["exact"] = False
    assert bench.compact_band(sec)["exact"] is False
    assert bench.compact_band(None) is None


def test_other_summaries_keep_their_keys(bench):
    plan = {"small": {"eager_us": 130.0, "graph_us": 52.0, "exact": True},
            "large": {"graph_step_ms": 14.3, "eager_step_ms": 14.2, "exact": True}}
    assert bench.compact_plan(plan) == {"small_eager_us": 130.0, "small_graph_us": 52.0,
                                        "large_graph_ms": 14.3, "large_eager_ms": 14.2, "exact": True}
    prot = {"gcups": 6330.123, "roofline": {"frac": 0.72261, "frac_alu_mix": 0.5665},
            "pairs_int32_rerun": 0, "exact_vs_int32_sample": True}
    assert bench.compact_protein(prot) == {"gcups": 6330.0, "frac": 0.7226, "frac_alu_mix": 0.5665,
                                           "rerun": 0, "exact": True}
    serve = {"p50_ms": 0.47, "p99_ms": 7.86, "max_ms": 29.7, "gcups": 2238.0, "capacity_gcups": 3090.0,
             "exact": True, "extra": 1}
    assert set(bench.compact_serve(serve)) == {"p50_ms", "p99_ms", "max_ms", "gcups", "capacity_gcups", "exact"}
