"""The host-side helpers of bench.py (no GPU): default step counts, the peak
table's fallback, the launch count per step, and the reading of the committed
DRAM-traffic files (a file taken on other sources must read as unknown)."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_defaults_meet_the_timing_rules(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1
    assert a.workload == "planted" and a.form == "gather" and a.impl == "gpga"


def test_peaks_name_their_source(bench):
    d, src = bench.peaks()
    assert src in ("measured", "fallback")
    assert d["hbm_gbs"] > 0


def test_launches_per_step(bench):
    # prelude 7, start 3 + score + select, then one fused kernel + selection per
    # generation (gather) or evolve + score + selection (plain: 2, tensor: 4)
    assert bench.launches_per_step("gather", 100) == 7 + 5 + 200
    assert bench.launches_per_step("plain", 10) == 7 + 6 + 40
    assert bench.launches_per_step("tensor", 10) == 7 + 8 + 60


@pytest.mark.parametrize("kernel,sources", [
    ("gather_generation_n500_p4096", ("gather.cu", "gpga_internal.cuh")),
    ("tc_mma_n500_p4096", ("score_tc.cu", "gpga_internal.cuh")),
    ("pair_plain_n500_p4096", ("score.cu", "gpga_internal.cuh")),
])
def test_traffic_files_parse(bench, kernel, sources):
    got = bench.profiled_traffic(kernel, bench.source_hash(*sources))
    assert got is None or got > 0
    assert bench.profiled_traffic(kernel, "0" * 16) is None  # other sources: unknown
