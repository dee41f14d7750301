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


def test_first_recovery_reads_the_records(bench):
    """Recovery along a run's records: the first generation whose best
    configuration matches the planted clusters over their members (noise series
    left out), its device time, and the final configuration's merged and split
    planted clusters."""
    import numpy as np
    truth = np.array([0, 0, 0, 1, 1, 1, 2, 2, 3, 4])  # clusters 0-2, noise 3 and 4
    merged = np.array([5, 5, 5, 5, 5, 5, 7, 7, 1, 5])  # 0 and 1 together
    split = np.array([5, 5, 6, 3, 3, 3, 7, 7, 5, 5])   # 0 in two pieces
    exact = np.array([9, 9, 9, 2, 2, 2, 4, 4, 9, 2])   # noise placed anywhere
    h = {"labels": [merged, split, exact, exact], "t_ns": np.array([0, 10, 20, 35, 50]),
         "best_L": np.array([1.0, 2.0, 3.0, 3.0])}
    r = bench.first_recovery(h, truth)
    assert r["generation"] == 2 and r["ms"] == 35e-6
    assert r["best_ari_members"] == 1.0 and r["best_ari_members_generation"] == 2
    assert r["final_planted_clusters_merged"] == 0 and r["final_planted_clusters_split"] == 0
    r = bench.first_recovery({**h, "labels": [exact, merged]}, truth)
    assert r["final_planted_clusters_merged"] == 2 and r["final_planted_clusters_split"] == 0
    r = bench.first_recovery({**h, "labels": [split]}, truth)
    assert r["generation"] is None and r["ms"] is None
    assert r["final_planted_clusters_merged"] == 0 and r["final_planted_clusters_split"] == 1
