"""The benchmark's CPU-oracle legs (host only): the single-process sample and
the all-core run of the same oracle in one process per core."""

import os
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KW = {"n": 64, "n_bodies": 12}


def test_single_sample_counts_its_markers():
    with tempfile.TemporaryDirectory() as td:
        r = bench.run_oracle_sample("c2", "exact", [0, 2], 1, os.path.join(td, "s.npz"), KW)
    assert r["markers"] == 2 * 1280 and len(r["times"]) == 1 and r["times"][0] > 0


def test_all_cores_runs_one_process_per_core():
    value, procs = bench.run_oracle_all_cores("c2", "exact", 2, KW)
    assert procs == max(1, os.cpu_count() or 1)
    assert value > 0
    # a sample larger than the workload is refused rather than truncated
    assert bench.run_oracle_all_cores("c2", "exact", 13, KW) is None


def test_reference_arm_reports_the_measured_sample(capsys):
    class A:
        workload, grid, bodies, method, steps, warmup = "c2", 64, 12, "exact", 1, 0
    bench.run_reference(A, 0, 1)
    import json
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    procs = max(1, os.cpu_count() or 1)
    assert line["impl"] == "reference" and line["config"]["markers_per_step"] == procs * 12 * 1280
    # value is the sample's markers over the measured step time
    assert abs(line["value"] - line["config"]["markers_per_step"] / (line["ms_per_step"] / 1e3)) <= 1e-6 * line["value"]
