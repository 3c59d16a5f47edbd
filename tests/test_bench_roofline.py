"""The benchmark's roofline entry (host arithmetic, no GPU): the dominant phase
is picked by device time, its algorithmic bytes per launch come from the
per-unit table and the workload, and the committed DRAM-traffic record is
used only for the launch parameters it was taken with."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def workload():
    trees = [dict(n=1 << 24, u=np.zeros(1 << 24, np.int32)) for _ in range(3)]
    graphs = [dict(n=1 << 22, m=(1 << 25) - 1), dict(n=1 << 22, m=(1 << 22) - 1 + (1 << 24))]
    return trees, graphs


def test_dominant_phase_and_algorithmic_bytes():
    trees, graphs = workload()
    steps = 4
    # walk0: 5 launches per step (3 trees + 2 graphs), 1 ms each; query: 3 launches of 0.5 ms
    phases = {"rank.walk0": (5 * steps * 1.0, 5 * steps), "lca.query": (3 * steps * 0.5, 3 * steps)}
    r = bench.roofline_from_phases(phases, trees, graphs, steps)
    assert r["kernel"] == "rank.walk0" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    want = (3 * 2 * (1 << 24) * 12 + 2 * (2 * (1 << 22) - 1) * 12) / 5
    assert r["bytes_per_launch"] == pytest.approx(want)
    assert r["avg_launch_ms"] == pytest.approx(1.0)
    assert r["achieved"] == pytest.approx(want / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["launches_per_step"] == 5


def test_traffic_record_needs_its_launch_parameters():
    import paper_2103_15217_gb300 as etl
    etl.build()
    etl.load_library()
    old = etl.tune_get()
    try:
        t = bench.committed_traffic("rank.walk0", 3, 2)
        assert t is None or t > 0
        etl.tune_set(rank_k0_log2=3 if old["rank_k0_log2"] != 3 else 4)  # not the capture's setting
        assert bench.committed_traffic("rank.walk0", 3, 2) is None
    finally:
        etl.tune_set(**old)
    assert bench.committed_traffic("lca.query", 3, 2) is None  # the record is for the walk only
    assert bench.committed_traffic("rank.walk0", 1, 2) is None  # and for the bench's workload only


def test_step_statistics_and_seeds():
    s = bench.step_stats([3.0, 1.0, 2.0, 6.0])
    assert s == {"mean": 3.0, "std": pytest.approx(np.std([3.0, 1.0, 2.0, 6.0])), "min": 1.0, "median": 2.5,
                 "max": 6.0, "n": 4}
    assert bench.replica_seed(0) == 1 and bench.replica_seed(3, base=5) == 8


def test_every_phase_with_a_byte_figure_gets_a_roofline_row():
    trees, graphs = workload()
    steps = 2
    phases = {"rank.walk0": (10.0, 10), "lca.query": (3.0, 6), "rmq.top": (1.0, 30), "br.hook": (4.0, 8)}
    rows = bench.phase_rooflines(phases, trees, graphs, steps)
    assert set(rows) == {"rank.walk0", "lca.query", "br.hook"}  # rmq.top has no per-unit figure
    q = rows["lca.query"]
    assert q["bytes_per_launch"] == (1 << 24) * 32 and q["avg_launch_ms"] == 0.5 and q["launches_per_step"] == 3
    assert abs(q["achieved_gbs"] - (1 << 24) * 32 / 0.5e-3 / 1e9) < 1e-9
    hook = rows["br.hook"]  # graph-only phase: the mean edge count of the two graphs
    assert hook["bytes_per_launch"] == ((1 << 25) - 1 + (1 << 22) - 1 + (1 << 24)) / 2 * 17
    # the dominant-kernel entry is the same arithmetic as its row
    top = bench.roofline_from_phases(phases, trees, graphs, steps)
    assert top["kernel"] == "rank.walk0" and abs(top["achieved"] - rows["rank.walk0"]["achieved_gbs"]) < 1e-9
