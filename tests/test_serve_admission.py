"""Admission and batch formation of the request server (host logic, no GPU):
arrival order, the HBM byte budget, the per-batch caps, one request per
launch without batching, and a request larger than the whole budget running
alone once the device is otherwise idle."""

from collections import deque

import numpy as np

from paper_2103_15217_gb300.serve import GRAPH_BYTES_PER_EDGE, GRAPH_BYTES_PER_NODE, LCA_BYTES_PER_QUERY, \
    Request, form_batch


def lca(q, rid):
    return Request("lca", 0.0, tree=0, u=np.zeros(q, np.int32), v=np.zeros(q, np.int32), rid=rid)


def graph(n, m, rid):
    return Request("bridges", 0.0, n=n, edges=np.zeros((m, 2), np.int32), rid=rid)


def test_request_bytes():
    assert lca(100, 0).bytes() == 100 * LCA_BYTES_PER_QUERY
    assert graph(10, 40, 0).bytes() == 40 * GRAPH_BYTES_PER_EDGE + 10 * GRAPH_BYTES_PER_NODE


def test_fifo_until_the_budget():
    q = deque(lca(100, i) for i in range(5))
    batch, nb = form_batch(q, used=0, budget=3 * 100 * LCA_BYTES_PER_QUERY, batching=True, max_q=10 ** 9,
                           max_g=16, idle=False)
    assert [r.rid for r in batch] == [0, 1, 2] and nb == 3 * 100 * LCA_BYTES_PER_QUERY
    assert [r.rid for r in q] == [3, 4]


def test_budget_counts_what_is_in_use():
    q = deque([lca(100, 0)])
    budget = 100 * LCA_BYTES_PER_QUERY
    assert form_batch(q, used=1, budget=budget, batching=True, max_q=10 ** 9, max_g=16, idle=False) == ([], 0)
    assert len(q) == 1


def test_caps_per_batch():
    q = deque([lca(60, 0), lca(60, 1), graph(10, 40, 2), graph(10, 40, 3), lca(10, 4)])
    batch, _ = form_batch(q, used=0, budget=10 ** 12, batching=True, max_q=100, max_g=1, idle=False)
    assert [r.rid for r in batch] == [0]          # the second LCA request would pass 100 queries
    batch, _ = form_batch(q, used=0, budget=10 ** 12, batching=True, max_q=100, max_g=1, idle=False)
    assert [r.rid for r in batch] == [1, 2]       # then one graph; the next graph waits
    batch, _ = form_batch(q, used=0, budget=10 ** 12, batching=True, max_q=100, max_g=1, idle=False)
    assert [r.rid for r in batch] == [3, 4]


def test_one_request_per_launch_without_batching():
    q = deque(lca(10, i) for i in range(3))
    for i in range(3):
        batch, _ = form_batch(q, used=0, budget=10 ** 12, batching=False, max_q=10 ** 9, max_g=16, idle=False)
        assert [r.rid for r in batch] == [i]
    assert not q


def test_oversize_request_runs_alone_when_idle():
    big = lca(1000, 0)
    q = deque([big, lca(1, 1)])
    budget = 10 * LCA_BYTES_PER_QUERY
    assert form_batch(q, used=0, budget=budget, batching=True, max_q=10 ** 9, max_g=16, idle=False) == ([], 0)
    batch, nb = form_batch(q, used=0, budget=budget, batching=True, max_q=10 ** 9, max_g=16, idle=True)
    assert batch == [big] and nb == big.bytes()
    assert [r.rid for r in q] == [1]


def test_summary_percentiles_and_throughput():
    from paper_2103_15217_gb300.serve import Result, summarize
    res = [Result(i, "lca", np.zeros(10, np.int32), t_arrive=0.01 * i, t_admit=0.01 * i,
                  t_done=0.01 * i + 0.001 * (i + 1)) for i in range(100)]
    s = summarize(res)
    assert s["requests"] == 100 and s["units"] == 1000
    assert abs(s["seconds"] - (0.99 + 0.1)) < 1e-12 and abs(s["throughput"] - 1000 / 1.09) < 1e-6
    assert abs(s["p50_ms"] - 50.5) < 1e-9 and abs(s["p99_ms"] - 99.01) < 1e-9  # latencies 1..100 ms
    assert abs(s["mean_ms"] - 50.5) < 1e-9
    assert summarize(res, wall_units=7)["units"] == 7


def test_resident_table_forms():
    from paper_2103_15217_gb300.serve import resident_bytes
    sizes = [1 << 20, 1 << 16, 1 << 10]
    n = sum(sizes)
    blocked, full = resident_bytes(sizes, True), resident_bytes(sizes, False)
    # both hold at least pre, depth, size and order; the blocked form also a 16-byte record per node
    assert blocked >= 32 * n and full >= 16 * n
    # the full sparse table grows with log n per node, the blocked one does not
    assert full > blocked
    assert resident_bytes([1 << 22], False) / (1 << 22) > resident_bytes([1 << 12], False) / (1 << 12)
    assert abs(resident_bytes([1 << 22], True) / (1 << 22) - resident_bytes([1 << 12], True) / (1 << 12)) < 2
