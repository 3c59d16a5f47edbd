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
