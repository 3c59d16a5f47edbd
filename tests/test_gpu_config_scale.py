"""The batched and served workloads at their full configured scale, every
result compared with the CPU oracle (bit-exact: all of it is integer work).

* Batched (Sec. 3.3 "Batch Size" is the motivation): 2048 trees with n
  log-uniform in [2^6, 2^18] (grasp 1, 1024 and unlimited, round robin), n
  uniform queries each, and 2048 graphs with n log-uniform in [2^6, 2^16],
  m = 4n, small- and large-diameter alternating -- the inputs the benchmark
  times. They run through lca_preprocess_batch / lca_query_batch and
  find_bridges_batch, first eagerly and then replayed from one captured CUDA
  graph with the tree batch and the graph batch on two parallel streams (the
  benchmark runs them one after the other on one stream; the forked capture
  also checks that the two batches share no scratch). At this scale the chained tour of all trees is a
  list far larger than L2, so the walk runs with the launch shape of large
  lists, and the connectivity pass spreads its edge chunks over 2048 graphs.
* Served: 256 resident trees with n log-uniform in [2^10, 2^22] and the
  600-request Poisson stream (LCA batches of 2^4..2^20 queries, bridge
  requests on fresh graphs of 2^10..2^22 nodes with m = 4n), served with
  continuous batching in real time and with every request already arrived.

The oracle (Tarjan's offline LCA, DFS low-link bridges) runs on host threads:
its C functions are called through ctypes, which releases the interpreter
lock, and they keep no global state.
"""

import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _pool():
    return cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))


def test_batched_config_matches_oracle():
    import bench
    import paper_2103_15217_gb300 as etl
    B = bench.make_batch_inputs(small=False)
    assert len(B["trees"]) == 2048 and len(B["graphs"]) == 2048
    dev = torch.device("cuda", 0)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    P, O = T(np.concatenate(B["tp"])), T(B["toff"])
    I, U, V = T(np.concatenate(B["ti"])), T(np.concatenate(B["tu"])), T(np.concatenate(B["tv"]))
    E, EO, NO = T(np.concatenate(B["ge"])), T(B["eoff"]), T(B["noff"])
    max_n = max(d["n"] for d in B["trees"])
    total_gn = int(B["noff"][-1])
    out = torch.full_like(U, -9)
    mask = torch.full((E.shape[0],), 7, dtype=torch.uint8, device=dev)
    st_t, st_g = etl.new_status(dev), etl.new_status(dev)
    stream, side = torch.cuda.Stream(), torch.cuda.Stream()

    def step():
        main = torch.cuda.current_stream()
        side.wait_stream(main)
        h = etl.lca_preprocess_batch(P, O, max_n)
        h.query_batch(I, U, V, out=out, status=st_t)
        h.free()
        with torch.cuda.stream(side):
            mask.copy_(etl.find_bridges_batch(E, EO, NO, total_gn, status=st_g))
        main.wait_stream(side)

    # the oracle's answers, on host threads while the GPU works
    with _pool() as pool:
        want_lca = [pool.submit(oracle.lca_offline, p, u, v) for p, u, v in zip(B["tp"], B["tu"], B["tv"])]
        want_br = [pool.submit(oracle.bridges_dfs, d["n"], e) for d, e in zip(B["graphs"], B["ge"])]
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            step()
        torch.cuda.synchronize()
        eager = (out.cpu().numpy(), mask.cpu().numpy())
        assert int(st_t.item()) == 0 and int(st_g.item()) == 0
        out.fill_(-9)
        mask.fill_(7)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            step()
        g.replay()
        torch.cuda.synchronize()
        replayed = (out.cpu().numpy(), mask.cpu().numpy())
        del g
        want = (np.concatenate([f.result() for f in want_lca]), np.concatenate([f.result() for f in want_br]))
    qoff = np.cumsum([0] + [u.shape[0] for u in B["tu"]])
    for got in (eager, replayed):
        bad = np.flatnonzero(got[0] != want[0])
        if bad.size:
            ti = int(np.searchsorted(qoff, bad[0], side="right") - 1)
            raise AssertionError(f"batched LCA differs from the oracle on {bad.size} queries, first in tree {ti} "
                                 f"({B['trees'][ti]})")
        bad = np.flatnonzero(got[1] != want[1])
        if bad.size:
            gi = int(np.searchsorted(B["eoff"], bad[0], side="right") - 1)
            raise AssertionError(f"batched bridges differ from the oracle on {bad.size} edges, first in graph {gi} "
                                 f"({B['graphs'][gi]})")
    assert int(st_t.item()) == 0 and int(st_g.item()) == 0


def _submit_serving_oracle(parents, reqs, pool):
    """Oracle work for every request: one offline-LCA call per tree over all of its queries."""
    by_tree = {}
    for r in reqs:
        if r.kind == "lca":
            by_tree.setdefault(r.tree, []).append(r)
    futs = {}
    for tree, rs in by_tree.items():
        u = np.concatenate([r.u for r in rs])
        v = np.concatenate([r.v for r in rs])
        futs[("t", tree)] = (rs, pool.submit(oracle.lca_offline, parents[tree], u, v))
    for r in reqs:
        if r.kind == "bridges":
            futs[("g", r.rid)] = ([r], pool.submit(oracle.bridges_dfs, r.n, r.edges))
    return futs


def _collect(futs):
    want = {}
    for (kind, _), (rs, f) in futs.items():
        ans = f.result()
        if kind == "g":
            want[rs[0].rid] = ans
            continue
        pos = 0
        for r in rs:
            want[r.rid] = ans[pos:pos + r.u.shape[0]]
            pos += r.u.shape[0]
    return want


def test_serving_config_matches_oracle():
    import bench
    from paper_2103_15217_gb300.serve import Server
    parents, reqs = bench.make_serving_inputs(small=False)
    assert len(parents) == 256 and len(reqs) == 600
    with _pool() as pool:
        futs = _submit_serving_oracle(parents, reqs, pool)
        srv = Server(parents, budget_bytes=40 << 30, slots=4)
        live = srv.serve(reqs, batching=True, realtime=True)
        offline = srv.serve(reqs, batching=True, realtime=False)
        srv.close()
        want = _collect(futs)
    assert sorted(want) == sorted(r.rid for r in reqs)
    for results in (live, offline):
        assert [x.rid for x in results] == sorted(r.rid for r in reqs)
        for x in results:
            w = want[x.rid]
            assert x.out.shape == w.shape and (x.out == w).all(), f"request {x.rid} ({x.kind}) differs from the oracle"
