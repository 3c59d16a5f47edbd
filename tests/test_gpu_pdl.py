"""Programmatic dependent launch (ETL_TUNE_PDL) on and off: the same results.

With the knob on, each kernel of the library may be scheduled while the one
before it on the stream is finishing and waits on the device for its
writes; the chains of dependent passes of Sec. 2 (tour, ranking, prefix
sums), Sec. 3 (tables, queries) and Sec. 4.1 (connectivity, forest tour,
low/high) must give the oracle's answers either way, eagerly and replayed
from a captured CUDA graph.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture
def etl():
    import paper_2103_15217_gb300 as etl
    etl.build()
    etl.load_library()
    old = etl.tune_get()
    yield etl
    etl.tune_set(**old)


@pytest.mark.parametrize("pdl", [0, 1])
def test_results_do_not_depend_on_pdl(etl, pdl):
    etl.tune_set(pdl=pdl)
    n, q, gn = 70001, 90000, 30000
    parent = synth.tree_parent(n, 1024, seed=pdl + 3)
    u, v = synth.lca_queries(n, q, seed=pdl + 3)
    e = synth.hard_graph(gn, 3 * gn, gn // 64, seed=pdl + 3)
    P, U, V, E = dev(parent), dev(u), dev(v), dev(e)
    want_lca = oracle.lca_offline(parent, u, v)
    want_br = oracle.bridges_dfs(gn, e)
    h = etl.lca_preprocess(P)
    assert (host(h.query(U, V)) == want_lca).all()
    pre, depth, size, _ = oracle.tree_tour(parent)
    arr = {k: host(t) for k, t in h.arrays().items()}
    assert (arr["pre"] == pre).all() and (arr["depth"] == depth).all() and (arr["size"] == size).all()
    h.free()
    assert (host(etl.find_bridges(E, gn)) == want_br).all()
    order = np.random.default_rng(pdl).permutation(n).astype(np.int32)
    succ = np.full(n, -1, np.int32)
    succ[order[:-1]] = order[1:]
    rank = host(etl.list_rank(dev(succ), int(order[0])))
    assert (rank[order] == np.arange(n)).all()

    # the same chain captured into one graph and replayed twice
    ws_t = etl.new_workspace(etl.workspace_size("lca_preprocess", n))
    ws_g = etl.new_workspace(etl.workspace_size("find_bridges", gn, e.shape[0]))
    out = torch.full_like(U, -5)
    mask = torch.full((e.shape[0],), 9, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        hg = etl.lca_preprocess(P, workspace=ws_t)
        hg.query(U, V, out=out)
        etl.find_bridges(E, gn, out=mask, workspace=ws_g)
    for _ in range(2):
        out.fill_(-5)
        mask.fill_(9)
        g.replay()
        torch.cuda.synchronize()
        assert (host(out) == want_lca).all()
        assert (host(mask) == want_br).all()
    hg.free()
    del g
