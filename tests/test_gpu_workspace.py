"""Caller-owned workspaces (the _ws entry points and etl_workspace_size).

Every _ws call runs on a buffer of exactly the size etl_workspace_size reports,
gives the oracle's answers (bit-exact), and requests no device allocation from
the library (etl_alloc_count does not move) -- also while the calls are being
captured into a CUDA graph, whose replays give the same answers. A buffer one
byte short is refused with ETL_ENOMEM. The problem statements are those of
Sec. 3 (LCA) and Sec. 4.1 (bridges); list ranking is Sec. 2.2.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _etl():
    import paper_2103_15217_gb300 as etl
    etl.build()
    etl.load_library()
    return etl


def test_sizes_are_positive_and_grow():
    etl = _etl()
    for kind, args in (("list_rank", (1,)), ("lca_preprocess", (1,)), ("find_bridges", (2, 1))):
        small = etl.workspace_size(kind, *args)
        big = etl.workspace_size(kind, *(a * 4096 for a in args))
        assert 0 < small < big
    assert etl.workspace_size("lca_query", 1000, 1 << 20) == 0
    assert etl.workspace_size("find_bridges", 10, 0) == 0        # no edges: the call does nothing
    with pytest.raises(etl.EtlError):
        etl.workspace_size("lca_preprocess", 0)


@pytest.mark.parametrize("n", [1, 2, 33, 4099, 70001])
def test_list_rank_in_workspace(n):
    etl = _etl()
    order = np.random.default_rng(n).permutation(n).astype(np.int32)
    succ = np.full(n, -1, np.int32)
    succ[order[:-1]] = order[1:]
    want = np.empty(n, np.int32)
    want[order] = np.arange(n, dtype=np.int32)
    ws = etl.new_workspace(etl.workspace_size("list_rank", n))
    s = dev(succ)
    a0 = etl.alloc_count()
    st = etl.new_status()
    got = etl.list_rank(s, int(order[0]), status=st, workspace=ws)
    assert etl.alloc_count() == a0
    assert etl.status_get(st) == 0
    assert (host(got) == want).all()


@pytest.mark.parametrize("n,grasp", [(1, None), (2, None), (1000, 1), (65537, None), (100003, 1024)])
def test_lca_in_workspace(n, grasp):
    etl = _etl()
    parent = synth.tree_parent(n, grasp, seed=n)
    u, v = synth.lca_queries(n, 2 * n + 5, seed=n)
    P, U, V = dev(parent), dev(u), dev(v)
    ws = etl.new_workspace(etl.workspace_size("lca_preprocess", n))
    a0 = etl.alloc_count()
    h = etl.lca_preprocess(P, workspace=ws)
    out = torch.empty_like(U)
    h.query(U, V, out=out)
    assert etl.alloc_count() == a0
    assert h.status() == 0
    pre, depth, size, _ = oracle.tree_tour(parent)
    arr = {k: host(t) for k, t in h.arrays().items()}
    assert (arr["pre"] == pre).all() and (arr["depth"] == depth).all() and (arr["size"] == size).all()
    assert (host(out) == oracle.lca_offline(parent, u, v)).all()
    h.free()


@pytest.mark.parametrize("kind,n", [("easy", 5000), ("hard", 20000), ("easy", 3)])
def test_bridges_in_workspace(kind, n):
    etl = _etl()
    e = synth.easy_graph(n, 4 * n, seed=n) if kind == "easy" else synth.hard_graph(n, 3 * n, max(1, n // 64), seed=n)
    ws = etl.new_workspace(etl.workspace_size("find_bridges", n, e.shape[0]))
    E = dev(e)
    a0 = etl.alloc_count()
    st = etl.new_status()
    mask = etl.find_bridges(E, n, status=st, workspace=ws)
    assert etl.alloc_count() == a0
    assert etl.status_get(st) == 0
    assert (host(mask) == oracle.bridges_dfs(n, e)).all()


def test_batches_in_workspace():
    etl = _etl()
    sizes = [1, 700, 3000, 64]
    parents = [synth.tree_parent(k, g, seed=k) for k, g in zip(sizes, (None, 1, 16, None))]
    node_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    total = int(node_off[-1])
    ws = etl.new_workspace(etl.workspace_size_batch("lca_preprocess", len(sizes), total, max(sizes)))
    inst = np.repeat(np.arange(len(sizes), dtype=np.int32), 300)
    rng = np.random.default_rng(1)
    bu = (rng.integers(0, 1 << 30, inst.size) % np.array(sizes)[inst]).astype(np.int32)
    bv = (rng.integers(0, 1 << 30, inst.size) % np.array(sizes)[inst]).astype(np.int32)
    a0 = etl.alloc_count()
    h = etl.lca_preprocess_batch(dev(np.concatenate(parents)), dev(node_off), max(sizes), workspace=ws)
    got = host(h.query_batch(dev(inst), dev(bu), dev(bv)))
    assert etl.alloc_count() == a0
    for i, par in enumerate(parents):
        sel = inst == i
        assert (got[sel] == oracle.lca_offline(par, bu[sel], bv[sel])).all()
    h.free()

    graphs = [(n_, synth.easy_graph(n_, 4 * n_, seed=n_) if n_ % 2 else synth.hard_graph(n_, 3 * n_, 5, seed=n_))
              for n_ in (64, 301, 1000)]
    eoff = np.concatenate([[0], np.cumsum([g.shape[0] for _, g in graphs])]).astype(np.int32)
    noff = np.concatenate([[0], np.cumsum([n_ for n_, _ in graphs])]).astype(np.int32)
    ws = etl.new_workspace(etl.workspace_size_batch("find_bridges", len(graphs), int(noff[-1]), int(eoff[-1])))
    a0 = etl.alloc_count()
    st = etl.new_status()
    got = host(etl.find_bridges_batch(dev(np.concatenate([g for _, g in graphs])), dev(eoff), dev(noff),
                                      int(noff[-1]), status=st, workspace=ws))
    assert etl.alloc_count() == a0
    assert etl.status_get(st) == 0
    assert (got == np.concatenate([oracle.bridges_dfs(n_, g) for n_, g in graphs])).all()


def test_captured_graph_allocates_nothing():
    # preprocessing, queries and bridges captured into one CUDA graph with caller workspaces: no
    # allocation request reaches the library's allocator (so the graph has no memory nodes of ours),
    # the library's pool does not grow, and every replay gives the oracle's answers
    etl = _etl()
    n, q, gn = 50_000, 80_000, 20_000
    parent = synth.tree_parent(n, None, seed=3)
    u, v = synth.lca_queries(n, q, seed=3)
    e = synth.hard_graph(gn, 3 * gn, gn // 64, seed=3)
    P, U, V, E = dev(parent), dev(u), dev(v), dev(e)
    ws_t = etl.new_workspace(etl.workspace_size("lca_preprocess", n))
    ws_g = etl.new_workspace(etl.workspace_size("find_bridges", gn, e.shape[0]))
    out = torch.full_like(U, -5)
    mask = torch.full((e.shape[0],), 9, dtype=torch.uint8, device="cuda")
    st = etl.new_status()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    pool0 = etl.pool_stats()
    a0 = etl.alloc_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        h = etl.lca_preprocess(P, workspace=ws_t)
        h.query(U, V, out=out)
        etl.find_bridges(E, gn, status=st, out=mask, workspace=ws_g)
    assert etl.alloc_count() == a0
    want_lca = oracle.lca_offline(parent, u, v)
    want_br = oracle.bridges_dfs(gn, e)
    for _ in range(2):
        out.fill_(-5)
        mask.fill_(9)
        g.replay()
        torch.cuda.synchronize()
        assert (host(out) == want_lca).all()
        assert (host(mask) == want_br).all()
        assert int(st.item()) == 0
    assert etl.alloc_count() == a0
    assert etl.pool_stats()["reserved"] == pool0["reserved"]
    h.free()
    del g


def test_short_workspace_is_refused():
    etl = _etl()
    n = 10_000
    parent = synth.tree_parent(n, None, seed=2)
    need = etl.workspace_size("lca_preprocess", n)
    ws = etl.new_workspace(need)
    assert ws.data_ptr() % 256 == 0
    # the size includes 256 bytes of room to align an arbitrary base; on an aligned base the call
    # uses need - 256 bytes, so this buffer is one byte short of it
    short = ws[: need - 257]
    with pytest.raises(etl.EtlError) as err:
        etl.lca_preprocess(dev(parent), workspace=short)
    assert err.value.code == 2                     # ETL_ENOMEM
    torch.cuda.synchronize()
    h = etl.lca_preprocess(dev(parent), workspace=ws)  # the exact size is enough
    assert h.status() == 0
    h.free()


def test_data_errors_in_workspace():
    # malformed inputs through the _ws entry points: the same device status codes and outputs as the
    # plain calls (not one tree -> ETL_EBADTREE and -1 answers; endpoint out of range -> ETL_EBADGRAPH
    # and an all-zero mask), and nothing allocated
    etl = _etl()
    u = dev(np.array([0, 1, 2], np.int32))
    a0 = etl.alloc_count()
    for parent in ([-1, -1, 0], [-1, 2, 1], [-1, 7, 0], [1, 0, 0]):
        ws = etl.new_workspace(etl.workspace_size("lca_preprocess", len(parent)))
        h = etl.lca_preprocess(dev(np.array(parent, np.int32)), workspace=ws)
        assert h.status() == 4
        assert (host(h.query(u, u)) == -1).all()
        h.free()
    n = 50000   # a long cycle hidden in a big tree
    parent = synth.tree_parent(n, None, seed=3)
    kids = np.nonzero(parent >= 0)[0]
    parent[kids[10]], parent[kids[20]] = kids[20], kids[10]
    ws = etl.new_workspace(etl.workspace_size("lca_preprocess", n))
    h = etl.lca_preprocess(dev(parent), workspace=ws)
    assert h.status() == 4
    h.free()
    e = np.array([[0, 1], [1, 4], [2, 3]], np.int32)
    ws = etl.new_workspace(etl.workspace_size("find_bridges", 4, 3))
    st = etl.new_status()
    mask = host(etl.find_bridges(dev(e), 4, status=st, workspace=ws))
    assert etl.status_get(st) == 6 and (mask == 0).all()
    assert etl.alloc_count() == a0

