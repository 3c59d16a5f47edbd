"""GPU LCA (preprocess + query through the C ABI) against the CPU oracle.

Every answer is compared element by element (bit-exact, integer work), as are
the per-node arrays pre / depth / size (unique, since children are visited in
ascending label order on both sides). Sizes span several tiles and ragged
tails; the full-size tree of the benchmark (n = 2^24) is checked on all
queries with the oracle's offline LCA.
"""

import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run_gpu(parent, u, v):
    import paper_2103_15217_gb300 as etl
    h = etl.lca_preprocess(dev(parent))
    st = etl.new_status()
    out = host(h.query(dev(u), dev(v), status=st))
    arrays = {k: host(t) for k, t in h.arrays().items()}
    hst = h.status()
    h.free()
    return out, arrays, hst, int(host(st)[0])


def check_tree(parent, u, v, full_arrays=True):
    out, arr, hst, qst = run_gpu(parent, u, v)
    assert hst == 0 and qst == 0
    pre, depth, size, _ = oracle.tree_tour(parent)
    if full_arrays:
        assert (arr["pre"] == pre).all()
        assert (arr["depth"] == depth).all()
        assert (arr["size"] == size).all()
        order = np.empty_like(pre)
        order[pre] = np.arange(pre.shape[0], dtype=np.int32)
        assert (arr["order"] == order).all()
    want = oracle.lca_offline(parent, u, v)
    assert (out == want).all(), f"{(out != want).sum()} mismatches"


def test_fig1():
    g = json.load(open(os.path.join(GOLDEN, "fig1_euler_tour.json")))
    parent = np.array(g["parent"], np.int32)
    u = np.array([x[0] for x in g["lca"]], np.int32)
    v = np.array([x[1] for x in g["lca"]], np.int32)
    out, arr, hst, _ = run_gpu(parent, u, v)
    assert hst == 0
    assert out.tolist() == [x[2] for x in g["lca"]]
    assert [arr["pre"][int(k)] for k in g["pre"]] == list(g["pre"].values())
    assert [arr["depth"][int(k)] for k in g["depth"]] == list(g["depth"].values())
    assert [arr["size"][int(k)] for k in g["size"]] == list(g["size"].values())


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 255, 256, 257, 2047, 2048, 2049, 4097, 10007, 65537])
@pytest.mark.parametrize("grasp", [1, 3, 1024, None])
def test_random_trees(n, grasp):
    parent = synth.tree_parent(n, grasp, seed=n * 7 + (grasp or 0))
    u, v = synth.lca_queries(n, 3 * n + 11, seed=n)
    check_tree(parent, u, v)


def test_all_small_trees_exhaustive():
    import test_oracle_pins as pins
    for n in (2, 3, 4, 5):
        pairs = np.array([(a, b) for a in range(n) for b in range(n)], np.int32)
        for edges in pins.prufer_trees(n):
            for root in range(n):
                parent = pins.root_tree(n, edges, root)
                out, arr, hst, _ = run_gpu(parent, pairs[:, 0].copy(), pairs[:, 1].copy())
                assert hst == 0
                assert out.tolist() == oracle.lca_offline(parent, pairs[:, 0], pairs[:, 1]).tolist()


def test_star_and_unpermuted_path():
    n = 100003
    star = np.full(n, 77, np.int32)
    star[77] = -1
    u, v = synth.lca_queries(n, n, seed=1)
    check_tree(star, u, v)
    path = synth.tree_parent(n, 1, seed=1, permute=False)
    check_tree(path, u, v)
    out, _, _, _ = run_gpu(path, u, v)
    assert (out == np.minimum(u, v)).all()   # closed form on the path 0-1-2-...


def test_config_small():
    # the small LCA workload: random recursive tree n = 2^16, permuted labels, 2^16 uniform queries
    n = 1 << 16
    parent = synth.tree_parent(n, None, seed=1)
    u, v = synth.lca_queries(n, n, seed=1)
    check_tree(parent, u, v)
    _, depth, _, _ = oracle.tree_tour(parent)
    out, _, _, _ = run_gpu(parent, u, v)
    assert (out == oracle.lca_climb(parent, depth, u, v)).all()


@pytest.mark.parametrize("grasp", [None, 1024, 1])
def test_config_full_size(grasp):
    # the benchmark workload: n = 2^24, 2^24 uniform queries, all answers checked
    n = 1 << 24
    parent = synth.tree_parent(n, grasp, seed=1)
    u, v = synth.lca_queries(n, n, seed=1)
    check_tree(parent, u, v, full_arrays=(grasp is None))


def test_bad_trees_flagged():
    import paper_2103_15217_gb300 as etl
    u = np.array([0, 1, 2], np.int32)
    for parent in ([-1, -1, 0], [-1, 2, 1], [-1, 7, 0], [1, 0, 0], [-1, 1, 0]):
        h = etl.lca_preprocess(dev(np.array(parent, np.int32)))
        assert h.status() == 4
        out = host(h.query(dev(u), dev(u)))
        assert (out == -1).all()
        h.free()
    n = 50000   # a long cycle hidden in a big tree
    parent = synth.tree_parent(n, None, seed=3)
    kids = np.nonzero(parent >= 0)[0]
    a, b = kids[10], kids[20]
    parent[a], parent[b] = b, a
    h = etl.lca_preprocess(dev(parent))
    assert h.status() == 4
    h.free()


def test_bad_queries_flagged():
    import paper_2103_15217_gb300 as etl
    n = 1000
    parent = synth.tree_parent(n, None, seed=2)
    h = etl.lca_preprocess(dev(parent))
    u = np.array([0, -1, 5, n], np.int32)
    v = np.array([1, 2, n + 5, 3], np.int32)
    st = etl.new_status()
    out = host(h.query(dev(u), dev(v), status=st))
    assert out[1] == -1 and out[2] == -1 and out[3] == -1
    assert out[0] == oracle.lca_offline(parent, u[:1], v[:1])[0]
    assert host(st)[0] == 5
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    assert h.query(empty, empty).numel() == 0
    h.free()


def test_queries_on_other_stream_after_event():
    import paper_2103_15217_gb300 as etl
    n = 1 << 18
    parent = synth.tree_parent(n, 1024, seed=5)
    u, v = synth.lca_queries(n, n, seed=5)
    h = etl.lca_preprocess(dev(parent))
    ev = torch.cuda.Event()
    ev.record()
    s = torch.cuda.Stream()
    s.wait_event(ev)
    with torch.cuda.stream(s):
        du, dv = dev(u), dev(v)
        out = h.query(du, dv)
    s.synchronize()
    assert (out.cpu().numpy() == oracle.lca_offline(parent, u, v)).all()
    h.free()


@pytest.mark.parametrize("hub", [2, 63, 64, 65, 200, 5000])
def test_child_group_sizes(hub):
    # one node with `hub` children inside a random tree: exercises both the
    # in-place ordering of small sibling groups and the sorted fallback
    rng = np.random.default_rng(hub)
    n = 20000
    parent = synth.tree_parent(n, None, seed=hub)
    kids = rng.choice(np.nonzero(parent >= 0)[0], size=hub, replace=False)
    root = int(np.nonzero(parent == -1)[0][0])
    h_node = int(rng.choice(np.setdiff1d(np.arange(n), np.concatenate([kids, [root]]))))
    # re-hang the chosen nodes under h_node unless that would create a cycle (h_node below one of them)
    anc = set()
    x = h_node
    while x != -1:
        anc.add(x)
        x = int(parent[x])
    for c in kids:
        if int(c) not in anc:
            parent[c] = h_node
    u, v = synth.lca_queries(n, 3 * n, seed=hub)
    check_tree(parent, u, v)
