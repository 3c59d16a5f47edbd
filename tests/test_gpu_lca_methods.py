"""The paper's two other LCA methods on the GPU -- Inlabel (Schieber-Vishkin,
built on the Euler-tour results) and the naive climbing method -- against the
CPU oracle, element by element, and against the RMQ path."""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def all_methods(parent, u, v):
    import paper_2103_15217_gb300 as etl
    P, U, V = dev(parent), dev(u), dev(v)
    h = etl.lca_preprocess(P)
    h.build_inlabel(P)
    st = etl.new_status()
    rmq = host(h.query(U, V, status=st))
    inl = host(h.query_inlabel(U, V, status=st))
    assert h.status() == 0 and int(host(st)[0]) == 0
    h.free()
    st2 = etl.new_status()
    nv = etl.NaiveLca(P, status=st2)
    naive = host(nv.query(U, V, status=st2))
    assert int(host(st2)[0]) == 0
    return rmq, inl, naive


def test_fig1_all_methods():
    g = json.load(open(os.path.join(GOLDEN, "fig1_euler_tour.json")))
    parent = np.array(g["parent"], np.int32)
    u = np.array([x[0] for x in g["lca"]], np.int32)
    v = np.array([x[1] for x in g["lca"]], np.int32)
    want = [x[2] for x in g["lca"]]
    for out in all_methods(parent, u, v):
        assert out.tolist() == want


def test_exhaustive_small_trees():
    import test_oracle_pins as pins
    for n in (2, 3, 4, 5):
        pairs = np.array([(a, b) for a in range(n) for b in range(n)], np.int32)
        for edges in pins.prufer_trees(n):
            for root in range(n):
                parent = pins.root_tree(n, edges, root)
                want = oracle.lca_offline(parent, pairs[:, 0], pairs[:, 1]).tolist()
                for out in all_methods(parent, pairs[:, 0].copy(), pairs[:, 1].copy()):
                    assert out.tolist() == want


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1000, 4096, 4097, 65536, 100003])
@pytest.mark.parametrize("grasp", [1, 7, 1024, None])
def test_random_trees(n, grasp):
    parent = synth.tree_parent(n, grasp, seed=n + (grasp or 0))
    u, v = synth.lca_queries(n, 2 * n + 5, seed=n)
    want = oracle.lca_offline(parent, u, v)
    for out in all_methods(parent, u, v):
        assert (out == want).all()


def test_scale_free_star_and_path():
    for parent in (synth.ba_tree(50000, seed=3),
                   np.where(np.arange(30000) == 17, -1, 17).astype(np.int32),
                   synth.tree_parent(30000, 1, seed=2, permute=False)):
        n = parent.shape[0]
        u, v = synth.lca_queries(n, 3 * n, seed=4)
        want = oracle.lca_offline(parent, u, v)
        for out in all_methods(parent, u, v):
            assert (out == want).all()


@pytest.mark.parametrize("grasp", [None, 1024, 1])
def test_inlabel_full_size(grasp):
    import paper_2103_15217_gb300 as etl
    n = 1 << 24
    parent = synth.tree_parent(n, grasp, seed=1)
    u, v = synth.lca_queries(n, n, seed=1)
    P = dev(parent)
    h = etl.lca_preprocess(P)
    h.build_inlabel(P)
    out = host(h.query_inlabel(dev(u), dev(v)))
    h.free()
    assert (out == oracle.lca_offline(parent, u, v)).all()


def test_naive_full_size_shallow():
    import paper_2103_15217_gb300 as etl
    n = 1 << 24
    parent = synth.tree_parent(n, None, seed=1)
    u, v = synth.lca_queries(n, n, seed=1)
    out = host(etl.NaiveLca(dev(parent)).query(dev(u), dev(v)))
    assert (out == oracle.lca_offline(parent, u, v)).all()


def test_errors():
    import paper_2103_15217_gb300 as etl
    st = etl.new_status()
    nv = etl.NaiveLca(dev(np.array([-1, 2, 1], np.int32)), status=st)   # cycle 1 <-> 2
    assert int(host(st)[0]) == 4
    st = etl.new_status()
    etl.NaiveLca(dev(np.array([-1, -1, 0], np.int32)), status=st)        # two roots
    assert int(host(st)[0]) == 4
    h = etl.lca_preprocess_batch(dev(np.array([-1, 0, -1], np.int32)), dev(np.array([0, 2, 3], np.int32)), 2)
    with pytest.raises(etl.EtlError):
        h.build_inlabel(dev(np.array([-1, 0, -1], np.int32)))
    h.free()
    parent = synth.tree_parent(1000, None, seed=1)
    h = etl.lca_preprocess(dev(parent))
    with pytest.raises(etl.EtlError):                                     # structures not built yet
        h.query_inlabel(dev(np.zeros(4, np.int32)), dev(np.zeros(4, np.int32)))
    h.free()
    del nv


def test_inlabel_only_handle():
    import paper_2103_15217_gb300 as etl
    n = 70000
    parent = synth.tree_parent(n, 64, seed=9)
    u, v = synth.lca_queries(n, 2 * n, seed=9)
    h = etl.lca_preprocess(dev(parent), methods=("inlabel",))
    assert h.status() == 0
    out = host(h.query_inlabel(dev(u), dev(v)))
    assert (out == oracle.lca_offline(parent, u, v)).all()
    with pytest.raises(etl.EtlError):          # no sparse table in this handle
        h.query(dev(u), dev(v))
    arr = {k: host(t) for k, t in h.arrays().items()}
    pre, depth, size, _ = oracle.tree_tour(parent)
    assert (arr["pre"] == pre).all() and (arr["size"] == size).all()
    h.free()
    etl.trim()
