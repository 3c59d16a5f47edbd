"""The seeded generators (host logic): the same seed gives the same arrays,
different seeds or streams give different ones, and every array has the
shape, dtype, value range and structure its recipe states."""

import numpy as np
import pytest

import synth
from synth.generators import batched_instances, make_graph, make_tree, serving_stream


@pytest.mark.parametrize("grasp", [1, 7, None])
def test_tree_parent_recipe(grasp):
    n = 5000
    a = synth.tree_parent(n, grasp, seed=3)
    assert a.dtype == np.int32 and a.shape == (n,)
    assert (a == synth.tree_parent(n, grasp, seed=3)).all()
    assert not (a == synth.tree_parent(n, grasp, seed=4)).all()
    assert (a == -1).sum() == 1 and ((a >= -1) & (a < n)).all()
    raw = synth.tree_parent(n, grasp, seed=3, permute=False)
    i = np.arange(1, n)
    lo = 0 if grasp is None else np.maximum(0, i - grasp)
    assert raw[0] == -1 and ((raw[1:] >= lo) & (raw[1:] < i)).all()  # parent(i) in [max(0, i - grasp), i)
    # the permuted tree is the unpermuted one relabelled: same multiset of child counts
    assert sorted(np.bincount(a[a >= 0], minlength=n)) == sorted(np.bincount(raw[raw >= 0], minlength=n))


def test_queries_and_graphs():
    u, v = synth.lca_queries(1000, 3000, seed=5)
    assert u.dtype == v.dtype == np.int32 and u.shape == v.shape == (3000,)
    assert ((u >= 0) & (u < 1000) & (v >= 0) & (v < 1000)).all()
    e = synth.easy_graph(1000, 4000, seed=5)
    assert e.dtype == np.int32 and e.shape == (4000, 2) and ((e >= 0) & (e < 1000)).all()
    assert (e == synth.easy_graph(1000, 4000, seed=5)).all()
    h = synth.hard_graph(1000, 2000, 10, seed=5)
    assert h.shape == (999 + 2000, 2)
    d = np.abs(h[:, 0].astype(np.int64) - h[:, 1])
    assert ((d >= 1) & (d <= 16)).all() and (d == 1).sum() == 999  # the path plus chords of length 2..16
    b = synth.ba_tree(2000, seed=5)
    assert (b == -1).sum() == 1 and b.dtype == np.int32


def test_batched_and_serving_descriptors():
    trees, graphs = batched_instances(seed=2, ntrees=30, ngraphs=30)
    assert len(trees) == len(graphs) == 30
    assert all(2 ** 6 <= t["n"] <= 2 ** 18 and t["q"] == t["n"] for t in trees)
    assert [t["grasp"] for t in trees[:3]] == [1, 1024, None]
    assert all(g["m"] == 4 * g["n"] and g["kind"] == ("easy" if i % 2 == 0 else "hard") for i, g in enumerate(graphs))
    p, u, v = make_tree(trees[0])
    assert p.shape == (trees[0]["n"],) and u.shape == (trees[0]["q"],)
    assert make_graph(graphs[1]).shape == (graphs[1]["m"], 2)
    rt, reqs = serving_stream(seed=2, nrequests=200, ntrees=16)
    assert len(rt) == 16 and len(reqs) == 200
    ts = [r["t"] for r in reqs]
    assert ts == sorted(ts) and ts[0] == 0.0
    assert all(r["kind"] in ("lca", "bridges") for r in reqs)
