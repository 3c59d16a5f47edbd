"""LCA by range minimum over the depth-annotated Euler tour (the classical
reduction named in Sec. 3.1), through the C ABI, against the CPU oracle: the
worked example of Fig. 1, every small rooted tree, random trees of all shapes
with sizes around the 32-entry blocks of the table (the tour has 2n
positions), error cases, and the full-size benchmark tree."""

import json
import os

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tour_lca(parent, u, v, methods=("tour_rmq",)):
    import paper_2103_15217_gb300 as etl
    h = etl.lca_preprocess(dev(parent), methods=methods)
    st = etl.new_status()
    out = host(h.query_tour(dev(u), dev(v), status=st))
    hst = h.status()
    h.free()
    return out, hst, int(host(st)[0])


def test_fig1():
    g = json.load(open(os.path.join(GOLDEN, "fig1_euler_tour.json")))
    parent = np.array(g["parent"], np.int32)
    u = np.array([x[0] for x in g["lca"]], np.int32)
    v = np.array([x[1] for x in g["lca"]], np.int32)
    out, hst, qst = tour_lca(parent, u, v)
    assert hst == 0 and qst == 0
    assert out.tolist() == [x[2] for x in g["lca"]]


def test_all_small_trees_exhaustive():
    import test_oracle_pins as pins
    for n in (1, 2, 3, 4, 5):
        pairs = np.array([(a, b) for a in range(n) for b in range(n)], np.int32)
        for edges in (pins.prufer_trees(n) if n > 1 else [[]]):
            for root in range(n):
                parent = pins.root_tree(n, edges, root) if n > 1 else np.array([-1], np.int32)
                out, hst, qst = tour_lca(parent, pairs[:, 0].copy(), pairs[:, 1].copy())
                assert hst == 0 and qst == 0
                assert out.tolist() == oracle.lca_offline(parent, pairs[:, 0], pairs[:, 1]).tolist()


@pytest.mark.parametrize("n", [2, 15, 16, 17, 31, 32, 33, 1000, 1024, 4097, 65537])
@pytest.mark.parametrize("grasp", [1, 4, None])
def test_random_trees(n, grasp):
    parent = synth.tree_parent(n, grasp, seed=3 * n + (grasp or 0))
    u, v = synth.lca_queries(n, 3 * n + 5, seed=n + 1)
    out, hst, qst = tour_lca(parent, u, v, methods=("rmq", "tour_rmq"))
    assert hst == 0 and qst == 0
    want = oracle.lca_offline(parent, u, v)
    assert (out == want).all(), f"{(out != want).sum()} mismatches"


def test_star_and_scale_free():
    n = 40000
    star = np.full(n, 5, np.int32)
    star[5] = -1
    u, v = synth.lca_queries(n, n, seed=2)
    out, hst, _ = tour_lca(star, u, v)
    assert hst == 0 and (out == oracle.lca_offline(star, u, v)).all()
    ba = synth.ba_tree(n, seed=2)
    out, hst, _ = tour_lca(ba, u, v)
    assert hst == 0 and (out == oracle.lca_offline(ba, u, v)).all()


def test_errors():
    import paper_2103_15217_gb300 as etl
    parent = synth.tree_parent(1000, None, seed=1)
    h = etl.lca_preprocess(dev(parent))                       # no tour table in this handle
    with pytest.raises(etl.EtlError):
        h.query_tour(dev(np.zeros(4, np.int32)), dev(np.zeros(4, np.int32)))
    h.free()
    with pytest.raises(ValueError):
        etl.lca_preprocess(dev(parent), methods=("tour",))
    out, _, qst = tour_lca(parent, np.array([0, 1000], np.int32), np.array([1, 2], np.int32))
    assert qst == 5 and out[1] == -1                          # id out of range: ETL_EBADQUERY, -1
    bad = np.array([-1, 2, 1, 0], np.int32)                   # a cycle 1 <-> 2 beside the root
    out, hst, _ = tour_lca(bad, np.array([0, 3], np.int32), np.array([3, 1], np.int32))
    assert hst == 4 and (out == -1).all()


def test_full_size():
    # the benchmark's random recursive tree: n = 2^24, 2^22 uniform queries, all checked
    n = 1 << 24
    parent = synth.tree_parent(n, None, seed=1)
    u, v = synth.lca_queries(n, 1 << 22, seed=1)
    out, hst, qst = tour_lca(parent, u, v)
    assert hst == 0 and qst == 0
    assert (out == oracle.lca_offline(parent, u, v)).all()
