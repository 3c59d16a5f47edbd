"""The radix passes that group children by parent give the same, oracle-equal
preorder under every tile size and digit-ranking method (ballots or
__match_any_sync): the grouping is a stable sort, so pre / depth / size and
the LCA answers do not depend on how it is computed."""

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture
def restore_tuning():
    import paper_2103_15217_gb300 as etl
    old = etl.tune_get()
    yield
    etl.tune_set(sort_rounds=old["sort_rounds"], sort_ballot=old["sort_ballot"])


@pytest.mark.parametrize("rounds", [8, 16])
@pytest.mark.parametrize("ballot", [0, 1])
def test_sort_forms(restore_tuning, rounds, ballot):
    import paper_2103_15217_gb300 as etl
    etl.tune_set(sort_rounds=rounds, sort_ballot=ballot)
    for n, grasp in ((1, None), (2047, None), (2049, 3), (4097, 1), (70001, None), (300000, 1024)):
        parent = synth.tree_parent(n, grasp, seed=n + rounds)
        u, v = synth.lca_queries(n, n + 3, seed=n)
        h = etl.lca_preprocess(dev(parent))
        out = host(h.query(dev(u), dev(v)))
        arr = {k: host(t) for k, t in h.arrays().items()}
        assert h.status() == 0
        h.free()
        pre, depth, size, _ = oracle.tree_tour(parent)
        assert (arr["pre"] == pre).all() and (arr["depth"] == depth).all() and (arr["size"] == size).all()
        assert (out == oracle.lca_offline(parent, u, v)).all()
    star = np.full(5000, 0, np.int32)   # one parent with every other node as a child: one long digit run
    star[0] = -1
    h = etl.lca_preprocess(dev(star))
    pre = host(h.arrays()["pre"])
    h.free()
    assert (pre == oracle.tree_tour(star)[0]).all()
