"""Both range-minimum table forms (blocked two-level, full sparse table) give
the oracle's answers: LCA queries whose preorder ranges fall inside one block
of 32, straddle two blocks, or span many, on trees whose sizes sit around the
block size; and bridge masks, where most subtree ranges are short."""

import numpy as np
import pytest

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(params=[1, 0], ids=["blocked", "full"])
def rmq_form(request):
    import paper_2103_15217_gb300 as etl
    old = etl.tune_get()["rmq_blocked"]
    etl.tune_set(rmq_blocked=request.param)
    yield request.param
    etl.tune_set(rmq_blocked=old)


def near_pairs(pre, count, span, seed):
    """Node pairs whose preorder numbers differ by at most span."""
    n = pre.shape[0]
    order = np.empty_like(pre)
    order[pre] = np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, count)
    b = np.clip(a + rng.integers(-span, span + 1, count), 0, n - 1)
    return order[a].astype(np.int32), order[b].astype(np.int32)


@pytest.mark.parametrize("n", [2, 31, 32, 33, 63, 64, 65, 95, 1023, 1024, 1025, 4095, 33000])
@pytest.mark.parametrize("grasp", [1, 8, None])
def test_lca_both_forms(rmq_form, n, grasp):
    import paper_2103_15217_gb300 as etl
    parent = synth.tree_parent(n, grasp, seed=n + (grasp or 0))
    pre, _, _, _ = oracle.tree_tour(parent)
    u1, v1 = synth.lca_queries(n, 2 * n + 7, seed=n)
    u2, v2 = near_pairs(pre, 2 * n + 7, 40, seed=n)
    u = np.concatenate([u1, u2])
    v = np.concatenate([v1, v2])
    h = etl.lca_preprocess(dev(parent))
    st = etl.new_status()
    out = host(h.query(dev(u), dev(v), status=st))
    assert h.status() == 0 and int(host(st)[0]) == 0
    h.free()
    want = oracle.lca_offline(parent, u, v)
    assert (out == want).all(), f"{(out != want).sum()} mismatches"


def test_lca_batch_both_forms(rmq_form):
    import paper_2103_15217_gb300 as etl
    sizes = [1, 2, 31, 32, 33, 100, 1000, 5000, 64]
    parents, us, vs, insts, off = [], [], [], [], [0]
    for i, n in enumerate(sizes):
        p = synth.tree_parent(n, [1, 8, None][i % 3], seed=i)
        u, v = synth.lca_queries(n, 3 * n, seed=i)
        parents.append(p)
        us.append(u)
        vs.append(v)
        insts.append(np.full(u.shape[0], i, np.int32))
        off.append(off[-1] + n)
    h = etl.lca_preprocess_batch(dev(np.concatenate(parents)), dev(np.array(off, np.int32)), max(sizes))
    out = host(h.query_batch(dev(np.concatenate(insts)), dev(np.concatenate(us)), dev(np.concatenate(vs))))
    assert h.status() == 0
    h.free()
    pos = 0
    for p, u, v in zip(parents, us, vs):
        k = u.shape[0]
        assert (out[pos:pos + k] == oracle.lca_offline(p, u, v)).all()
        pos += k


@pytest.mark.parametrize("n", [3, 33, 65, 1025, 20000])
@pytest.mark.parametrize("kind", ["easy", "hard", "tree"])
def test_bridges_both_forms(rmq_form, n, kind):
    import paper_2103_15217_gb300 as etl
    if kind == "hard" and n < 20:
        pytest.skip("chords of length up to 16 need n >= 20")
    if kind == "easy":
        edges = synth.easy_graph(n, 2 * n, seed=n)
    elif kind == "hard":
        edges = synth.hard_graph(n, n, max(1, n // 32), seed=n)
    else:
        p = synth.tree_parent(n, 4, seed=n)
        c = np.nonzero(p >= 0)[0]
        edges = np.stack([c, p[c]], 1).astype(np.int32)
    st = etl.new_status()
    got = host(etl.find_bridges(dev(edges), n, status=st))
    assert int(host(st)[0]) == 0
    want = oracle.bridges_dfs(n, edges)
    assert (got == want).all(), f"{(got != want).sum()} mismatches"
