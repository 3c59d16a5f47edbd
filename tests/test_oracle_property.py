"""Property-based pins of the oracle (CPU only): hypothesis draws small trees
and multigraphs -- including the degenerate ones: one node, no edges, only
self-loops, stacks of parallel edges, many components -- and the oracle must
agree with brute force from the definitions (ancestor sets for LCA, deleting
each edge for bridges, pairwise reachability for 2-edge-connected
components) and with its own invariants (Sec. 2: tour length, preorder a
permutation, subtrees are preorder intervals)."""

import numpy as np
import pytest

pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

from oracle import brute  # noqa: E402
import oracle  # noqa: E402


@st.composite
def trees(draw, max_n=24):
    """A parent array: node labels permuted, parents drawn among earlier nodes of the permutation."""
    n = draw(st.integers(1, max_n))
    order = draw(st.permutations(list(range(n))))
    parent = [-1] * n
    for i in range(1, n):
        parent[order[i]] = order[draw(st.integers(0, i - 1))]
    return np.array(parent, np.int32)


@st.composite
def multigraphs(draw, max_n=9, max_m=14):
    n = draw(st.integers(1, max_n))
    m = draw(st.integers(0, max_m))
    ends = st.integers(0, n - 1)
    edges = [(draw(ends), draw(ends)) for _ in range(m)]
    return n, np.array(edges, np.int32).reshape(-1, 2)


@settings(max_examples=300, deadline=None)
@given(trees(), st.data())
def test_lca_oracles_match_ancestor_sets(parent, data):
    n = parent.shape[0]
    q = data.draw(st.integers(1, 40))
    u = np.array(data.draw(st.lists(st.integers(0, n - 1), min_size=q, max_size=q)), np.int32)
    v = np.array(data.draw(st.lists(st.integers(0, n - 1), min_size=q, max_size=q)), np.int32)
    want = [brute.lca(parent.tolist(), int(a), int(b)) for a, b in zip(u, v)]
    assert oracle.lca_offline(parent, u, v).tolist() == want
    pre, depth, size, tour = oracle.tree_tour(parent)
    assert oracle.lca_climb(parent, depth, u, v).tolist() == want
    # Sec. 2 invariants: 2n brackets, each once; preorder is a permutation; subtree = preorder interval
    assert sorted(tour.tolist()) == list(range(2 * n))
    assert sorted(pre.tolist()) == list(range(n))
    for c in range(n):
        p = parent[c]
        if p >= 0:
            assert depth[c] == depth[p] + 1
            assert pre[p] < pre[c] < pre[p] + size[p] and pre[c] + size[c] <= pre[p] + size[p]


@settings(max_examples=400, deadline=None)
@given(multigraphs())
def test_bridge_oracles_match_edge_deletion(g):
    n, edges = g
    want = brute.bridges(n, edges.tolist())
    assert oracle.bridges_dfs(n, edges).tolist() == want
    assert oracle.bridges_tv(n, edges).tolist() == want
    assert oracle.two_edge_cc(n, edges).tolist() == brute.two_edge_cc(n, edges.tolist())
