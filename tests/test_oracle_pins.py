"""Pins of the CPU oracle against things other than itself.

The oracle is checked here against the paper's worked example (Figures 1-2),
brute force on tiny inputs (all labelled rooted trees up to 6 nodes, random
multigraphs), closed forms (paths, stars, trees-as-graphs, cycles, the
planted cuts of the large-diameter graph) and invariants of the Euler tour
(Sec. 2). No GPU is involved.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import brute
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fig1():
    with open(os.path.join(GOLDEN, "fig1_euler_tour.json")) as f:
        return json.load(f)


def bracket_to_arc(parent, b):
    """Bracket 2v = arc (parent(v), v) going down, 2v+1 = arc (v, parent(v)) going up."""
    v = b // 2
    return (int(parent[v]), v) if b % 2 == 0 else (v, int(parent[v]))


# --------------------------------------------------------------------------- worked example


def test_fig1_tour_pre_depth_size():
    g = _fig1()
    parent = np.array(g["parent"], np.int32)
    pre, depth, size, tour = oracle.tree_tour(parent)
    root = g["root"]
    # the tour without the root's two virtual brackets is exactly the printed list of Figure 1
    arcs = [bracket_to_arc(parent, b) for b in tour if b // 2 != root]
    assert arcs == [tuple(a) for a in g["tour"]]
    assert tour[0] == 2 * root and tour[-1] == 2 * root + 1
    for k, val in g["pre"].items():
        assert pre[int(k)] == val
    for k, val in g["depth"].items():
        assert depth[int(k)] == val
    for k, val in g["size"].items():
        assert size[int(k)] == val


def test_fig2_dcel_arrays_and_successor():
    g = _fig1()
    A = g["A"]
    edges = np.array(A[0::2], np.int32)  # A holds the two halves of each undirected edge side by side
    succ, tour, B = oracle.dcel_tour(6, edges, g["root"])
    halves = [tuple(A[i]) for i in range(len(A))]
    assert [halves[b] for b in B] == [tuple(x) for x in g["B"]]
    # first[x]: the first half-edge of each source in B
    firsts = []
    seen = set()
    for b in B:
        if halves[b][0] not in seen:
            seen.add(halves[b][0])
            firsts.append(halves[b])
    assert firsts == [tuple(x) for x in g["first"]]
    assert [halves[a] for a in tour] == [tuple(x) for x in g["tour"]]
    # succ(6) = next(twin(6)) = next(1) = 7, with list positions numbered from 1
    pos = {int(a): i + 1 for i, a in enumerate(tour)}
    a6 = int(tour[g["succ_example"]["arc"] - 1])
    assert pos[int(succ[a6])] == g["succ_example"]["succ"]
    assert pos[a6 ^ 1] == g["succ_example"]["twin"]


def test_fig1_lca():
    g = _fig1()
    parent = np.array(g["parent"], np.int32)
    _, depth, _, _ = oracle.tree_tour(parent)
    u = np.array([x[0] for x in g["lca"]], np.int32)
    v = np.array([x[1] for x in g["lca"]], np.int32)
    want = np.array([x[2] for x in g["lca"]], np.int32)
    assert (oracle.lca_climb(parent, depth, u, v) == want).all()
    assert (oracle.lca_offline(parent, u, v) == want).all()
    assert [brute.lca(parent, a, b) for a, b in zip(u, v)] == list(want)


# --------------------------------------------------------------------------- exhaustive tiny trees


def prufer_trees(n):
    """All labelled trees on n >= 2 nodes (Pruefer decoding), as edge lists."""
    for seq in itertools.product(range(n), repeat=n - 2):
        degree = [1] * n
        for x in seq:
            degree[x] += 1
        edges = []
        for x in seq:
            leaf = min(i for i in range(n) if degree[i] == 1)
            edges.append((leaf, x))
            degree[leaf] -= 1
            degree[x] -= 1
        u, w = [i for i in range(n) if degree[i] == 1]
        edges.append((u, w))
        yield edges


def root_tree(n, edges, root):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    parent = [-2] * n
    parent[root] = -1
    stack = [root]
    while stack:
        x = stack.pop()
        for w in adj[x]:
            if parent[w] == -2:
                parent[w] = x
                stack.append(w)
    return np.array(parent, np.int32)


def check_tree_invariants(parent, pre, depth, size, tour):
    n = parent.shape[0]
    root = int(np.nonzero(parent == -1)[0][0])
    assert sorted(pre.tolist()) == list(range(n))           # preorder is a permutation
    assert size[root] == n and pre[root] == 0 and depth[root] == 0
    assert tour.shape[0] == 2 * n and sorted(tour.tolist()) == list(range(2 * n))  # every bracket once
    nonroot = np.nonzero(parent >= 0)[0]
    p = parent[nonroot]
    assert (depth[nonroot] == depth[p] + 1).all()
    assert ((pre[p] < pre[nonroot]) & (pre[nonroot] < pre[p] + size[p])).all()  # subtree = interval
    child_sum = np.zeros(n, np.int64)
    np.add.at(child_sum, p, size[nonroot])
    assert (child_sum == size.astype(np.int64) - 1).all()
    # Sec. 2: prefix sums of weights 1 (down) / 0 (up) give preorder, 1 / -1 give levels
    down = (tour % 2 == 0).astype(np.int64)
    pos = np.empty(2 * n, np.int64)
    pos[tour] = np.arange(2 * n)
    pre_scan = np.cumsum(down) - 1
    lvl_scan = np.cumsum(np.where(down == 1, 1, -1)) - 1
    assert (pre_scan[pos[2 * np.arange(n)]] == pre).all()
    assert (lvl_scan[pos[2 * np.arange(n)]] == depth).all()
    # a half-edge goes down iff it appears before its twin (Sec. 2, footnote)
    assert (pos[2 * np.arange(n)] < pos[2 * np.arange(n) + 1]).all()
    # subtree size from the two bracket positions
    assert ((pos[2 * np.arange(n) + 1] - pos[2 * np.arange(n)] + 1) // 2 == size).all()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_all_rooted_trees_bruteforce(n):
    trees = [[]] if n == 1 else list(prufer_trees(n))
    pairs = np.array(list(itertools.product(range(n), repeat=2)), np.int32)
    u, v = pairs[:, 0].copy(), pairs[:, 1].copy()
    count = 0
    for edges in trees:
        for root in range(n):
            parent = root_tree(n, edges, root) if n > 1 else np.array([-1], np.int32)
            pre, depth, size, tour = oracle.tree_tour(parent)
            check_tree_invariants(parent, pre, depth, size, tour)
            want = [brute.lca(parent, a, b) for a, b in pairs]
            assert oracle.lca_climb(parent, depth, u, v).tolist() == want
            assert oracle.lca_offline(parent, u, v).tolist() == want
            count += 1
    assert count == n ** (n - 1)  # Cayley: n^(n-1) rooted labelled trees


def test_all_rooted_trees_n7_lca():
    # every rooted labelled tree on 7 nodes (7^6 = 117,649) and all 49 query pairs: both LCA oracles
    # against the definition, the deepest common element of the two ancestor sets (kept as bit masks)
    n = 7
    pairs = np.array(list(itertools.product(range(n), repeat=2)), np.int32)
    u, v = pairs[:, 0].copy(), pairs[:, 1].copy()
    count = 0
    for edges in prufer_trees(n):
        for root in range(n):
            parent = root_tree(n, edges, root)
            anc, dep = [0] * n, [0] * n
            for x in range(n):  # ancestor set (x included) and depth by climbing
                y, d = x, 0
                while y != -1:
                    anc[x] |= 1 << y
                    y = int(parent[y])
                    d += 1
                dep[x] = d
            want = []
            for a_, b_ in pairs.tolist():
                common = anc[a_] & anc[b_]
                want.append(max((z for z in range(n) if common >> z & 1), key=lambda z: dep[z]))
            pre, depth, size, tour = oracle.tree_tour(parent)
            assert oracle.lca_climb(parent, depth, u, v).tolist() == want
            assert oracle.lca_offline(parent, u, v).tolist() == want
            count += 1
    assert count == n ** (n - 1)


# --------------------------------------------------------------------------- random trees


@pytest.mark.parametrize("grasp", [1, 2, 16, 1024, None])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_trees(grasp, seed):
    n = 3000
    parent = synth.tree_parent(n, grasp, seed=seed)
    pre, depth, size, tour = oracle.tree_tour(parent)
    check_tree_invariants(parent, pre, depth, size, tour)
    u, v = synth.lca_queries(n, 5000, seed=seed)
    a = oracle.lca_climb(parent, depth, u, v)
    b = oracle.lca_offline(parent, u, v)
    assert (a == b).all()
    idx = np.random.default_rng(seed).choice(5000, 60, replace=False)
    assert [brute.lca(parent, u[i], v[i]) for i in idx] == a[idx].tolist()
    # the answer is a common ancestor no deeper than either endpoint (interval test)
    for x in (u, v):
        assert ((pre[a] <= pre[x]) & (pre[x] < pre[a] + size[a])).all()
    assert (depth[a] <= np.minimum(depth[u], depth[v])).all()


@pytest.mark.parametrize("grasp", [1, 4, None])
def test_rmq_reading_over_preorder(grasp):
    # the RMQ form the GPU path uses, checked against brute-force LCAs: with Q[i] = pre(parent(node at
    # preorder i)), min Q over (pre x, pre y] is pre(LCA) for pre x < pre y; when x is not an ancestor
    # of y, Q[pre x] >= pre(LCA) too, so the range may start at pre x; when it is, x is the LCA
    n = 400
    parent = synth.tree_parent(n, grasp, seed=11)
    pre, depth, size, _ = oracle.tree_tour(parent)
    order = np.empty(n, np.int64)
    order[pre] = np.arange(n)
    Q = np.array([pre[parent[order[i]]] if parent[order[i]] >= 0 else -1 for i in range(n)])
    u, v = synth.lca_queries(n, 600, seed=12)
    for a, b in zip(u.tolist(), v.tolist()):
        if a == b:
            continue
        x, y = (a, b) if pre[a] < pre[b] else (b, a)
        want = brute.lca(parent, a, b)
        assert order[Q[pre[x] + 1: pre[y] + 1].min()] == want
        if pre[y] < pre[x] + size[x]:
            assert want == x
        else:
            assert order[Q[pre[x]: pre[y] + 1].min()] == want


@pytest.mark.parametrize("grasp", [1, 3, 1024, None])
def test_original_label_climbing(grasp):
    # before the relabelling every parent has a smaller label than its child, so climbing from the
    # larger of the two labels until they meet is exact and needs no depths (an independent LCA)
    n = 20000
    parent = synth.tree_parent(n, grasp, seed=21, permute=False)
    u, v = synth.lca_queries(n, 3000, seed=22)
    want = []
    for a, b in zip(u.tolist(), v.tolist()):
        while a != b:
            if a > b:
                a = int(parent[a])
            else:
                b = int(parent[b])
        want.append(a)
    assert oracle.lca_offline(parent, u, v).tolist() == want
    _, depth, _, _ = oracle.tree_tour(parent)
    assert oracle.lca_climb(parent, depth, u, v).tolist() == want


def test_path_closed_form():
    n = 5000
    parent = synth.tree_parent(n, 1, seed=4, permute=False)
    assert (parent[1:] == np.arange(n - 1)).all()   # grasp 1 gives the path 0-1-2-...
    u, v = synth.lca_queries(n, 20000, seed=4)
    want = np.minimum(u, v)                         # on a path rooted at 0 the LCA is the smaller label
    pre, depth, size, _ = oracle.tree_tour(parent)
    assert (oracle.lca_climb(parent, depth, u, v) == want).all()
    assert (oracle.lca_offline(parent, u, v) == want).all()
    assert (depth == np.arange(n)).all() and (size == n - np.arange(n)).all()


def test_star_closed_form():
    n = 4000
    center = 1234
    parent = np.full(n, center, np.int32)
    parent[center] = -1
    u, v = synth.lca_queries(n, 20000, seed=5)
    want = np.where(u == v, u, center)
    pre, depth, size, _ = oracle.tree_tour(parent)
    assert (oracle.lca_climb(parent, depth, u, v) == want).all()
    assert (oracle.lca_offline(parent, u, v) == want).all()
    leaves = np.delete(np.arange(n), center)
    assert (pre[leaves] == np.arange(1, n)).all()   # ascending child order


def test_bad_trees_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.tree_tour(np.array([-1, -1, 0], np.int32))   # two roots
    with pytest.raises(oracle.OracleError):
        oracle.tree_tour(np.array([-1, 2, 1], np.int32))    # cycle 1 <-> 2
    with pytest.raises(oracle.OracleError):
        oracle.tree_tour(np.array([-1, 7, 0], np.int32))    # out of range
    with pytest.raises(oracle.OracleError):
        oracle.tree_tour(np.array([0, 0], np.int32))        # no root / self-parent


def test_generator_average_depth():
    # Sec. 3.2: expected average depth ln n for unlimited grasp and n/(grasp+1) + O(1) for a
    # finite grasp. With a 0-based root, node i has expected depth H_i, so the exact mean of
    # the average is H_{n-1} - 1 + 1/n; the average of one tree fluctuates by about 0.6, so
    # several seeds are averaged.
    n = 1 << 14
    seeds = range(1, 9)
    avg = np.mean([oracle.tree_tour(synth.tree_parent(n, None, seed=s))[1].mean() for s in seeds])
    exact = sum(1.0 / k for k in range(1, n)) - 1 + 1 / n
    assert abs(avg - exact) < 0.75
    assert abs(avg - math.log(n)) < 0.42 + 0.75
    for grasp in (16, 256):
        avg = np.mean([oracle.tree_tour(synth.tree_parent(n, grasp, seed=s))[1].mean() for s in seeds])
        assert abs(avg - n / (grasp + 1)) < 3 + 0.05 * n / (grasp + 1)


# --------------------------------------------------------------------------- bridges


def random_multigraph(rng, n, m):
    e = rng.integers(0, n, size=(m, 2)).astype(np.int32)
    if m >= 2 and rng.random() < 0.5:
        e[1] = e[0][::-1]               # a parallel pair
    if m >= 3 and rng.random() < 0.5:
        e[2] = [e[2][0], e[2][0]]       # a self-loop
    return e


def random_spanning_forest(rng, n, edges):
    """A spanning forest picked by Kruskal over a random edge order."""
    order = rng.permutation(edges.shape[0])
    uf = list(range(n))

    def find(x):
        while uf[x] != x:
            uf[x] = uf[uf[x]]
            x = uf[x]
        return x

    tree = np.zeros(edges.shape[0], np.uint8)
    for e in order:
        a, b = find(int(edges[e, 0])), find(int(edges[e, 1]))
        if a != b:
            uf[a] = b
            tree[e] = 1
    return tree


def test_bridges_bruteforce_random_multigraphs():
    rng = np.random.default_rng(11)
    for trial in range(600):
        n = int(rng.integers(1, 11))
        m = int(rng.integers(0, 16))
        edges = random_multigraph(rng, n, m)
        want = brute.bridges(n, edges)
        assert oracle.bridges_dfs(n, edges).tolist() == want, (n, edges)
        assert oracle.bridges_tv(n, edges).tolist() == want
        for _ in range(3):
            tree = random_spanning_forest(rng, n, edges)
            assert oracle.bridges_tv(n, edges, tree).tolist() == want


def test_bridges_closed_forms():
    rng = np.random.default_rng(3)
    # a tree: every edge is a bridge
    parent = synth.tree_parent(2000, None, seed=3)
    child = np.nonzero(parent >= 0)[0]
    tree_edges = np.stack([child, parent[child]], 1).astype(np.int32)
    assert oracle.bridges_dfs(2000, tree_edges).all()
    assert oracle.bridges_tv(2000, tree_edges).all()
    # a cycle: no bridges; plus a pendant path: exactly its edges
    n = 1000
    cyc = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    assert not oracle.bridges_dfs(n, cyc).any()
    tail = np.array([[0, n], [n, n + 1]], np.int32)
    g = np.concatenate([cyc, tail])[rng.permutation(n + 2)]
    got = oracle.bridges_dfs(n + 2, g)
    assert got.sum() == 2 and set(map(tuple, g[got == 1].tolist())) == {(0, n), (n, n + 1)}
    # a parallel copy of a tree edge makes it a non-bridge
    dup = np.concatenate([tree_edges, tree_edges[:1]])
    got = oracle.bridges_dfs(2000, dup)
    assert got[0] == 0 and got[-1] == 0 and got[1:-1].all()


def path_coverage_bridges(n, edges):
    """Closed form for the large-diameter graph: path edge (j, j+1) is a bridge iff
    no chord (i, i+d) with i <= j < i+d covers it (difference array over j)."""
    a = np.minimum(edges[:, 0], edges[:, 1]).astype(np.int64)
    b = np.maximum(edges[:, 0], edges[:, 1]).astype(np.int64)
    chord = (b - a) >= 2
    diff = np.zeros(n + 1, np.int64)
    np.add.at(diff, a[chord], 1)
    np.add.at(diff, b[chord], -1)
    covered = np.cumsum(diff)[: n - 1] > 0
    is_path = (b - a) == 1
    want = np.zeros(edges.shape[0], np.uint8)
    want[is_path] = ~covered[a[is_path]]
    return want


@pytest.mark.parametrize("seed", [1, 2])
def test_hard_graph_closed_form(seed):
    n = 1 << 14
    edges = synth.hard_graph(n, 1 << 16, 1 << 8, seed=seed)
    want = path_coverage_bridges(n, edges)
    assert want.sum() >= 1 << 8
    assert (oracle.bridges_dfs(n, edges) == want).all()
    assert (oracle.bridges_tv(n, edges) == want).all()


def test_easy_graph_agreement_and_count_identity():
    n = 1 << 13
    edges = synth.easy_graph(n, 3 * n, seed=7)
    a = oracle.bridges_dfs(n, edges)
    b = oracle.bridges_tv(n, edges)
    assert (a == b).all()
    # removing all bridges raises the component count by exactly their number
    keep = edges[a == 0]
    assert brute.components(n, keep) - brute.components(n, edges) == int(a.sum())
    # a vertex of degree 1 hangs on a bridge
    deg = np.bincount(edges.ravel(), minlength=n)
    for e in np.nonzero((deg[edges[:, 0]] == 1) | (deg[edges[:, 1]] == 1))[0]:
        if edges[e, 0] != edges[e, 1]:
            assert a[e] == 1


def test_bad_graph_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.bridges_dfs(3, np.array([[0, 3]], np.int32))
    with pytest.raises(oracle.OracleError):   # marked edges with a cycle are not a forest
        oracle.bridges_tv(3, np.array([[0, 1], [1, 2], [2, 0]], np.int32), np.ones(3, np.uint8))


# --------------------------------------------------------------------------- 2-edge-connected components


def test_two_edge_cc_bruteforce():
    rng = np.random.default_rng(17)
    for trial in range(300):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, 12))
        edges = random_multigraph(rng, n, m)
        assert oracle.two_edge_cc(n, edges).tolist() == brute.two_edge_cc(n, edges), (n, edges.tolist())


def test_two_edge_cc_closed_forms():
    # a cycle is one component; a tree is all singletons; two cycles joined by a bridge: two components
    n = 500
    cyc = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int32)
    assert (oracle.two_edge_cc(n, cyc) == 0).all()
    parent = synth.tree_parent(n, None, seed=2)
    c = np.nonzero(parent >= 0)[0]
    assert (oracle.two_edge_cc(n, np.stack([c, parent[c]], 1)) == np.arange(n)).all()
    two = np.concatenate([cyc[:, :] % 250 + 0, (cyc % 250) + 250, [[3, 400]]]).astype(np.int32)
    lab = oracle.two_edge_cc(500, two)
    assert (lab[:250] == 0).all() and (lab[250:] == 250).all()
