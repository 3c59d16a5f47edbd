"""Seeded generators for the paper's synthetic workloads.

Trees follow the paper's LCA dataset recipe (Sec. 3.2, "Datasets"): node 0 is
the root and every later node i picks its parent uniformly from the previous
``grasp`` nodes (all previous nodes when the grasp is unlimited); the labels are
then mapped through a random permutation and queries are uniform pairs.

Graphs stand in for the bridge datasets of Table 1 (Sec. 4.2), which are not
available here: ``easy_graph`` is a random spanning tree plus uniform extra
edges (small diameter, like the Kronecker and social graphs), ``hard_graph`` is
a path with short chords and planted uncovered path edges (large diameter and
many bridges, like the road graphs).

Everything is int32 and drawn from numpy's PCG64, seeded from (seed, stream)
so that independent draws never share a stream.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "tree_parent",
    "lca_queries",
    "easy_graph",
    "hard_graph",
    "ba_tree",
    "batched_instances",
    "serving_stream",
    "make_tree",
    "make_graph",
]

# stream ids: one per kind of draw, so that changing one draw never shifts another
_S_TREE, _S_PERM, _S_QUERY, _S_GRAPH, _S_BATCH, _S_SERVE, _S_BA = range(7)


def _rng(seed: int, stream: int, *extra: int) -> np.random.Generator:
    ss = np.random.SeedSequence([int(seed) & 0xFFFFFFFF, int(stream), *[int(x) for x in extra]])
    return np.random.Generator(np.random.PCG64(ss))


def tree_parent(n: int, grasp: int | None = None, seed: int = 1, permute: bool = True) -> np.ndarray:
    """Parent array of a random tree with ``n`` nodes (root marked by -1).

    Before relabelling, node 0 is the root and node i >= 1 has its parent drawn
    uniformly from ``[max(0, i - grasp), i)``; ``grasp=None`` means unlimited,
    i.e. ``[0, i)`` (random recursive tree, expected average depth about ln n),
    ``grasp=1`` gives a path. This is the paper's grasp model (Sec. 3.2) with
    0-based labels. With ``permute`` the labels are mapped through a seeded
    random permutation, as the paper does before handing trees to algorithms.
    """
    n = int(n)
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = _rng(seed, _S_TREE, n, 0 if grasp is None else int(grasp))
    i = np.arange(1, n, dtype=np.int64)
    lo = np.zeros_like(i) if grasp is None else np.maximum(0, i - int(grasp))
    par = lo + rng.integers(0, i - lo) if n > 1 else np.zeros(0, dtype=np.int64)
    parent = np.empty(n, dtype=np.int64)
    parent[0] = -1
    parent[1:] = par
    if permute:
        perm = _rng(seed, _S_PERM, n).permutation(n)  # old label -> new label
        out = np.empty(n, dtype=np.int64)
        out[perm[1:]] = perm[par]
        out[perm[0]] = -1
        parent = out
    return parent.astype(np.int32)


def lca_queries(n: int, q: int, seed: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """``q`` query pairs drawn uniformly from [0, n) x [0, n) (Sec. 3.2)."""
    rng = _rng(seed, _S_QUERY, int(n), int(q))
    u = rng.integers(0, n, size=int(q), dtype=np.int64).astype(np.int32)
    v = rng.integers(0, n, size=int(q), dtype=np.int64).astype(np.int32)
    return u, v


def _shuffle_orient(rng: np.random.Generator, edges: np.ndarray) -> np.ndarray:
    m = edges.shape[0]
    edges = edges[rng.permutation(m)]
    flip = rng.integers(0, 2, size=m).astype(bool)
    edges[flip] = edges[flip][:, ::-1]
    return np.ascontiguousarray(edges.astype(np.int32))


def easy_graph(n: int, m: int, seed: int = 1) -> np.ndarray:
    """Small-diameter graph: random spanning tree plus ``m - (n - 1)`` uniform edges.

    The spanning tree is a random recursive tree on permuted labels; the extra
    endpoints are independent and uniform, so self-loops and parallel edges are
    kept. The edge list is shuffled and each edge randomly oriented. Returns an
    int32 array of shape (m, 2).
    """
    n, m = int(n), int(m)
    if n < 1 or m < n - 1:
        raise ValueError("need n >= 1 and m >= n - 1")
    rng = _rng(seed, _S_GRAPH, 0, n, m)
    parent = tree_parent(n, None, seed=int(rng.integers(0, 2**31)), permute=True)
    child = np.nonzero(parent >= 0)[0]
    tree = np.stack([child, parent[child]], axis=1).astype(np.int64)
    k = m - (n - 1)
    extra = rng.integers(0, n, size=(k, 2), dtype=np.int64)
    return _shuffle_orient(rng, np.concatenate([tree, extra], axis=0))


def hard_graph(n: int, extra: int, ncut: int, seed: int = 1, dmin: int = 2, dmax: int = 16) -> np.ndarray:
    """Large-diameter graph: path 0..n-1 plus ``extra`` chords (i, i+d).

    ``ncut`` distinct path edges (j, j+1) are chosen first; every chord is drawn
    with d uniform in [dmin, dmax] and i uniform in [0, n-1-d], and redrawn if
    it would jump over a chosen path edge, so those stay uncovered and are
    bridges. Labels are not permuted; the edge list is shuffled and randomly
    oriented. Returns an int32 array of shape (n - 1 + extra, 2).
    """
    n, extra, ncut = int(n), int(extra), int(ncut)
    if n < dmax + 2:
        raise ValueError("n too small for the chord lengths")
    if not 0 <= ncut <= n - 1:
        raise ValueError("ncut out of range")
    rng = _rng(seed, _S_GRAPH, 1, n, extra, ncut)
    cuts = np.sort(rng.choice(n - 1, size=ncut, replace=False)).astype(np.int64)
    chords = np.empty((0, 2), dtype=np.int64)
    need = extra
    while need > 0:
        k = int(need * 1.25) + 64
        d = rng.integers(dmin, dmax + 1, size=k, dtype=np.int64)
        i = rng.integers(0, n - d, dtype=np.int64)  # i in [0, n-1-d]
        if ncut:
            idx = np.searchsorted(cuts, i, side="left")
            nxt = np.where(idx < ncut, cuts[np.minimum(idx, ncut - 1)], np.iinfo(np.int64).max)
            ok = nxt > i + d - 1  # no chosen path edge j with i <= j <= i+d-1
        else:
            ok = np.ones(k, dtype=bool)
        acc = np.stack([i[ok], i[ok] + d[ok]], axis=1)[:need]
        chords = np.concatenate([chords, acc], axis=0)
        need = extra - chords.shape[0]
    j = np.arange(n - 1, dtype=np.int64)
    path = np.stack([j, j + 1], axis=1)
    return _shuffle_orient(rng, np.concatenate([path, chords], axis=0))


def ba_tree(n: int, seed: int = 1, permute: bool = True) -> np.ndarray:
    """Scale-free (Barabasi-Albert) tree: node i attaches to an earlier node
    chosen with probability proportional to its degree (Sec. 3.2). Picking a
    uniform entry of the list of all edge endpoints realises that choice."""
    n = int(n)
    rng = _rng(seed, _S_BA, n)
    parent = np.full(n, -1, dtype=np.int64)
    if n > 1:
        parent[1] = 0
        ends = np.empty(2 * (n - 1), dtype=np.int64)
        ends[0], ends[1] = 0, 1
        r = rng.random(n)
        for i in range(2, n):
            p = int(ends[int(r[i] * (2 * (i - 1)))])
            parent[i] = p
            ends[2 * (i - 1)] = i
            ends[2 * (i - 1) + 1] = p
    if permute:
        perm = _rng(seed, _S_PERM, n, 7).permutation(n)
        out = np.empty(n, dtype=np.int64)
        out[perm[1:]] = perm[parent[1:]]
        out[perm[0]] = -1
        parent = out
    return parent.astype(np.int32)


def _log_uniform_sizes(rng: np.random.Generator, count: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    return np.floor(np.exp2(rng.uniform(lo_exp, hi_exp, size=count))).astype(np.int64)


def batched_instances(seed: int = 1, ntrees: int = 2048, ngraphs: int = 2048,
                      tree_exp=(6, 18), graph_exp=(6, 16), edges_per_node: int = 4):
    """Descriptors of a batched workload of independent instances.

    Trees: n log-uniform in 2^tree_exp, shapes round-robin over grasp 1, grasp
    1024 and unlimited grasp, each with n uniform queries. Graphs: n log-uniform
    in 2^graph_exp, m = edges_per_node * n, easy and hard alternating (the hard
    generator plants n/64 uncovered path edges). Returns two lists of dicts; the
    arrays are produced by ``materialize``-style calls on each descriptor so
    that a caller can bound memory.
    """
    rng = _rng(seed, _S_BATCH, ntrees, ngraphs)
    tn = _log_uniform_sizes(rng, ntrees, *tree_exp)
    gn = _log_uniform_sizes(rng, ngraphs, *graph_exp)
    shapes = (1, 1024, None)
    trees = [dict(kind="tree", n=int(tn[t]), grasp=shapes[t % 3], q=int(tn[t]),
                  seed=int(seed) * 1_000_003 + t) for t in range(ntrees)]
    graphs = []
    for g in range(ngraphs):
        n = max(int(gn[g]), 18)
        m = edges_per_node * n
        graphs.append(dict(kind="easy" if g % 2 == 0 else "hard", n=n, m=m,
                           seed=int(seed) * 1_000_033 + g))
    return trees, graphs


def make_tree(desc) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Materialise a tree descriptor into (parent, u, v)."""
    parent = tree_parent(desc["n"], desc["grasp"], seed=desc["seed"])
    u, v = lca_queries(desc["n"], desc["q"], seed=desc["seed"])
    return parent, u, v


def make_graph(desc) -> np.ndarray:
    """Materialise a graph descriptor into an (m, 2) int32 edge list."""
    n, m = desc["n"], desc["m"]
    if desc["kind"] == "easy":
        return easy_graph(n, m, seed=desc["seed"])
    return hard_graph(n, m - (n - 1), max(1, n // 64), seed=desc["seed"])


def serving_stream(seed: int = 1, nrequests: int = 2000, rate_hz: float = 2000.0, ntrees: int = 256,
                   tree_exp=(10, 22), batch_exp=(4, 20), graph_exp=(10, 22), p_bridge: float = 0.1,
                   edges_per_node: int = 4):
    """A seeded Poisson request stream over ``ntrees`` resident trees.

    Returns (trees, requests). Each tree is a descriptor (n log-uniform in
    2^tree_exp, unlimited grasp). Each request has an arrival time (exponential
    gaps at ``rate_hz``) and is either an LCA batch on a uniform resident tree
    (size log-uniform in 2^batch_exp) or, with probability ``p_bridge``, a
    bridge-finding request on a fresh easy or hard graph (n log-uniform in
    2^graph_exp, m = edges_per_node * n).
    """
    rng = _rng(seed, _S_SERVE, ntrees, nrequests)
    tn = _log_uniform_sizes(rng, ntrees, *tree_exp)
    trees = [dict(kind="tree", n=int(tn[t]), grasp=None, q=0, seed=int(seed) * 7_000_003 + t)
             for t in range(ntrees)]
    gaps = rng.exponential(1.0 / rate_hz, size=nrequests)
    arrival = np.cumsum(gaps) - gaps[0]
    is_bridge = rng.random(nrequests) < p_bridge
    sizes = _log_uniform_sizes(rng, nrequests, *batch_exp)
    tree_ids = rng.integers(0, ntrees, size=nrequests)
    gsz = _log_uniform_sizes(rng, nrequests, *graph_exp)
    reqs = []
    for r in range(nrequests):
        if is_bridge[r]:
            n = max(int(gsz[r]), 18)
            reqs.append(dict(kind="bridges", t=float(arrival[r]), n=n, m=edges_per_node * n,
                             graph="easy" if r % 2 == 0 else "hard", seed=int(seed) * 9_000_011 + r))
        else:
            reqs.append(dict(kind="lca", t=float(arrival[r]), tree=int(tree_ids[r]), q=int(sizes[r]),
                             seed=int(seed) * 9_000_049 + r))
    return trees, reqs

