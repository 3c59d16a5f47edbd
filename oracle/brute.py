"""Brute force for tiny inputs (test infrastructure only).

Straight from the definitions, with no cleverness at all:

* LCA(x, y): of all common ancestors of x and y (a node is its own ancestor),
  the one furthest from the root (Sec. 3, problem statement).
* bridge: an edge whose deletion increases the number of connected components
  (Sec. 4, problem statement); counted by a BFS over the graph without it.
* 2-edge-connected: u and v are in the same 2-edge-connected component iff no
  single edge deletion separates them (Menger: two edge-disjoint paths).
"""

from __future__ import annotations

from collections import deque


def ancestors(parent, x):
    """Path from x up to the root, x first."""
    out = [x]
    while parent[out[-1]] != -1:
        out.append(int(parent[out[-1]]))
        if len(out) > len(parent):
            raise ValueError("parent array has a cycle")
    return out


def lca(parent, x, y):
    ax = ancestors(parent, int(x))
    common = set(ax) & set(ancestors(parent, int(y)))
    return max(common, key=lambda z: len(ancestors(parent, z)))


def components(n, edges, skip=-1):
    adj = [[] for _ in range(n)]
    for e, (a, b) in enumerate(edges):
        if e != skip:
            adj[int(a)].append(int(b))
            adj[int(b)].append(int(a))
    seen = [False] * n
    count = 0
    for s in range(n):
        if seen[s]:
            continue
        count += 1
        seen[s] = True
        dq = deque([s])
        while dq:
            x = dq.popleft()
            for w in adj[x]:
                if not seen[w]:
                    seen[w] = True
                    dq.append(w)
    return count


def bridges(n, edges):
    base = components(n, edges)
    return [int(components(n, edges, skip=e) > base) for e in range(len(edges))]


def reach(n, edges, s, skip=-1):
    adj = [[] for _ in range(n)]
    for e, (a, b) in enumerate(edges):
        if e != skip:
            adj[int(a)].append(int(b))
            adj[int(b)].append(int(a))
    seen = [False] * n
    seen[s] = True
    dq = deque([s])
    while dq:
        x = dq.popleft()
        for w in adj[x]:
            if not seen[w]:
                seen[w] = True
                dq.append(w)
    return seen


def two_edge_cc(n, edges):
    """label[v] = smallest u that no single edge deletion separates from v."""
    cut = [reach(n, edges, s) for s in range(n)]
    per_edge = [[reach(n, edges, s, skip=e) for s in range(n)] for e in range(len(edges))]
    label = []
    for v in range(n):
        for u in range(n):
            if cut[v][u] and all(pe[v][u] for pe in per_edge):
                label.append(u)
                break
    return label
