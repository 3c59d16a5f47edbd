"""The entry points at the largest sizes their contracts allow.

* list ranking (Sec. 2.2) of a list of 2^31 - 2 elements, the longest a
  signed 32-bit rank can describe, visited in a random order;
* LCA preprocessing and queries (Sec. 3) on trees of 2^30 - 1 nodes, whose
  Euler tours (two brackets per node) are lists of 2^31 - 2 elements: a
  random recursive tree and the path, the shallowest and deepest shapes;
* bridges (Sec. 4.1) with the most edges (2^31 - 2) and with the most
  vertices (2^30 - 1): a path with chords, the large-diameter family.

At these sizes the oracle's DFS takes minutes, so each result is checked
against what defines it exactly, computed from the inputs alone:

* ranks: the list is built from a known order, so rank[order[i]] = i;
* pre / depth / size of a tree whose children carry larger labels than their
  parents: depth(root) = 0 and depth(c) = depth(parent(c)) + 1; with the
  children of each node taken in ascending label order, the first child c of
  p has pre(c) = pre(p) + 1, each later child follows its predecessor c' at
  pre(c') + size(c'), the last one ends where p ends (pre(c) + size(c) =
  pre(p) + size(p)), a leaf has size 1, and pre(root) = 0. These relations
  determine preorder and subtree sizes completely (top-down and bottom-up
  induction), so checking all of them is checking the definition;
* LCA: every answer is a common ancestor of its pair (an interval test on the
  checked preorder), and on a sample it equals climbing by labels (the parent
  of a node has the smaller label, so the larger of the two labels steps to its
  parent until they meet); min(u, v) on the path rooted at 0;
* bridges of a path 0 - 1 - ... - (n-1) with chords (i, i + d), d >= 2: a
  chord is on a cycle and never a bridge; path edge (j, j + 1) is a bridge
  exactly when no chord spans it (i <= j < i + d). The chords are drawn so
  that the edges no chord spans are a chosen set of cuts.

Inputs are drawn on the device from seeded generators; every call runs in a
caller-owned workspace, so nothing stays cached between the tests. These
sizes need about 200 GB of device memory (the largest case) and run only on a
device with more than that.
"""

import gc

import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

MAX_LIST = (1 << 31) - 2
MAX_NODES = (1 << 30) - 1
MAX_EDGES = (1 << 31) - 2
NEED_BYTES = 230 << 30


def _etl():
    import paper_2103_15217_gb300 as etl
    etl.build()
    etl.load_library()
    return etl


@pytest.fixture(autouse=True)
def _fresh_device():
    gc.collect()
    torch.cuda.empty_cache()
    if torch.cuda.get_device_properties(0).total_memory < NEED_BYTES:
        pytest.skip("the largest inputs need a device with more than 230 GB of memory")
    yield
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _gen(seed):
    return torch.Generator(device="cuda").manual_seed(seed)


def _perm(m, g, dtype=torch.int64):
    """A random permutation of [0, m): the order that sorts m random 62-bit keys (torch.randperm is far
    slower at these lengths)."""
    keys = torch.randint(0, 1 << 62, (m,), generator=g, device="cuda", dtype=torch.int64)
    idx = torch.sort(keys)[1]
    del keys
    return idx.to(dtype)


def test_list_rank_longest_list():
    etl = _etl()
    L = MAX_LIST
    order = _perm(L, _gen(1))  # visiting order of the list
    succ = torch.empty(L, dtype=torch.int32, device="cuda")
    succ[order[:-1]] = order[1:].to(torch.int32)
    succ[order[-1]] = -1
    head = int(order[0])
    ws = etl.new_workspace(etl.workspace_size("list_rank", L))
    st = etl.new_status()
    rank = etl.list_rank(succ, head, status=st, workspace=ws)
    assert etl.status_get(st) == 0
    del ws, succ
    got = rank[order]
    del rank
    assert torch.equal(got, torch.arange(L, dtype=torch.int32, device="cuda"))


def _random_recursive_tree(n, seed):
    """parent(i) uniform in [0, i) for i >= 1, parent(0) = -1 (labels not permuted)."""
    i = torch.arange(n, dtype=torch.float64, device="cuda")
    p = torch.floor(torch.rand(n, dtype=torch.float64, generator=_gen(seed), device="cuda") * i)
    p = torch.minimum(p, i - 1).to(torch.int32)  # rounding of u * i can reach i when u is close to 1
    del i
    p[0] = -1
    return p


def _climb(parent, u, v):
    """LCA by labels: the larger label steps to its parent until the two meet."""
    u, v = u.astype(np.int64), v.astype(np.int64)
    out = np.empty(u.size, np.int64)
    idx = np.arange(u.size)
    for _ in range(1 << 12):
        met = u == v
        out[idx[met]] = u[met]
        if met.all():
            return out.astype(np.int32)
        idx, u, v = idx[~met], u[~met], v[~met]
        a = u > v
        u = np.where(a, parent[u], u)
        v = np.where(a, v, parent[v])
    raise AssertionError("climbing did not meet")


def _check_tree_arrays(parent, arr, n):
    pre, depth, size, order = arr["pre"], arr["depth"], arr["size"], arr["order"]
    assert int(pre[0]) == 0 and int(depth[0]) == 0 and int(size[0]) == n
    p = parent[1:].to(torch.int64)
    assert torch.equal(depth[1:], depth[p] + 1)
    del p
    # children of every node in ascending label order: a stable sort by parent keeps the labels ascending
    pv, idx = torch.sort(parent[1:], stable=True)
    kids = idx + 1
    del idx
    pv = pv.to(torch.int64)
    first = torch.ones(n - 1, dtype=torch.bool, device="cuda")
    first[1:] = pv[1:] != pv[:-1]
    last = torch.ones(n - 1, dtype=torch.bool, device="cuda")
    last[:-1] = first[1:]
    pre_k, size_k = pre[kids], size[kids]
    pre_p, size_p = pre[pv], size[pv]
    assert torch.equal(pre_k[first], pre_p[first] + 1)
    follow = pre_k[:-1] + size_k[:-1]
    assert torch.equal(pre_k[1:][~first[1:]], follow[~first[1:]])
    del follow
    assert torch.equal((pre_k + size_k)[last], (pre_p + size_p)[last])
    del pre_k, size_k, pre_p, size_p, first, last, kids
    has_child = torch.zeros(n, dtype=torch.bool, device="cuda")
    has_child[pv] = True
    assert bool((size[~has_child] == 1).all())
    del has_child, pv
    assert torch.equal(order[pre.to(torch.int64)], torch.arange(n, dtype=torch.int32, device="cuda"))


def test_lca_largest_random_tree():
    etl = _etl()
    n = MAX_NODES
    parent = _random_recursive_tree(n, seed=2)
    ws = etl.new_workspace(etl.workspace_size("lca_preprocess", n))
    h = etl.lca_preprocess(parent, workspace=ws)
    q = 1 << 22
    u = torch.randint(0, n, (q,), generator=_gen(3), device="cuda", dtype=torch.int32)
    v = torch.randint(0, n, (q,), generator=_gen(4), device="cuda", dtype=torch.int32)
    got = h.query(u, v)
    assert h.status() == 0
    arr = h.arrays()
    h.free()
    del ws
    _check_tree_arrays(parent, arr, n)
    # with pre and size checked, every answer must be a common ancestor of its pair (interval test)
    pre, size = arr["pre"], arr["size"]
    pw, sw = pre[got.long()], size[got.long()]
    pu, pv = pre[u.long()], pre[v.long()]
    assert bool(((pw <= pu) & (pu < pw + sw) & (pw <= pv) & (pv < pw + sw)).all())
    del arr, pre, size
    # ... and the deepest one: exact by label climbing on the first 2^16 queries
    k = 1 << 16
    want = _climb(parent.cpu().numpy(), u[:k].cpu().numpy(), v[:k].cpu().numpy())
    assert (got[:k].cpu().numpy() == want).all()


def test_lca_longest_path():
    etl = _etl()
    n = MAX_NODES
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    parent = ids - 1  # the path 0 - 1 - ... - (n-1) rooted at 0, parent(0) = -1
    ws = etl.new_workspace(etl.workspace_size("lca_preprocess", n))
    h = etl.lca_preprocess(parent, workspace=ws)
    q = 1 << 24
    u = torch.randint(0, n, (q,), generator=_gen(5), device="cuda", dtype=torch.int32)
    v = torch.randint(0, n, (q,), generator=_gen(6), device="cuda", dtype=torch.int32)
    got = h.query(u, v)
    assert h.status() == 0
    assert torch.equal(got, torch.minimum(u, v))
    arr = h.arrays()
    h.free()
    del ws, parent
    assert torch.equal(arr["pre"], ids) and torch.equal(arr["depth"], ids) and torch.equal(arr["order"], ids)
    assert torch.equal(arr["size"], n - ids)


def _path_with_chords(n, extra, ncut, seed):
    """A path 0 - 1 - ... - (n-1) with chords (i, i + d), d >= 2, whose bridges are known by
    construction: ncut path edges are chosen as cuts (4r + 2 for distinct r, so no two are closer
    than 4 and none is near an end); every other path edge j gets one covering chord of length 2,
    (j, j + 2) or, when j + 1 is a cut, (j - 1, j + 1), which spans no cut; then `extra` random chords
    (d uniform in [2, 16], i uniform in [0, n - 1 - d]) are drawn, and drawn again when they would span
    a cut. Each chord lies on a cycle with the path; a path edge is a bridge exactly when no chord
    spans it, which here means exactly the cuts. Returns the shuffled, randomly oriented edge list
    (device int32 [m, 2], path edges first before the shuffle, then the chords), the permutation that
    shuffled it and the cut mask of the path edges (device bool [n - 1])."""
    g = _gen(seed)
    r = _perm((n - 10) // 4, g)[:ncut]
    cut = torch.zeros(n + 1, dtype=torch.bool, device="cuda")
    cut[4 * r + 2] = True
    del r
    cut_pre = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    cut_pre[1:] = torch.cumsum(cut[:n].to(torch.int32), 0, dtype=torch.int32)  # cuts below x
    j = torch.arange(n - 1, dtype=torch.int32, device="cuda")
    keep = ~cut[: n - 1]
    lo = torch.where(cut[1:n] | (j + 2 > n - 1), j - 1, j)[keep]
    del j, keep
    cover = torch.stack([lo, lo + 2], 1)
    del lo
    chords = [cover]
    have, batch = 0, 1 << 28
    while have < extra:
        d = torch.randint(2, 17, (batch,), generator=g, device="cuda", dtype=torch.int64)
        i = torch.floor(torch.rand(batch, dtype=torch.float64, generator=g, device="cuda") * (n - d)).to(torch.int64)
        i = torch.minimum(i, n - 1 - d)
        ok = cut_pre[i + d] == cut_pre[i]  # no cut among the path edges i .. i + d - 1
        i, d = i[ok][: extra - have], d[ok][: extra - have]
        chords.append(torch.stack([i, i + d], 1).to(torch.int32))
        have += i.numel()
        del i, d, ok
    del cut_pre
    j = torch.arange(n - 1, dtype=torch.int32, device="cuda")
    edges = torch.cat([torch.stack([j, j + 1], 1)] + chords)
    del j, chords, cover
    m = edges.shape[0]
    flip = torch.randint(0, 2, (m,), generator=g, device="cuda", dtype=torch.int8).bool()
    edges[flip] = edges[flip].flip(1)
    del flip
    perm = _perm(m, g, torch.int32)
    edges = edges[perm]
    return edges, perm, cut[: n - 1].clone()


def _check_bridges(etl, edges, perm, want_path, n):
    m = edges.shape[0]
    ws = etl.new_workspace(etl.workspace_size("find_bridges", n, m))
    st = etl.new_status()
    mask = etl.find_bridges(edges, n, status=st, workspace=ws)
    assert etl.status_get(st) == 0
    del ws, edges
    got = torch.empty_like(mask)
    got[perm] = mask  # back to the unshuffled order: path edges first, then the chords
    del mask, perm
    assert int(got[n - 1:].sum()) == 0
    assert torch.equal(got[: n - 1].bool(), want_path)


def test_bridges_most_edges():
    etl = _etl()
    n = 1 << 26
    ncut = 1 << 16
    cover = n - 1 - ncut
    edges, perm, want = _path_with_chords(n, MAX_EDGES - (n - 1) - cover, ncut, seed=7)
    assert edges.shape[0] == MAX_EDGES
    _check_bridges(etl, edges, perm, want, n)


def test_bridges_most_vertices():
    etl = _etl()
    n = MAX_NODES
    ncut = 1 << 16
    cover = n - 1 - ncut
    edges, perm, want = _path_with_chords(n, MAX_EDGES - (n - 1) - cover - 2, ncut, seed=8)
    assert edges.shape[0] == MAX_EDGES - 2
    _check_bridges(etl, edges, perm, want, n)
