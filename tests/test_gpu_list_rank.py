"""GPU list ranking (the ruling-set ranker behind both paths) against the
definition: a list built from a permutation has rank[perm[i]] = i."""

import numpy as np
import pytest

from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


def list_from_order(order):
    """succ array of the list that visits elements in the given order."""
    n = order.shape[0]
    succ = np.full(n, -1, np.int32)
    succ[order[:-1]] = order[1:]
    rank = np.empty(n, np.int32)
    rank[order] = np.arange(n, dtype=np.int32)
    return succ, int(order[0]), rank


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 1000, 8191, 8192, 8193, 70000, 1 << 20, (1 << 20) + 7])
def test_random_lists(n):
    import paper_2103_15217_gb300 as etl
    order = np.random.default_rng(n).permutation(n).astype(np.int32)
    succ, head, want = list_from_order(order)
    st = etl.new_status()
    got = host(etl.list_rank(dev(succ), head, status=st))
    assert (got == want).all()
    assert host(st)[0] == 0


@pytest.mark.parametrize("kind", ["identity", "reversed", "evens_then_odds", "stride17", "blocks"])
def test_structured_lists(kind):
    import paper_2103_15217_gb300 as etl
    n = 1 << 18
    idx = np.arange(n, dtype=np.int32)
    order = {
        "identity": idx,
        "reversed": idx[::-1].copy(),
        "evens_then_odds": np.concatenate([idx[0::2], idx[1::2][::-1]]),
        "stride17": np.argsort((idx.astype(np.int64) * 17) % n).astype(np.int32),
        "blocks": idx.reshape(-1, 64)[np.random.default_rng(1).permutation(n // 64)].ravel(),
    }[kind]
    succ, head, want = list_from_order(order)
    got = host(etl.list_rank(dev(succ), head))
    assert (got == want).all()


# The ranker picks splitters by a multiplicative hash of the element index: e
# opens a sublist iff (e * KMUL mod 2^b) < 2^b / 2^k, with 2^b the smallest
# power of two >= the level's capacity (at least 2^k). A walk that reaches
# KLCAP elements without meeting a splitter opens a "dynamic" one. Random
# lists never come near that (gaps of a few hundred), so the lists below are
# laid out from the same rule to make walks far longer than KLCAP, at level 0
# (k_walk0) and at the first reduced level (k_walk).
KMUL = 0x9E3779B1
KLCAP = 4096


def _rule(cap, k_log2):
    b = max(int(cap - 1).bit_length() if cap > 1 else 0, k_log2)
    return (1 << b) - 1, 1 << (b - k_log2)


def _level0_density(length, tuned):
    """The ranker's level-0 density: the tuned value above 2^22 elements, denser below (one in 4 up to
    2^15 elements, 8 up to 2^20, 16 up to 2^22, or the tuned value where that is denser)."""
    if length > 1 << 22:
        return tuned
    return min(4 if length > 1 << 20 else 3 if length > 1 << 15 else 2, tuned)


def _hashed(x, mask):
    return ((np.asarray(x, np.uint64) * np.uint64(KMUL)) & np.uint64(mask)).astype(np.int64)


def _splitter_mask(n, cap, k_log2):
    mask, s0 = _rule(cap, k_log2)
    return _hashed(np.arange(n), mask) < s0


def _longest_unsplit_run(order, split):
    """Longest run of list positions, starting at the head or at a splitter, before the next splitter."""
    pos = np.flatnonzero(split[order])
    starts = np.concatenate([[0], pos])
    ends = np.concatenate([pos, [order.shape[0]]])
    return int((ends - starts).max())


@pytest.mark.slow
@pytest.mark.parametrize("n", [1 << 20, 1 << 25])
def test_level0_walk_opens_dynamic_splitters(n):
    # every non-splitter first, then the splitters: the head's walk crosses
    # ~31/32 of the list and has to open a dynamic splitter every KLCAP elements
    import paper_2103_15217_gb300 as etl
    k0 = _level0_density(n, etl.tune_get()["rank_k0_log2"])
    split = _splitter_mask(n, n, k0)
    rng = np.random.default_rng(n)
    idx = np.arange(n, dtype=np.int32)
    non, spl = idx[~split], idx[split]
    if n <= 1 << 20:
        non = rng.permutation(non)   # random addresses on the small list, index order on the large one
    order = np.concatenate([non, rng.permutation(spl)]).astype(np.int32)
    assert _longest_unsplit_run(order, split) > 100 * KLCAP   # the branch is taken many times
    succ, head, want = list_from_order(order)
    st = etl.new_status()
    got = host(etl.list_rank(dev(succ), head, status=st))
    assert host(st)[0] == 0
    assert (got == want).all()


@pytest.mark.slow
@pytest.mark.parametrize("n", [1 << 20, 1 << 25])
def test_upper_level_walk_opens_dynamic_splitters(n):
    # short level-0 sublists whose ids, in list order, give first every
    # reduced-list element that is not a level-1 splitter: the walk of the
    # reduced list from its head crosses ~15/16 of it
    import paper_2103_15217_gb300 as etl
    t = etl.tune_get()
    k0, k1 = _level0_density(n, t["rank_k0_log2"]), t["rank_k_log2"]
    mask0, s00 = _rule(n, k0)
    split0 = _hashed(np.arange(n), mask0) < s00
    cap1 = s00 + 1 + (n // KLCAP + 2)
    mask1, s01 = _rule(cap1, k1)
    idx = np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(n + 1)
    spl = rng.permutation(idx[split0])
    sid = _hashed(spl, mask0)
    up_split = _hashed(sid, mask1) < s01
    spl = np.concatenate([spl[~up_split], spl[up_split]])     # level-1 non-splitters' sublists first
    non = rng.permutation(idx[~split0])      # each splitter followed by an equal share of them
    chunk = np.arange(non.shape[0]) * spl.shape[0] // non.shape[0]
    keys = np.concatenate([2 * np.arange(spl.shape[0]), 2 * chunk + 1])
    order = np.concatenate([spl, non])[np.argsort(keys, kind="stable")].astype(np.int32)
    assert _longest_unsplit_run(order, split0) < KLCAP         # no dynamic splitter at level 0
    sid_order = _hashed(spl, mask0)                             # the reduced list, in list order
    assert _longest_unsplit_run(np.arange(sid_order.shape[0]), _hashed(sid_order, mask1) < s01) > 5 * KLCAP
    succ, head, want = list_from_order(order)
    st = etl.new_status()
    got = host(etl.list_rank(dev(succ), head, status=st))
    assert host(st)[0] == 0
    assert (got == want).all()


def test_tree_tour_opens_dynamic_splitters():
    # a path whose nodes are ordered so that the opening brackets 2v met first
    # are not splitters: the ranking walk of the tour (brackets 2v / 2v + 1,
    # counting opening brackets as it goes) opens dynamic splitters
    import oracle
    import paper_2103_15217_gb300 as etl
    n = 1 << 20
    k0 = _level0_density(2 * n, etl.tune_get()["rank_k0_log2"])
    split = _splitter_mask(2 * n, 2 * n, k0)
    labels = np.arange(n, dtype=np.int32)
    open_split = split[2 * labels]
    rng = np.random.default_rng(5)
    path = np.concatenate([rng.permutation(labels[~open_split]), rng.permutation(labels[open_split])])
    assert (~open_split).sum() > 100 * KLCAP
    parent = np.empty(n, np.int32)
    parent[path[0]] = -1
    parent[path[1:]] = path[:-1]
    h = etl.lca_preprocess(dev(parent))
    u = rng.integers(0, n, 1 << 18).astype(np.int32)
    v = rng.integers(0, n, 1 << 18).astype(np.int32)
    out = host(h.query(dev(u), dev(v)))
    arr = {k: host(t) for k, t in h.arrays().items()}
    assert h.status() == 0
    h.free()
    pre, depth, size, _ = oracle.tree_tour(parent)
    assert (arr["pre"] == pre).all() and (arr["depth"] == depth).all() and (arr["size"] == size).all()
    assert (out == oracle.lca_offline(parent, u, v)).all()
    where = np.empty(n, np.int64)
    where[path] = np.arange(n)
    assert (out == np.where(where[u] < where[v], u, v)).all()   # closed form on a path: the end nearer the root


def test_two_lists_is_an_error():
    import paper_2103_15217_gb300 as etl
    n = 5000
    order = np.random.default_rng(3).permutation(n).astype(np.int32)
    succ, head, _ = list_from_order(order)
    succ[order[2499]] = -1          # split into two lists
    st = etl.new_status()
    etl.list_rank(dev(succ), head, status=st)
    assert host(st)[0] == 4         # ETL_EBADTREE


def test_cycle_is_an_error_and_terminates():
    import paper_2103_15217_gb300 as etl
    n = 100000
    order = np.random.default_rng(4).permutation(n).astype(np.int32)
    succ, head, _ = list_from_order(order)
    succ[order[-1]] = order[n // 2]   # tail points back into the list: a rho shape
    st = etl.new_status()
    etl.list_rank(dev(succ), head, status=st)
    assert host(st)[0] != 0
