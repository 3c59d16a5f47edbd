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


def test_long_path_forces_dynamic_splitters():
    # a list laid out so that hashed splitters are sparse is still ranked exactly;
    # 3 million elements visited in index order
    import paper_2103_15217_gb300 as etl
    n = 3_000_000
    order = np.arange(n, dtype=np.int32)
    succ, head, want = list_from_order(order)
    got = host(etl.list_rank(dev(succ), head))
    assert (got == want).all()


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
