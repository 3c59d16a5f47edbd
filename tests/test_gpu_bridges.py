"""GPU bridge finding (through the C ABI) against the CPU oracle's DFS
low-function method, on brute-force-sized multigraphs, the two synthetic
graph families (small sizes spanning several tiles, and the full size of the
benchmark), and degenerate inputs. Masks must match bit for bit."""

import numpy as np
import pytest

import oracle
from oracle import brute
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


def gpu_bridges(n, edges):
    import paper_2103_15217_gb300 as etl
    st = etl.new_status()
    mask = host(etl.find_bridges(dev(np.asarray(edges, np.int32).reshape(-1, 2)), n, status=st))
    return mask, int(host(st)[0])


def test_tiny_multigraphs_bruteforce():
    rng = np.random.default_rng(5)
    for trial in range(300):
        n = int(rng.integers(1, 12))
        m = int(rng.integers(1, 18))
        edges = rng.integers(0, n, size=(m, 2)).astype(np.int32)
        got, st = gpu_bridges(n, edges)
        assert st == 0
        assert got.tolist() == brute.bridges(n, edges), (n, edges.tolist())


@pytest.mark.parametrize("n", [20, 257, 2049, 10007, 65536])
@pytest.mark.parametrize("kind", ["easy", "hard", "tree", "forest"])
def test_graph_families(n, kind):
    if kind == "easy":
        edges = synth.easy_graph(n, 3 * n, seed=n)
    elif kind == "hard":
        edges = synth.hard_graph(n, 2 * n, max(1, n // 64), seed=n)
    elif kind == "tree":
        p = synth.tree_parent(n, None, seed=n)
        c = np.nonzero(p >= 0)[0]
        edges = np.stack([c, p[c]], 1).astype(np.int32)
    else:  # many components, isolated vertices, self-loops and parallel edges
        rng = np.random.default_rng(n)
        edges = rng.integers(0, n, size=(n // 2, 2)).astype(np.int32)
        edges = np.concatenate([edges, edges[: n // 20], np.stack([np.arange(5), np.arange(5)], 1)]).astype(np.int32)
    got, st = gpu_bridges(n, edges)
    assert st == 0
    want = oracle.bridges_dfs(n, edges)
    assert (got == want).all(), f"{(got != want).sum()} mismatches"


def test_degenerate():
    assert gpu_bridges(1, [[0, 0]]) == (np.array([0], np.uint8), 0)
    got, st = gpu_bridges(2, [[0, 1]])
    assert got.tolist() == [1] and st == 0
    got, st = gpu_bridges(2, [[0, 1], [1, 0]])
    assert got.tolist() == [0, 0]
    got, st = gpu_bridges(5, [[3, 4]])
    assert got.tolist() == [1]
    got, st = gpu_bridges(4, [[0, 1], [1, 4]])   # endpoint out of range
    assert st == 6 and got.tolist() == [0, 0]


def test_config_full_size_hard():
    # large-diameter graph at the benchmark size: closed form + DFS oracle
    import test_oracle_pins as pins
    n = 1 << 22
    edges = synth.hard_graph(n, 1 << 24, 1 << 16, seed=1)
    got, st = gpu_bridges(n, edges)
    assert st == 0
    assert (got == pins.path_coverage_bridges(n, edges)).all()


def test_config_full_size_easy():
    n = 1 << 22
    edges = synth.easy_graph(n, (1 << 25) - 1, seed=1)
    got, st = gpu_bridges(n, edges)
    assert st == 0
    assert (got == oracle.bridges_dfs(n, edges)).all()


def test_two_edge_cc_matches_oracle():
    import paper_2103_15217_gb300 as etl
    from oracle import brute
    rng = np.random.default_rng(31)
    for trial in range(100):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, 12))
        edges = rng.integers(0, n, size=(m, 2)).astype(np.int32)
        got = host(etl.two_edge_cc(dev(edges.reshape(-1, 2)), n)) if m else host(etl.two_edge_cc(dev(np.zeros((0, 2), np.int32)), n))
        assert got.tolist() == brute.two_edge_cc(n, edges), (n, edges.tolist())
    for n, edges in ((1 << 14, synth.easy_graph(1 << 14, 3 << 14, seed=2)),
                     (1 << 14, synth.hard_graph(1 << 14, 1 << 15, 256, seed=2)),
                     (1 << 20, synth.hard_graph(1 << 20, 1 << 21, 1 << 14, seed=3))):
        st = etl.new_status()
        got = host(etl.two_edge_cc(dev(edges), n, status=st))
        assert int(host(st)[0]) == 0
        assert (got == oracle.two_edge_cc(n, edges)).all()


def test_hybrid_method_matches_oracle():
    import paper_2103_15217_gb300 as etl
    rng = np.random.default_rng(41)
    for trial in range(150):
        n = int(rng.integers(1, 12))
        m = int(rng.integers(1, 18))
        edges = rng.integers(0, n, size=(m, 2)).astype(np.int32)
        got = host(etl.find_bridges(dev(edges), n, method="hybrid"))
        assert got.tolist() == brute.bridges(n, edges), (n, edges.tolist())
    for n, edges in ((20000, synth.easy_graph(20000, 80000, seed=5)),
                     (20000, synth.hard_graph(20000, 60000, 300, seed=5)),
                     (1 << 18, synth.easy_graph(1 << 18, 1 << 21, seed=6))):
        st = etl.new_status()
        got = host(etl.find_bridges(dev(edges), n, status=st, method="hybrid"))
        assert int(host(st)[0]) == 0
        assert (got == oracle.bridges_dfs(n, edges)).all()
