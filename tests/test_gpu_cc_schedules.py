"""Every hooking schedule of the connectivity pass (first slice size, doubling
slices or one launch for the rest, the giant-root priority, and the spread
order used for batches) gives the oracle's bridge masks: the spanning forest
changes, the bridges do not."""

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
    etl.tune_set(**{k: old[k] for k in ("cc_first_slice", "cc_doubling", "cc_giant")})


@pytest.mark.parametrize("first", [1, 2, 4, 64])
@pytest.mark.parametrize("doubling", [0, 1])
@pytest.mark.parametrize("giant", [0, 1])
def test_single_graphs(restore_tuning, first, doubling, giant):
    import paper_2103_15217_gb300 as etl
    etl.tune_set(cc_first_slice=first, cc_doubling=doubling, cc_giant=giant)
    for n, kind in ((3000, "easy"), (3001, "hard"), (70000, "easy"), (70001, "hard")):
        e = synth.easy_graph(n, 6 * n, seed=n) if kind == "easy" else synth.hard_graph(n, 3 * n, n // 50, seed=n)
        st = etl.new_status()
        got = host(etl.find_bridges(dev(e), n, status=st))
        assert int(host(st)[0]) == 0
        assert (got == oracle.bridges_dfs(n, e)).all(), (n, kind)
        lab = host(etl.two_edge_cc(dev(e), n))
        assert (lab == oracle.two_edge_cc(n, e)).all(), (n, kind)


@pytest.mark.parametrize("doubling", [0, 1])
@pytest.mark.parametrize("giant", [0, 1])
def test_batches(restore_tuning, doubling, giant):
    import paper_2103_15217_gb300 as etl
    etl.tune_set(cc_first_slice=1, cc_doubling=doubling, cc_giant=giant)
    rng = np.random.default_rng(doubling)
    parts, eoff, noff, want = [], [0], [0], []
    for i in range(300):
        n = int(rng.integers(20, 400))
        e = synth.easy_graph(n, 3 * n, seed=i) if i % 2 else synth.hard_graph(n, 2 * n, max(1, n // 20), seed=i)
        parts.append(e)
        eoff.append(eoff[-1] + e.shape[0])
        noff.append(noff[-1] + n)
        want.append(oracle.bridges_dfs(n, e))
    st = etl.new_status()
    got = host(etl.find_bridges_batch(dev(np.concatenate(parts)), dev(np.array(eoff, np.int32)),
                                      dev(np.array(noff, np.int32)), noff[-1], status=st))
    assert int(host(st)[0]) == 0
    assert (got == np.concatenate(want)).all()
