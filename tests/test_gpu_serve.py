"""Continuous-batching server: every result must be the same in the mix as
alone (integer outputs, so exactly the same), and equal to the CPU oracle."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def workload(seed=3, ntrees=12, nreq=90, rate=20000.0):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp2(rng.uniform(10, 14, size=ntrees))).astype(int)
    trees = [synth.tree_parent(int(n), (None, 1024, 1)[i % 3], seed=seed * 100 + i) for i, n in enumerate(sizes)]
    from paper_2103_15217_gb300.serve import Request
    reqs, t = [], 0.0
    for r in range(nreq):
        t += rng.exponential(1.0 / rate)
        if r % 9 == 4:
            n = int(np.floor(np.exp2(rng.uniform(10, 13))))
            e = synth.easy_graph(n, 4 * n, seed=seed + r) if r % 2 else synth.hard_graph(n, 3 * n + 1, n // 64, seed=seed + r)
            reqs.append(Request("bridges", t, n=n, edges=e, rid=r))
        else:
            tree = int(rng.integers(0, ntrees))
            q = int(np.floor(np.exp2(rng.uniform(4, 12))))
            u, v = synth.lca_queries(int(sizes[tree]), q, seed=seed * 1000 + r)
            reqs.append(Request("lca", t, tree=tree, u=u, v=v, rid=r))
    return trees, reqs


def check_oracle(trees, reqs, results):
    for r, res in zip(reqs, results):
        assert res.rid == r.rid
        if r.kind == "lca":
            assert (res.out == oracle.lca_offline(trees[r.tree], r.u, r.v)).all()
        else:
            assert (res.out == oracle.bridges_dfs(r.n, r.edges)).all()


def test_mixed_equals_alone_and_oracle():
    from paper_2103_15217_gb300.serve import Server, summarize
    trees, reqs = workload()
    srv = Server(trees, budget_bytes=8 << 30, slots=4)
    mixed = srv.serve(reqs, batching=True)
    check_oracle(trees, reqs, mixed)
    batched_launches = {round(x.t_admit, 9) for x in mixed}
    assert len(batched_launches) < len(reqs)          # requests really were batched together
    for r, m in zip(reqs, mixed):
        alone = srv.serve([r], batching=False, realtime=False)[0]
        assert alone.out.dtype == m.out.dtype and (alone.out == m.out).all()
    s = summarize(mixed)
    assert s["requests"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0
    srv.close()


def test_tight_budget_and_plain_mode_agree():
    from paper_2103_15217_gb300.serve import Server, resident_bytes
    trees, reqs = workload(seed=5, nreq=40)
    budget = resident_bytes([t.shape[0] for t in trees]) + max(r.bytes() for r in reqs)
    srv = Server(trees, budget_bytes=budget, slots=3)
    tight = srv.serve(reqs, batching=True)
    plain = srv.serve(reqs, batching=False)
    check_oracle(trees, reqs, tight)
    for a, b in zip(tight, plain):
        assert (a.out == b.out).all()
    srv.close()
