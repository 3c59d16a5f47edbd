"""Batched trees and graphs in one launch sequence (and one CUDA graph)
against the CPU oracle per instance, and against the single-instance entry
points on the GPU: every answer and every mask bit must be identical."""

import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu_util import dev, host

pytestmark = pytest.mark.gpu


def make_tree_batch(sizes, seed):
    parents, us, vs, insts = [], [], [], []
    for i, n in enumerate(sizes):
        grasp = (1, 1024, None, 3)[i % 4]
        p = synth.tree_parent(n, grasp, seed=seed * 1000 + i)
        u, v = synth.lca_queries(n, max(1, 2 * n), seed=seed * 1000 + i)
        parents.append(p)
        us.append(u)
        vs.append(v)
        insts.append(np.full(u.shape[0], i, np.int32))
    off = np.zeros(len(sizes) + 1, np.int32)
    off[1:] = np.cumsum(sizes)
    return parents, us, vs, insts, off


def shuffled(arrays, seed):
    perm = np.random.default_rng(seed).permutation(arrays[0].shape[0])
    return [a[perm] for a in arrays], perm


def test_tree_batch_matches_oracle_per_instance():
    import paper_2103_15217_gb300 as etl
    sizes = [1, 2, 3, 7, 64, 100, 1000, 4097, 5, 2048, 12345, 1, 300]
    parents, us, vs, insts, off = make_tree_batch(sizes, seed=3)
    h = etl.lca_preprocess_batch(dev(np.concatenate(parents)), dev(off), max(sizes))
    assert h.status() == 0
    (inst, u, v), perm = shuffled([np.concatenate(insts), np.concatenate(us), np.concatenate(vs)], 7)
    st = etl.new_status()
    out = host(h.query_batch(dev(inst), dev(u), dev(v), status=st))
    assert int(host(st)[0]) == 0
    arr = {k: host(t) for k, t in h.arrays().items()}
    qoff = np.zeros(len(sizes) + 1, np.int64)
    qoff[1:] = np.cumsum([x.shape[0] for x in us])
    unperm = np.empty_like(perm)
    unperm[perm] = np.arange(perm.shape[0])
    out = out[unperm]
    for i, p in enumerate(parents):
        want = oracle.lca_offline(p, us[i], vs[i])
        assert (out[qoff[i]:qoff[i + 1]] == want).all(), f"tree {i}"
        pre, depth, size, _ = oracle.tree_tour(p)
        assert (arr["pre"][off[i]:off[i + 1]] - off[i] == pre).all()
        assert (arr["depth"][off[i]:off[i + 1]] == depth).all()
        assert (arr["size"][off[i]:off[i + 1]] == size).all()
    h.free()


def test_tree_batch_equals_single_instance_calls():
    import paper_2103_15217_gb300 as etl
    sizes = list(np.random.default_rng(1).integers(1, 3000, size=40))
    parents, us, vs, insts, off = make_tree_batch(sizes, seed=5)
    h = etl.lca_preprocess_batch(dev(np.concatenate(parents)), dev(off), int(max(sizes)))
    out = host(h.query_batch(dev(np.concatenate(insts)), dev(np.concatenate(us)), dev(np.concatenate(vs))))
    pos = 0
    for i, p in enumerate(parents):
        hi = etl.lca_preprocess(dev(p))
        single = host(hi.query(dev(us[i]), dev(vs[i])))
        assert (out[pos:pos + single.shape[0]] == single).all()
        pos += single.shape[0]
        hi.free()
    h.free()


def test_tree_batch_errors():
    import paper_2103_15217_gb300 as etl
    parents = [np.array([-1, 0, 0], np.int32), np.array([-1, -1], np.int32)]   # second tree has two roots
    off = np.array([0, 3, 5], np.int32)
    h = etl.lca_preprocess_batch(dev(np.concatenate(parents)), dev(off), 3)
    assert h.status() == 4
    h.free()
    parents = [np.array([-1, 5, 0], np.int32)]                                   # parent outside its tree
    h = etl.lca_preprocess_batch(dev(parents[0]), dev(np.array([0, 3], np.int32)), 3)
    assert h.status() == 4
    h.free()
    p = np.array([-1, 0, -1, 0], np.int32)                                        # offsets not ending at n
    h = etl.lca_preprocess_batch(dev(p), dev(np.array([0, 2, 3], np.int32)), 2)
    assert h.status() == 1
    h.free()
    h = etl.lca_preprocess_batch(dev(p), dev(np.array([0, 2, 4], np.int32)), 2)
    assert h.status() == 0
    st = etl.new_status()
    out = host(h.query_batch(dev(np.array([0, 1, 2, -1, 1], np.int32)), dev(np.array([1, 1, 0, 0, 2], np.int32)),
                             dev(np.array([0, 0, 0, 0, 0], np.int32)), status=st))
    assert out.tolist() == [0, 0, -1, -1, -1] and int(host(st)[0]) == 5
    h.free()


def make_graph_batch(sizes, seed):
    edges, eoff, noff = [], [0], [0]
    for i, n in enumerate(sizes):
        if n < 18:
            e = np.random.default_rng(seed + i).integers(0, n, size=(2 * n, 2)).astype(np.int32)
        elif i % 2 == 0:
            e = synth.easy_graph(n, 3 * n, seed=seed + i)
        else:
            e = synth.hard_graph(n, 2 * n, max(1, n // 64), seed=seed + i)
        edges.append(e)
        eoff.append(eoff[-1] + e.shape[0])
        noff.append(noff[-1] + n)
    return edges, np.array(eoff, np.int32), np.array(noff, np.int32)


def test_graph_batch_matches_oracle_and_single_calls():
    import paper_2103_15217_gb300 as etl
    sizes = [1, 2, 5, 17, 64, 1000, 5000, 20, 333, 18, 4096]
    edges, eoff, noff = make_graph_batch(sizes, seed=11)
    st = etl.new_status()
    mask = host(etl.find_bridges_batch(dev(np.concatenate(edges)), dev(eoff), dev(noff), int(noff[-1]), status=st))
    assert int(host(st)[0]) == 0
    for i, e in enumerate(edges):
        want = oracle.bridges_dfs(sizes[i], e)
        assert (mask[eoff[i]:eoff[i + 1]] == want).all(), f"graph {i}"
        single = host(etl.find_bridges(dev(e), sizes[i]))
        assert (single == want).all()


def test_graph_batch_errors():
    import paper_2103_15217_gb300 as etl
    e = np.array([[0, 1], [1, 2], [0, 3]], np.int32)                 # third edge leaves graph 0 (3 nodes)
    st = etl.new_status()
    mask = host(etl.find_bridges_batch(dev(e), dev(np.array([0, 3], np.int32)), dev(np.array([0, 3], np.int32)),
                                       3, status=st))
    assert int(host(st)[0]) == 6 and not mask.any()
    st = etl.new_status()
    etl.find_bridges_batch(dev(e), dev(np.array([0, 2], np.int32)), dev(np.array([0, 3], np.int32)), 3, status=st)
    assert int(host(st)[0]) == 1                                      # edge offsets do not end at m


def test_batch_pipeline_in_one_cuda_graph():
    import paper_2103_15217_gb300 as etl
    sizes = [50, 3000, 1, 777, 64]
    parents, us, vs, insts, off = make_tree_batch(sizes, seed=21)
    edges, eoff, noff = make_graph_batch([100, 2000, 40], seed=23)
    P, O = dev(np.concatenate(parents)), dev(off)
    I, U, V = dev(np.concatenate(insts)), dev(np.concatenate(us)), dev(np.concatenate(vs))
    E, EO, NO = dev(np.concatenate(edges)), dev(eoff), dev(noff)
    out = torch.empty_like(U)
    mask = torch.empty(E.shape[0], dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())

    def pipeline():
        h = etl.lca_preprocess_batch(P, O, max(sizes))
        h.query_batch(I, U, V, out=out)
        h.free()
        mask.copy_(etl.find_bridges_batch(E, EO, NO, int(noff[-1])))

    with torch.cuda.stream(s):
        pipeline()   # eager once (first-call set-up outside capture)
    torch.cuda.synchronize()
    want_out, want_mask = host(out).copy(), host(mask).copy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pipeline()
    for _ in range(2):
        out.fill_(-9)
        mask.fill_(9)
        g.replay()
        torch.cuda.synchronize()
        assert (host(out) == want_out).all() and (host(mask) == want_mask).all()
    qoff = np.zeros(len(sizes) + 1, np.int64)
    qoff[1:] = np.cumsum([x.shape[0] for x in us])
    for i, p in enumerate(parents):
        assert (want_out[qoff[i]:qoff[i + 1]] == oracle.lca_offline(p, us[i], vs[i])).all()
