"""CPU oracle for the Euler-tour path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library under
``paper_2103_15217_gb300`` never does, and the two share no code: the oracle is
plain C (``etl_oracle.c``) compiled with gcc and called through ctypes, plus
pure-Python brute force for tiny inputs (``brute.py``).

Every function takes and returns numpy int32 / uint8 arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "etl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EBADTREE, EBADQUERY, EBADGRAPH = 0, 1, 2, 4, 5, 6


class OracleError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed with oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no GPU, no CUDA) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def bind(lib):
    """Declare the C signatures on a loaded oracle library (also used by the
    planted-mistake tests, which load mutated copies of the oracle)."""
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    lib.oracle_tree_tour.argtypes = [i32, P, P, P, P, P]
    lib.oracle_dcel_tour.argtypes = [i32, i64, P, i32, P, P, P]
    lib.oracle_lca_climb.argtypes = [i32, P, P, i64, P, P, P]
    lib.oracle_lca_offline.argtypes = [i32, P, i64, P, P, P]
    lib.oracle_bridges_dfs.argtypes = [i32, i64, P, P]
    lib.oracle_bridges_tv.argtypes = [i32, i64, P, P, P]
    lib.oracle_two_edge_cc.argtypes = [i32, i64, P, P]
    for f in ("oracle_tree_tour", "oracle_dcel_tour", "oracle_lca_climb", "oracle_lca_offline",
              "oracle_bridges_dfs", "oracle_bridges_tv", "oracle_two_edge_cc"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(fn, rc, allow=()):
    if rc != OK and rc not in allow:
        raise OracleError(fn, rc)
    return rc


def tree_tour(parent):
    """(pre, depth, size, tour) of the rooted tree (Sec. 2): DFS visiting
    children in ascending label order; tour lists bracket ids 2v (enter v) and
    2v+1 (leave v) in order, 2n entries including the root's two brackets."""
    parent = _i32(parent)
    n = parent.shape[0]
    pre, depth, size = (np.empty(n, np.int32) for _ in range(3))
    tour = np.empty(2 * n, np.int32)
    _check("oracle_tree_tour", _load().oracle_tree_tour(n, _p(parent), _p(pre), _p(depth), _p(size), _p(tour)))
    return pre, depth, size, tour


def dcel_tour(n, edges, root):
    """The paper's DCEL construction (Sec. 2.1): returns (succ, tour, B) over
    half-edges 2i=(x_i,y_i), 2i+1=(y_i,x_i); B is the lexicographically sorted
    order of the half-edges, tour the list from first[root]."""
    edges = _i32(edges).reshape(-1, 2)
    k = edges.shape[0]
    succ, tour, B = (np.empty(2 * k, np.int32) for _ in range(3))
    _check("oracle_dcel_tour", _load().oracle_dcel_tour(int(n), k, _p(edges), int(root), _p(succ), _p(tour), _p(B)))
    return succ, tour, B


def lca_climb(parent, depth, u, v):
    """LCA by climbing (Sec. 3.1 naive method = the definition)."""
    parent, depth, u, v = _i32(parent), _i32(depth), _i32(u), _i32(v)
    out = np.empty(u.shape[0], np.int32)
    rc = _load().oracle_lca_climb(parent.shape[0], _p(parent), _p(depth), u.shape[0], _p(u), _p(v), _p(out))
    _check("oracle_lca_climb", rc, allow=(EBADQUERY,))
    return out


def lca_offline(parent, u, v):
    """Tarjan's offline union-find LCA (exact, near-linear)."""
    parent, u, v = _i32(parent), _i32(u), _i32(v)
    out = np.empty(u.shape[0], np.int32)
    rc = _load().oracle_lca_offline(parent.shape[0], _p(parent), u.shape[0], _p(u), _p(v), _p(out))
    _check("oracle_lca_offline", rc, allow=(EBADQUERY,))
    return out


def bridges_dfs(n, edges):
    """Bridge mask by the sequential DFS low-function method (Sec. 4.1)."""
    edges = _i32(edges).reshape(-1, 2)
    out = np.empty(edges.shape[0], np.uint8)
    _check("oracle_bridges_dfs", _load().oracle_bridges_dfs(int(n), edges.shape[0], _p(edges), _p(out)))
    return out


def bridges_tv(n, edges, tree=None):
    """Bridge mask by the Tarjan-Vishkin low/high criterion over a given
    spanning forest (uint8 mask per edge), or Kruskal in input order if None."""
    edges = _i32(edges).reshape(-1, 2)
    t = None if tree is None else np.ascontiguousarray(tree, dtype=np.uint8)
    out = np.empty(edges.shape[0], np.uint8)
    _check("oracle_bridges_tv", _load().oracle_bridges_tv(int(n), edges.shape[0], _p(edges), _p(t), _p(out)))
    return out


def two_edge_cc(n, edges):
    """Label of every vertex's 2-edge-connected component (its smallest vertex)."""
    edges = _i32(edges).reshape(-1, 2)
    out = np.empty(int(n), np.int32)
    _check("oracle_two_edge_cc", _load().oracle_two_edge_cc(int(n), edges.shape[0], _p(edges), _p(out)))
    return out
