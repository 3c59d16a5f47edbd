"""Python binding of the GB300 Euler-tour library (``include/etl.h``).

Thin ctypes marshalling over ``_build/libetl.so``: every step of the path runs
in the library's CUDA kernels; PyTorch only provides device memory and the
current stream. There is no fallback: if the library is not built, or a
tensor is not a CUDA int32 tensor, the call raises.

    import paper_2103_15217_gb300 as etl
    h = etl.lca_preprocess(parent)          # parent: int32 CUDA tensor, root = -1
    out = h.query(u, v)                     # LCA per query pair
    mask = etl.find_bridges(edges, n)       # edges: (m, 2) int32 CUDA tensor
    rank = etl.list_rank(succ, head)
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libetl.so")

STATUS = {0: "ETL_OK", 1: "ETL_EINVAL", 2: "ETL_ENOMEM", 3: "ETL_ECUDA", 4: "ETL_EBADTREE",
          5: "ETL_EBADQUERY", 6: "ETL_EBADGRAPH", 7: "ETL_ETIMEOUT"}
EXPORTS = ("etl_status_string", "etl_list_rank", "etl_list_rank_static", "lca_preprocess", "lca_query", "lca_status", "lca_arrays",
           "lca_export", "lca_free", "find_bridges", "lca_preprocess_batch", "lca_query_batch", "find_bridges_batch",
           "lca_build_inlabel", "lca_query_inlabel", "lca_query_tour", "lca_naive_preprocess", "lca_naive_query",
           "lca_preprocess_ex", "etl_trim", "etl_pool_stats", "two_edge_cc", "find_bridges_hybrid", "etl_profile_enable", "etl_profile_reset",
           "etl_profile_count", "etl_profile_get", "etl_launch_count", "etl_tune_set", "etl_tune_get",
           "etl_workspace_size", "etl_workspace_size_batch", "etl_list_rank_ws", "lca_preprocess_ws",
           "lca_preprocess_batch_ws", "find_bridges_ws", "find_bridges_batch_ws", "etl_status_get",
           "etl_alloc_count", "etl_probe_gather_scatter")
WS_KINDS = {"list_rank": 1, "lca_preprocess": 2, "lca_query": 3, "find_bridges": 4}
TUNE_KEYS = {"rank_k0_log2": 1, "rank_k_log2": 2, "rank_block": 3, "rank_blocks_per_sm": 4,
             "rmq_levels_per_pass": 5, "rmq_block": 6, "cc_first_slice": 7,
             "rmq_blocked": 8, "sort_rounds": 9, "cc_doubling": 10,
             "cc_giant": 11, "sort_ballot": 12, "pdl": 13}

_lock = threading.Lock()
_lib = None


class EtlError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a) if its sources changed."""
    from . import buildlib  # a submodule named like this function would replace it on import
    return buildlib.build(force=force)


def load_library(path: str | None = None):
    """Load (once) and declare the C ABI. Raises if the library is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build the CUDA library first (paper_2103_15217_gb300.build())")
        lib = ctypes.CDLL(p)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        PP = ctypes.POINTER(ctypes.c_void_p)
        lib.etl_status_string.argtypes = [i32]
        lib.etl_status_string.restype = ctypes.c_char_p
        lib.etl_list_rank.argtypes = [P, i64, i32, P, P, P]
        lib.etl_list_rank_static.argtypes = [P, i64, i32, P, P, P]
        lib.lca_preprocess.argtypes = [P, i32, P, PP]
        lib.lca_query.argtypes = [P, P, P, i64, P, P, P]
        lib.lca_status.argtypes = [P, ctypes.POINTER(i32)]
        lib.lca_arrays.argtypes = [P, PP, PP, PP, PP]
        lib.lca_export.argtypes = [P, P, P, P, P, P]
        lib.lca_free.argtypes = [P]
        lib.find_bridges.argtypes = [P, i64, i32, P, P, P]
        lib.lca_preprocess_batch.argtypes = [P, P, i32, i32, i32, P, PP]
        lib.lca_build_inlabel.argtypes = [P, P, P]
        lib.lca_preprocess_ex.argtypes = [P, i32, i32, P, PP]
        lib.two_edge_cc.argtypes = [P, i64, i32, P, P, P]
        lib.find_bridges_hybrid.argtypes = [P, i64, i32, P, P, P]
        lib.etl_trim.argtypes = []
        lib.etl_pool_stats.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.lca_naive_preprocess.argtypes = [P, i32, P, P, P]
        lib.lca_naive_query.argtypes = [P, i32, P, P, i64, P, P, P]
        lib.lca_query_inlabel.argtypes = [P, P, P, i64, P, P, P]
        lib.lca_query_tour.argtypes = [P, P, P, i64, P, P, P]
        lib.lca_query_batch.argtypes = [P, P, P, P, i64, P, P, P]
        lib.find_bridges_batch.argtypes = [P, P, P, i32, i64, i32, P, P, P]
        lib.etl_launch_count.argtypes = [ctypes.POINTER(i64)]
        lib.etl_tune_set.argtypes = [i32, i32]
        lib.etl_tune_get.argtypes = [i32, ctypes.POINTER(i32)]
        lib.etl_profile_enable.argtypes = [i32]
        lib.etl_profile_reset.argtypes = []
        lib.etl_profile_count.argtypes = [ctypes.POINTER(i32)]
        lib.etl_profile_get.argtypes = [i32, ctypes.c_char_p, i32, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(i64)]
        SZ = ctypes.c_size_t
        lib.etl_workspace_size.argtypes = [i32, i64, i64, ctypes.POINTER(SZ)]
        lib.etl_workspace_size_batch.argtypes = [i32, i32, i64, i64, ctypes.POINTER(SZ)]
        lib.etl_list_rank_ws.argtypes = [P, i64, i32, P, P, P, SZ, P]
        lib.lca_preprocess_ws.argtypes = [P, i32, P, SZ, P, PP]
        lib.lca_preprocess_batch_ws.argtypes = [P, P, i32, i32, i32, P, SZ, P, PP]
        lib.find_bridges_ws.argtypes = [P, i64, i32, P, P, P, SZ, P]
        lib.find_bridges_batch_ws.argtypes = [P, P, P, i32, i64, i32, P, P, P, SZ, P]
        lib.etl_status_get.argtypes = [P, P, ctypes.POINTER(i32)]
        lib.etl_alloc_count.argtypes = [ctypes.POINTER(i64)]
        lib.etl_probe_gather_scatter.argtypes = [P, P, i64, P, P]
        for f in EXPORTS[1:]:
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(fn: str, rc: int):
    if rc != 0:
        raise EtlError(fn, rc)


def _dev_i32(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int32 CUDA tensor")
    return t.data_ptr()


def _status_ptr(status) -> int | None:
    if status is None:
        return None
    return _dev_i32(status, "status")


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def new_status(device=None) -> torch.Tensor:
    """A zeroed device status word (int32[1])."""
    return torch.zeros(1, dtype=torch.int32, device=device or "cuda")


def _workspace(ws) -> tuple[int, int]:
    """(pointer, bytes) of a caller-owned device workspace (any contiguous CUDA tensor)."""
    if not isinstance(ws, torch.Tensor) or not ws.is_cuda or not ws.is_contiguous():
        raise TypeError("workspace must be a contiguous CUDA tensor")
    return ws.data_ptr(), ws.numel() * ws.element_size()


def workspace_size(kind: str, n: int, m_or_q: int = 0) -> int:
    """Bytes of caller-owned workspace a ``workspace=`` call of this kind needs (exact, for the tuning
    parameters in force); kind is one of WS_KINDS."""
    b = ctypes.c_size_t(0)
    _check("etl_workspace_size", load_library().etl_workspace_size(WS_KINDS[kind], int(n), int(m_or_q),
                                                                   ctypes.byref(b)))
    return b.value


def workspace_size_batch(kind: str, k: int, total_n: int, max_n_or_total_m: int) -> int:
    """Workspace bytes of a batched call: kind "lca_preprocess" (third size = max_n) or "find_bridges"
    (third size = total_m)."""
    b = ctypes.c_size_t(0)
    _check("etl_workspace_size_batch", load_library().etl_workspace_size_batch(
        WS_KINDS[kind], int(k), int(total_n), int(max_n_or_total_m), ctypes.byref(b)))
    return b.value


def new_workspace(nbytes: int, device=None) -> torch.Tensor:
    """A device buffer of at least nbytes bytes to pass as ``workspace=``."""
    return torch.empty(max(1, int(nbytes)), dtype=torch.uint8, device=device or "cuda")


def probe_gather_scatter(order: torch.Tensor, succ: torch.Tensor, out: torch.Tensor, stream=None):
    """Measurement aid: out[order[i]] = (succ[order[i]], i) with independent random accesses (the
    access pattern of the ranking walk without its dependent chain); out is int32[2n] or int64[n]."""
    if out.numel() * out.element_size() < 8 * order.numel() or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA tensor of 8 bytes per element")
    if succ.numel() < order.numel():
        raise ValueError("succ must have at least as many entries as order")
    _check("etl_probe_gather_scatter", load_library().etl_probe_gather_scatter(
        _dev_i32(order, "order"), _dev_i32(succ, "succ"), order.numel(), out.data_ptr(), _stream(stream)))


def alloc_count() -> int:
    """Device allocations the library has requested so far (workspace carving excluded)."""
    c = ctypes.c_int64(0)
    _check("etl_alloc_count", load_library().etl_alloc_count(ctypes.byref(c)))
    return c.value


def status_get(status: torch.Tensor, stream=None) -> int:
    """Waits for the stream, then reads a device status word."""
    v = ctypes.c_int32(-1)
    _check("etl_status_get", load_library().etl_status_get(_stream(stream), _dev_i32(status, "status"),
                                                           ctypes.byref(v)))
    return v.value


def list_rank(succ: torch.Tensor, head: int, status: torch.Tensor | None = None, stream=None,
              workspace: torch.Tensor | None = None) -> torch.Tensor:
    """rank[e] = distance of element e from ``head`` along ``succ`` (-1 = end). With ``workspace``
    (a device buffer of workspace_size("list_rank", len) bytes) the call allocates nothing."""
    lib = load_library()
    p = _dev_i32(succ, "succ")
    rank = torch.empty_like(succ)
    if workspace is None:
        _check("etl_list_rank", lib.etl_list_rank(p, succ.numel(), int(head), rank.data_ptr(), _status_ptr(status),
                                                  _stream(stream)))
    else:
        wp, wb = _workspace(workspace)
        _check("etl_list_rank_ws", lib.etl_list_rank_ws(p, succ.numel(), int(head), rank.data_ptr(),
                                                        _status_ptr(status), wp, wb, _stream(stream)))
    return rank


class Lca:
    """A preprocessed tree, or a batch of trees: wraps an ``etl_lca_t`` handle."""

    def __init__(self, parent: torch.Tensor, stream=None, node_off: torch.Tensor | None = None,
                 max_n: int | None = None, methods: tuple = ("rmq",), workspace: torch.Tensor | None = None):
        lib = load_library()
        self._lib = lib
        _dev_i32(parent, "parent")  # refuse host tensors before touching any stream
        self.n = parent.numel()
        self.batched = node_off is not None
        self._h = ctypes.c_void_p()
        self._stream = _stream(stream)
        if workspace is not None:
            # the handle's tables live in the caller's workspace, which this object keeps alive
            if tuple(methods) != ("rmq",):
                raise ValueError("a handle in a caller-owned workspace holds the RMQ structure only")
            wp, wb = _workspace(workspace)
            if self.batched:
                self.k = node_off.numel() - 1
                _check("lca_preprocess_batch_ws", lib.lca_preprocess_batch_ws(
                    _dev_i32(parent, "parent"), _dev_i32(node_off, "node_off"), self.k, self.n,
                    int(max_n if max_n is not None else self.n), wp, wb, self._stream, ctypes.byref(self._h)))
            else:
                self.k = 1
                _check("lca_preprocess_ws", lib.lca_preprocess_ws(_dev_i32(parent, "parent"), self.n, wp, wb,
                                                                  self._stream, ctypes.byref(self._h)))
            self._refs = (parent, node_off, workspace)
            return
        if self.batched:
            self.k = node_off.numel() - 1
            _check("lca_preprocess_batch", lib.lca_preprocess_batch(
                _dev_i32(parent, "parent"), _dev_i32(node_off, "node_off"), self.k, self.n,
                int(max_n if max_n is not None else self.n), self._stream, ctypes.byref(self._h)))
        else:
            self.k = 1
            unknown = set(methods) - {"rmq", "inlabel", "tour_rmq"}
            if unknown:
                raise ValueError(f"unknown LCA methods {sorted(unknown)}")
            flags = (1 if "rmq" in methods else 0) | (2 if "inlabel" in methods else 0) | \
                (4 if "tour_rmq" in methods else 0)
            _check("lca_preprocess_ex", lib.lca_preprocess_ex(_dev_i32(parent, "parent"), self.n, flags,
                                                              self._stream, ctypes.byref(self._h)))
        self._refs = (parent, node_off)  # keep the inputs alive until preprocessing has run

    def query(self, u: torch.Tensor, v: torch.Tensor, out: torch.Tensor | None = None,
              status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if u.numel() != v.numel():
            raise ValueError("u and v must have the same length")
        if out is None:
            out = torch.empty_like(u)
        _check("lca_query", self._lib.lca_query(self._h, _dev_i32(u, "u"), _dev_i32(v, "v"), u.numel(),
                                                _dev_i32(out, "out"), _status_ptr(status), _stream(stream)))
        return out

    def query_batch(self, inst: torch.Tensor, u: torch.Tensor, v: torch.Tensor, out: torch.Tensor | None = None,
                    status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Queries of a batch handle: tree ``inst[i]``, local ids in and out."""
        if not (u.numel() == v.numel() == inst.numel()):
            raise ValueError("inst, u and v must have the same length")
        if out is None:
            out = torch.empty_like(u)
        _check("lca_query_batch", self._lib.lca_query_batch(self._h, _dev_i32(inst, "inst"), _dev_i32(u, "u"),
                                                            _dev_i32(v, "v"), u.numel(), _dev_i32(out, "out"),
                                                            _status_ptr(status), _stream(stream)))
        return out

    def build_inlabel(self, parent: torch.Tensor, stream=None):
        """Add the Inlabel (Schieber-Vishkin) structures; parent = the array the handle was built from."""
        _check("lca_build_inlabel", self._lib.lca_build_inlabel(self._h, _dev_i32(parent, "parent"), _stream(stream)))
        self._refs = self._refs + (parent,)
        return self

    def query_inlabel(self, u: torch.Tensor, v: torch.Tensor, out: torch.Tensor | None = None,
                      status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """LCA by the Inlabel method (needs build_inlabel)."""
        if u.numel() != v.numel():
            raise ValueError("u and v must have the same length")
        if out is None:
            out = torch.empty_like(u)
        _check("lca_query_inlabel", self._lib.lca_query_inlabel(self._h, _dev_i32(u, "u"), _dev_i32(v, "v"), u.numel(),
                                                                _dev_i32(out, "out"), _status_ptr(status),
                                                                _stream(stream)))
        return out

    def query_tour(self, u: torch.Tensor, v: torch.Tensor, out: torch.Tensor | None = None,
                   status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """LCA by range minimum over the Euler tour (needs methods including "tour_rmq")."""
        if u.numel() != v.numel():
            raise ValueError("u and v must have the same length")
        if out is None:
            out = torch.empty_like(u)
        _check("lca_query_tour", self._lib.lca_query_tour(self._h, _dev_i32(u, "u"), _dev_i32(v, "v"), u.numel(),
                                                          _dev_i32(out, "out"), _status_ptr(status), _stream(stream)))
        return out

    def status(self) -> int:
        st = ctypes.c_int32(-1)
        _check("lca_status", self._lib.lca_status(self._h, ctypes.byref(st)))
        return st.value

    def arrays(self, stream=None) -> dict:
        """Copies of the per-node arrays: pre, depth, size, order (int32[n])."""
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {k: torch.empty(self.n, dtype=torch.int32, device=dev) for k in ("pre", "depth", "size", "order")}
        _check("lca_export", self._lib.lca_export(self._h, out["pre"].data_ptr(), out["depth"].data_ptr(),
                                                  out["size"].data_ptr(), out["order"].data_ptr(),
                                                  _stream(stream)))
        return out

    def free(self):
        if self._h:
            self._lib.lca_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def profile_enable(on: bool = True):
    """Turn the library's per-phase CUDA-event timers on or off."""
    _check("etl_profile_enable", load_library().etl_profile_enable(1 if on else 0))


def tune_set(**params):
    """Set launch parameters and table forms (no effect on results); names as in TUNE_KEYS."""
    lib = load_library()
    for k, v in params.items():
        _check(f"etl_tune_set({k})", lib.etl_tune_set(TUNE_KEYS[k], int(v)))


def tune_get() -> dict:
    lib = load_library()
    out = {}
    for k, key in TUNE_KEYS.items():
        v = ctypes.c_int32(0)
        _check("etl_tune_get", lib.etl_tune_get(key, ctypes.byref(v)))
        out[k] = v.value
    return out


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    c = ctypes.c_int64(0)
    _check("etl_launch_count", load_library().etl_launch_count(ctypes.byref(c)))
    return c.value


def profile_reset():
    _check("etl_profile_reset", load_library().etl_profile_reset())


def profile_read() -> dict:
    """{phase: (total_ms, launches)} accumulated since the last reset (waits for the events)."""
    lib = load_library()
    cnt = ctypes.c_int32(0)
    _check("etl_profile_count", lib.etl_profile_count(ctypes.byref(cnt)))
    out = {}
    buf = ctypes.create_string_buffer(64)
    for i in range(cnt.value):
        ms, k = ctypes.c_double(0), ctypes.c_int64(0)
        _check("etl_profile_get", lib.etl_profile_get(i, buf, 64, ctypes.byref(ms), ctypes.byref(k)))
        out[buf.value.decode()] = (ms.value, k.value)
    return out


def lca_preprocess(parent: torch.Tensor, stream=None, methods: tuple = ("rmq",),
                   workspace: torch.Tensor | None = None) -> Lca:
    """Preprocess one tree; methods: any of "rmq" (query), "inlabel" (query_inlabel) and "tour_rmq"
    (query_tour). With ``workspace`` (workspace_size("lca_preprocess", n) bytes; RMQ only) nothing is
    allocated and the handle's tables live in that buffer."""
    return Lca(parent, stream, methods=methods, workspace=workspace)


def pool_stats() -> dict:
    """Bytes reserved and in use in the library's memory pool on the current device."""
    r, u = ctypes.c_int64(0), ctypes.c_int64(0)
    _check("etl_pool_stats", load_library().etl_pool_stats(ctypes.byref(r), ctypes.byref(u)))
    return {"reserved": r.value, "used": u.value}


def trim():
    """Give back the device memory the library keeps reserved for reuse."""
    _check("etl_trim", load_library().etl_trim())


def lca_preprocess_batch(parent: torch.Tensor, node_off: torch.Tensor, max_n: int, stream=None,
                         workspace: torch.Tensor | None = None) -> Lca:
    """Trees concatenated in local ids; node_off (device int32[k+1]) delimits them."""
    return Lca(parent, stream, node_off=node_off, max_n=max_n, workspace=workspace)


class NaiveLca:
    """The paper's naive GPU LCA (levels by pointer jumping, queries by climbing)."""

    def __init__(self, parent: torch.Tensor, status: torch.Tensor | None = None, stream=None):
        self._lib = load_library()
        self.n = parent.numel()
        self.rec = torch.empty(2 * self.n, dtype=torch.int32, device=parent.device)
        _check("lca_naive_preprocess", self._lib.lca_naive_preprocess(_dev_i32(parent, "parent"), self.n,
                                                                      self.rec.data_ptr(), _status_ptr(status),
                                                                      _stream(stream)))

    def query(self, u: torch.Tensor, v: torch.Tensor, out: torch.Tensor | None = None,
              status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(u)
        _check("lca_naive_query", self._lib.lca_naive_query(self.rec.data_ptr(), self.n, _dev_i32(u, "u"),
                                                            _dev_i32(v, "v"), u.numel(), _dev_i32(out, "out"),
                                                            _status_ptr(status), _stream(stream)))
        return out


def find_bridges_batch(edges: torch.Tensor, edge_off: torch.Tensor, node_off: torch.Tensor, total_n: int,
                       status: torch.Tensor | None = None, stream=None,
                       workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Bridge masks of k graphs concatenated in local ids (edge_off / node_off: device int32[k+1],
    total_n = node_off[k] given by the caller so that nothing is read back from the device)."""
    lib = load_library()
    if edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("edges must have shape (m, 2)")
    k = node_off.numel() - 1
    m = edges.shape[0]
    mask = torch.empty(m, dtype=torch.uint8, device=edges.device)
    if workspace is None:
        _check("find_bridges_batch", lib.find_bridges_batch(
            _dev_i32(edges, "edges"), _dev_i32(edge_off, "edge_off"), _dev_i32(node_off, "node_off"), k, m, total_n,
            mask.data_ptr(), _status_ptr(status), _stream(stream)))
    else:
        wp, wb = _workspace(workspace)
        _check("find_bridges_batch_ws", lib.find_bridges_batch_ws(
            _dev_i32(edges, "edges"), _dev_i32(edge_off, "edge_off"), _dev_i32(node_off, "node_off"), k, m, total_n,
            mask.data_ptr(), _status_ptr(status), wp, wb, _stream(stream)))
    return mask


def find_bridges(edges: torch.Tensor, n: int, status: torch.Tensor | None = None, stream=None,
                 method: str = "tv", out: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None) -> torch.Tensor:
    """uint8 mask, 1 for every bridge of the undirected multigraph (m, 2).
    method: "tv" (Tarjan-Vishkin low/high) or "hybrid" (tour levels + Chaitanya-Kothapalli marking).
    out: optional contiguous uint8 device tensor of m entries to write the mask into.
    workspace: a device buffer of workspace_size("find_bridges", n, m) bytes ("tv" only): nothing is
    allocated."""
    lib = load_library()
    if edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("edges must have shape (m, 2)")
    m = edges.shape[0]
    if out is None:
        mask = torch.empty(m, dtype=torch.uint8, device=edges.device)
    else:
        if out.dtype != torch.uint8 or out.numel() != m or not out.is_contiguous() or out.device != edges.device:
            raise ValueError("out must be a contiguous uint8 tensor of m entries on the edges' device")
        mask = out
    if workspace is not None:
        if method != "tv":
            raise ValueError("a caller-owned workspace is supported by the Tarjan-Vishkin method only")
        wp, wb = _workspace(workspace)
        _check("find_bridges_ws", lib.find_bridges_ws(_dev_i32(edges, "edges"), m, int(n), mask.data_ptr(),
                                                      _status_ptr(status), wp, wb, _stream(stream)))
        return mask
    fn = {"tv": lib.find_bridges, "hybrid": lib.find_bridges_hybrid}[method]
    _check("find_bridges", fn(_dev_i32(edges, "edges"), m, int(n), mask.data_ptr(), _status_ptr(status),
                              _stream(stream)))
    return mask


def two_edge_cc(edges: torch.Tensor, n: int, status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """2-edge-connected component label (smallest vertex) of every vertex."""
    lib = load_library()
    if edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("edges must have shape (m, 2)")
    label = torch.empty(int(n), dtype=torch.int32, device=edges.device)
    _check("two_edge_cc", lib.two_edge_cc(_dev_i32(edges, "edges"), edges.shape[0], int(n), label.data_ptr(),
                                          _status_ptr(status), _stream(stream)))
    return label
