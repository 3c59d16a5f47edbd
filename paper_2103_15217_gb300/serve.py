"""Continuous-batching request server for LCA queries and bridge finding.

Trees are preprocessed once and stay resident on the device (one batched LCA
handle: Euler tour, preorder, range-minimum table for all of them). Requests arrive
over time: an LCA request carries a batch of (u, v) pairs for one resident
tree; a bridge request carries a fresh graph. The server loop

  * admits arrived requests in arrival order while the bytes they need fit
    the HBM budget (resident tables are charged once, up front);
  * merges every admitted LCA request into one ``lca_query_batch`` launch
    (queries of different trees mixed, tagged by tree) and every admitted
    bridge request into one ``find_bridges_batch`` launch;
  * runs each such batch on its own CUDA stream ("slot"), so batches overlap
    on the device, and keeps forming new batches from requests that arrive
    while earlier ones are still running: requests join as soon as a slot
    and budget are free rather than waiting for a fixed batch to fill.

Per-request latency is measured on the device clock: completion = the CUDA
event recorded after the request's result copy, relative to an event
recorded when the server started. With ``batching=False`` and one slot the
same loop serves one request per launch in arrival order ("plain per-request
launches"), the baseline the batched server is compared against.

Results never depend on what else is in a batch: queries are answered
independently and the bridges of a disjoint union are the union of the
bridges of its parts.
"""

from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np
import torch

from . import find_bridges_batch, lca_preprocess_batch

LCA_BYTES_PER_QUERY = 16          # inst, u, v, out (int32)
GRAPH_BYTES_PER_EDGE = 48         # edges, flags, prefix sums, masks, staging
GRAPH_BYTES_PER_NODE = 520        # union-find, tour, ranking, low / high tables over 2n positions (full form)


@dataclasses.dataclass
class Request:
    kind: str                     # "lca" or "bridges"
    t: float                      # arrival, seconds after the server starts
    tree: int = -1                # lca: resident tree index
    u: np.ndarray | None = None   # lca: local ids
    v: np.ndarray | None = None
    n: int = 0                    # bridges: nodes
    edges: np.ndarray | None = None  # bridges: (m, 2) local ids
    rid: int = -1

    def units(self) -> int:
        return int(self.u.shape[0]) if self.kind == "lca" else int(self.edges.shape[0])

    def bytes(self) -> int:
        if self.kind == "lca":
            return LCA_BYTES_PER_QUERY * int(self.u.shape[0])
        return GRAPH_BYTES_PER_EDGE * int(self.edges.shape[0]) + GRAPH_BYTES_PER_NODE * int(self.n)


@dataclasses.dataclass
class Result:
    rid: int
    kind: str
    out: np.ndarray
    t_arrive: float
    t_admit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


class _Batch:
    def __init__(self, reqs, stream, nbytes):
        self.reqs = reqs
        self.stream = stream
        self.nbytes = nbytes
        self.done = torch.cuda.Event(enable_timing=True)
        self.keep = []            # device / pinned buffers alive until the batch is done
        self.outs = []            # (request, pinned host view)
        self.t_admit = 0.0


def resident_bytes(sizes, blocked: bool = True) -> int:
    """Device bytes of a resident batch handle over trees of these sizes: pre, depth, size, order and
    the range-minimum table (blocked: three int32 arrays of n plus a sparse table over blocks of 32,
    and a 16-byte query record per node; full: one int32 row of n per level)."""
    n = int(sum(sizes))
    if blocked:
        nblk = (n + 31) // 32
        levels = int(np.ceil(np.log2(max(2, (max(sizes) + 31) // 32 + 1)))) + 1
        return 32 * n + 4 * (3 * nblk * 32 + nblk * levels)  # + one 16-byte query record per node
    levels = int(np.ceil(np.log2(max(2, max(sizes))))) + 1
    return 16 * n + 4 * ((n + 3) // 4 * 4) * levels


def form_batch(queue, used: int, budget: int, batching: bool, max_q: int, max_g: int, idle: bool):
    """Take the next batch from the head of the arrival-ordered queue (a deque, consumed in place):
    requests join in order while their bytes fit the budget next to `used`, at most max_q LCA queries
    and max_g graphs per batch (one request when not batching). A request too large for the whole
    budget runs alone once nothing else is resident (`idle`). Returns (batch, bytes)."""
    batch, nb, nq, ng = [], 0, 0, 0
    while queue:
        r = queue[0]
        rb = r.bytes()
        if used + nb + rb > budget:
            break
        if batch and not batching:
            break
        if r.kind == "lca" and batch and nq + r.units() > max_q:
            break
        if r.kind == "bridges" and batch and ng + 1 > max_g:
            break
        batch.append(queue.popleft())
        nb += rb
        if r.kind == "lca":
            nq += r.units()
        else:
            ng += 1
    if not batch and idle and queue:
        r = queue.popleft()  # larger than the whole budget: run it alone
        batch, nb = [r], r.bytes()
    return batch, nb


class Server:
    def __init__(self, tree_parents, budget_bytes: int = 40 << 30, slots: int = 4,
                 max_batch_queries: int = 1 << 23, max_batch_graphs: int = 16, device=None):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        sizes = [int(p.shape[0]) for p in tree_parents]
        self.sizes = np.array(sizes, np.int64)
        off = np.zeros(len(sizes) + 1, np.int32)
        off[1:] = np.cumsum(sizes)
        self.budget = int(budget_bytes)
        from . import tune_get
        self.resident = resident_bytes(sizes, blocked=bool(tune_get()["rmq_blocked"]))
        if self.resident > self.budget:
            raise ValueError("resident trees alone exceed the HBM budget")
        parent = torch.from_numpy(np.concatenate(tree_parents).astype(np.int32)).to(self.dev)
        self.handle = lca_preprocess_batch(parent, torch.from_numpy(off).to(self.dev), int(max(sizes)))
        if self.handle.status() != 0:
            raise ValueError(f"resident trees rejected (status {self.handle.status()})")
        self.slots = [torch.cuda.Stream(self.dev) for _ in range(max(1, slots))]
        self.max_q = max_batch_queries
        self.max_g = max_batch_graphs

    def close(self):
        self.handle.free()

    # -------------------------------------------------------------- launches

    def _launch(self, reqs, stream) -> _Batch:
        b = _Batch(reqs, stream, sum(r.bytes() for r in reqs))
        with torch.cuda.stream(stream):
            lca = [r for r in reqs if r.kind == "lca"]
            gr = [r for r in reqs if r.kind == "bridges"]
            if lca:
                q = sum(r.u.shape[0] for r in lca)
                host = torch.empty((3, q), dtype=torch.int32).pin_memory()
                pos = 0
                for r in lca:
                    k = r.u.shape[0]
                    host[0, pos:pos + k] = r.tree
                    host[1, pos:pos + k] = torch.from_numpy(r.u)
                    host[2, pos:pos + k] = torch.from_numpy(r.v)
                    pos += k
                d = host.to(self.dev, non_blocking=True)
                out = self.handle.query_batch(d[0], d[1], d[2])
                out_h = torch.empty(q, dtype=torch.int32).pin_memory()
                out_h.copy_(out, non_blocking=True)
                b.keep += [host, d, out]
                pos = 0
                for r in lca:
                    k = r.u.shape[0]
                    b.outs.append((r, out_h[pos:pos + k]))
                    pos += k
            if gr:
                m = sum(r.edges.shape[0] for r in gr)
                eh = torch.empty((m, 2), dtype=torch.int32).pin_memory()
                offs = np.zeros((2, len(gr) + 1), np.int32)
                pos = 0
                for i, r in enumerate(gr):
                    k = r.edges.shape[0]
                    eh[pos:pos + k] = torch.from_numpy(r.edges)
                    pos += k
                    offs[0, i + 1] = pos
                    offs[1, i + 1] = offs[1, i] + r.n
                oh = torch.from_numpy(offs).pin_memory()
                de = eh.to(self.dev, non_blocking=True)
                do = oh.to(self.dev, non_blocking=True)
                mask = find_bridges_batch(de, do[0], do[1], int(offs[1, -1]))
                mh = torch.empty(m, dtype=torch.uint8).pin_memory()
                mh.copy_(mask, non_blocking=True)
                b.keep += [eh, oh, de, do, mask]
                pos = 0
                for r in gr:
                    k = r.edges.shape[0]
                    b.outs.append((r, mh[pos:pos + k]))
                    pos += k
            b.done.record(stream)
        return b

    # -------------------------------------------------------------- the loop

    def serve(self, requests, batching: bool = True, realtime: bool = True):
        """Serve requests (arrival times in seconds from now); returns results in request order."""
        reqs = sorted(requests, key=lambda r: r.t)
        for i, r in enumerate(reqs):
            if r.rid < 0:
                r.rid = i
        slots = self.slots if batching else self.slots[:1]
        torch.cuda.synchronize(self.dev)
        t0_ev = torch.cuda.Event(enable_timing=True)
        t0_ev.record(slots[0])
        t0_ev.synchronize()
        t0 = time.perf_counter()
        pending = deque(reqs)
        queue = deque()
        inflight = {}                 # slot index -> batch
        used = self.resident
        results = {}

        def now():
            return time.perf_counter() - t0

        while pending or queue or inflight:
            t = now() if realtime else float("inf")
            while pending and pending[0].t <= t:
                queue.append(pending.popleft())
            for si, b in list(inflight.items()):
                if b.done.query():
                    t_done = t0_ev.elapsed_time(b.done) / 1e3
                    for r, h in b.outs:
                        results[r.rid] = Result(r.rid, r.kind, h.numpy().copy(), r.t, b.t_admit, t_done)
                    used -= b.nbytes
                    del inflight[si]
            free = [i for i in range(len(slots)) if i not in inflight]
            while free and queue:
                batch, nb = form_batch(queue, used, self.budget, batching, self.max_q, self.max_g,
                                       idle=not inflight and used == self.resident)
                if not batch:
                    break
                si = free.pop(0)
                b = self._launch(batch, slots[si])
                b.t_admit = now()
                used += nb
                inflight[si] = b
            if not (queue and free):
                if inflight and not (pending and pending[0].t <= now()):
                    time.sleep(20e-6)
                elif not inflight and pending:
                    wait = pending[0].t - now()
                    if wait > 0:
                        time.sleep(min(wait, 1e-3))
        torch.cuda.synchronize(self.dev)
        return [results[r.rid] for r in sorted(reqs, key=lambda r: r.rid)]


def summarize(results, wall_units=None) -> dict:
    lat = np.array([r.latency for r in results])
    units = sum(int(r.out.shape[0]) for r in results) if wall_units is None else wall_units
    t_first = min(r.t_arrive for r in results)
    t_last = max(r.t_done for r in results)
    return {"requests": len(results), "units": int(units), "seconds": t_last - t_first,
            "throughput": units / max(t_last - t_first, 1e-9),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
