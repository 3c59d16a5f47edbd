"""Autotuner for the launch parameters of the Euler-tour library.

The knobs change no result, only speed (``etl_tune_set``): the list ranker's
splitter densities and walk-kernel shape (threads per block and resident
blocks per SM of the walks over lists larger than L2), the range tables'
form and build shape, the radix passes' tile size and ranking, and the
connectivity pass's hooking schedule, and whether kernels are launched as
programmatic dependents of the one before. ``autotune`` times candidate settings
with CUDA events on the caller's own work -- a callable that enqueues one
representative run (for example one batch of trees and graphs of the mix to
be served), with its inputs already on the device -- and keeps the fastest.
Results are cached per (GPU name, caller's key) in ``_build/tune_cache.json``
so later runs start from the tuned values.

The search is coordinate-wise: ranking density first (it sets the length of
the longest dependent walk), then the walk kernel's shape, then the other
knobs in the order of SPACE; each coordinate keeps the best value found before
moving on.
"""

from __future__ import annotations

import json
import os
import statistics

import torch

from . import load_library, tune_get, tune_set

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")

SPACE = [
    ("rank_k0_log2", [2, 3, 4, 5]),
    ("rank_k_log2", [3, 4, 5]),
    ("rank_block", [128, 256, 512]),
    ("rank_blocks_per_sm", [4, 8, 16]),
    ("rmq_levels_per_pass", [1, 2, 3]),
    ("rmq_block", [256, 512]),
    ("cc_first_slice", [1, 2, 4, 8]),
    ("cc_doubling", [0, 1]),
    ("cc_giant", [0, 1]),
    ("rmq_blocked", [0, 1]),
    ("sort_rounds", [8, 16]),
    ("sort_ballot", [0, 1]),
    ("pdl", [0, 1]),
]


def _key(key: str) -> str:
    return f"{torch.cuda.get_device_name()}|{key}"


def _load_cache() -> dict:
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c: dict):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def _time(fn, reps: int) -> float:
    s = torch.cuda.current_stream()
    fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def valid(params: dict) -> bool:
    """Settings the library accepts together (each knob's own range is checked by etl_tune_set)."""
    return params["rank_block"] * params["rank_blocks_per_sm"] <= 2048


def coordinate_search(space, start: dict, measure, is_valid=lambda p: True):
    """Coordinate-wise search: for each (name, values) of space in turn, try every value with the
    other knobs at the best setting so far and keep the fastest; measure(params) returns a time
    (lower is better) or None for a setting to skip. Returns (best, best_time, trials)."""
    best = dict(start)
    best_t = measure(best)
    trials = [(dict(best), best_t)]
    for name, values in space:
        for v in values:
            if v == best[name]:
                continue
            cand = dict(best, **{name: v})
            if not is_valid(cand):
                continue
            t = measure(cand)
            if t is None:
                continue
            trials.append((dict(cand), t))
            if t < best_t:
                best, best_t = cand, t
    return best, best_t, trials


def autotune(workload, key: str, reps: int = 3, use_cache: bool = True, verbose: bool = False,
             space=SPACE) -> dict:
    """Tune on the caller's work: workload() enqueues one representative run on the current stream
    (inputs already on the device; every call must do the same work). key names the workload in the
    cache. Applies the best setting and returns {"params", "ms", "default_ms", "trials"}."""
    load_library()
    ckey = _key(key)
    cache = _load_cache() if use_cache else {}
    if ckey in cache:
        tune_set(**cache[ckey]["params"])
        return dict(cache[ckey], cached=True)

    def measure(params):
        try:
            tune_set(**params)
        except Exception:
            return None  # rejected by the library
        ms = _time(workload, reps)
        if verbose:
            print(f"  {params}: {ms:.3f} ms")
        return ms

    best, best_ms, trials = coordinate_search(space, tune_get(), measure, valid)
    tune_set(**best)
    res = {"params": best, "ms": best_ms, "key": key, "trials": len(trials), "default_ms": trials[0][1]}
    cache[ckey] = res
    _save_cache(cache)
    return res
