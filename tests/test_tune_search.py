"""The autotuner's coordinate search (host logic, no GPU): it finds the
optimum of a separable cost, keeps the starting point when nothing is
faster, skips settings that are invalid or that the library rejects, and
every knob it searches exists in the library's key table."""

import itertools

from paper_2103_15217_gb300 import TUNE_KEYS
from paper_2103_15217_gb300.tune import SPACE, coordinate_search, valid


def test_finds_separable_optimum():
    space = [("a", [1, 2, 3, 4]), ("b", [10, 20, 30]), ("c", [0, 1])]
    target = {"a": 3, "b": 20, "c": 1}
    cost = lambda p: sum((p[k] - target[k]) ** 2 for k in target)  # noqa: E731
    best, t, trials = coordinate_search(space, {"a": 1, "b": 10, "c": 0}, cost)
    assert best == target and t == 0
    assert len(trials) == 1 + 3 + 2 + 1  # the start, then every other value of each knob once


def test_keeps_start_when_nothing_is_faster():
    space = [("a", [1, 2]), ("b", [5, 6])]
    best, t, _ = coordinate_search(space, {"a": 1, "b": 5}, lambda p: 1.0 + (p != {"a": 1, "b": 5}))
    assert best == {"a": 1, "b": 5} and t == 1.0


def test_skips_invalid_and_rejected_settings():
    space = [("a", [1, 2, 3]), ("b", [1, 2, 3])]
    seen = []

    def measure(p):
        seen.append(dict(p))
        return None if p["a"] == 3 else -p["a"] - p["b"]  # the library rejects a = 3
    best, _, trials = coordinate_search(space, {"a": 1, "b": 1}, measure, lambda p: p["a"] + p["b"] <= 4)
    assert best == {"a": 2, "b": 2}
    assert all(p["a"] + p["b"] <= 4 for p in seen)
    assert all(p["a"] != 3 for p, _ in trials)


def test_space_matches_library_keys():
    for name, values in SPACE:
        assert name in TUNE_KEYS and len(values) >= 2
    # the shape constraint admits the library's default walk shape and rejects oversubscription
    assert valid({"rank_block": 128, "rank_blocks_per_sm": 4})
    assert not valid({"rank_block": 512, "rank_blocks_per_sm": 8})
    names = [n for n, _ in SPACE]
    assert len(names) == len(set(names))
    assert all(a != b for a, b in itertools.combinations(names, 2))
