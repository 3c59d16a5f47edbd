"""Planted mistakes: each mutation of the C oracle must be caught by the pins.

A copy of the oracle source gets one plausible bug (a dropped term, a wrong
comparison, a swapped operand, the paper's garbled bridge criterion taken
literally), is compiled with gcc into a temporary directory and swapped in for
the real oracle; at least one pin of ``test_oracle_pins`` must then fail.
Everything runs on the CPU. Every mutation keeps the oracle's loops bounded.
"""

import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "etl_oracle.c")

MUTATIONS = {
    "children_descending": (
        "for (int32_t c = 0; c < n; ++c)\n        if (parent[c] >= 0) kids[fill[parent[c]]++] = c;",
        "for (int32_t c = n - 1; c >= 0; --c)\n        if (parent[c] >= 0) kids[fill[parent[c]]++] = c;"),
    "size_off_by_one": ("size[v] = visited - pre[v];", "size[v] = visited - pre[v] - 1;"),
    "climb_one_step_too_far": ("        out[i] = a;\n    }\n    return rc;", "        out[i] = parent[a] >= 0 ? parent[a] : a;\n    }\n    return rc;"),
    "offline_wrong_ancestor": ("anc[rp] = p;", "anc[rp] = x;"),
    "dcel_succ_without_twin": ("int64_t t = a ^ 1;                 /* twin(a) */", "int64_t t = a;"),
    "dfs_strict_low_test": ("(uint8_t)(low[x] >= pre[x])", "(uint8_t)(low[x] > pre[x])"),
    "dfs_skip_no_edge": ("if (eid[j] == in_edge[x]) continue; /* the tree edge x was entered by */", ""),
    "tv_literal_garbled_criterion": (
        "(uint8_t)(lo >= pre[x] && hi < pre[x] + size[x])",
        "(uint8_t)(lo < pre[x] || hi >= pre[x] + size[x])"),
    "tv_high_off_by_one": ("hi < pre[x] + size[x])", "hi <= pre[x] + size[x])"),
    "tv_drop_high": ("(uint8_t)(lo >= pre[x] && hi < pre[x] + size[x])", "(uint8_t)(lo >= pre[x])"),
    "depth_not_incremented": ("depth[c] = depth[v] + 1;", "depth[c] = depth[v];"),
    "dcel_sort_by_target_first": ("if (ax != bx) return ax < bx ? -1 : 1;\n    if (ay != by) return ay < by ? -1 : 1;",
                                  "if (ay != by) return ay < by ? -1 : 1;\n    if (ax != bx) return ax < bx ? -1 : 1;"),
    "dcel_wrap_to_following_entry": (": B[first[x]];", ": B[(i + 1) % na];"),
    "tv_non_tree_edge_one_end_only": ("        if (pre[a] < nlo[b]) nlo[b] = pre[a];\n        if (pre[a] > nhi[b]) nhi[b] = pre[a];\n",
                                      ""),
    "tv_no_subtree_aggregation": ("            if (nlo[x] < nlo[p]) nlo[p] = nlo[x];\n            if (nhi[x] > nhi[p]) nhi[p] = nhi[x];\n",
                                  "            (void)p;\n"),
    "two_edge_cc_keeps_bridges": ("        if (br[e]) continue;\n", ""),
    "two_edge_cc_largest_label": ("if (a < b) uf[b] = a; else uf[a] = b;", "if (a < b) uf[a] = b; else uf[b] = a;"),
}

PINS = [
    pins.test_fig1_tour_pre_depth_size,
    pins.test_fig2_dcel_arrays_and_successor,
    pins.test_fig1_lca,
    lambda: pins.test_all_rooted_trees_bruteforce(5),
    lambda: pins.test_random_trees(16, 1),
    pins.test_path_closed_form,
    pins.test_bridges_bruteforce_random_multigraphs,
    lambda: pins.test_hard_graph_closed_form(1),
    pins.test_two_edge_cc_closed_forms,
    pins.test_two_edge_cc_bruteforce,
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found in the oracle source"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    lib_path = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-w", "-shared", "-fPIC", str(mutated), "-o", str(lib_path)])
    lib = oracle.bind(ctypes.CDLL(str(lib_path)))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, oracle.OracleError, IndexError, ValueError):
            caught += 1
            break
    assert caught, f"planted mistake {name!r} passed every pin"
