"""The CUDA library builds, loads without a GPU, exports every function that
include/etl.h declares, and rejects bad host-side arguments before touching
the device (no compute call is made here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "etl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_][a-z_0-9]*)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_2103_15217_gb300 as etl
    etl.build()
    return etl.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("lca_preprocess", "lca_query", "lca_free", "find_bridges", "etl_list_rank"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2103_15217_gb300 as etl
    names = declared_functions()
    for f in names:
        assert hasattr(lib, f), f"{f} declared in etl.h but not exported"
    assert set(names) <= set(etl.EXPORTS)


def test_status_strings(lib):
    assert lib.etl_status_string(0) == b"ETL_OK"
    assert lib.etl_status_string(4) == b"ETL_EBADTREE"
    assert lib.etl_status_string(99) == b"ETL_UNKNOWN"


def test_host_side_validation(lib):
    h = ctypes.c_void_p()
    assert lib.lca_preprocess(None, 5, None, ctypes.byref(h)) == 1
    assert lib.lca_preprocess(ctypes.c_void_p(16), 0, None, ctypes.byref(h)) == 1
    assert lib.lca_preprocess(ctypes.c_void_p(16), 5, None, None) == 1
    assert lib.lca_query(None, None, None, 5, None, None, None) == 1
    assert lib.find_bridges(None, 3, 0, None, None, None) == 1
    assert lib.find_bridges(None, -1, 4, None, None, None) == 1
    assert lib.find_bridges(None, 0, 4, None, None, None) == 0      # no edges: nothing to do
    assert lib.etl_list_rank(None, 4, 0, None, None, None) == 1
    assert lib.etl_list_rank(ctypes.c_void_p(16), 4, 4, ctypes.c_void_p(16), None, None) == 1
    assert lib.lca_free(None) == 0
    big = 1 << 30  # one past the largest tree (2^30 - 1 nodes: two list elements per node in 31 bits)
    assert lib.lca_preprocess(ctypes.c_void_p(16), big, None, ctypes.byref(h)) == 1

    for flags in (0, 8, 16, -1):  # no method, or an unknown bit
        assert lib.lca_preprocess_ex(ctypes.c_void_p(16), 5, flags, None, ctypes.byref(h)) == 1
    assert lib.lca_preprocess_ex(ctypes.c_void_p(16), big, 1, None, ctypes.byref(h)) == 1
    fake = ctypes.c_void_p(16)  # never dereferenced: each call below is refused on the host
    assert lib.find_bridges(fake, 3, big, fake, None, None) == 1           # forest tour past 2^31 - 2
    assert lib.find_bridges_hybrid(fake, 3, big, fake, None, None) == 1
    assert lib.two_edge_cc(fake, 3, big, fake, None, None) == 1
    assert lib.find_bridges_batch(fake, fake, fake, 1, 3, big, fake, None, None) == 1
    off = ctypes.c_void_p(32)
    assert lib.lca_preprocess_batch(ctypes.c_void_p(16), off, 0, 5, 5, None, ctypes.byref(h)) == 1   # k < 1
    assert lib.lca_preprocess_batch(ctypes.c_void_p(16), off, 2, 5, 6, None, ctypes.byref(h)) == 1   # max_n > n
    assert lib.lca_preprocess_batch(ctypes.c_void_p(16), off, 6, 5, 1, None, ctypes.byref(h)) == 1   # k > n
    assert lib.lca_preprocess_batch(ctypes.c_void_p(16), None, 2, 5, 3, None, ctypes.byref(h)) == 1
    assert lib.lca_query_inlabel(None, None, None, 4, None, None, None) == 1   # no handle
    assert lib.lca_query_tour(None, None, None, 4, None, None, None) == 1
    assert lib.lca_query_batch(None, None, None, None, 4, None, None, None) == 1
    assert lib.find_bridges_batch(None, None, None, 1, 4, 4, None, None, None) == 1
    assert lib.two_edge_cc(None, 3, 4, None, None, None) == 1
    assert lib.etl_pool_stats(None, None) == 1
    v = ctypes.c_int32(0)
    assert lib.etl_tune_get(999, ctypes.byref(v)) == 1
    assert lib.etl_tune_set(999, 1) == 1
    for key, bad in ((1, 0), (1, 9), (3, 100), (5, 4), (7, 0), (8, 2), (9, 12), (12, 2), (13, 2)):
        assert lib.etl_tune_set(key, bad) == 1, (key, bad)
    for key in range(1, 14):  # every key reads back, and writing back its value is accepted
        assert lib.etl_tune_get(key, ctypes.byref(v)) == 0
        assert lib.etl_tune_set(key, v.value) == 0


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2103_15217_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "etl_oracle" not in src, f


def test_workspace_entry_points_validate_on_the_host(lib):
    # refused before any CUDA call: unknown kinds, sizes out of range, a missing workspace
    b = ctypes.c_size_t(123)
    assert lib.etl_workspace_size(99, 10, 10, ctypes.byref(b)) == 1 and b.value == 0
    assert lib.etl_workspace_size(2, 0, 0, ctypes.byref(b)) == 1              # n < 1
    assert lib.etl_workspace_size(4, 10, -1, ctypes.byref(b)) == 1            # m < 0
    assert lib.etl_workspace_size(3, 10, 5, ctypes.byref(b)) == 0 and b.value == 0   # queries: no scratch
    assert lib.etl_workspace_size(2, 10, 0, None) == 1
    assert lib.etl_workspace_size_batch(2, 0, 10, 5, ctypes.byref(b)) == 1     # k < 1
    assert lib.etl_workspace_size_batch(2, 3, 10, 11, ctypes.byref(b)) == 1    # max_n > total_n
    h = ctypes.c_void_p(77)
    assert lib.lca_preprocess_ws(ctypes.c_void_p(16), 5, None, 1 << 20, None, ctypes.byref(h)) == 1
    assert h.value is None                                                    # *out cleared
    assert lib.etl_list_rank_ws(ctypes.c_void_p(16), 4, 0, ctypes.c_void_p(16), None, None, 1 << 20, None) == 1
    assert lib.find_bridges_ws(ctypes.c_void_p(16), 3, 4, ctypes.c_void_p(16), None, None, 1 << 20, None) == 1
    assert lib.find_bridges_batch_ws(ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 3, 4,
                                     ctypes.c_void_p(16), None, None, 1 << 20, None) == 1
    assert lib.lca_preprocess_batch_ws(ctypes.c_void_p(16), ctypes.c_void_p(16), 1, 5, 5, None, 1 << 20, None,
                                       ctypes.byref(h)) == 1
    v = ctypes.c_int32(0)
    assert lib.etl_status_get(None, None, ctypes.byref(v)) == 1
    c = ctypes.c_int64(-1)
    assert lib.etl_alloc_count(ctypes.byref(c)) == 0 and c.value >= 0
    assert lib.etl_alloc_count(None) == 1
