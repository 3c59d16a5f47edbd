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


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2103_15217_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src and "etl_oracle" not in src, f
