"""The boundary is plain C: include/etl.h compiles as strict C11 and as C++,
a C program that takes the address of every declared entry point links
against the library, and its host-side argument checks answer as the header
says. Nothing here needs a GPU: every call below is refused on the host."""

import os
import subprocess

import pytest

from test_abi_exports import ROOT, declared_functions

CHECKS = r"""
    etl_lca_t h = 0;
    int32_t v = 0;
    if (lca_preprocess(NULL, 5, NULL, &h) != ETL_EINVAL) return 10;
    if (lca_preprocess((const int32_t *)16, 0, NULL, &h) != ETL_EINVAL) return 11;
    if (lca_query(NULL, NULL, NULL, 5, NULL, NULL, NULL) != ETL_EINVAL) return 12;
    if (find_bridges(NULL, 3, 0, NULL, NULL, NULL) != ETL_EINVAL) return 13;
    if (find_bridges(NULL, 0, 4, NULL, NULL, NULL) != ETL_OK) return 14;
    if (etl_list_rank(NULL, 4, 0, NULL, NULL, NULL) != ETL_EINVAL) return 15;
    if (lca_free(NULL) != ETL_OK) return 16;
    if (etl_tune_get(999, &v) != ETL_EINVAL) return 17;
    if (strcmp(etl_status_string(ETL_EBADTREE), "ETL_EBADTREE") != 0) return 18;
    if (strcmp(etl_status_string(ETL_ETIMEOUT), "ETL_ETIMEOUT") != 0) return 19;
    {
        size_t b = 1;
        if (etl_workspace_size(99, 10, 10, &b) != ETL_EINVAL || b != 0) return 20;
        if (etl_workspace_size(ETL_WS_LCA_QUERY, 10, 5, &b) != ETL_OK || b != 0) return 21;
        if (lca_preprocess_ws((const int32_t *)16, 5, NULL, 1024, NULL, &h) != ETL_EINVAL) return 22;
        if (find_bridges_ws((const int32_t *)16, 3, 4, (uint8_t *)16, NULL, NULL, 1024, NULL) != ETL_EINVAL)
            return 23;
        if (etl_status_get(NULL, NULL, &v) != ETL_EINVAL) return 24;
    }
    puts("ok");
    return 0;
"""


def client_source():
    fns = declared_functions()
    table = ",\n        ".join(f"(fn_t){f}" for f in fns)
    return (f'#include <stdio.h>\n#include <string.h>\n#include "etl.h"\n'
            f"typedef void (*fn_t)(void);\n"
            f"int main(void) {{\n"
            f"    fn_t entry[] = {{\n        {table}\n    }};\n"
            f"    for (size_t i = 0; i < sizeof entry / sizeof entry[0]; ++i)\n"
            f"        if (!entry[i]) return 1;\n"
            f"{CHECKS}}}\n")


@pytest.fixture(scope="module")
def libdir():
    import paper_2103_15217_gb300 as etl
    return os.path.dirname(etl.build())


def test_header_is_plain_c_and_cxx(tmp_path):
    inc = os.path.join(ROOT, "include")
    for compiler, ext, std in (("gcc", "c", "-std=c11"), ("g++", "cpp", "-std=c++17")):
        src = tmp_path / f"h.{ext}"
        src.write_text('#include "etl.h"\nint etl_header_only;\n')
        subprocess.check_call([compiler, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, "-c", str(src),
                               "-o", str(tmp_path / f"h_{ext}.o")])


def test_c_client_links_and_checks_arguments(tmp_path, libdir):
    src = tmp_path / "client.c"
    src.write_text(client_source())
    exe = tmp_path / "client"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                           str(src), "-L", libdir, "-letl", f"-Wl,-rpath,{libdir}", "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
