"""A plain C program computes on the GPU through include/etl.h alone.

The program is compiled with gcc against the library and the CUDA runtime,
allocates device memory with cudaMalloc, and runs the worked example of
Figures 1-2 (Sec. 2): lca_preprocess / lca_query / lca_export on the tree of
Figure 1, the same with a caller-owned workspace (lca_preprocess_ws), and
find_bridges / find_bridges_ws on a small graph whose bridges are known in
closed form (a cycle with a pendant path: only the path edges are bridges).
Its printed answers are compared with the golden values read off the figures
and with the oracle.
"""

import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from test_abi_exports import ROOT

pytestmark = pytest.mark.gpu

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime_api.h>
#include "etl.h"

#define CK(x) do { int rc_ = (int)(x); if (rc_) { printf("fail %s = %d\n", #x, rc_); return 1; } } while (0)

static int32_t *to_dev(const int32_t *h, size_t n) {
    void *d = NULL;
    if (cudaMalloc(&d, n * sizeof(int32_t) + 4) != cudaSuccess) return NULL;
    if (cudaMemcpy(d, h, n * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) return NULL;
    return (int32_t *)d;
}

static void print_arr(const char *name, const int32_t *d, size_t n) {
    int32_t *h = (int32_t *)malloc(n * sizeof(int32_t));
    cudaMemcpy(h, d, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    printf("%s", name);
    for (size_t i = 0; i < n; ++i) printf(" %d", h[i]);
    printf("\n");
    free(h);
}

int main(void) {
    const int32_t parent[] = {PARENT};
    const int32_t n = (int32_t)(sizeof parent / sizeof parent[0]);
    const int32_t qu[] = {QU}, qv[] = {QV};
    const int64_t q = (int64_t)(sizeof qu / sizeof qu[0]);
    const int32_t edges[] = {EDGES};
    const int64_t m = (int64_t)(sizeof edges / sizeof edges[0]) / 2;
    const int32_t gn = GN;

    int32_t *d_parent = to_dev(parent, (size_t)n), *d_u = to_dev(qu, (size_t)q), *d_v = to_dev(qv, (size_t)q);
    int32_t *d_edges = to_dev(edges, (size_t)(2 * m));
    int32_t *d_out = NULL, *d_status = NULL, *d_arr = NULL;
    uint8_t *d_mask = NULL;
    if (!d_parent || !d_u || !d_v || !d_edges) { printf("fail cudaMalloc\n"); return 1; }
    CK(cudaMalloc((void **)&d_out, (size_t)q * sizeof(int32_t)));
    CK(cudaMalloc((void **)&d_status, sizeof(int32_t)));
    CK(cudaMalloc((void **)&d_arr, 3 * (size_t)n * sizeof(int32_t)));
    CK(cudaMalloc((void **)&d_mask, (size_t)m));
    CK(cudaMemset(d_status, 0, sizeof(int32_t)));

    /* the plain entry points */
    etl_lca_t h = NULL;
    int32_t st = -1;
    CK(lca_preprocess(d_parent, n, NULL, &h));
    CK(lca_query(h, d_u, d_v, q, d_out, d_status, NULL));
    CK(lca_export(h, d_arr, d_arr + n, d_arr + 2 * n, NULL, NULL));
    CK(lca_status(h, &st));
    printf("tree_status %d\n", st);
    print_arr("lca", d_out, (size_t)q);
    print_arr("pre", d_arr, (size_t)n);
    print_arr("depth", d_arr + n, (size_t)n);
    print_arr("size", d_arr + 2 * n, (size_t)n);
    CK(lca_free(h));
    CK(find_bridges(d_edges, m, gn, d_mask, d_status, NULL));
    CK(etl_status_get(NULL, d_status, &st));
    printf("graph_status %d\n", st);
    {
        uint8_t *mk = (uint8_t *)malloc((size_t)m);
        cudaMemcpy(mk, d_mask, (size_t)m, cudaMemcpyDeviceToHost);
        printf("bridges");
        for (int64_t i = 0; i < m; ++i) printf(" %d", mk[i]);
        printf("\n");
        free(mk);
    }

    /* the same with caller-owned workspaces: nothing allocated by the library */
    size_t bt = 0, bg = 0;
    int64_t a0 = 0, a1 = 0;
    void *ws_t = NULL, *ws_g = NULL;
    CK(etl_workspace_size(ETL_WS_LCA_PREPROCESS, n, 0, &bt));
    CK(etl_workspace_size(ETL_WS_FIND_BRIDGES, gn, m, &bg));
    CK(cudaMalloc(&ws_t, bt));
    CK(cudaMalloc(&ws_g, bg));
    CK(cudaMemset(d_out, 0xff, (size_t)q * sizeof(int32_t)));
    CK(cudaMemset(d_mask, 7, (size_t)m));
    CK(etl_alloc_count(&a0));
    CK(lca_preprocess_ws(d_parent, n, ws_t, bt, NULL, &h));
    CK(lca_query(h, d_u, d_v, q, d_out, d_status, NULL));
    CK(find_bridges_ws(d_edges, m, gn, d_mask, d_status, ws_g, bg, NULL));
    CK(etl_status_get(NULL, d_status, &st));
    CK(etl_alloc_count(&a1));
    printf("ws_status %d allocs %lld\n", st, (long long)(a1 - a0));
    print_arr("ws_lca", d_out, (size_t)q);
    {
        uint8_t *mk = (uint8_t *)malloc((size_t)m);
        cudaMemcpy(mk, d_mask, (size_t)m, cudaMemcpyDeviceToHost);
        printf("ws_bridges");
        for (int64_t i = 0; i < m; ++i) printf(" %d", mk[i]);
        printf("\n");
        free(mk);
    }
    CK(lca_free(h));
    cudaFree(ws_t);
    cudaFree(ws_g);
    printf("done\n");
    return 0;
}
"""


def _graph():
    # a 6-cycle 0..5 with a pendant path 5-6-7-8, a parallel copy of edge 1-2 and a self-loop at 3:
    # the bridges are exactly the three path edges (Sec. 4: deleting one disconnects the graph)
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (5, 6), (6, 7), (7, 8), (2, 1), (3, 3)]
    return 9, np.array(edges, np.int32)


def test_c_program_on_the_gpu(tmp_path):
    import paper_2103_15217_gb300 as etl
    libdir = os.path.dirname(etl.build())
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "fig1_euler_tour.json")))
    gn, edges = _graph()
    src = (PROGRAM.replace("PARENT", ", ".join(map(str, g["parent"])))
           .replace("QU", ", ".join(str(x[0]) for x in g["lca"]))
           .replace("QV", ", ".join(str(x[1]) for x in g["lca"]))
           .replace("EDGES", ", ".join(map(str, edges.ravel())))
           .replace("GN", str(gn)))
    (tmp_path / "client.c").write_text(src)
    cuda = os.path.dirname(os.path.dirname(shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"))
    exe = tmp_path / "client"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(cuda, "include"), str(tmp_path / "client.c"),
                           "-L", libdir, "-letl", f"-Wl,-rpath,{libdir}",
                           "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}",
                           "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.stdout, r.stderr)
    out = {ln.split()[0]: ln.split()[1:] for ln in r.stdout.splitlines() if ln.strip()}
    assert "done" in out
    assert out["tree_status"] == ["0"] and out["graph_status"] == ["0"]
    want_lca = [str(x[2]) for x in g["lca"]]
    assert out["lca"] == want_lca and out["ws_lca"] == want_lca
    for key in ("pre", "depth", "size"):
        assert [int(out[key][int(v)]) for v in g[key]] == list(g[key].values())
    want_br = [str(int(x)) for x in oracle.bridges_dfs(gn, edges)]
    assert want_br == ["0"] * 6 + ["1"] * 3 + ["0", "0"]   # the closed form of this graph
    assert out["bridges"] == want_br and out["ws_bridges"] == want_br
    assert out["ws_status"] == ["0", "allocs", "0"]
