// LCA by range minimum over the depth-annotated Euler tour: the classical
// reduction of LCA to RMQ that Sec. 3.1 names (the second of its two families
// of LCA algorithms), on the 2n brackets of the tour rather than on the
// preorder sequence of the main path.
//
// The tour visits a node at each of its brackets: at the opening bracket of v
// (tour position r0(v) = 2 pre(v) - depth(v)) it is at v, and at the closing
// bracket of v (position r1(v) = r0(v) + 2 size(v) - 1) it is back at
// parent(v). Entry E[r] holds the key depth << 32 | node of the node the tour
// is at after position r. For nodes u, v with r0(u) <= r0(v), the tour between
// the two positions stays inside the subtree of LCA(u, v) and passes through
// the LCA itself (at r0(u) if u is the LCA, else at the closing bracket of
// the LCA's child towards u), so the minimal key over [r0(u), r0(v)] has the
// least depth in that window, the LCA's, and every entry of that depth names
// the LCA: its low half is the answer. No tie-breaking is needed.
//
// Built on a preprocessed handle (preorder, depth, size); one blocked range
// table of 64-bit keys over 2n positions (rmq.cu) and the node -> position
// array. A query reads two positions, two per-position table entries and two
// L2-resident top-table entries.
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * int64_t(blockDim.x) + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

__device__ __forceinline__ long long tour_key(int32_t depth, int32_t node) {
    return (static_cast<long long>(depth) << 32) | uint32_t(node);
}

__global__ void k_tour_keys(const int32_t *__restrict__ parent, const int32_t *__restrict__ pre,
                            const int32_t *__restrict__ depth, const int32_t *__restrict__ size, int32_t n,
                            long long *__restrict__ keys, int32_t *__restrict__ tpos) {
    pdl_prologue();
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int32_t p = pre[v], d = depth[v], sz = size[v];
        const int64_t r0 = 2 * int64_t(p) - d, r1 = r0 + 2 * int64_t(sz) - 1;
        if (p < 0 || d < 0 || sz < 1 || r0 < 0 || r1 >= 2 * int64_t(n) || r0 >= r1) {  // flagged tree
            tpos[v] = 0;
            continue;
        }
        tpos[v] = int32_t(r0);
        keys[r0] = tour_key(d, int32_t(v));
        const int32_t up = parent[v];
        keys[r1] = (up >= 0 && up < n) ? tour_key(d - 1, up) : INT64_MAX;  // the root's closing bracket
    }
}

struct TourView {
    int32_t n;
    const int32_t *tpos, *hstatus;
    BlockedView<OpMinKey> bv;
};

constexpr int kIlp = 4;

__global__ void __launch_bounds__(256)
    k_tour_query(TourView h, const int32_t *__restrict__ u, const int32_t *__restrict__ v, int64_t q,
                 int32_t *__restrict__ out, int32_t *__restrict__ status) {
    pdl_prologue();
    const bool bad_tree = *h.hstatus != 0;
    const int64_t stride = gstride();
    for (int64_t base = gtid(); base < q; base += stride * kIlp) {
        int32_t a[kIlp], b[kIlp], res[kIlp];
        bool go[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const int64_t i = base + k * stride;
            go[k] = false;
            res[k] = -1;
            a[k] = b[k] = 0;
            if (i < q) {
                a[k] = __ldcs(u + i);
                b[k] = __ldcs(v + i);
                if (a[k] < 0 || a[k] >= h.n || b[k] < 0 || b[k] >= h.n) {
                    set_status(status, ETL_EBADQUERY);
                } else if (!bad_tree) {
                    if (a[k] == b[k]) res[k] = a[k];
                    else go[k] = true;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            if (!go[k]) continue;
            const int32_t x = __ldg(h.tpos + a[k]), y = __ldg(h.tpos + b[k]);
            res[k] = int32_t(uint32_t(blocked_query<OpMinKey>(h.bv, min(x, y), max(x, y))));
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const int64_t i = base + k * stride;
            if (i < q) __stcs(out + i, res[k]);
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t blocks = ceil_div(work, threads);
    const int64_t cap = int64_t(num_sms()) * (2048 / threads) * 4;
    if (blocks > cap) blocks = cap;
    return int(blocks < 1 ? 1 : blocks);
}

}  // namespace
}  // namespace etl

using namespace etl;

etl_status lca_build_tour_impl(etl_lca_t h, const int32_t *parent, cudaStream_t s) {
    if (!h || !parent || h->node_off || h->tour_table) return ETL_EINVAL;
    const int32_t n = h->n;
    const int64_t P = 2 * int64_t(n);
    h->tbl = blocked_layout(P, P);
    if (dev_alloc(&h->tour_table, size_t(h->tbl.elems()) * sizeof(long long), s) != cudaSuccess) return ETL_ENOMEM;
    if (dev_alloc((void **)&h->tpos, size_t(n) * sizeof(int32_t), s) != cudaSuccess) return ETL_ENOMEM;
    long long *keys = static_cast<long long *>(h->tour_table);
    {
        PhaseTimer pt("tour_rmq.keys", s);
        launch(k_tour_keys, grid_for(n, 256), 256, 0, s, parent, h->pre, h->depth, h->size, n, keys, h->tpos);
        note_launch();
    }
    etl_status st = last_launch();
    if (!st) st = blocked_build<OpMinKey>(keys, P, h->tbl, s);
    return st;
}

extern "C" etl_status lca_query_tour(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                                     int32_t *status, void *stream) {
    if (!h || !h->tour_table || q < 0 || q > (int64_t(1) << 40)) return ETL_EINVAL;
    if (q == 0) return ETL_OK;
    if (!u || !v || !out) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TourView view{h->n, h->tpos, h->status,
                  blocked_view<OpMinKey>(static_cast<const long long *>(h->tour_table), h->tbl)};
    PhaseTimer pt("tour_rmq.query", s);
    launch(k_tour_query, grid_for(ceil_div(q, kIlp), 256), 256, 0, s, view, u, v, q, out, status);
    note_launch();
    return last_launch();
}
