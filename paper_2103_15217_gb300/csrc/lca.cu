// Lowest common ancestors by RMQ over the Euler tour (Sec. 3.1), for a tree
// given as a parent array (the input format of Sec. 3.2).
//
// Preprocessing (all on one stream, no host synchronisation):
//   1. k_count_children: child counts, root detection, validation.
//   2. scan -> CSR offsets; stable radix sort of (parent, child) -> children of
//      each node in ascending label order (the grouping step of Sec. 2.1).
//   3. k_tour_succ: successor array of the Euler tour in bracket form. Node v
//      owns two list elements, 2v (the arc entering v from its parent, an
//      opening bracket) and 2v+1 (the arc leaving v, a closing bracket); the
//      root's two brackets start and end the list. succ(2v) = 2*firstchild(v)
//      or 2v+1; succ(2c+1) = 2*nextsibling(c) or 2*parent(c)+1. This is
//      succ(e) = next(twin(e)) of Sec. 2.1 with the cyclic list already cut at
//      the root (head = 2*root).
//   4. list ranking (rank.cu), counting opening brackets on the way.
//   5. k_node_stats: preorder = opening brackets before 2v; depth =
//      2*pre - rank(2v) (opening minus closing brackets before it, the +1/-1
//      prefix sum of Sec. 2); size = (rank(2v+1) - rank(2v) + 1) / 2.
//   6. k_parent_pre: Q[pre(v)] = pre(parent(v)), level 0 of the sparse table.
//   7. sparse table over Q (rmq.cu).
//
// Query: for u != v with i = min(pre u, pre v), j = max(...), every node with
// preorder in (i, j] is a proper descendant of LCA(u, v), and the child of the
// LCA on the path to the deeper end lies in that range; so the minimum of Q
// over (i, j] is pre(LCA). This is the depth-minimum of the RMQ reduction
// (the node of least depth in the range is a child of the LCA) with the
// answer read directly: one min, no argmin and no tie-breaking.
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

__global__ void k_count_children(const int32_t *__restrict__ parent, int32_t n, int32_t *__restrict__ cnt,
                                 int32_t *__restrict__ misc, int32_t *__restrict__ status) {
    // misc[0] = number of roots, misc[1] = root, misc[2] = list head (2*root)
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int32_t p = parent[v];
        if (p == -1) {
            atomicAdd(&misc[0], 1);
            misc[1] = int32_t(v);
            misc[2] = 2 * int32_t(v);
        } else if (p < 0 || p >= n) {
            set_status(status, ETL_EBADTREE);
        } else {
            if (p == v) set_status(status, ETL_EBADTREE);
            atomicAdd(&cnt[p], 1);
        }
    }
}

__global__ void k_tour_succ(const int32_t *__restrict__ keys, const int32_t *__restrict__ kids,
                            const int32_t *__restrict__ coff, int32_t n, const int32_t *__restrict__ misc,
                            int32_t *__restrict__ succ, int32_t *__restrict__ status) {
    const int32_t kept = coff[n];  // number of (parent, child) pairs
    if (blockIdx.x == 0 && threadIdx.x == 0 && misc[0] != 1) set_status(status, ETL_EBADTREE);
    const int32_t root = misc[1];
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t v = int32_t(t);
        const int32_t b = coff[v], e = coff[v + 1];
        succ[2 * v] = (b < e) ? 2 * kids[b] : 2 * v + 1;  // enter v -> enter first child, or leave v
        if (v == root) succ[2 * v + 1] = ETL_END;
        if (t < kept) {  // position t of the grouped children
            const int32_t c = kids[t], p = keys[t];
            if (c >= 0 && c < n && p >= 0 && p < n) {
                const int32_t sib = (t + 1 < coff[p + 1]) ? kids[t + 1] : -1;
                succ[2 * c + 1] = sib >= 0 ? 2 * sib : 2 * p + 1;  // leave c -> enter next sibling, or leave p
            }
        }
    }
}

__global__ void k_node_stats(RankResult rr, int32_t n, const int32_t *__restrict__ misc,
                             int32_t *__restrict__ pre, int32_t *__restrict__ depth, int32_t *__restrict__ size,
                             int32_t *__restrict__ order, int32_t *__restrict__ status) {
    const uint4 *pk = reinterpret_cast<const uint4 *>(rr.packed);  // brackets 2v and 2v+1 side by side
    const int32_t root = misc[1];
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        const uint4 q = pk[t];
        if (q.x >= rr.rcap || q.z >= rr.rcap) {  // not on the list from the root: malformed input
            set_status(status, ETL_EBADTREE);
            pre[t] = depth[t] = size[t] = -1;
            continue;
        }
        const uint2 in = make_uint2(q.x, q.y), out = make_uint2(q.z, q.w);
        const int32_t r0 = rank_of(rr, in), r1 = rank_of(rr, out);
        const int32_t p = evens_before(rr, in);
        pre[t] = p;
        depth[t] = 2 * p - r0;
        size[t] = (r1 - r0 + 1) >> 1;
        if (p >= 0 && p < n) order[p] = int32_t(t);
        if (t == root && (r0 != 0 || int64_t(r1) != 2 * int64_t(n) - 1)) set_status(status, ETL_EBADTREE);
    }
}

__global__ void k_parent_pre(const int32_t *__restrict__ parent, const int32_t *__restrict__ pre, int32_t n,
                             int32_t *__restrict__ q0) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int32_t i = pre[v], p = parent[v];
        if (i >= 0 && i < n) q0[i] = (p >= 0 && p < n) ? __ldg(pre + p) : -1;
    }
}

struct LcaView {
    int32_t n;
    const int32_t *pre, *order, *table, *hstatus;
};

constexpr int kQueryIlp = 4;

// Each thread answers kQueryIlp queries at once so that their dependent
// gathers (pre, table, order) overlap in flight.
__global__ void __launch_bounds__(256)
    k_lca_query(LcaView h, const int32_t *__restrict__ u, const int32_t *__restrict__ v, int64_t q,
                int32_t *__restrict__ out, int32_t *__restrict__ status) {
    const bool bad_tree = *h.hstatus != 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; base < q; base += stride * kQueryIlp) {
        int32_t a[kQueryIlp], b[kQueryIlp], lo[kQueryIlp], hi[kQueryIlp], res[kQueryIlp];
        bool need[kQueryIlp];
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k) {
            const int64_t i = base + k * stride;
            need[k] = false;
            res[k] = -1;
            if (i < q) {
                a[k] = __ldcs(u + i);
                b[k] = __ldcs(v + i);
            } else {
                a[k] = b[k] = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k) {
            const int64_t i = base + k * stride;
            if (i >= q) continue;
            if (a[k] < 0 || a[k] >= h.n || b[k] < 0 || b[k] >= h.n) {
                set_status(status, ETL_EBADQUERY);
            } else if (!bad_tree) {
                if (a[k] == b[k]) {
                    res[k] = a[k];
                } else {
                    const int32_t pa = __ldg(h.pre + a[k]), pb = __ldg(h.pre + b[k]);
                    lo[k] = min(pa, pb) + 1;
                    hi[k] = max(pa, pb);
                    need[k] = true;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k)
            if (need[k]) lo[k] = sparse_query<false>(h.table, h.n, lo[k], hi[k]);
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k) {
            const int64_t i = base + k * stride;
            if (i >= q) continue;
            if (need[k]) res[k] = __ldg(h.order + lo[k]);
            __stcs(out + i, res[k]);
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t blocks = ceil_div(work, threads);
    const int64_t cap = int64_t(num_sms()) * (2048 / threads) * 4;
    if (blocks > cap) blocks = cap;
    return int(blocks < 1 ? 1 : blocks);
}

void free_handle(etl_lca_s *h) {
    if (!h) return;
    cudaStream_t s = h->stream;
    for (int32_t *p : {h->pre, h->depth, h->size, h->order, h->table, h->status})
        if (p) cudaFreeAsync(p, s);
    delete h;
}

}  // namespace
}  // namespace etl

using namespace etl;

extern "C" etl_status lca_preprocess(const int32_t *parent, int32_t n, void *stream, etl_lca_t *out) {
    if (!out) return ETL_EINVAL;
    *out = nullptr;
    if (!parent || n < 1 || n > (1 << 30)) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    etl_lca_s *h = new etl_lca_s;
    h->n = n;
    h->stream = s;
    h->levels = n > 1 ? sparse_levels(n - 1) : 1;
    const size_t nb = size_t(n) * sizeof(int32_t);
    bool ok = cudaMallocAsync((void **)&h->pre, nb, s) == cudaSuccess;
    ok = ok && cudaMallocAsync((void **)&h->depth, nb, s) == cudaSuccess;
    ok = ok && cudaMallocAsync((void **)&h->size, nb, s) == cudaSuccess;
    ok = ok && cudaMallocAsync((void **)&h->order, nb, s) == cudaSuccess;
    ok = ok && cudaMallocAsync((void **)&h->table, nb * size_t(h->levels), s) == cudaSuccess;
    ok = ok && cudaMallocAsync((void **)&h->status, sizeof(int32_t), s) == cudaSuccess;
    if (!ok) {
        free_handle(h);
        return ETL_ENOMEM;
    }
    cudaMemsetAsync(h->status, 0, sizeof(int32_t), s);
    etl_status st = ETL_OK;
    {
        Workspace ws(s);
        int32_t *cnt = ws.get<int32_t>(n);
        int32_t *coff = ws.get<int32_t>(int64_t(n) + 1);
        int32_t *misc = ws.get<int32_t>(4);
        int32_t *succ = ws.get<int32_t>(2 * int64_t(n));
        if (!ws.ok()) st = ETL_ENOMEM;
        if (!st) {
            cudaMemsetAsync(cnt, 0, nb, s);
            cudaMemsetAsync(misc, 0, 4 * sizeof(int32_t), s);
            PhaseTimer pt("lca.count", s);
            k_count_children<<<grid_for(n, 256), 256, 0, s>>>(parent, n, cnt, misc, h->status);
        note_launch();
            st = last_launch();
        }
        if (!st) st = scan_exclusive_i32(cnt, coff, n, ws);
        SortResult sr{};
        if (!st) st = radix_sort_pairs(parent, nullptr, nullptr, n, ceil_log2(uint64_t(n)), n, ws, &sr);
        if (!st) {
            PhaseTimer pt("lca.succ", s);
            k_tour_succ<<<grid_for(n, 256), 256, 0, s>>>(sr.keys, sr.vals, coff, n, misc, succ, h->status);
        note_launch();
            st = last_launch();
        }
        RankResult rr{};
        if (!st) st = list_rank(succ, 2 * int64_t(n), nullptr, misc + 2, true, 2 * int64_t(n), h->status, ws, &rr);
        if (!st) {
            PhaseTimer pt("lca.node_stats", s);
            k_node_stats<<<grid_for(n, 256), 256, 0, s>>>(rr, n, misc, h->pre, h->depth, h->size, h->order,
                                                          h->status);
        note_launch();
            st = last_launch();
        }
        if (!st) {
            PhaseTimer pt("lca.parent_pre", s);
            k_parent_pre<<<grid_for(n, 256), 256, 0, s>>>(parent, h->pre, n, h->table);
        note_launch();
            st = last_launch();
        }
        if (!st) st = sparse_table_build<false>(h->table, n, h->levels, s);
    }
    if (st) {
        free_handle(h);
        return st;
    }
    *out = h;
    return ETL_OK;
}

extern "C" etl_status lca_query(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                                int32_t *status, void *stream) {
    if (!h || q < 0 || q > (int64_t(1) << 40)) return ETL_EINVAL;
    if (q == 0) return ETL_OK;
    if (!u || !v || !out) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LcaView view{h->n, h->pre, h->order, h->table, h->status};
    PhaseTimer pt("lca.query", s);
    k_lca_query<<<grid_for(ceil_div(q, kQueryIlp), 256), 256, 0, s>>>(view, u, v, q, out, status);
        note_launch();
    return last_launch();
}

extern "C" etl_status lca_status(etl_lca_t h, int32_t *status) {
    if (!h || !status) return ETL_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return ETL_ECUDA;
    if (cudaMemcpy(status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) return ETL_ECUDA;
    return ETL_OK;
}

extern "C" etl_status lca_arrays(etl_lca_t h, const int32_t **pre, const int32_t **depth, const int32_t **size,
                                 const int32_t **order) {
    if (!h) return ETL_EINVAL;
    if (pre) *pre = h->pre;
    if (depth) *depth = h->depth;
    if (size) *size = h->size;
    if (order) *order = h->order;
    return ETL_OK;
}

extern "C" etl_status lca_export(etl_lca_t h, int32_t *pre, int32_t *depth, int32_t *size, int32_t *order,
                                 void *stream) {
    if (!h) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nb = size_t(h->n) * sizeof(int32_t);
    int32_t *dst[4] = {pre, depth, size, order};
    const int32_t *src[4] = {h->pre, h->depth, h->size, h->order};
    for (int i = 0; i < 4; ++i)
        if (dst[i] && cudaMemcpyAsync(dst[i], src[i], nb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return ETL_ECUDA;
    return ETL_OK;
}

extern "C" etl_status lca_free(etl_lca_t h) {
    if (!h) return ETL_OK;
    free_handle(h);
    return cudaGetLastError() == cudaSuccess ? ETL_OK : ETL_ECUDA;
}
