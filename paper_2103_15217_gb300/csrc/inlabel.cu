// Inlabel LCA (Schieber and Vishkin), the paper's GPU LCA method (Sec. 3.1,
// "The Inlabel Algorithm"), built on the Euler-tour results of a preprocessed
// handle (preorder, subtree size, depth). With preorder numbers counted from 1:
//
//  * inlabel(v) is the number in v's preorder interval [pre(v), pre(v) +
//    size(v) - 1] with the most trailing zeros: with a = pre(v) - 1 and
//    b = pre(v) + size(v) - 1, h = floor(log2(a xor b)) and inlabel(v) =
//    (b >> h) << h. Nodes with equal inlabels form top-down paths, and an
//    ancestor's inlabel is an ancestor of v's inlabel in the complete binary
//    tree numbered in inorder (the two properties Sec. 3.1 states).
//  * A node is the head of its path if its parent's inlabel differs (or it is
//    the root). ascendant(v) has bit k set iff some ancestor of v (v included)
//    has an inlabel of height k (k trailing zeros). Only path heads contribute
//    new bits and their heights strictly grow towards the root, so the OR over
//    ancestors is a plain SUM of lowbit(inlabel(u)) over the heads u on the
//    root path -- a prefix sum over the Euler tour with +lowbit at a head's
//    opening bracket and -lowbit at its closing bracket. The bracket positions
//    come from pre, depth and size (rank(2v) = 2 pre(v) - depth(v), rank(2v+1)
//    = rank(2v) + 2 size(v) - 1), so one scatter, one scan and one gather
//    replace the per-level propagation.
//  * For every path (indexed by its inlabel) the parent of its head and that
//    parent's depth are stored, so leaving a path is one load.
//
// Query LCA(x, y), ix = inlabel(x), iy = inlabel(y): if ix == iy the
// shallower of x, y. Otherwise the binary-tree LCA of ix and iy has height
// j = max(floor(log2(ix xor iy)), height(ix), height(iy)); the lowest common
// set bit of ascendant(x) and ascendant(y) at or above j is the height of
// inlabel(z), z the answer. On each side, if the side's inlabel is not
// inlabel(z), the side leaves its path below z at the highest ascendant bit
// under that height: that path's head's parent. z is the shallower of the two
// entry points. Every step is O(1); a query reads two 16-byte node records
// and at most two 8-byte path records.
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * int64_t(blockDim.x) + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }
__device__ __forceinline__ uint32_t lowbit(uint32_t x) { return x & (0u - x); }

__global__ void k_inlabel(const int32_t *__restrict__ pre, const int32_t *__restrict__ size, int32_t n,
                          uint32_t *__restrict__ inl) {
    pdl_prologue();
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int32_t p = pre[v], sz = size[v];
        if (p < 0 || sz < 1 || int64_t(p) + sz > n) {  // only on a tree the handle already flagged as bad
            inl[v] = 0;
            continue;
        }
        const uint32_t a = uint32_t(p);       // pre(v) - 1 with 1-based preorder
        const uint32_t b = uint32_t(p + sz);  // last preorder number of the subtree, 1-based
        const int h = 31 - __clz(int(a ^ b));
        inl[v] = (b >> h) << h;
    }
}

// heads: tour values +-lowbit(inlabel) at their brackets, and the path record of their inlabel
__global__ void k_inlabel_heads(const int32_t *__restrict__ parent, const int32_t *__restrict__ pre,
                                const int32_t *__restrict__ depth, const int32_t *__restrict__ size,
                                const uint32_t *__restrict__ inl, int32_t n, int32_t *__restrict__ tourval,
                                int2 *__restrict__ pathrec) {
    pdl_prologue();
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int32_t p = parent[v];
        const uint32_t iv = inl[v];
        if (iv == 0) continue;
        const bool head = p < 0 || p >= n || inl[p] != iv;
        const int64_t open = 2 * int64_t(pre[v]) - depth[v], close = open + 2 * int64_t(size[v]) - 1;
        if (open < 0 || close >= 2 * int64_t(n) || open >= close) continue;
        const int32_t w = head ? int32_t(lowbit(iv)) : 0;
        tourval[open] = w;
        tourval[close] = -w;
        if (head && iv <= uint32_t(n)) pathrec[iv] = (p >= 0 && p < n) ? make_int2(p, depth[p]) : make_int2(-1, -1);
    }
}

__global__ void k_inlabel_records(const uint32_t *__restrict__ inl, const int32_t *__restrict__ pre,
                                  const int32_t *__restrict__ depth, const int32_t *__restrict__ parent,
                                  const int32_t *__restrict__ excl, int32_t n, int4 *__restrict__ rec) {
    pdl_prologue();
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int64_t open = 2 * int64_t(pre[v]) - depth[v];
        const int32_t asc = (open >= 0 && open < 2 * int64_t(n)) ? excl[open + 1] : 0;  // inclusive prefix at open
        rec[v] = make_int4(int32_t(inl[v]), asc, depth[v], parent[v]);
    }
}

struct InView {
    int32_t n;
    const int4 *rec;
    const int2 *path;
    const int32_t *hstatus;
};

__device__ __forceinline__ uint32_t label_at(uint32_t x, int k) {  // ancestor of x at height k in the binary tree
    return ((x >> (k + 1)) << (k + 1)) | (1u << k);
}

__global__ void __launch_bounds__(256)
    k_inlabel_query(InView h, const int32_t *__restrict__ u, const int32_t *__restrict__ v, int64_t q,
                    int32_t *__restrict__ out, int32_t *__restrict__ status) {
    pdl_prologue();
    const bool bad_tree = *h.hstatus != 0;
    for (int64_t i = gtid(); i < q; i += gstride()) {
        const int32_t x = __ldcs(u + i), y = __ldcs(v + i);
        int32_t res = -1;
        if (x < 0 || x >= h.n || y < 0 || y >= h.n) {
            set_status(status, ETL_EBADQUERY);
        } else if (!bad_tree) {
            if (x == y) {
                res = x;
            } else {
                const int4 rx = __ldg(h.rec + x), ry = __ldg(h.rec + y);
                const uint32_t ix = uint32_t(rx.x), iy = uint32_t(ry.x);
                if (ix == iy) {
                    res = rx.z <= ry.z ? x : y;  // same path: the shallower one
                } else {
                    const int hi = 31 - __clz(int(ix ^ iy));
                    const int j = max(hi, max(__ffs(int(ix)) - 1, __ffs(int(iy)) - 1));
                    const uint32_t common = uint32_t(rx.y) & uint32_t(ry.y) & (0xffffffffu << j);
                    if (common == 0) {  // structures not built from this tree's parent array
                        set_status(status, ETL_EINVAL);
                        __stcs(out + i, -1);
                        continue;
                    }
                    const int jz = __ffs(int(common)) - 1;
                    const uint32_t iz = label_at(ix, jz);
                    int32_t xh = x, xd = rx.z, yh = y, yd = ry.z;
                    if (ix != iz) {  // leave x's path at the highest ascendant bit below height jz
                        const int k = 31 - __clz(int(uint32_t(rx.y) & ((1u << jz) - 1u)));
                        const uint32_t w = k >= 0 ? label_at(ix, k) : 0u;
                        const int2 pr = (w >= 1 && w <= uint32_t(h.n)) ? __ldg(h.path + w) : make_int2(-1, INT_MAX);
                        xh = pr.x;
                        xd = pr.y;
                    }
                    if (iy != iz) {
                        const int k = 31 - __clz(int(uint32_t(ry.y) & ((1u << jz) - 1u)));
                        const uint32_t w = k >= 0 ? label_at(iy, k) : 0u;
                        const int2 pr = (w >= 1 && w <= uint32_t(h.n)) ? __ldg(h.path + w) : make_int2(-1, INT_MAX);
                        yh = pr.x;
                        yd = pr.y;
                    }
                    res = xd <= yd ? xh : yh;
                }
            }
        }
        __stcs(out + i, res);
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

etl_status lca_build_inlabel_impl(etl_lca_t h, const int32_t *parent, cudaStream_t s) {
    if (!h || !parent || h->node_off) return ETL_EINVAL;
    const int32_t n = h->n;
    if (!h->inrec) {
        if (dev_alloc((void **)&h->inrec, size_t(n) * sizeof(int4), s) != cudaSuccess) return ETL_ENOMEM;
        if (dev_alloc((void **)&h->inpath, (size_t(n) + 1) * sizeof(int2), s) != cudaSuccess) return ETL_ENOMEM;
    }
    Workspace ws(s);
    uint32_t *inl = ws.get<uint32_t>(n);
    int32_t *tourval = ws.get<int32_t>(2 * int64_t(n));
    int32_t *excl = ws.get<int32_t>(2 * int64_t(n) + 1);
    if (!ws.ok()) return ETL_ENOMEM;
    const int g = grid_for(n, 256);
    {
        PhaseTimer pt("inlabel.build", s);
        launch(k_inlabel, g, 256, 0, s, h->pre, h->size, n, inl);
        note_launch();
        launch(k_inlabel_heads, g, 256, 0, s, parent, h->pre, h->depth, h->size, inl, n, tourval,
               reinterpret_cast<int2 *>(h->inpath));
        note_launch();
    }
    etl_status st = last_launch();
    if (!st) st = scan_exclusive_i32(tourval, excl, 2 * int64_t(n), ws);
    if (!st) {
        PhaseTimer pt("inlabel.build", s);
        launch(k_inlabel_records, g, 256, 0, s, inl, h->pre, h->depth, parent, excl, n,
               reinterpret_cast<int4 *>(h->inrec));
        note_launch();
        st = last_launch();
    }
    return st;
}

extern "C" etl_status lca_build_inlabel(etl_lca_t h, const int32_t *parent, void *stream) {
    if (h && h->arena) return ETL_EINVAL;  // a handle inside a caller's workspace takes no more tables
    return lca_build_inlabel_impl(h, parent, static_cast<cudaStream_t>(stream));
}

extern "C" etl_status lca_query_inlabel(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                                        int32_t *status, void *stream) {
    if (!h || !h->inrec || q < 0 || q > (int64_t(1) << 40)) return ETL_EINVAL;
    if (q == 0) return ETL_OK;
    if (!u || !v || !out) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    InView view{h->n, reinterpret_cast<const int4 *>(h->inrec), reinterpret_cast<const int2 *>(h->inpath),
                h->status};
    PhaseTimer pt("inlabel.query", s);
    launch(k_inlabel_query, grid_for(q, 256), 256, 0, s, view, u, v, q, out, status);
    note_launch();
    return last_launch();
}
