// Lowest common ancestors by RMQ over the Euler tour (Sec. 3.1), for a tree
// given as a parent array (the input format of Sec. 3.2), or for a batch of
// independent trees preprocessed and queried together.
//
// Preprocessing (all on one stream, no host synchronisation):
//   1. k_count_children: child counts, roots, validation (and, for a batch,
//      local parent ids turned into global ones: node v of instance i has
//      global id node_off[i] + v).
//   2. scan -> CSR offsets; stable radix sort of (parent, child) -> children of
//      each node in ascending label order (the grouping step of Sec. 2.1).
//   3. k_tour_succ: successor array of the Euler tour in bracket form. Node v
//      owns two list elements, 2v (the arc entering v from its parent, an
//      opening bracket) and 2v+1 (the arc leaving v, a closing bracket).
//      succ(2v) = 2*firstchild(v) or 2v+1; succ(2c+1) = 2*nextsibling(c) or
//      2*parent(c)+1. This is succ(e) = next(twin(e)) of Sec. 2.1 with the
//      cyclic list cut at the root: the root's two brackets start and end
//      its tour. k_link_roots chains the tours of a batch, root i's closing
//      bracket -> root i+1's opening bracket, so one list covers all trees.
//      The two halves are written apart (the closing brackets' successors at
//      random places into an array of n entries that L2 holds) and
//      interleaved by k_tour_assemble, which also contracts the leaves.
//   4. list ranking (rank.cu), counting opening brackets on the way.
//   5. k_node_stats: preorder = opening brackets before 2v; depth =
//      2*pre - rank(2v) (opening minus closing brackets before it, the +1/-1
//      prefix sum of Sec. 2); size = (rank(2v+1) - rank(2v) + 1) / 2. In a
//      chained batch, tree i occupies preorder positions node_off[i] ..
//      node_off[i+1]-1 and depth / size come out per tree.
//   6. k_parent_pre: Q[i] = pre(parent(order[i])), level 0 of the range-minimum
//      table, written in preorder (a separate pass: gathering pre[] is cheaper
//      than re-deriving the parent's preorder from its bracket record).
//   7. range-minimum table over Q (rmq.cu): by default the blocked two-level
//      table (in-block prefix / suffix minima plus a sparse table over blocks
//      of 32), else a full sparse table; sized for the largest tree.
//
// Query: for u != v with i = min(pre u, pre v), j = max(...), every node with
// preorder in (i, j] is a proper descendant of LCA(u, v), and the child of the
// LCA on the path to the later end lies in that range; so the minimum of Q
// over (i, j] is pre(LCA). This is the depth-minimum of the RMQ reduction
// (the node of least depth in the range is a child of the LCA) with the
// answer read directly: one min, no argmin and no tie-breaking.
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * int64_t(blockDim.x) + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

// node_off must be 0 = off[0] < off[1] < ... < off[k] = total (every instance non-empty)
__global__ void k_check_offsets(const int32_t *__restrict__ off, int32_t k, int32_t total,
                                int32_t *__restrict__ bad, int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t i = gtid(); i < k; i += gstride()) {
        const int32_t b = off[i], e = off[i + 1];
        if (b < 0 || e > total || b >= e || (i == 0 && b != 0) || (i == k - 1 && e != total)) {
            set_status(status, ETL_EINVAL);
            *bad = 1;
        }
    }
}

// inst_of[v] = instance of node v; one block per instance, coalesced writes
__global__ void k_fill_inst(const int32_t *__restrict__ off, int32_t k, const int32_t *__restrict__ bad,
                            int32_t *__restrict__ inst_of) {
    pdl_prologue();
    if (*bad) return;
    for (int64_t i = blockIdx.x; i < k; i += gridDim.x) {
        const int32_t b = off[i], e = off[i + 1];
        for (int32_t v = b + threadIdx.x; v < e; v += blockDim.x) inst_of[v] = int32_t(i);
    }
}

template <bool BATCH>
__global__ void k_count_children(const int32_t *__restrict__ parent, int32_t n, const int32_t *__restrict__ off,
                                 const int32_t *__restrict__ inst_of, const int32_t *__restrict__ bad,
                                 int32_t *__restrict__ gparent, int32_t *__restrict__ cnt,
                                 int32_t *__restrict__ root_cnt, int32_t *__restrict__ root_of,
                                 int32_t *__restrict__ status) {
    pdl_prologue();
    const bool bad_offsets = BATCH && *bad;
    for (int64_t t = gtid(); t < n; t += gstride()) {
        const int32_t v = int32_t(t);
        if (bad_offsets) {  // instance ids unusable: drop every node (status is already set)
            gparent[v] = -2;
            continue;
        }
        const int32_t p = __ldcs(parent + v);
        int32_t inst = 0, base = 0, size = n;
        if (BATCH) {
            inst = inst_of[v];
            base = off[inst];
            size = off[inst + 1] - base;
        }
        int32_t g = -2;
        if (p == -1) {
            atomicAdd(&root_cnt[inst], 1);
            root_of[inst] = v;
            g = -1;
        } else if (p < 0 || p >= size) {
            set_status(status, ETL_EBADTREE);
        } else {
            g = p + base;
            if (g == v) set_status(status, ETL_EBADTREE);
            atomicAdd(&cnt[g], 1);
        }
        if (BATCH) gparent[v] = g;
    }
}

// kv[t] = (parent, child), grouped by parent with children ascending. Child c at position t has a
// next sibling iff position t + 1 holds the same parent (the groups are contiguous), which the
// coalesced read of kv[t + 1] shows without a gather of the parent's group end. The successors of
// the opening brackets go to so[v] (coalesced), those of the closing brackets to sc[c]: written at
// random places, they stay within n entries, which L2 holds while they are written (in place, at
// succ[2c + 1], they spread over twice the memory and the kernel ran 2.2x slower);
// k_tour_assemble interleaves the two.
__global__ void k_tour_succ(const int2 *__restrict__ kv, const int32_t *__restrict__ coff, int32_t n,
                            int32_t *__restrict__ so, int32_t *__restrict__ sc) {
    pdl_prologue();
    const int32_t kept = coff[n];  // number of (parent, child) pairs
    for (int64_t t = gtid(); t < n; t += gstride()) {
        const int32_t v = int32_t(t);
        const int32_t b = __ldcs(coff + v), e = __ldcs(coff + v + 1);
        __stcs(so + v, (b < e) ? 2 * kv[b].y : 2 * v + 1);  // enter v -> enter first child, or leave v
        if (t < kept) {                                      // position t of the grouped children
            const int2 pc = kv[t];
            const int32_t c = pc.y, p = pc.x;
            if (c >= 0 && c < n && p >= 0 && p < n) {
                int32_t sib = -1;
                if (t + 1 < kept) {
                    const int2 nx = kv[t + 1];
                    if (nx.x == p) sib = nx.y;
                }
                sc[c] = sib >= 0 ? 2 * sib : 2 * p + 1;  // leave c -> enter next sibling, or leave p
            }
        }
    }
}

// succ[2v] = so[v], succ[2v + 1] = sc[v], one 8-byte store per node. A leaf v's brackets are
// adjacent in the tour: 2v jumps straight to the successor of 2v+1 with weight 2 (top bit set), and
// 2v+1 leaves the list. Roots are never contracted.
__global__ void k_tour_assemble(const int32_t *__restrict__ coff, const int32_t *__restrict__ par,
                                const int32_t *__restrict__ so, const int32_t *__restrict__ sc, int32_t n,
                                int32_t *__restrict__ succ) {
    pdl_prologue();
    int2 *pair = reinterpret_cast<int2 *>(succ);
    for (int64_t t = gtid(); t < n; t += gstride()) {
        const bool leaf = __ldcs(coff + t) == __ldcs(coff + t + 1) && __ldcs(par + t) >= 0;  // no children, no root
        const int32_t a = __ldcs(so + t), c = __ldcs(sc + t);
        // a malformed close successor (c < 0) stays uncontracted: the validity checks see it
        pair[t] = (leaf && c >= 0) ? make_int2(int32_t(uint32_t(c) | 0x80000000u), ETL_END) : make_int2(a, c);
    }
}

// exactly one root per instance; leave root i -> enter root i+1 (or end of the list after the last
// tree); the list starts at the first root's opening bracket
__global__ void k_link_roots(const int32_t *__restrict__ root_cnt, const int32_t *__restrict__ root_of, int32_t k,
                             int32_t n, int32_t *__restrict__ sc, int32_t *__restrict__ head,
                             int32_t *__restrict__ status) {
    pdl_prologue();
    if (gtid() == 0) *head = 2 * root_of[0];
    for (int64_t i = gtid(); i < k; i += gstride()) {
        if (root_cnt[i] != 1) set_status(status, ETL_EBADTREE);
        const int32_t r = root_of[i];
        if (r < 0 || r >= n) continue;
        const int32_t nr = (i + 1 < k) ? root_of[i + 1] : -1;
        sc[r] = (nr >= 0 && nr < n) ? 2 * nr : ETL_END;
    }
}

__global__ void k_node_stats(RankResult rr, const int32_t *__restrict__ succ, int32_t n, int32_t *__restrict__ pre,
                             int32_t *__restrict__ depth, int32_t *__restrict__ size, int32_t *__restrict__ order,
                             int32_t *__restrict__ status) {
    pdl_prologue();
    const uint4 *pk = reinterpret_cast<const uint4 *>(rr.packed);  // brackets 2v and 2v+1 side by side
    for (int64_t t = gtid(); t < n; t += gstride()) {
        const bool leaf = __ldcs(succ + 2 * t) < ETL_END;  // contracted: the closing bracket is ranked right after
        uint4 q;
        if (leaf) {
            const uint2 a = __ldcs(rr.packed + 2 * t);
            q = make_uint4(a.x, a.y, a.x, 0u);
        } else {
            q = __ldcs(pk + t);
        }
        if (q.x >= rr.rcap || q.z >= rr.rcap) {  // not on the list from the root: malformed input
            set_status(status, ETL_EBADTREE);
            pre[t] = depth[t] = size[t] = -1;
            continue;
        }
        const uint2 in = make_uint2(q.x, q.y), out = make_uint2(q.z, q.w);
        const int32_t r0 = rank_of(rr, in), r1 = leaf ? r0 + 1 : rank_of(rr, out);
        const int32_t p = evens_before(rr, in);
        __stcs(pre + t, p);
        __stcs(depth + t, 2 * p - r0);
        __stcs(size + t, (r1 - r0 + 1) >> 1);
        if (p >= 0 && p < n) order[p] = int32_t(t);
    }
}

// Q in preorder: position i holds pre(parent(order[i])); two gathers and a coalesced write (a
// scatter to pre(v) would cost a read-for-fill and a write-back per random sector). The root is
// never inside a query range.
constexpr int kGatherIlp = 4;  // positions per thread per step whose dependent gathers are in flight together

__global__ void k_parent_pre(const int32_t *__restrict__ parent, const int32_t *__restrict__ pre,
                             const int32_t *__restrict__ order, int32_t n, int32_t *__restrict__ q0) {
    pdl_prologue();
    const int64_t step = gstride() * kGatherIlp;
    for (int64_t base = blockIdx.x * int64_t(blockDim.x) * kGatherIlp + threadIdx.x; base < n; base += step) {
        int32_t v[kGatherIlp], p[kGatherIlp];
#pragma unroll
        for (int j = 0; j < kGatherIlp; ++j) {
            const int64_t i = base + int64_t(j) * blockDim.x;
            v[j] = i < n ? __ldcs(order + i) : -1;
        }
#pragma unroll
        for (int j = 0; j < kGatherIlp; ++j) p[j] = (v[j] >= 0 && v[j] < n) ? __ldg(parent + v[j]) : -1;
#pragma unroll
        for (int j = 0; j < kGatherIlp; ++j) {
            const int64_t i = base + int64_t(j) * blockDim.x;
            if (i < n) __stcs(q0 + i, (p[j] >= 0 && p[j] < n) ? __ldg(pre + p[j]) : -1);
        }
    }
}

// root i must open its tree at preorder off[i] and span the whole instance
__global__ void k_check_instances(const int32_t *__restrict__ root_of, const int32_t *__restrict__ off, int32_t k,
                                  int32_t n, const int32_t *__restrict__ pre, const int32_t *__restrict__ size,
                                  int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t i = gtid(); i < k; i += gstride()) {
        const int32_t b = off ? off[i] : 0, e = off ? off[i + 1] : n;
        const int32_t r = root_of[i];
        if (r < 0 || r >= n || pre[r] != b || size[r] != e - b) set_status(status, ETL_EBADTREE);
    }
}

struct LcaView {
    int32_t n, k, levels;
    int64_t ld;
    const int32_t *pre, *order, *table, *hstatus, *off;
    BlockedView<OpMin> bv;  // the blocked table (when built instead of the full one)
    int64_t max_len;        // longest range the table answers
    const int4 *nrec;       // blocked table: per node (pre, pm[pre], sm[pre], size)
};

// Per node w with p = pre(w): the per-position entries of the blocked table that a query can need
// from w's side, pm[p] (w has the larger preorder number) and sm[p] (the smaller one), with p and
// size(w), so that a query reads two 16-byte records instead of pre[] twice, then pm and sm. The
// table stores (pm, sm) pairs, so this is one 8-byte gather per node.
__global__ void k_node_rec(const int32_t *__restrict__ pre, const int32_t *__restrict__ size,
                           const int2 *__restrict__ pmsm, int32_t n, int4 *__restrict__ nrec) {
    pdl_prologue();
    constexpr int kIlp = 4;  // nodes per thread per step, their gathers in flight together
    const int64_t step = gstride() * kIlp;
    for (int64_t base = blockIdx.x * int64_t(blockDim.x) * kIlp + threadIdx.x; base < n; base += step) {
        int32_t p[kIlp];
        int2 e[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const int64_t w = base + int64_t(j) * blockDim.x;
            p[j] = w < n ? __ldcs(pre + w) : -1;
            e[j] = (p[j] >= 0 && p[j] < n) ? __ldg(pmsm + p[j]) : make_int2(INT_MAX, INT_MAX);  // bad tree: flagged
        }
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const int64_t w = base + int64_t(j) * blockDim.x;
            if (w < n) __stcs(nrec + w, make_int4(p[j], e[j].x, e[j].y, __ldcs(size + w)));
        }
    }
}

constexpr int kQueryIlp = 4;

// min of x[lo..hi], a range inside one block of the blocked table (at most 32 entries, one line)
__device__ __forceinline__ int32_t inblock_min(const int32_t *__restrict__ x, int32_t lo, int32_t hi) {
    int32_t m = __ldg(x + lo);
    for (int32_t j = lo + 1; j <= hi; ++j) m = min(m, __ldg(x + j));
    return m;
}

// Each thread answers kQueryIlp queries at once so that their dependent
// gathers (pre, table, order) overlap in flight. BATCH: ids are local to the
// instance inst[i] and so is the answer.
template <bool BATCH, bool BLOCKED>
__global__ void __launch_bounds__(256)
    k_lca_query(LcaView h, const int32_t *__restrict__ inst, const int32_t *__restrict__ u,
                const int32_t *__restrict__ v, int64_t q, int32_t *__restrict__ out, int32_t *__restrict__ status) {
    pdl_prologue();
    const bool bad_tree = *h.hstatus != 0;
    const int64_t stride = gstride();
    for (int64_t base = gtid(); base < q; base += stride * kQueryIlp) {
        int32_t a[kQueryIlp], b[kQueryIlp], lo[kQueryIlp], hi[kQueryIlp], res[kQueryIlp], ofs[kQueryIlp];
        bool need[kQueryIlp], ok[kQueryIlp];
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k) {
            const int64_t i = base + k * stride;
            need[k] = false;
            ok[k] = false;
            res[k] = -1;
            ofs[k] = 0;
            a[k] = b[k] = 0;
            if (i < q) {
                a[k] = __ldcs(u + i);
                b[k] = __ldcs(v + i);
                int32_t lim = h.n;
                if (BATCH) {
                    const int32_t t = __ldcs(inst + i);
                    if (t >= 0 && t < h.k) {
                        ofs[k] = __ldg(h.off + t);
                        lim = __ldg(h.off + t + 1) - ofs[k];
                    } else {
                        lim = 0;
                    }
                }
                ok[k] = a[k] >= 0 && a[k] < lim && b[k] >= 0 && b[k] < lim;
                if (!ok[k]) set_status(status, ETL_EBADQUERY);
            }
        }
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k) {
            if (!ok[k] || bad_tree) continue;
            if (a[k] == b[k]) {
                res[k] = a[k];
            } else if (BLOCKED) {
                const int4 ra = __ldg(h.nrec + ofs[k] + a[k]), rb = __ldg(h.nrec + ofs[k] + b[k]);
                const bool a_first = ra.x < rb.x;
                const int4 x = a_first ? ra : rb, y = a_first ? rb : ra;  // x earlier in preorder
                lo[k] = x.x + 1;
                hi[k] = y.x;
                need[k] = hi[k] - lo[k] + 1 <= h.max_len;  // cannot fail unless max_n was understated
                if (!need[k]) {
                    set_status(status, ETL_EINVAL);
                } else if (y.x < x.x + x.w) {  // y lies in x's subtree: x is the answer
                    need[k] = false;
                    res[k] = a_first ? a[k] : b[k];
                } else if ((x.x >> kRmqBlockLog2) != (hi[k] >> kRmqBlockLog2)) {
                    // across blocks: x is no ancestor of y, so Q at pre(x) (x's parent, the LCA or below
                    // it) cannot lower the minimum and the range may start at pre(x) itself: sm[pre x]
                    // and pm[pre y] come with the records, whole blocks between from the top table
                    int32_t m = min(x.z, y.y);
                    const int32_t bl = (x.x >> kRmqBlockLog2) + 1, bh = (hi[k] >> kRmqBlockLog2) - 1;
                    if (bl <= bh) {
                        const int l = 31 - __clz(bh - bl + 1);
                        const int32_t *row = h.bv.top + int64_t(l) * h.bv.nblk;
                        m = min(m, min(__ldg(row + bl), __ldg(row + bh - (1 << l) + 1)));
                    }
                    lo[k] = m;
                    hi[k] = -1;  // answered
                }
            } else {
                const int32_t pa = __ldg(h.pre + ofs[k] + a[k]), pb = __ldg(h.pre + ofs[k] + b[k]);
                lo[k] = min(pa, pb) + 1;
                hi[k] = max(pa, pb);
                need[k] = hi[k] - lo[k] + 1 <= h.max_len;  // cannot fail unless max_n was understated
                if (!need[k]) set_status(status, ETL_EINVAL);
            }
        }
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k)
            if (need[k] && hi[k] >= 0)  // in one block (blocked table), or the full table
                lo[k] = BLOCKED ? inblock_min(h.bv.x, lo[k], hi[k]) : sparse_query<false>(h.table, h.ld, lo[k], hi[k]);
#pragma unroll
        for (int k = 0; k < kQueryIlp; ++k) {
            const int64_t i = base + k * stride;
            if (i >= q) continue;
            if (need[k]) res[k] = __ldg(h.order + lo[k]) - ofs[k];
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
    if (h->arena) {  // the device arrays belong to the caller's workspace
        delete h;
        return;
    }
    cudaStream_t s = h->stream;
    for (int32_t *p : {h->pre, h->depth, h->size, h->order, h->table, h->status, h->node_off})
        if (p) cudaFreeAsync(p, s);
    for (void *p : {h->inrec, h->inpath, h->tour_table, static_cast<void *>(h->tpos), h->nrec})
        if (p) cudaFreeAsync(p, s);
    delete h;
}

// n nodes in k >= 1 trees; node_off (device, k+1 entries) is null for one tree
etl_status lca_build(const int32_t *parent, int32_t n, const int32_t *node_off, int32_t k, int32_t max_n,
                     bool with_table, cudaStream_t s, etl_lca_t *out) {
    const bool batch = node_off != nullptr;
    etl_lca_s *h = new etl_lca_s;
    h->arena = current_arena() != nullptr;
    h->n = n;
    h->k = k;
    h->stream = s;
    h->levels = max_n > 1 ? sparse_levels(max_n - 1) : 1;
    h->has_table = with_table;
    h->ld = sparse_ld(n);
    h->blocked = rmq_params().blocked;
    h->bl = blocked_layout(n, max_n);
    const size_t table_bytes = (h->blocked ? size_t(h->bl.elems()) : size_t(h->ld) * size_t(h->levels)) * 4;
    const size_t nb = size_t(n) * sizeof(int32_t);
    bool ok = dev_alloc((void **)&h->pre, nb, s) == cudaSuccess;
    ok = ok && dev_alloc((void **)&h->depth, nb, s) == cudaSuccess;
    ok = ok && dev_alloc((void **)&h->size, nb, s) == cudaSuccess;
    ok = ok && dev_alloc((void **)&h->order, nb, s) == cudaSuccess;
    if (with_table)
        ok = ok && dev_alloc((void **)&h->table, table_bytes, s) == cudaSuccess;
    if (with_table && h->blocked)
        ok = ok && dev_alloc((void **)&h->nrec, size_t(n) * sizeof(int4), s) == cudaSuccess;
    ok = ok && dev_alloc((void **)&h->status, sizeof(int32_t), s) == cudaSuccess;
    if (ok && batch)
        ok = dev_alloc((void **)&h->node_off, size_t(k + 1) * sizeof(int32_t), s) == cudaSuccess;
    if (!ok) {
        free_handle(h);
        return ETL_ENOMEM;
    }
    memset_async(h->status, 0, sizeof(int32_t), s);
    if (batch) copy_d2d_async(h->node_off, node_off, size_t(k + 1) * sizeof(int32_t), s);
    etl_status st = ETL_OK;
    {
        Workspace ws(s);
        int32_t *cnt = ws.get<int32_t>(n);
        int32_t *coff = ws.get<int32_t>(int64_t(n) + 1);
        int32_t *misc = ws.get<int32_t>(4);  // [0] list head, [1] offsets invalid
        int32_t *succ = ws.get<int32_t>(2 * int64_t(n));
        int32_t *sc = ws.get<int32_t>(n);  // successors of the closing brackets; those of the opening ones reuse cnt
        int32_t *root_cnt = ws.get<int32_t>(k), *root_of = ws.get<int32_t>(k);
        int32_t *inst_of = batch ? ws.get<int32_t>(n) : nullptr;
        int32_t *gparent = batch ? ws.get<int32_t>(n) : nullptr;
        if (!ws.ok()) st = ETL_ENOMEM;
        const int32_t *par = batch ? gparent : parent;
        if (!st) {
            memset_async(cnt, 0, nb, s);
            memset_async(misc, 0, 4 * sizeof(int32_t), s);
            memset_async(root_cnt, 0, size_t(k) * sizeof(int32_t), s);
            memset_async(root_of, 0, size_t(k) * sizeof(int32_t), s);
            PhaseTimer pt("lca.count", s);
            if (batch) {
                launch(k_check_offsets, grid_for(k, 256), 256, 0, s, h->node_off, k, n, misc + 1, h->status);
                note_launch();
                launch(k_fill_inst, k < 8192 ? k : 8192, 256, 0, s, h->node_off, k, misc + 1, inst_of);
                note_launch();
                launch(k_count_children<true>, grid_for(n, 256), 256, 0, s, parent, n, h->node_off, inst_of, misc + 1,
                       gparent, cnt, root_cnt, root_of, h->status);
                note_launch();
            } else {
                launch(k_count_children<false>, grid_for(n, 256), 256, 0, s, parent, n, nullptr, nullptr, nullptr,
                       nullptr, cnt, root_cnt, root_of, h->status);
                note_launch();
            }
            st = last_launch();
        }
        if (!st) st = scan_exclusive_i32(cnt, coff, n, ws);
        SortResult sr{};
        if (!st) st = radix_sort_pairs(par, nullptr, nullptr, n, ceil_log2(uint64_t(n)), n, ws, &sr);
        if (!st) {
            PhaseTimer pt("lca.succ", s);
            int32_t *so = cnt;  // the child counts are no longer needed once the offsets are scanned
            launch(k_tour_succ, grid_for(n, 256), 256, 0, s, sr.kv, coff, n, so, sc);
            note_launch();
            launch(k_link_roots, grid_for(k, 256), 256, 0, s, root_cnt, root_of, k, n, sc, misc, h->status);
            note_launch();
            launch(k_tour_assemble, grid_for(n, 256), 256, 0, s, coff, par, so, sc, n, succ);
            note_launch();
            st = last_launch();
        }
        RankResult rr{};
        if (!st) st = list_rank(succ, 2 * int64_t(n), nullptr, misc, true, 2 * int64_t(n), h->status, ws, &rr);
        if (!st) {
            PhaseTimer pt("lca.node_stats", s);
            launch(k_node_stats, grid_for(n, 256), 256, 0, s, rr, succ, n, h->pre, h->depth, h->size, h->order,
                   h->status);
            note_launch();
            launch(k_check_instances, grid_for(k, 256), 256, 0, s, root_of, batch ? h->node_off : nullptr, k, n, h->pre,
                   h->size, h->status);
            note_launch();
            st = last_launch();
        }
        if (!st && with_table) {
            PhaseTimer pt("lca.parent_pre", s);
            launch(k_parent_pre, grid_for(n, 256), 256, 0, s, par, h->pre, h->order, n, h->table);
            note_launch();
            st = last_launch();
        }
        if (!st && with_table)
            st = h->blocked ? blocked_build<OpMin>(h->table, n, h->bl, s, /*pairs=*/true)
                            : sparse_table_build<false>(h->table, n, h->levels, s);
        if (!st && with_table && h->blocked) {
            PhaseTimer pt("lca.node_rec", s);
            launch(k_node_rec, grid_for(n, 256), 256, 0, s, h->pre, h->size,
                   reinterpret_cast<const int2 *>(h->table + h->bl.nblk * kRmqBlock), n, static_cast<int4 *>(h->nrec));
            note_launch();
            st = last_launch();
        }
    }
    if (st) {
        free_handle(h);
        return st;
    }
    *out = h;
    return ETL_OK;
}

etl_status query_launch(etl_lca_t h, const int32_t *inst, const int32_t *u, const int32_t *v, int64_t q,
                        int32_t *out, int32_t *status, cudaStream_t s) {
    LcaView view{h->n,     h->k,      h->levels, h->ld,
                 h->pre,   h->order,  h->table,  h->status,
                 h->node_off, blocked_view<OpMin>(h->table, h->bl),
                 h->blocked ? blocked_max_len(h->bl) : (int64_t(1) << h->levels) - 1,
                 static_cast<const int4 *>(h->nrec)};
    PhaseTimer pt("lca.query", s);
    const int grid = grid_for(ceil_div(q, kQueryIlp), 256);
    if (h->blocked) {
        if (inst)
            launch(k_lca_query<true, true>, grid, 256, 0, s, view, inst, u, v, q, out, status);
        else
            launch(k_lca_query<false, true>, grid, 256, 0, s, view, nullptr, u, v, q, out, status);
    } else {
        if (inst)
            launch(k_lca_query<true, false>, grid, 256, 0, s, view, inst, u, v, q, out, status);
        else
            launch(k_lca_query<false, false>, grid, 256, 0, s, view, nullptr, u, v, q, out, status);
    }
    note_launch();
    return last_launch();
}

}  // namespace
}  // namespace etl

using namespace etl;

extern "C" etl_status lca_preprocess(const int32_t *parent, int32_t n, void *stream, etl_lca_t *out) {
    if (!out) return ETL_EINVAL;
    *out = nullptr;
    if (!parent || n < 1 || n > (1 << 30) - 1) return ETL_EINVAL;
    return lca_build(parent, n, nullptr, 1, n, true, static_cast<cudaStream_t>(stream), out);
}

etl_status lca_build_inlabel_impl(etl_lca_t h, const int32_t *parent, cudaStream_t s);
etl_status lca_build_tour_impl(etl_lca_t h, const int32_t *parent, cudaStream_t s);

extern "C" etl_status lca_preprocess_ex(const int32_t *parent, int32_t n, int32_t flags, void *stream,
                                        etl_lca_t *out) {
    if (!out) return ETL_EINVAL;
    *out = nullptr;
    constexpr int32_t kAll = ETL_LCA_RMQ | ETL_LCA_INLABEL | ETL_LCA_TOUR_RMQ;
    if (!parent || n < 1 || n > (1 << 30) - 1 || !(flags & kAll) || (flags & ~kAll)) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    etl_status st = lca_build(parent, n, nullptr, 1, n, (flags & ETL_LCA_RMQ) != 0, s, out);
    if (!st && (flags & ETL_LCA_INLABEL)) st = lca_build_inlabel_impl(*out, parent, s);
    if (!st && (flags & ETL_LCA_TOUR_RMQ)) st = lca_build_tour_impl(*out, parent, s);
    if (st && *out) {
        free_handle(*out);
        *out = nullptr;
    }
    return st;
}

extern "C" etl_status lca_preprocess_batch(const int32_t *parent, const int32_t *node_off, int32_t k,
                                           int32_t total_n, int32_t max_n, void *stream, etl_lca_t *out) {
    if (!out) return ETL_EINVAL;
    *out = nullptr;
    if (!parent || !node_off || k < 1 || total_n < k || total_n > (1 << 30) - 1 || max_n < 1 || max_n > total_n)
        return ETL_EINVAL;
    return lca_build(parent, total_n, node_off, k, max_n, true, static_cast<cudaStream_t>(stream), out);
}

extern "C" etl_status lca_query(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                                int32_t *status, void *stream) {
    if (!h || h->node_off || !h->has_table || q < 0 || q > (int64_t(1) << 40)) return ETL_EINVAL;
    if (q == 0) return ETL_OK;
    if (!u || !v || !out) return ETL_EINVAL;
    return query_launch(h, nullptr, u, v, q, out, status, static_cast<cudaStream_t>(stream));
}

extern "C" etl_status lca_query_batch(etl_lca_t h, const int32_t *inst, const int32_t *u, const int32_t *v,
                                      int64_t q, int32_t *out, int32_t *status, void *stream) {
    if (!h || !h->node_off || q < 0 || q > (int64_t(1) << 40)) return ETL_EINVAL;
    if (q == 0) return ETL_OK;
    if (!inst || !u || !v || !out) return ETL_EINVAL;
    return query_launch(h, inst, u, v, q, out, status, static_cast<cudaStream_t>(stream));
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
        if (dst[i] && copy_d2d_async(dst[i], src[i], nb, s) != cudaSuccess) return ETL_ECUDA;
    return ETL_OK;
}

extern "C" etl_status lca_free(etl_lca_t h) {
    if (!h) return ETL_OK;
    free_handle(h);
    return cudaGetLastError() == cudaSuccess ? ETL_OK : ETL_ECUDA;
}
