// Bridges by the Tarjan-Vishkin method (Sec. 4.1) on one GPU.
//
// Phase 1, spanning forest: a lock-free hook-and-compress connected-components
//   pass in the style the paper takes from Jaiganesh and Burtscher: every edge
//   finds the roots of its two ends (with path halving) and hooks the larger
//   root under the smaller one with a CAS. A CAS that succeeds joins two
//   different trees, so its edge is a forest edge; exactly n - c succeed.
// Phase 2, Euler tour of the forest (Sec. 2.1): forest edge t owns half-edges
//   2t = (u_t, v_t) and 2t+1 = (v_t, u_t), so twin(a) = a ^ 1. A counting
//   sort by tail (atomic slots; the order inside a vertex's group is free,
//   any cyclic order gives an Euler tour) groups the half-edges of every
//   vertex (array B); next(a) is
//   the following entry of B with the same tail, cyclically; succ(a) =
//   next(twin(a)). Each component's cyclic list is cut in front of the first
//   half-edge of its root (the smallest vertex, which is where hooking ends),
//   and the component lists are chained into one list behind a virtual head,
//   which is ranked once (rank.cu).
// Phase 3, low / high: with tin(x) = rank of the half-edge entering x (a root
//   gets the position just before its component), the subtree of u is the
//   tour interval [tin(u), tout(u)], tout(u) = rank of the half-edge leaving
//   u. nlo(x) / nhi(x) = min / max of tin(x) and tin(w) over non-forest
//   edges (x, w), by atomics (the paper uses a segmented reduction);
//   placed at tin(x) in tour order, low(u) / high(u) are range-min / -max
//   queries over [tin(u), tout(u)]: one blocked table of (L, H) pairs by
//   default, else two full sparse tables (rmq.cu).
// Phase 4, the test: forest edge {u, parent(u)} is a bridge iff
//   low(u) >= tin(u) and high(u) <= tout(u), i.e. no non-forest edge leaves
//   the subtree of u. (Sec. 4.1 states the condition the other way round;
//   low or high escaping the subtree's interval is the NON-bridge case,
//   since such an edge reconnects the subtree with the rest of the graph.)
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

constexpr int64_t kFindCap = int64_t(1) << 26;  // bound on pointer-chasing steps of one edge

__global__ void k_init(int32_t n, int32_t *__restrict__ par, int32_t *__restrict__ deg, int32_t *__restrict__ tin) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        par[v] = int32_t(v);
        deg[v] = 0;
        tin[v] = 0;
    }
}

// root of x with path halving; -1 if the step budget runs out
__device__ __forceinline__ int32_t find_root(int32_t *par, int32_t x, int64_t &budget) {
    while (budget-- > 0) {
        const int32_t p = __ldcg(par + x);
        if (p == x) return x;
        const int32_t gp = __ldcg(par + p);
        if (gp == p) return p;
        par[x] = gp;  // only non-roots are rewritten, always to an ancestor
        x = gp;
    }
    return -1;
}

// The edges are cut into chunks of kHookChunk consecutive edges, one chunk per block step; one
// launch hooks positions c0 .. c1 - 1 of the chunk sequence. With `spread` (batches of graphs) the
// chunks are grouped into superchunks of kHookSuper that are visited in a permuted order
// (superchunk s of the sequence is s * P mod nsuper, P = 2^31 - 1, a prime above any superchunk
// count, so the map is a bijection), the chunks of a superchunk in order. The blocks running at one
// time then work on ~150 regions of 64 KB of edges spread over the whole list: in a batch of many
// small graphs, a contiguous sweep puts thousands of threads on one graph's few roots, where their
// CAS attempts collide and retry (measured: 11.4 -> 4 ms on 2048 graphs), and a first slice of the
// sequence samples every graph of the batch, not the first ones only. A single graph keeps the
// contiguous order, which measured faster on it (0.7 against 1.3 ms on 2^25 shuffled edges).
constexpr int kHookChunk = 256;
constexpr int kHookSuper = 32;

// number of positions of the chunk sequence over m edges (whole superchunks)
inline int64_t hook_positions(int64_t m) {
    return ceil_div(ceil_div(m, kHookChunk), kHookSuper) * kHookSuper;
}

__device__ __forceinline__ int64_t hook_chunk(int64_t c, int64_t nsuper, bool spread) {
    constexpr int64_t kP = 2147483647;
    return spread ? ((c / kHookSuper) * kP % nsuper) * kHookSuper + c % kHookSuper : c;
}

// Roots are hooked under roots of higher priority: a smaller id, except that the root named by
// *giant (if any: the most frequent root after a compression, i.e. the giant component's) ranks above
// all. Priorities are a strict total order, so the forest stays acyclic, and the giant root never
// moves: once the giant component has formed, every later hook leaves the paths of its members as
// they are (with plain smaller-id order the giant root moves whenever a smaller one joins, and every
// member's path grows by a step).
__device__ __forceinline__ bool hook_above(int32_t a, int32_t b, int32_t giant) {  // a ranks above b
    return a == giant || (b != giant && a < b);
}

// skip (may be null): edges to leave out; is_tree (may be null): 1 for edges whose hook succeeded
__global__ void __launch_bounds__(kHookChunk)
    k_hook(const int32_t *__restrict__ edges, int64_t m, int64_t c0, int64_t c1, bool spread, int32_t n,
           int32_t *__restrict__ par, uint8_t *__restrict__ is_tree, const uint8_t *__restrict__ skip,
           const int32_t *__restrict__ d_giant, int32_t *__restrict__ status) {
    pdl_prologue();
    const int32_t giant = d_giant ? *d_giant : -1;
    const int64_t nsuper = ((m + kHookChunk - 1) / kHookChunk + kHookSuper - 1) / kHookSuper;
    for (int64_t c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const int64_t e = hook_chunk(c, nsuper, spread) * kHookChunk + threadIdx.x;
        if (e >= m) continue;
        int32_t a = __ldcs(edges + 2 * e), b = __ldcs(edges + 2 * e + 1);
        uint8_t tree = 0;
        if (skip && skip[e]) {
            // left out
        } else if (a < 0 || a >= n || b < 0 || b >= n) {
            set_status(status, ETL_EBADGRAPH);
        } else {
            int64_t budget = kFindCap;
            // both ends already point at the same node: same set, nothing to hook
            const bool same = __ldcg(par + a) == __ldcg(par + b);
            while (!same) {
                const int32_t ra = find_root(par, a, budget), rb = find_root(par, b, budget);
                if (ra < 0 || rb < 0) {
                    set_status(status, ETL_ETIMEOUT);
                    break;
                }
                if (ra == rb) break;
                const bool a_up = hook_above(ra, rb, giant);
                const int32_t hi = a_up ? rb : ra, lo = a_up ? ra : rb;  // hi goes under lo
                if (atomicCAS(par + hi, hi, lo) == hi) {
                    tree = 1;
                    break;
                }
                a = ra;  // someone hooked one of the roots meanwhile: retry from them
                b = rb;
            }
        }
        if (is_tree) is_tree[e] = tree;
    }
}

__global__ void k_compress(int32_t n, int32_t *__restrict__ par, int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        int64_t budget = kFindCap;
        const int32_t r = find_root(par, int32_t(v), budget);
        if (r < 0)
            set_status(status, ETL_ETIMEOUT);
        else
            par[v] = r;
    }
}

// The most frequent root among kGiantSample vertices spread over [0, n) (one block; par must be
// compressed, so par[v] is v's root): the giant component's root when there is one.
constexpr int kGiantSample = 1024;

__global__ void __launch_bounds__(kGiantSample) k_giant(const int32_t *__restrict__ par, int32_t n,
                                                         int32_t *__restrict__ giant) {
    pdl_prologue();
    constexpr int kSlots = 2 * kGiantSample;  // open-addressing table of (root, count)
    __shared__ int32_t key[kSlots], cnt[kSlots];
    __shared__ unsigned long long best;
    const int i = threadIdx.x;
    for (int j = i; j < kSlots; j += kGiantSample) {
        key[j] = -1;
        cnt[j] = 0;
    }
    if (i == 0) best = 0;
    __syncthreads();
    const int32_t v = int32_t((uint64_t(i) * 2654435761u + 12345u) % uint64_t(n));
    const int32_t r = __ldcg(par + v);
    int slot = -1;
    uint32_t h = (uint32_t(r) * 2654435761u) >> 21;  // 11 bits: kSlots = 2048
    for (int probe = 0; probe < kSlots; ++probe, h = (h + 1) & (kSlots - 1)) {
        const int32_t prev = atomicCAS(&key[h], -1, r);
        if (prev == -1 || prev == r) {
            slot = int(h);
            atomicAdd(&cnt[h], 1);
            break;
        }
    }
    __syncthreads();
    // largest count, then smallest root id: pack (count, ~root) and take the maximum
    if (slot >= 0)
        atomicMax(&best, (static_cast<unsigned long long>(cnt[slot]) << 32) | uint32_t(~uint32_t(r)));
    __syncthreads();
    if (i == 0) *giant = best ? int32_t(~uint32_t(best & 0xffffffffu)) : -1;
}

// forest edges packed in edge order: tuv[2t] = u, tuv[2t+1] = v, tedge[t] = e
__global__ void k_forest_edges(const int32_t *__restrict__ edges, int64_t m, const uint8_t *__restrict__ is_tree,
                               const int32_t *__restrict__ tpos, int32_t *__restrict__ tuv,
                               int32_t *__restrict__ tedge, int32_t *__restrict__ n_arcs) {
    pdl_prologue();
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_arcs = 2 * tpos[m];
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        if (is_tree[e]) {
            const int32_t t = tpos[e];
            tuv[2 * t] = edges[2 * e];
            tuv[2 * t + 1] = edges[2 * e + 1];
            tedge[t] = int32_t(e);
        }
    }
}

// half-edges per tail vertex
__global__ void k_arc_count(const int32_t *__restrict__ tuv, const int32_t *__restrict__ d_len,
                            int32_t *__restrict__ deg) {
    pdl_prologue();
    const int64_t len = *d_len;
    for (int64_t a = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; a < len; a += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&deg[tuv[a]], 1);
}

// B[i] = (half-edge, tail) grouped by tail: off[x] .. off[x+1]-1 are the half-edges leaving x
__global__ void k_arc_scatter(const int32_t *__restrict__ tuv, const int32_t *__restrict__ d_len,
                              const int32_t *__restrict__ off, int32_t *__restrict__ deg, int2 *__restrict__ B) {
    pdl_prologue();
    const int64_t len = *d_len;
    for (int64_t a = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; a < len; a += int64_t(gridDim.x) * blockDim.x) {
        const int32_t x = tuv[a];
        const int32_t k = atomicSub(&deg[x], 1) - 1;
        B[off[x] + k] = make_int2(int32_t(a), x);
    }
}

// succ(twin(b)) := next(b) for every half-edge b at position i of B; half-edge
// slots beyond the forest (and the virtual head, set later) are inert
__global__ void k_forest_succ(const int2 *__restrict__ B, const int32_t *__restrict__ d_len, int64_t cap,
                              const int32_t *__restrict__ off, int32_t *__restrict__ succ) {
    pdl_prologue();
    const int64_t len = *d_len;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < cap; i += int64_t(gridDim.x) * blockDim.x) {
        if (i < len) {
            const int2 bx = B[i];
            // the group of tail bx.y continues at i + 1 iff that entry has the same tail; only the last
            // entry of a group reads the group's start
            const int2 nx = i + 1 < len ? B[i + 1] : make_int2(-1, -1);
            const int32_t nb = nx.y == bx.y ? nx.x : B[off[bx.y]].x;
            succ[bx.x ^ 1] = nb;
        } else {
            succ[i] = ETL_END;
        }
    }
}

__global__ void k_root_flags(int32_t n, const int32_t *__restrict__ par, const int32_t *__restrict__ off,
                             uint8_t *__restrict__ flag) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        flag[v] = (par[v] == v && off[v + 1] > off[v]) ? 1 : 0;
}

__global__ void k_root_list(int32_t n, const uint8_t *__restrict__ flag, const int32_t *__restrict__ rpos,
                            int32_t *__restrict__ roots) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        if (flag[v]) roots[rpos[v]] = int32_t(v);
}

// cut each component's cyclic tour in front of its root's first half-edge and
// chain the components: virtual head -> comp 0 -> comp 1 -> ... -> end
__global__ void k_chain(int32_t n, const int32_t *__restrict__ rpos, const int32_t *__restrict__ roots,
                        const int2 *__restrict__ B, const int32_t *__restrict__ off, int32_t vhead,
                        int32_t *__restrict__ succ) {
    pdl_prologue();
    const int32_t c = rpos[n];
    if (blockIdx.x == 0 && threadIdx.x == 0) succ[vhead] = c > 0 ? B[off[roots[0]]].x : ETL_END;
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < c; k += int64_t(gridDim.x) * blockDim.x) {
        const int32_t r = roots[k];
        const int32_t tail = B[off[r + 1] - 1].x ^ 1;  // the half-edge whose successor was the head
        succ[tail] = (k + 1 < c) ? B[off[roots[k + 1]]].x : ETL_END;
    }
}

// tour positions of forest edges: the half-edge ranked first goes down into the child
__global__ void k_forest_tin(RankResult rr, const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ tuv,
                             int32_t *__restrict__ tin, int32_t *__restrict__ child, int32_t *__restrict__ etin,
                             int32_t *__restrict__ etout) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    const uint4 *pk = reinterpret_cast<const uint4 *>(rr.packed);
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const uint4 q = pk[t];
        if (q.x >= rr.rcap || q.z >= rr.rcap) {  // cannot happen for a forest built above; keep memory safe
            child[t] = 0;
            etin[t] = etout[t] = -1;
            continue;
        }
        const int32_t r0 = rank_of(rr, make_uint2(q.x, q.y)), r1 = rank_of(rr, make_uint2(q.z, q.w));
        const int32_t c = r0 < r1 ? tuv[2 * t + 1] : tuv[2 * t];
        const int32_t a = min(r0, r1), b = max(r0, r1);
        tin[c] = a;
        child[t] = c;
        etin[t] = a;
        etout[t] = b;
    }
}

__global__ void k_root_tin(int32_t n, const int32_t *__restrict__ rpos, const int32_t *__restrict__ roots,
                           const int2 *__restrict__ B, const int32_t *__restrict__ off, RankResult rr,
                           int32_t *__restrict__ tin) {
    pdl_prologue();
    const int32_t c = rpos[n];
    for (int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; k < c; k += int64_t(gridDim.x) * blockDim.x) {
        const int32_t r = roots[k];
        const uint2 p = rr.packed[B[off[r]].x];
        tin[r] = p.x < rr.rcap ? rank_of(rr, p) - 1 : -1;
    }
}

__global__ void k_nlo_init(int32_t n, const int32_t *__restrict__ tin, int32_t *__restrict__ nlo,
                           int32_t *__restrict__ nhi) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        const int32_t x = tin[v];
        nlo[v] = x;
        nhi[v] = x;
    }
}

__global__ void k_nontree_minmax(const int32_t *__restrict__ edges, int64_t m, int32_t n,
                                 const uint8_t *__restrict__ is_tree, const int32_t *__restrict__ tin,
                                 int32_t *__restrict__ nlo, int32_t *__restrict__ nhi) {
    pdl_prologue();
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        if (__ldcs(is_tree + e)) continue;
        const int32_t a = __ldcs(edges + 2 * e), b = __ldcs(edges + 2 * e + 1);
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) continue;
        const int32_t ta = __ldg(tin + a), tb = __ldg(tin + b);
        // nlo(x) and nhi(x) start at tin(x): of the four updates only the one lowering the later
        // end's nlo and the one raising the earlier end's nhi can change anything
        if (ta < tb) {
            atomicMax(nhi + a, tb);
            atomicMin(nlo + b, ta);
        } else if (tb < ta) {
            atomicMax(nhi + b, ta);
            atomicMin(nlo + a, tb);
        }
    }
}

// nlo / nhi of every non-root vertex at its tour position; identities at the
// positions of half-edges going up and at the virtual head (position 0)
__global__ void k_place(const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ child,
                        const int32_t *__restrict__ etin, const int32_t *__restrict__ etout,
                        const int32_t *__restrict__ nlo, const int32_t *__restrict__ nhi, int64_t P,
                        int32_t *__restrict__ L, int32_t *__restrict__ H) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        L[0] = INT_MAX;
        H[0] = INT_MIN;
    }
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = child[t], a = etin[t], b = etout[t];
        if (a < 0 || b >= P || a >= b) continue;
        L[a] = nlo[c];
        H[a] = nhi[c];
        L[b] = INT_MAX;
        H[b] = INT_MIN;
    }
}

// blocked form: L and H interleaved (x = L, y = H) in one table of int2
__global__ void k_place2(const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ child,
                         const int32_t *__restrict__ etin, const int32_t *__restrict__ etout,
                         const int32_t *__restrict__ nlo, const int32_t *__restrict__ nhi, int64_t P,
                         int2 *__restrict__ LH) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    const int2 id = make_int2(INT_MAX, INT_MIN);
    if (blockIdx.x == 0 && threadIdx.x == 0) LH[0] = id;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = child[t], a = etin[t], b = etout[t];
        if (a < 0 || b >= P || a >= b) continue;
        LH[a] = make_int2(nlo[c], nhi[c]);
        LH[b] = id;
    }
}

__global__ void k_bridge_test2(const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ etin,
                               const int32_t *__restrict__ etout, BlockedView<OpMinMax> lh, int64_t P,
                               uint8_t *__restrict__ tflag) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t a = etin[t], b = etout[t];
        if (a < 0 || b >= P || a >= b) {
            tflag[t] = 0;
            continue;
        }
        const int2 r = blocked_query<OpMinMax>(lh, a, b);  // (low, high) of the subtree
        tflag[t] = (r.x >= a && r.y <= b) ? 1 : 0;
    }
}

__global__ void k_bridge_test(const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ etin,
                              const int32_t *__restrict__ etout, const int32_t *__restrict__ Lt,
                              const int32_t *__restrict__ Ht, int64_t P, int64_t ld, uint8_t *__restrict__ tflag) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t a = etin[t], b = etout[t];
        if (a < 0 || b >= P || a >= b) {
            tflag[t] = 0;
            continue;
        }
        const int32_t low = sparse_query<false>(Lt, ld, a, b);
        const int32_t high = sparse_query<true>(Ht, ld, a, b);
        tflag[t] = (low >= a && high <= b) ? 1 : 0;
    }
}

__global__ void k_finalize(int64_t m, const uint8_t *__restrict__ is_tree, const int32_t *__restrict__ tpos,
                           const uint8_t *__restrict__ tflag, const int32_t *__restrict__ status,
                           uint8_t *__restrict__ is_bridge) {
    pdl_prologue();
    const bool bad = *status != 0;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x)
        is_bridge[e] = (!bad && is_tree[e]) ? tflag[tpos[e]] : 0;
}

}  // namespace

CcParams &cc_params() {
    static CcParams p;
    return p;
}

namespace {

int grid_for(int64_t work, int threads) {
    int64_t blocks = ceil_div(work, threads);
    const int64_t cap = int64_t(num_sms()) * (2048 / threads) * 4;
    if (blocks > cap) blocks = cap;
    return int(blocks < 1 ? 1 : blocks);
}

}  // namespace
}  // namespace etl

namespace etl {
namespace {

// ---- the hybrid of Sec. 4.3: parents and levels of the rooted forest from its Euler tour, then
// Chaitanya-Kothapalli marking: every non-tree edge walks both ends up to their LCA and marks the
// tree edges on the way (a tree edge is named by its child); unmarked tree edges are bridges

__global__ void k_tour_pm(const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ etin,
                          const int32_t *__restrict__ etout, int64_t P, int32_t *__restrict__ val) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    if (blockIdx.x == 0 && threadIdx.x == 0) val[0] = 0;  // the virtual head
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t a = etin[t], b = etout[t];
        if (a < 0 || b >= P || a >= b) continue;
        val[a] = 1;   // down into the child: one level deeper
        val[b] = -1;  // back up
    }
}

__global__ void k_tree_records(int32_t n, const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ tuv,
                               const int32_t *__restrict__ child, const int32_t *__restrict__ etin,
                               const int32_t *__restrict__ excl, int64_t P, int2 *__restrict__ trec,
                               uint8_t *__restrict__ mark) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t c = child[t], a = etin[t];
        if (a < 0 || a >= P) continue;
        const int32_t p = tuv[2 * t] == c ? tuv[2 * t + 1] : tuv[2 * t];
        trec[c] = make_int2(p, excl[a + 1]);  // (parent, level): level = prefix of +-1 at the child's entry
        mark[c] = 0;
    }
}

__global__ void k_tree_records_init(int32_t n, int2 *__restrict__ trec) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        trec[v] = make_int2(-1, 0);  // roots and isolated vertices
}

__global__ void k_ck_mark(const int32_t *__restrict__ edges, int64_t m, int32_t n, const uint8_t *__restrict__ is_tree,
                          const int2 *__restrict__ trec, uint8_t *__restrict__ mark, int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        if (is_tree[e]) continue;
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) continue;
        int2 ra = __ldg(trec + a), rb = __ldg(trec + b);
        int64_t steps = 0;
        while (a != b) {
            if (++steps > 2 * int64_t(n)) {
                set_status(status, ETL_ETIMEOUT);
                break;
            }
            if (ra.y >= rb.y) {
                mark[a] = 1;
                a = ra.x;
                if (a < 0 || a >= n) break;
                ra = __ldg(trec + a);
            } else {
                mark[b] = 1;
                b = rb.x;
                if (b < 0 || b >= n) break;
                rb = __ldg(trec + b);
            }
        }
    }
}

__global__ void k_ck_flags(const int32_t *__restrict__ d_arcs, const int32_t *__restrict__ child,
                           const uint8_t *__restrict__ mark, uint8_t *__restrict__ tflag) {
    pdl_prologue();
    const int64_t T = *d_arcs / 2;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < T; t += int64_t(gridDim.x) * blockDim.x)
        tflag[t] = mark[child[t]] ? 0 : 1;
}

etl_status hybrid_marking(const int32_t *edges, int64_t m, int32_t n, const uint8_t *is_tree, const int32_t *tpos,
                          const int32_t *tuv, const int32_t *n_arcs, const int32_t *child, const int32_t *etin,
                          const int32_t *etout, int64_t P, uint8_t *tflag, int32_t *st, Workspace &ws) {
    (void)tpos;
    cudaStream_t s = ws.stream();
    int32_t *val = ws.get<int32_t>(P), *excl = ws.get<int32_t>(P + 1);
    int2 *trec = ws.get<int2>(n);
    uint8_t *mark = ws.get<uint8_t>(n);
    if (!ws.ok()) return ETL_ENOMEM;
    const int gn = grid_for(n, 256);
    {
        PhaseTimer pt("hybrid.levels", s);
        launch(k_tour_pm, gn, 256, 0, s, n_arcs, etin, etout, P, val);
        note_launch();
    }
    etl_status rc = last_launch();
    if (!rc) rc = scan_exclusive_i32(val, excl, P, ws);
    if (rc) return rc;
    PhaseTimer pt("hybrid.mark", s);
    launch(k_tree_records_init, gn, 256, 0, s, n, trec);
    note_launch();
    launch(k_tree_records, gn, 256, 0, s, n, n_arcs, tuv, child, etin, excl, P, trec, mark);
    note_launch();
    launch(k_ck_mark, grid_for(m, 256), 256, 0, s, edges, m, n, is_tree, trec, mark, st);
    note_launch();
    launch(k_ck_flags, gn, 256, 0, s, n_arcs, child, mark, tflag);
    note_launch();
    return last_launch();
}

// the whole Tarjan-Vishkin pipeline on a graph with global ids; st is a zeroed device status word.
// hybrid: instead of low / high, the Chaitanya-Kothapalli marking on the same rooted forest
etl_status bridges_core(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge, int32_t *st,
                        Workspace &ws, bool hybrid = false, bool spread = false) {
    cudaStream_t s = ws.stream();
    const int64_t A = 2 * int64_t(n - 1);  // half-edge capacity of a spanning forest
    const int64_t N = A + 1;                // + the virtual head, at index A
    const int64_t P = N;                    // tour positions 0 .. A
    const int levels = sparse_levels(P);
    const int64_t ld = sparse_ld(P);
    const bool blocked = rmq_params().blocked;
    const BlockedLayout bl = blocked_layout(P, P);
    int32_t *par = ws.get<int32_t>(n), *deg = ws.get<int32_t>(n), *off = ws.get<int32_t>(int64_t(n) + 1);
    int2 *B = ws.get<int2>(A > 0 ? A : 1);
    int32_t *tin = ws.get<int32_t>(n), *nlo = ws.get<int32_t>(n), *nhi = ws.get<int32_t>(n);
    uint8_t *is_tree = ws.get<uint8_t>(m), *rflag = ws.get<uint8_t>(n);
    int32_t *tpos = ws.get<int32_t>(m + 1), *rpos = ws.get<int32_t>(int64_t(n) + 1), *roots = ws.get<int32_t>(n);
    int32_t *tuv = ws.get<int32_t>(A > 0 ? A : 1), *tedge = ws.get<int32_t>(n);
    int32_t *n_arcs = ws.get<int32_t>(1), *vhead = ws.get<int32_t>(1), *giant = ws.get<int32_t>(1);
    int32_t *succ = ws.get<int32_t>(N);
    int32_t *child = ws.get<int32_t>(n), *etin = ws.get<int32_t>(n), *etout = ws.get<int32_t>(n);
    uint8_t *tflag = ws.get<uint8_t>(n);
    int32_t *Lt = (hybrid || blocked) ? nullptr : ws.get<int32_t>(ld * levels);
    int32_t *Ht = (hybrid || blocked) ? nullptr : ws.get<int32_t>(ld * levels);
    int2 *LH = (!hybrid && blocked) ? ws.get<int2>(bl.elems()) : nullptr;
    if (!ws.ok()) return ETL_ENOMEM;
    etl_status rc = ETL_OK;
    const int gn = grid_for(n, 256), gm = grid_for(m, 256), gA = grid_for(N, 256);
    {
        PhaseTimer pt("br.init", s);
        launch(k_init, gn, 256, 0, s, n, par, deg, tin);
        note_launch();
    }
    {
        // hook a first slice of the edges, compress every path to its root, then hook the rest:
        // after the compression most finds take one step and most edges meet equal roots at once.
        // With `doubling`, the rest goes in slices that double in size, each followed by a
        // compression, so that no phase builds long paths in a fresh part of the forest.
        const CcParams &C = cc_params();
        const int64_t slice = int64_t(C.first_slice_quarters) * n / 4;
        const int64_t nchunks = hook_positions(m);
        int64_t w = ceil_div(slice > 0 ? slice : 1, kHookChunk);  // chunks in the current slice
        PhaseTimer pt("br.hook", s);
        for (int64_t c0 = 0; c0 < nchunks;) {
            const int64_t c1 = (C.doubling || c0 == 0) ? (c0 + w < nchunks ? c0 + w : nchunks) : nchunks;
            if (c0 > 0) {
                launch(k_compress, gn, 256, 0, s, n, par, st);
                note_launch();
                if (C.giant) {
                    launch(k_giant, 1, kGiantSample, 0, s, par, n, giant);
                    note_launch();
                }
            }
            launch(k_hook, grid_for((c1 - c0) * kHookChunk, kHookChunk), kHookChunk, 0, s, edges, m, c0, c1, spread, n,
                   par, is_tree, nullptr, (c0 > 0 && C.giant) ? giant : nullptr, st);
            note_launch();
            c0 = c1;
            w *= 2;
        }
    }
    {
        PhaseTimer pt("br.compress", s);
        launch(k_compress, gn, 256, 0, s, n, par, st);
        note_launch();
    }
    rc = last_launch();
    if (!rc) rc = scan_exclusive_u8(is_tree, tpos, m, ws);
    if (!rc) {
        PhaseTimer pt("br.forest_edges", s);
        launch(k_forest_edges, gm, 256, 0, s, edges, m, is_tree, tpos, tuv, tedge, n_arcs);
        note_launch();
        rc = last_launch();
    }
    if (!rc) {
        PhaseTimer pt("br.group", s);
        launch(k_arc_count, gA, 256, 0, s, tuv, n_arcs, deg);
        note_launch();
        rc = last_launch();
    }
    if (!rc) rc = scan_exclusive_i32(deg, off, n, ws);
    if (!rc) {
        PhaseTimer pt("br.forest_succ", s);
        launch(k_arc_scatter, gA, 256, 0, s, tuv, n_arcs, off, deg, B);
        note_launch();
        launch(k_forest_succ, gA, 256, 0, s, B, n_arcs, N, off, succ);
        note_launch();
        launch(k_root_flags, gn, 256, 0, s, n, par, off, rflag);
        note_launch();
        rc = last_launch();
    }
    if (!rc) rc = scan_exclusive_u8(rflag, rpos, n, ws);
    if (!rc) {
        PhaseTimer pt("br.chain", s);
        launch(k_root_list, gn, 256, 0, s, n, rflag, rpos, roots);
        note_launch();
        launch(k_chain, gn, 256, 0, s, n, rpos, roots, B, off, int32_t(A), succ);
        note_launch();
        rc = last_launch();
    }
    if (!rc) rc = set_device_i32(vhead, int32_t(A), s);
    RankResult rr{};
    if (!rc) rc = list_rank(succ, N, nullptr, vhead, false, -1, st, ws, &rr);
    if (!rc) {
        const int gt = grid_for(n, 256);
        PhaseTimer pt("br.lowhigh_prep", s);
        launch(k_forest_tin, gt, 256, 0, s, rr, n_arcs, tuv, tin, child, etin, etout);
        note_launch();
        launch(k_root_tin, gn, 256, 0, s, n, rpos, roots, B, off, rr, tin);
        note_launch();
        rc = last_launch();
    }
    if (hybrid) {
        if (!rc) rc = hybrid_marking(edges, m, n, is_tree, tpos, tuv, n_arcs, child, etin, etout, P, tflag, st, ws);
        if (!rc) {
            launch(k_finalize, gm, 256, 0, s, m, is_tree, tpos, tflag, st, is_bridge);
            note_launch();
            rc = last_launch();
        }
        return rc;
    }
    if (!rc) {
        const int gt = grid_for(n, 256);
        PhaseTimer pt("br.lowhigh_prep", s);
        launch(k_nlo_init, gn, 256, 0, s, n, tin, nlo, nhi);
        note_launch();
        launch(k_nontree_minmax, gm, 256, 0, s, edges, m, n, is_tree, tin, nlo, nhi);
        note_launch();
        if (blocked)
            launch(k_place2, gt, 256, 0, s, n_arcs, child, etin, etout, nlo, nhi, P, LH);
        else
            launch(k_place, gt, 256, 0, s, n_arcs, child, etin, etout, nlo, nhi, P, Lt, Ht);
        note_launch();
        rc = last_launch();
    }
    if (blocked) {
        if (!rc) rc = blocked_build<OpMinMax>(LH, P, bl, s);
    } else {
        if (!rc) rc = sparse_table_build<false>(Lt, P, levels, s);
        if (!rc) rc = sparse_table_build<true>(Ht, P, levels, s);
    }
    if (!rc) {
        PhaseTimer pt("br.test", s);
        if (blocked)
            launch(k_bridge_test2, grid_for(n, 256), 256, 0, s, n_arcs, etin, etout, blocked_view<OpMinMax>(LH, bl), P,
                   tflag);
        else
            launch(k_bridge_test, grid_for(n, 256), 256, 0, s, n_arcs, etin, etout, Lt, Ht, P, ld, tflag);
        note_launch();
        launch(k_finalize, gm, 256, 0, s, m, is_tree, tpos, tflag, st, is_bridge);
        note_launch();
        rc = last_launch();
    }
    return rc;
}

__global__ void k_iota(int32_t n, int32_t *__restrict__ x) {
    pdl_prologue();
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        x[v] = int32_t(v);
}

__global__ void k_labels_on_error(int32_t n, const int32_t *__restrict__ status, int32_t *__restrict__ label) {
    pdl_prologue();
    if (*status == 0) return;
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        label[v] = -1;
}

// local edge ids of a batch -> global ids: edge e of instance i (edge_off[i] <= e < edge_off[i+1])
// joins node_off[i] + u and node_off[i] + v
__global__ void k_check_batch(const int32_t *__restrict__ eoff, const int32_t *__restrict__ noff, int32_t k,
                              int64_t m, int32_t n, int32_t *__restrict__ bad, int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < k; i += int64_t(gridDim.x) * blockDim.x) {
        const bool ok = eoff[i] >= 0 && eoff[i] <= eoff[i + 1] && eoff[i + 1] <= m && noff[i] >= 0 &&
                        noff[i] < noff[i + 1] && noff[i + 1] <= n && (i > 0 || (eoff[0] == 0 && noff[0] == 0)) &&
                        (i < k - 1 || (eoff[k] == m && noff[k] == n));
        if (!ok) {
            set_status(status, ETL_EINVAL);
            *bad = 1;
        }
    }
}

__global__ void k_globalize(const int32_t *__restrict__ edges, int64_t m, const int32_t *__restrict__ eoff,
                            const int32_t *__restrict__ noff, int32_t k, const int32_t *__restrict__ bad,
                            int32_t *__restrict__ gedges, int32_t *__restrict__ status) {
    pdl_prologue();
    const bool unusable = *bad != 0;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m; e += int64_t(gridDim.x) * blockDim.x) {
        int32_t gu = -1, gv = -1;
        if (!unusable) {
            int32_t lo = 0, hi = k;  // largest i with eoff[i] <= e (offsets checked monotone above)
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;
                if (__ldg(eoff + mid) <= e) lo = mid; else hi = mid - 1;
            }
            if (lo < k) {
                const int32_t base = __ldg(noff + lo), size = __ldg(noff + lo + 1) - base;
                const int32_t a = edges[2 * e], b = edges[2 * e + 1];
                if (a >= 0 && a < size && b >= 0 && b < size) {
                    gu = a + base;
                    gv = b + base;
                }
            }
            if (gu < 0) set_status(status, ETL_EBADGRAPH);
        }
        gedges[2 * e] = gu;
        gedges[2 * e + 1] = gv;
    }
}

}  // namespace
}  // namespace etl

using namespace etl;

extern "C" etl_status find_bridges(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge, int32_t *status,
                                   void *stream) {
    if (n < 1 || n > (1 << 30) - 1 || m < 0 || m > int64_t(INT32_MAX) - 1) return ETL_EINVAL;
    if (m == 0) return ETL_OK;
    if (!edges || !is_bridge) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    int32_t *st = status ? status : ws.get<int32_t>(1);
    if (!ws.ok()) return ETL_ENOMEM;
    memset_async(st, 0, sizeof(int32_t), s);
    return bridges_core(edges, m, n, is_bridge, st, ws);
}

extern "C" etl_status find_bridges_batch(const int32_t *edges, const int32_t *edge_off, const int32_t *node_off,
                                         int32_t k, int64_t total_m, int32_t total_n, uint8_t *is_bridge,
                                         int32_t *status, void *stream) {
    if (k < 1 || total_n < k || total_n > (1 << 30) - 1 || total_m < 0 || total_m > int64_t(INT32_MAX) - 1)
        return ETL_EINVAL;
    if (!edge_off || !node_off) return ETL_EINVAL;
    if (total_m == 0) return ETL_OK;
    if (!edges || !is_bridge) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    int32_t *st = status ? status : ws.get<int32_t>(1);
    int32_t *bad = ws.get<int32_t>(1);
    int32_t *gedges = ws.get<int32_t>(2 * total_m);
    if (!ws.ok()) return ETL_ENOMEM;
    memset_async(st, 0, sizeof(int32_t), s);
    memset_async(bad, 0, sizeof(int32_t), s);
    {
        PhaseTimer pt("br.globalize", s);
        launch(k_check_batch, grid_for(k, 256), 256, 0, s, edge_off, node_off, k, total_m, total_n, bad, st);
        note_launch();
        launch(k_globalize, grid_for(total_m, 256), 256, 0, s, edges, total_m, edge_off, node_off, k, bad, gedges, st);
        note_launch();
    }
    etl_status rc = last_launch();
    if (rc) return rc;
    return bridges_core(gedges, total_m, total_n, is_bridge, st, ws, false, true);
}

extern "C" etl_status two_edge_cc(const int32_t *edges, int64_t m, int32_t n, int32_t *label, int32_t *status,
                                  void *stream) {
    if (n < 1 || n > (1 << 30) - 1 || m < 0 || m > int64_t(INT32_MAX) - 1 || !label) return ETL_EINVAL;
    if (m > 0 && !edges) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    int32_t *st = status ? status : ws.get<int32_t>(1);
    uint8_t *is_bridge = ws.get<uint8_t>(m > 0 ? m : 1);
    if (!ws.ok()) return ETL_ENOMEM;
    memset_async(st, 0, sizeof(int32_t), s);
    etl_status rc = m > 0 ? bridges_core(edges, m, n, is_bridge, st, ws) : ETL_OK;
    if (rc) return rc;
    const int gn = grid_for(n, 256);
    PhaseTimer pt("br.two_edge_cc", s);
    launch(k_iota, gn, 256, 0, s, n, label);
    note_launch();
    if (m > 0) {  // connected components of the graph without its bridges; labels = smallest vertex
        launch(k_hook, grid_for(m, kHookChunk), kHookChunk, 0, s, edges, m, 0, hook_positions(m), false, n, label,
               nullptr, is_bridge, nullptr, st);
        note_launch();
        launch(k_compress, gn, 256, 0, s, n, label, st);
        note_launch();
    }
    launch(k_labels_on_error, gn, 256, 0, s, n, st, label);
    note_launch();
    return last_launch();
}

extern "C" etl_status find_bridges_hybrid(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge,
                                          int32_t *status, void *stream) {
    if (n < 1 || n > (1 << 30) - 1 || m < 0 || m > int64_t(INT32_MAX) - 1) return ETL_EINVAL;
    if (m == 0) return ETL_OK;
    if (!edges || !is_bridge) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    int32_t *st = status ? status : ws.get<int32_t>(1);
    if (!ws.ok()) return ETL_ENOMEM;
    memset_async(st, 0, sizeof(int32_t), s);
    return bridges_core(edges, m, n, is_bridge, st, ws, true);
}
