// List ranking on the GPU (Sec. 2.2): the successor array of the Euler tour is
// ranked once, and every later prefix sum over the tour is taken from these
// ranks. The paper uses the Wei-JaJa sparse-ruling-set method; this is a
// GB300-oriented ruling-set ranker:
//
//  * Splitters ("rulers") are picked by a multiplicative hash of the element
//    index: e is a splitter iff (e * M mod 2^b) < 2^b / K. The hashed value
//    is also the splitter's sublist id, so no table maps elements to sublists
//    and any structure in the labels (e.g. all opening brackets at even
//    indices) does not line up with the splitter pattern.
//  * The walk kernel is persistent: each lane walks one sublist, writing for
//    every element its sublist id and local offsets, and as soon as a lane's
//    walk ends it takes the next splitter from a warp-aggregated atomic
//    counter, so lanes stay busy despite the geometric spread of sublist
//    lengths. The hot loop is one dependent 4-byte load of succ[] per element,
//    so throughput comes from the number of walks in flight.
//  * A walk longer than kLcap elements opens a new sublist on the fly
//    ("dynamic splitter"), which bounds every local offset and every walk.
//  * The reduced list of sublists (weights = sublist length, and number of
//    even-indexed elements) is ranked recursively the same way; when it has
//    at most kPjCap elements one CTA finishes it with pointer jumping in
//    shared memory, then the prefixes are pushed back down level by level.
//
// The "dual" mode also counts even-indexed elements: in the bracket layout
// of a rooted tree (2v = entering v, 2v+1 = leaving v) that count is the
// preorder number, so preorder comes straight out of the ranking without a
// scatter + scan over the tour. In dual mode a successor with the top bit
// set (and not -1) marks a contracted leaf: element 2v of a leaf v stands for
// both of its brackets (weight 2), the low 31 bits are the successor of 2v+1,
// and 2v+1 itself is off the list.
#include <cstdio>
#include <mutex>

#include "etl_internal.cuh"

namespace etl {
namespace {

constexpr int32_t kLcap = 4096;    // longest walk before a dynamic splitter is opened (< 2^16 - 2)
constexpr int kPjCap = 8192;       // top level solved by one CTA in shared memory
constexpr int kPjThreads = 1024;
constexpr int kPjItems = kPjCap / kPjThreads;
constexpr uint32_t kMul = 0x9E3779B1u;  // odd, so multiplication is a bijection mod 2^b

struct Hash {
    uint32_t M, Minv, mask, S0;
    __device__ __forceinline__ bool split(uint32_t e) const { return ((e * M) & mask) < S0; }
    __device__ __forceinline__ int32_t sid(uint32_t e) const { return int32_t((e * M) & mask); }
    __device__ __forceinline__ uint32_t elem(uint32_t s) const { return (s * Minv) & mask; }
};

uint32_t inverse_mod_2_32(uint32_t a) {  // Newton iteration for a^-1 mod 2^32 (a odd)
    uint32_t x = a;
    for (int i = 0; i < 5; ++i) x *= 2u - a * x;
    return x;
}

Hash make_hash(int64_t cap, int k_log2) {
    int b = ceil_log2(uint64_t(cap > 1 ? cap : 1));
    if (b < k_log2) b = k_log2;
    Hash h;
    h.M = kMul;
    h.Minv = inverse_mod_2_32(kMul);
    h.mask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
    h.S0 = 1u << (b - k_log2);
    return h;
}

__device__ __forceinline__ int64_t level_len(int64_t base, const int32_t *d_add, int64_t cap) {
    int64_t l = base + (d_add ? int64_t(*d_add) : 0);
    return l < cap ? l : cap;
}

// ------------------------------------------------------------ level-0 walk

template <bool DUAL>
__global__ void k_walk0(const int32_t *__restrict__ succ, int64_t len, const int32_t *__restrict__ d_head, Hash H,
                        uint2 *__restrict__ packed, int32_t *__restrict__ rnext, int32_t *__restrict__ rw1,
                        int32_t *__restrict__ rw2, int32_t *__restrict__ ctr, int32_t dyn_cap,
                        int32_t *__restrict__ next_head, int32_t *__restrict__ status) {
    pdl_prologue();
    const int32_t head = *d_head;
    const bool head_split = H.split(uint32_t(head));
    if (blockIdx.x == 0 && threadIdx.x == 0) *next_head = head_split ? H.sid(uint32_t(head)) : int32_t(H.S0);
    const int64_t nwork = int64_t(H.S0) + 1;
    const int lane = threadIdx.x & 31;
    int32_t cur = 0, sid = 0;
    uint32_t lr = 0, lo = 0;
    int64_t steps = 0;
    bool active = false, exhausted = false;
    while (true) {
        unsigned idle = __ballot_sync(kFull, !active);
        if (idle && !exhausted) {
            const int leader = __ffs(idle) - 1;
            int32_t base = 0;
            if (lane == leader) base = atomicAdd(&ctr[0], __popc(idle));
            base = __shfl_sync(kFull, base, leader);
            if (int64_t(base) + __popc(idle) >= nwork) exhausted = true;
            if (!active) {
                const int64_t w = int64_t(base) + __popc(idle & lanemask_lt());
                if (w < nwork) {
                    int64_t e;
                    if (w < H.S0) {
                        e = H.elem(uint32_t(w));
                    } else {
                        e = head_split ? len : head;  // the head gets its own sublist unless it is a splitter
                    }
                    if (e >= len) {  // hole: no element behind this sublist id
                        rnext[w] = ETL_END;
                        rw1[w] = 0;
                        rw2[w] = 0;
                    } else {
                        cur = int32_t(e);
                        sid = int32_t(w);
                        lr = lo = 0;
                        steps = 0;
                        active = true;
                    }
                }
            }
        }
        if (__ballot_sync(kFull, active) == 0) {
            if (exhausted) break;
            continue;
        }
        if (active) {
            packed[cur] = make_uint2(uint32_t(sid), lr | (lo << 16));
            int32_t nxt = __ldg(succ + cur);
            lr += 1;
            if (DUAL) {
                lo += (cur & 1) == 0 ? 1u : 0u;
                if (nxt < ETL_END) {  // contracted leaf: its closing bracket follows at once
                    nxt &= 0x7fffffff;
                    lr += 1;
                }
            }
            ++steps;
            const bool bad = nxt >= len || nxt < ETL_END || steps > len;
            if (nxt == ETL_END || bad || H.split(uint32_t(nxt))) {
                if (bad) set_status(status, ETL_EBADTREE);
                rnext[sid] = (nxt == ETL_END || bad) ? ETL_END : H.sid(uint32_t(nxt));
                rw1[sid] = int32_t(lr);
                rw2[sid] = int32_t(lo);
                active = false;
            } else if (lr >= uint32_t(kLcap)) {
                const int32_t d = atomicAdd(&ctr[1], 1);
                if (d >= dyn_cap) {
                    set_status(status, ETL_ETIMEOUT);
                    rnext[sid] = ETL_END;
                    rw1[sid] = int32_t(lr);
                    rw2[sid] = int32_t(lo);
                    active = false;
                } else {
                    const int32_t ns = int32_t(H.S0) + 1 + d;
                    rnext[sid] = ns;
                    rw1[sid] = int32_t(lr);
                    rw2[sid] = int32_t(lo);
                    sid = ns;
                    lr = lo = 0;
                    cur = nxt;
                }
            } else {
                cur = nxt;
            }
        }
    }
}

// ------------------------------------------------------------ upper-level walk (explicit weights)

__global__ void k_walk(const int32_t *__restrict__ succ, const int32_t *__restrict__ w1in,
                       const int32_t *__restrict__ w2in, int64_t len_base, const int32_t *__restrict__ d_len_add,
                       int64_t cap, const int32_t *__restrict__ d_head, Hash H, int4 *__restrict__ loc,
                       int32_t *__restrict__ rnext, int32_t *__restrict__ rw1, int32_t *__restrict__ rw2,
                       int32_t *__restrict__ ctr, int32_t dyn_cap, int32_t *__restrict__ next_head,
                       int32_t *__restrict__ status) {
    pdl_prologue();
    const int64_t len = level_len(len_base, d_len_add, cap);
    const int32_t head = *d_head;
    const bool head_split = H.split(uint32_t(head));
    if (blockIdx.x == 0 && threadIdx.x == 0) *next_head = head_split ? H.sid(uint32_t(head)) : int32_t(H.S0);
    const int64_t nwork = int64_t(H.S0) + 1;
    const int lane = threadIdx.x & 31;
    int32_t cur = 0, sid = 0, a1 = 0, a2 = 0, lr = 0;
    int64_t steps = 0;
    bool active = false, exhausted = false;
    while (true) {
        unsigned idle = __ballot_sync(kFull, !active);
        if (idle && !exhausted) {
            const int leader = __ffs(idle) - 1;
            int32_t base = 0;
            if (lane == leader) base = atomicAdd(&ctr[0], __popc(idle));
            base = __shfl_sync(kFull, base, leader);
            if (int64_t(base) + __popc(idle) >= nwork) exhausted = true;
            if (!active) {
                const int64_t w = int64_t(base) + __popc(idle & lanemask_lt());
                if (w < nwork) {
                    int64_t e = (w < H.S0) ? int64_t(H.elem(uint32_t(w))) : (head_split ? len : head);
                    if (e >= len) {
                        rnext[w] = ETL_END;
                        rw1[w] = 0;
                        rw2[w] = 0;
                    } else {
                        cur = int32_t(e);
                        sid = int32_t(w);
                        a1 = a2 = lr = 0;
                        steps = 0;
                        active = true;
                    }
                }
            }
        }
        if (__ballot_sync(kFull, active) == 0) {
            if (exhausted) break;
            continue;
        }
        if (active) {
            loc[cur] = make_int4(sid, a1, a2, 0);
            a1 += w1in[cur];
            a2 += w2in[cur];
            ++lr;
            const int32_t nxt = succ[cur];
            ++steps;
            const bool bad = nxt >= len || nxt < ETL_END || steps > len;
            if (nxt == ETL_END || bad || H.split(uint32_t(nxt))) {
                if (bad) set_status(status, ETL_EBADTREE);
                rnext[sid] = (nxt == ETL_END || bad) ? ETL_END : H.sid(uint32_t(nxt));
                rw1[sid] = a1;
                rw2[sid] = a2;
                active = false;
            } else if (lr >= kLcap) {
                const int32_t d = atomicAdd(&ctr[1], 1);
                if (d >= dyn_cap) {
                    set_status(status, ETL_ETIMEOUT);
                    rnext[sid] = ETL_END;
                    rw1[sid] = a1;
                    rw2[sid] = a2;
                    active = false;
                } else {
                    const int32_t ns = int32_t(H.S0) + 1 + d;
                    rnext[sid] = ns;
                    rw1[sid] = a1;
                    rw2[sid] = a2;
                    sid = ns;
                    a1 = a2 = lr = 0;
                    cur = nxt;
                }
            } else {
                cur = nxt;
            }
        }
    }
}

// ------------------------------------------------------------ top level: pointer jumping in smem

// Q = predecessor pointer, V1/V2 = sums over the segment (Q, e], F = first
// element of that segment. A round replaces Q by Q[Q] and adds the
// predecessor segment; after ceil(log2 len) rounds every Q is -1 and V is the
// inclusive prefix from the list head, F the head itself.
__global__ void __launch_bounds__(kPjThreads)
    k_pointer_jump(const int32_t *__restrict__ succ, const int32_t *__restrict__ w1, const int32_t *__restrict__ w2,
                   int64_t len_base, const int32_t *__restrict__ d_len_add, int64_t cap,
                   const int32_t *__restrict__ d_head, int64_t expect_total, int32_t *__restrict__ R,
                   int32_t *__restrict__ O, int32_t *__restrict__ status) {
    pdl_prologue();
    extern __shared__ int32_t sm[];
    int32_t *Q = sm, *V1 = sm + kPjCap, *V2 = sm + 2 * kPjCap, *F = sm + 3 * kPjCap;
    __shared__ int found;
    const int len = int(level_len(len_base, d_len_add, cap));
    const int32_t head = *d_head;
    if (threadIdx.x == 0) found = 0;
    for (int e = threadIdx.x; e < len; e += kPjThreads) Q[e] = -1;
    __syncthreads();
    for (int e = threadIdx.x; e < len; e += kPjThreads) {
        const int32_t s = succ[e];
        if (s >= 0 && s < len) Q[s] = e;
        V1[e] = w1[e];
        V2[e] = w2[e];
        F[e] = e;
    }
    __syncthreads();
    int rounds = 0;
    while (true) {
        int32_t nq[kPjItems], n1[kPjItems], n2[kPjItems], nf[kPjItems];
        int any = 0;
#pragma unroll
        for (int k = 0; k < kPjItems; ++k) {
            const int e = threadIdx.x + k * kPjThreads;
            if (e < len) {
                const int32_t q = Q[e];
                if (q >= 0) {
                    nq[k] = Q[q];
                    n1[k] = V1[e] + V1[q];
                    n2[k] = V2[e] + V2[q];
                    nf[k] = F[q];
                    any = 1;
                } else {
                    nq[k] = -1;
                    n1[k] = V1[e];
                    n2[k] = V2[e];
                    nf[k] = F[e];
                }
            }
        }
        any = __syncthreads_or(any);
        if (!any) break;
        if (++rounds > 40) {  // cannot happen on a valid list of <= 2^31 elements
            if (threadIdx.x == 0) set_status(status, ETL_EBADTREE);
            break;
        }
#pragma unroll
        for (int k = 0; k < kPjItems; ++k) {
            const int e = threadIdx.x + k * kPjThreads;
            if (e < len) {
                Q[e] = nq[k];
                V1[e] = n1[k];
                V2[e] = n2[k];
                F[e] = nf[k];
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < len; e += kPjThreads) {
        R[e] = V1[e] - w1[e];
        O[e] = V2[e] - w2[e];
        if (expect_total >= 0 && succ[e] == ETL_END && F[e] == head && int64_t(V1[e]) == expect_total) found = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && expect_total >= 0 && !found) set_status(status, ETL_EBADTREE);
}

__global__ void k_expand(const int4 *__restrict__ loc, int64_t len_base, const int32_t *__restrict__ d_len_add,
                         int64_t cap, int64_t up_cap, const int32_t *__restrict__ Rup,
                         const int32_t *__restrict__ Oup, int32_t *__restrict__ R, int32_t *__restrict__ O) {
    pdl_prologue();
    const int64_t len = level_len(len_base, d_len_add, cap);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x) {
        const int4 l = loc[e];
        if (l.x >= 0 && l.x < up_cap) {  // elements off every list keep whatever was there
            R[e] = Rup[l.x] + l.y;
            O[e] = Oup[l.x] + l.z;
        }
    }
}

__global__ void k_set_i32(int32_t *p, int32_t v) {
    pdl_prologue();
    *p = v;
}

__global__ void k_final_rank(const uint2 *__restrict__ packed, int64_t len, const int32_t *__restrict__ R,
                             int64_t rcap, int32_t *__restrict__ rank) {
    pdl_prologue();
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < len; e += int64_t(gridDim.x) * blockDim.x) {
        const uint2 p = packed[e];
        rank[e] = p.x < rcap ? R[p.x] + int32_t(p.y & 0xffffu) : -1;
    }
}

}  // namespace

RankParams &rank_params() {
    static RankParams p;
    return p;
}

// Walks of a list whose successors and records (12 bytes per element) fit in about three quarters of
// the 129 MB L2 run with every SM full of walkers; on longer lists P.blocks_per_sm blocks per SM: with
// fewer random sectors in flight fewer are evicted before their reuse (measured on 2^25-element tours:
// 19% less DRAM traffic, and faster, with 512 walkers per SM than with 2048).
constexpr int64_t kWalkL2Bytes = int64_t(96) << 20;

// Level-0 splitter density (log2 of elements per splitter). A list longer than 2^22 elements takes
// the tuned value (P.k0_log2): its walks are bound by DRAM traffic, which sparser splitters reduce.
// A shorter list sits in L2 and its walk is bound by the latency of its longest sublist (about
// 2^k * ln(len / 2^k) dependent steps), so it takes denser splitters: one in 4 up to 2^15 elements,
// one in 8 up to 2^20, one in 16 up to 2^22, or the tuned value if that is denser (measured on
// random recursive trees of 2^11 .. 2^22 nodes and on forest tours of 2^12 .. 2^22-node graphs).
int level0_density(int64_t len, const RankParams &P) {
    if (len > (int64_t(1) << 22)) return P.k0_log2;
    const int k = len > (int64_t(1) << 20) ? 4 : len > (int64_t(1) << 15) ? 3 : 2;
    return k < P.k0_log2 ? k : P.k0_log2;
}

// ... and never more walkers than sublists: on a short list the surplus warps would only contend for
// the work counter before finding nothing to walk
int walk_grid(int64_t len, int64_t bytes_per_elem, int64_t sublists, const RankParams &P) {
    const int per_sm = len * bytes_per_elem > kWalkL2Bytes ? P.blocks_per_sm : 2048 / P.block;
    const int64_t grid = int64_t(num_sms()) * (per_sm > 0 ? per_sm : 1);
    const int64_t need = ceil_div(sublists, P.block);
    return int(need < grid ? (need > 0 ? need : 1) : grid);
}

etl_status list_rank(const int32_t *succ, int64_t n_cap, const int32_t *d_len, const int32_t *d_head, bool dual,
                     int64_t expect_len, int32_t *status, Workspace &ws, RankResult *out) {
    (void)d_len;  // level 0 always spans the whole array; inert slots carry succ = -1
    cudaStream_t s = ws.stream();
    const RankParams &P = rank_params();
    cudaFuncSetAttribute(k_pointer_jump, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kPjCap * 4);

    // ---- level 0: implicit weights, packed 16-bit local offsets
    const int64_t len0 = n_cap;
    Hash H = make_hash(len0, level0_density(len0, P));
    int32_t dyn_cap = int32_t(len0 / kLcap + 2);
    int64_t cap1 = int64_t(H.S0) + 1 + dyn_cap;
    uint2 *packed = ws.get<uint2>(len0);
    int32_t *rnext = ws.get<int32_t>(cap1), *rw1 = ws.get<int32_t>(cap1), *rw2 = ws.get<int32_t>(cap1);
    int32_t *ctr = ws.get<int32_t>(2);
    int32_t *head1 = ws.get<int32_t>(1);
    if (!ws.ok()) return ETL_ENOMEM;
    memset_async(ctr, 0, 2 * sizeof(int32_t), s);
    etl_status st;
    {
        PhaseTimer pt0("rank.walk0", s);
        const int grid = walk_grid(len0, 12, int64_t(H.S0) + 1, P);
        if (dual)
            launch(k_walk0<true>, grid, P.block, 0, s, succ, len0, d_head, H, packed, rnext, rw1, rw2, ctr, dyn_cap,
                   head1, status);
        else
            launch(k_walk0<false>, grid, P.block, 0, s, succ, len0, d_head, H, packed, rnext, rw1, rw2, ctr, dyn_cap,
                   head1, status);
        note_launch();
        st = last_launch();
    }
    if (st) return st;

    struct Level {
        const int32_t *succ, *w1, *w2;
        int64_t base, cap;
        const int32_t *d_add, *d_head;
        int4 *loc;
        int32_t *R, *O;
    };
    std::vector<Level> lv;
    lv.push_back(Level{rnext, rw1, rw2, int64_t(H.S0) + 1, cap1, ctr + 1, head1, nullptr, nullptr, nullptr});

    // ---- upper levels until one CTA can finish the reduced list
    while (lv.back().cap > kPjCap) {
        Level &L = lv.back();
        Hash h = make_hash(L.cap, P.k_log2);
        int32_t dcap = int32_t(L.cap / kLcap + 2);
        int64_t ncap = int64_t(h.S0) + 1 + dcap;
        L.loc = ws.get<int4>(L.cap);
        int32_t *nn = ws.get<int32_t>(ncap), *n1 = ws.get<int32_t>(ncap), *n2 = ws.get<int32_t>(ncap);
        int32_t *c = ws.get<int32_t>(2), *hd = ws.get<int32_t>(1);
        if (!ws.ok()) return ETL_ENOMEM;
        memset_async(c, 0, 2 * sizeof(int32_t), s);
        memset_async(L.loc, 0xff, size_t(L.cap) * sizeof(int4), s);
        {
            PhaseTimer ptw("rank.walk", s);
            const int grid = walk_grid(L.cap, 28, int64_t(h.S0) + 1, P);
            launch(k_walk, grid, P.block, 0, s, L.succ, L.w1, L.w2, L.base, L.d_add, L.cap, L.d_head, h, L.loc, nn, n1,
                   n2, c, dcap, hd, status);
        note_launch();
            st = last_launch();
        }
        if (st) return st;
        lv.push_back(Level{nn, n1, n2, int64_t(h.S0) + 1, ncap, c + 1, hd, nullptr, nullptr, nullptr});
    }

    // ---- top
    {
        Level &T = lv.back();
        T.R = ws.get<int32_t>(T.cap);
        T.O = ws.get<int32_t>(T.cap);
        if (!ws.ok()) return ETL_ENOMEM;
        PhaseTimer ptp("rank.pj", s);
        launch(k_pointer_jump, 1, kPjThreads, 4 * kPjCap * 4, s, T.succ, T.w1, T.w2, T.base, T.d_add, T.cap, T.d_head,
               expect_len, T.R, T.O, status);
        note_launch();
        st = last_launch();
        if (st) return st;
    }
    // ---- push prefixes back down
    for (int i = int(lv.size()) - 2; i >= 0; --i) {
        Level &L = lv[i];
        L.R = ws.get<int32_t>(L.cap);
        L.O = ws.get<int32_t>(L.cap);
        if (!ws.ok()) return ETL_ENOMEM;
        int blocks = int(ceil_div(L.cap, 256));
        if (blocks > num_sms() * 32) blocks = num_sms() * 32;  // four waves of full occupancy
        PhaseTimer pte("rank.expand", s);
        launch(k_expand, blocks, 256, 0, s, L.loc, L.base, L.d_add, L.cap, lv[i + 1].cap, lv[i + 1].R, lv[i + 1].O, L.R,
               L.O);
        note_launch();
        st = last_launch();
        if (st) return st;
    }
    out->packed = packed;
    out->R = lv[0].R;
    out->O = lv[0].O;
    out->rcap = lv[0].cap;
    return ETL_OK;
}

etl_status set_device_i32(int32_t *p, int32_t v, cudaStream_t s) {
    launch(k_set_i32, 1, 1, 0, s, p, v);
        note_launch();
    return last_launch();
}

etl_status final_rank(const RankResult &r, int64_t len, int32_t *rank, cudaStream_t s) {
    int blocks = int(ceil_div(len, 256));
    const int cap = num_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    PhaseTimer pt("rank.final", s);
    launch(k_final_rank, blocks, 256, 0, s, r.packed, len, r.R, r.rcap, rank);
        note_launch();
    return last_launch();
}

}  // namespace etl

// ------------------------------------------------------------------ list ranking without allocation
//
// etl_list_rank_static: the same ranking as etl_list_rank, but every byte of
// scratch it needs comes from one fixed array of device memory that the
// library reserves when it is loaded, so the call itself never allocates.
// It exists for callers that cannot allocate device memory at the point of
// the call: code that runs under an external memory manager that owns the
// whole device (so a cudaMalloc would fail or fragment its arena), code that
// must not block on the allocator's implicit synchronisation, and code with a
// fixed, pre-planned memory budget. Such callers still pass their own input
// and output arrays.
//
// Limits and rules (also in etl.h):
//  * len <= kStaticMaxLen (2^18 elements); larger lists are rejected with
//    ETL_EINVAL before anything is enqueued.
//  * The scratch array (kStaticBytes, 3 MiB) is a file-scope __device__
//    variable: every GPU on which the library is loaded holds it until the
//    process exits.
//  * All calls share it and it keeps the previous call's contents; the
//    counters that must start at zero are cleared by each call. Two calls
//    whose work overlaps on the GPU (different streams, or different host
//    threads) race on the same scratch and give wrong ranks: serialise them.
//  * The host cannot use the array's name as a device address, so the first
//    call on each device looks the address up with cudaGetSymbolAddress (with
//    that device current) and caches it with the id of the CUDA context it
//    belongs to; that first call should therefore come before any stream
//    capture on that device. When the context changes (cudaDeviceReset, or
//    the primary context destroyed and made again), the next call sees the
//    new context id and repeats the look-up instead of using a stale address.
namespace etl {
namespace {

constexpr int64_t kStaticMaxLen = int64_t(1) << 18;
constexpr size_t kStaticBytes = size_t(3) << 20;
constexpr int kStaticK0 = 4, kStaticK = 4;  // fixed splitter densities, so the layout is fixed

static __device__ __align__(256) unsigned char g_rank_scratch[kStaticBytes];

struct StaticArena {
    char *base;
    size_t used, cap;
    template <class T>
    T *take(int64_t count) {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = size_t(count > 0 ? count : 1) * sizeof(T);
        if (off + bytes > cap) return nullptr;
        used = off + bytes;
        return reinterpret_cast<T *>(base + off);
    }
};

std::mutex g_static_mu;
void *g_static_addr[64] = {nullptr};
unsigned long long g_static_ctx[64] = {0};

// The driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime (no link against libcuda).
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_ctx_fns_once;

// id of the calling thread's current CUDA context (unique over the process's lifetime); false when
// there is no current context or the driver entry points are unavailable
bool current_context_id(unsigned long long *id) {
    std::call_once(g_ctx_fns_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return false;
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return false;
    return g_ctx_get_id(ctx, id) == 0;
}

// with the device current: the device address of the scratch array, looked up once per device and
// context (and again after the context changed)
etl_status static_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ETL_ECUDA;
    std::lock_guard<std::mutex> g(g_static_mu);
    // without the driver's context ids (entry points not found) the address is cached per device only
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (!g_static_addr[dev] || (have_id && g_static_ctx[dev] != id)) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_rank_scratch) != cudaSuccess || !p) return ETL_ECUDA;
        if (cudaFuncSetAttribute(k_pointer_jump, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kPjCap * 4) !=
            cudaSuccess)
            return ETL_ECUDA;
        // the look-up made the device's primary context current if it was not yet
        g_static_ctx[dev] = current_context_id(&id) ? id : 0;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return ETL_OK;
}

}  // namespace
}  // namespace etl

extern "C" etl_status etl_list_rank_static(const int32_t *succ, int64_t len, int32_t head, int32_t *rank,
                                           int32_t *status, void *stream) {
    using namespace etl;
    if (!succ || !rank || len < 1 || head < 0 || head >= len) return ETL_EINVAL;
    if (len > kStaticMaxLen) return ETL_EINVAL;  // beyond the fixed scratch: documented limit
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    etl_status rc = static_scratch(&scratch);
    if (rc) return rc;
    StaticArena A{static_cast<char *>(scratch), 0, kStaticBytes};
    const int grid = num_sms() * 8;
    const int block = 256;

    int32_t *word = A.take<int32_t>(4);  // [0] head, [1] status when the caller passes none
    int32_t *st = status ? status : word + 1;
    Hash H = make_hash(len, kStaticK0);
    const int32_t dyn_cap = int32_t(len / kLcap + 2);
    const int64_t cap1 = int64_t(H.S0) + 1 + dyn_cap;
    uint2 *packed = A.take<uint2>(len);
    int32_t *rnext = A.take<int32_t>(cap1), *rw1 = A.take<int32_t>(cap1), *rw2 = A.take<int32_t>(cap1);
    int32_t *ctr = A.take<int32_t>(2), *head1 = A.take<int32_t>(1);
    if (!word || !packed || !rnext || !rw1 || !rw2 || !ctr || !head1) return ETL_ENOMEM;

    if (!status && cudaMemsetAsync(st, 0, sizeof(int32_t), s) != cudaSuccess) return ETL_ECUDA;
    if (cudaMemsetAsync(ctr, 0, 2 * sizeof(int32_t), s) != cudaSuccess) return ETL_ECUDA;
    launch(k_set_i32, 1, 1, 0, s, word, head);
    note_launch();
    launch(k_walk0<false>, grid, block, 0, s, succ, len, word, H, packed, rnext, rw1, rw2, ctr, dyn_cap, head1, st);
    note_launch();
    if ((rc = last_launch())) return rc;

    struct Level {
        const int32_t *succ, *w1, *w2;
        int64_t base, cap;
        const int32_t *d_add, *d_head;
        int4 *loc;
        int32_t *R, *O;
    };
    Level lv[8];
    int nl = 0;
    lv[nl++] = Level{rnext, rw1, rw2, int64_t(H.S0) + 1, cap1, ctr + 1, head1, nullptr, nullptr, nullptr};
    while (lv[nl - 1].cap > kPjCap) {
        if (nl >= 8) return ETL_ENOMEM;
        Level &L = lv[nl - 1];
        Hash h = make_hash(L.cap, kStaticK);
        const int32_t dcap = int32_t(L.cap / kLcap + 2);
        const int64_t ncap = int64_t(h.S0) + 1 + dcap;
        L.loc = A.take<int4>(L.cap);
        int32_t *nn = A.take<int32_t>(ncap), *n1 = A.take<int32_t>(ncap), *n2 = A.take<int32_t>(ncap);
        int32_t *c = A.take<int32_t>(2), *hd = A.take<int32_t>(1);
        if (!L.loc || !nn || !n1 || !n2 || !c || !hd) return ETL_ENOMEM;
        if (cudaMemsetAsync(c, 0, 2 * sizeof(int32_t), s) != cudaSuccess) return ETL_ECUDA;
        if (cudaMemsetAsync(L.loc, 0xff, size_t(L.cap) * sizeof(int4), s) != cudaSuccess) return ETL_ECUDA;
        launch(k_walk, grid, block, 0, s, L.succ, L.w1, L.w2, L.base, L.d_add, L.cap, L.d_head, h, L.loc, nn, n1, n2, c,
               dcap, hd, st);
        note_launch();
        if ((rc = last_launch())) return rc;
        lv[nl++] = Level{nn, n1, n2, int64_t(h.S0) + 1, ncap, c + 1, hd, nullptr, nullptr, nullptr};
    }
    Level &T = lv[nl - 1];
    T.R = A.take<int32_t>(T.cap);
    T.O = A.take<int32_t>(T.cap);
    if (!T.R || !T.O) return ETL_ENOMEM;
    launch(k_pointer_jump, 1, kPjThreads, 4 * kPjCap * 4, s, T.succ, T.w1, T.w2, T.base, T.d_add, T.cap, T.d_head, len,
           T.R, T.O, st);
    note_launch();
    if ((rc = last_launch())) return rc;
    for (int i = nl - 2; i >= 0; --i) {
        Level &L = lv[i];
        L.R = A.take<int32_t>(L.cap);
        L.O = A.take<int32_t>(L.cap);
        if (!L.R || !L.O) return ETL_ENOMEM;
        int blocks = int(ceil_div(L.cap, 256));
        if (blocks > grid * 4) blocks = grid * 4;
        launch(k_expand, blocks, 256, 0, s, L.loc, L.base, L.d_add, L.cap, lv[i + 1].cap, lv[i + 1].R, lv[i + 1].O, L.R,
               L.O);
        note_launch();
        if ((rc = last_launch())) return rc;
    }
    int blocks = int(ceil_div(len, 256));
    if (blocks > num_sms() * 16) blocks = num_sms() * 16;
    launch(k_final_rank, blocks, 256, 0, s, packed, len, lv[0].R, lv[0].cap, rank);
    note_launch();
    return last_launch();
}
