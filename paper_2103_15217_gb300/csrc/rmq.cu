// Sparse tables for range-minimum / range-maximum queries (Sec. 3.1 reduces
// LCA to RMQ; Sec. 4.1 aggregates low / high over subtrees by RMQ), full and
// blocked (two-level: in-block prefix / suffix results plus a full table over
// the blocks, declared in etl_internal.cuh).
//
// Full tables:
// Level l holds op over x[i .. i + 2^l). One streaming pass builds up to three
// consecutive levels l, l+1, l+2 from level l-1: with h = 2^(l-1),
//     T_l[i]   = op(p[i], p[i+h])
//     T_l+1[i] = op(p[i], p[i+h], p[i+2h], p[i+3h])
//     T_l+2[i] = op(p[i] .. p[i+7h] in steps of h)
// where p = T_(l-1). Every thread handles four consecutive entries with int4
// loads and stores; shifted operands whose offset is not a multiple of four
// are assembled from two aligned int4 loads. Only the unshifted stream comes
// from DRAM; the shifted ones trail it by at most 7h entries and hit in the
// 129 MB L2 for the sizes used here. Rows are padded to a multiple of four
// entries with the identity.
#include <climits>
#include <type_traits>

#include "etl_internal.cuh"

namespace etl {
namespace {

template <bool IS_MAX>
__device__ __forceinline__ int32_t op(int32_t a, int32_t b) {
    return IS_MAX ? max(a, b) : min(a, b);
}

template <bool IS_MAX>
__device__ __forceinline__ int4 op4(int4 a, int4 b) {
    return make_int4(op<IS_MAX>(a.x, b.x), op<IS_MAX>(a.y, b.y), op<IS_MAX>(a.z, b.z), op<IS_MAX>(a.w, b.w));
}

// elements [4i + s, 4i + s + 4) of a padded row (nv int4 vectors), identity past the end
template <bool IS_MAX>
__device__ __forceinline__ int4 shifted(const int4 *__restrict__ p, int64_t i, int64_t s, int64_t nv) {
    const int32_t id = IS_MAX ? INT_MIN : INT_MAX;
    const int4 I = make_int4(id, id, id, id);
    const int64_t q = i + (s >> 2);
    const int r = int(s & 3);
    const int4 a = q < nv ? p[q] : I;
    if (r == 0) return a;
    const int4 b = q + 1 < nv ? p[q + 1] : I;
    if (r == 1) return make_int4(a.y, a.z, a.w, b.x);
    if (r == 2) return make_int4(a.z, a.w, b.x, b.y);
    return make_int4(a.w, b.x, b.y, b.z);
}

template <bool IS_MAX>
__global__ void __launch_bounds__(1024) k_levels(int32_t *__restrict__ table, int64_t ld, int l, int count) {
    pdl_prologue();
    const int4 *p = reinterpret_cast<const int4 *>(table + int64_t(l - 1) * ld);
    int4 *o0 = reinterpret_cast<int4 *>(table + int64_t(l) * ld);
    int4 *o1 = reinterpret_cast<int4 *>(table + int64_t(l + 1) * ld);
    int4 *o2 = reinterpret_cast<int4 *>(table + int64_t(l + 2) * ld);
    const int64_t nv = ld >> 2, h = int64_t(1) << (l - 1);
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nv; i += int64_t(gridDim.x) * blockDim.x) {
        const int4 m01 = op4<IS_MAX>(p[i], shifted<IS_MAX>(p, i, h, nv));
        o0[i] = m01;
        if (count > 1) {
            const int4 m23 = op4<IS_MAX>(shifted<IS_MAX>(p, i, 2 * h, nv), shifted<IS_MAX>(p, i, 3 * h, nv));
            const int4 m03 = op4<IS_MAX>(m01, m23);
            o1[i] = m03;
            if (count > 2) {
                const int4 m45 = op4<IS_MAX>(shifted<IS_MAX>(p, i, 4 * h, nv), shifted<IS_MAX>(p, i, 5 * h, nv));
                const int4 m67 = op4<IS_MAX>(shifted<IS_MAX>(p, i, 6 * h, nv), shifted<IS_MAX>(p, i, 7 * h, nv));
                o2[i] = op4<IS_MAX>(m03, op4<IS_MAX>(m45, m67));
            }
        }
    }
}

template <bool IS_MAX>
__global__ void k_pad(int32_t *__restrict__ table, int64_t n, int64_t ld) {
    pdl_prologue();
    const int64_t i = n + threadIdx.x;
    if (i < ld) table[i] = IS_MAX ? INT_MIN : INT_MAX;
}

// ---- blocked tables

__device__ __forceinline__ int32_t shfl_up(int32_t v, int d) { return __shfl_up_sync(kFull, v, d); }
__device__ __forceinline__ int2 shfl_up(int2 v, int d) {
    return make_int2(__shfl_up_sync(kFull, v.x, d), __shfl_up_sync(kFull, v.y, d));
}
__device__ __forceinline__ long long shfl_up(long long v, int d) { return __shfl_up_sync(kFull, v, d); }
__device__ __forceinline__ int32_t shfl_down(int32_t v, int d) { return __shfl_down_sync(kFull, v, d); }
__device__ __forceinline__ long long shfl_down(long long v, int d) { return __shfl_down_sync(kFull, v, d); }
__device__ __forceinline__ int2 shfl_down(int2 v, int d) {
    return make_int2(__shfl_down_sync(kFull, v.x, d), __shfl_down_sync(kFull, v.y, d));
}

// one warp per block of 32 entries: prefix and suffix op by shuffles, block result -> top level 0;
// entries in [n, nblk * 32) are set to the identity first. PAIRS (int32 entries only): pm and sm are
// stored interleaved, (pm[i], sm[i]) as one 8-byte pair at position i of the 2N entries after x
template <class Op, bool PAIRS>
__global__ void k_block_scan(typename Op::T *__restrict__ x, int64_t n, int64_t nblk, typename Op::T *__restrict__ pm,
                             typename Op::T *__restrict__ sm, typename Op::T *__restrict__ top0) {
    pdl_prologue();
    using T = typename Op::T;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t b = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5; b < nblk; b += warps) {
        const int64_t i = b * kRmqBlock + lane;
        T v;
        if (i < n) {
            v = x[i];
        } else {
            v = Op::id();
            x[i] = v;
        }
        T p = v, q = v;
#pragma unroll
        for (int d = 1; d < kRmqBlock; d <<= 1) {
            const T up = shfl_up(p, d), dn = shfl_down(q, d);
            if (lane >= d) p = Op::f(p, up);
            if (lane + d < kRmqBlock) q = Op::f(q, dn);
        }
        if constexpr (PAIRS) {
            reinterpret_cast<int2 *>(pm)[i] = make_int2(p, q);
        } else {
            pm[i] = p;
            sm[i] = q;
        }
        if (lane == kRmqBlock - 1) top0[b] = p;
    }
}

// levels l .. l + count - 1 of the top table from level l - 1 (rows nblk apart, count <= 3)
template <class Op>
__global__ void k_top_levels(typename Op::T *__restrict__ top, int64_t nblk, int l, int count) {
    pdl_prologue();
    using T = typename Op::T;
    const T *p = top + int64_t(l - 1) * nblk;
    const int64_t h = int64_t(1) << (l - 1);
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nblk; i += int64_t(gridDim.x) * blockDim.x) {
        T m = Op::f(p[i], i + h < nblk ? p[i + h] : Op::id());
        top[int64_t(l) * nblk + i] = m;
        for (int c = 1; c < count; ++c) {
            const int64_t w = h << c;  // the next level adds the 2^c shifted entries w .. 2w - 1 (steps of h)
            for (int64_t j = w; j < 2 * w; j += h) m = Op::f(m, i + j < nblk ? p[i + j] : Op::id());
            top[int64_t(l + c) * nblk + i] = m;
        }
    }
}

}  // namespace

BlockedLayout blocked_layout(int64_t n, int64_t max_len) {
    BlockedLayout L;
    L.nblk = ceil_div(n < 1 ? 1 : n, kRmqBlock);
    const int64_t span = ceil_div(max_len < 1 ? 1 : max_len, kRmqBlock);  // whole blocks a range may cover, + 1
    L.tlevels = sparse_levels(span < L.nblk ? span : L.nblk);
    return L;
}

template <class Op>
etl_status blocked_build(typename Op::T *base, int64_t n, const BlockedLayout &L, cudaStream_t s, bool pairs) {
    using T = typename Op::T;
    const int64_t N = L.nblk * kRmqBlock;
    T *top = base + 3 * N;
    const int grid_cap = num_sms() * 8;
    {
        PhaseTimer pt("rmq.blocks", s);
        int blocks = int(ceil_div(N, 256));
        if (blocks > grid_cap) blocks = grid_cap;
        bool launched = false;
        if constexpr (std::is_same<T, int32_t>::value) {
            if (pairs) {
                launch(k_block_scan<Op, true>, blocks, 256, 0, s, base, n, L.nblk, base + N, base + 2 * N, top);
                launched = true;
            }
        }
        if (!launched) launch(k_block_scan<Op, false>, blocks, 256, 0, s, base, n, L.nblk, base + N, base + 2 * N, top);
        note_launch();
    }
    etl_status st = last_launch();
    for (int l = 1; !st && l < L.tlevels;) {
        const int count = L.tlevels - l >= 3 ? 3 : L.tlevels - l;
        int blocks = int(ceil_div(L.nblk, 256));
        if (blocks > grid_cap) blocks = grid_cap;
        PhaseTimer pt("rmq.top", s);
        launch(k_top_levels<Op>, blocks, 256, 0, s, top, L.nblk, l, count);
        note_launch();
        st = last_launch();
        l += count;
    }
    return st;
}

template etl_status blocked_build<OpMin>(int32_t *, int64_t, const BlockedLayout &, cudaStream_t, bool);
template etl_status blocked_build<OpMax>(int32_t *, int64_t, const BlockedLayout &, cudaStream_t, bool);
template etl_status blocked_build<OpMinMax>(int2 *, int64_t, const BlockedLayout &, cudaStream_t, bool);
template etl_status blocked_build<OpMinKey>(long long *, int64_t, const BlockedLayout &, cudaStream_t, bool);

RmqParams &rmq_params() {
    static RmqParams p;
    return p;
}

constexpr int64_t kL2ReuseBytes = int64_t(48) << 20;  // share of the 129 MB L2 one sweep may rely on

int64_t sparse_ld(int64_t n) { return (n + 3) & ~int64_t(3); }

int sparse_levels(int64_t max_len) {
    int L = 1;
    while ((int64_t(1) << L) <= max_len) ++L;
    return L;
}

template <bool IS_MAX>
etl_status sparse_table_build(int32_t *table, int64_t n, int levels, cudaStream_t s) {
    const int64_t ld = sparse_ld(n);
    if (ld > n) {
        launch(k_pad<IS_MAX>, 1, 4, 0, s, table, n, ld);
        note_launch();
    }
    const RmqParams &R = rmq_params();
    const int grid_cap = num_sms() * (2048 / R.block);
    for (int l = 1; l < levels;) {
        // fuse c levels only while the 2^c shifted streams stay inside L2: a pass re-reads each
        // entry of level l-1 at offsets up to (2^c - 1) * 2^(l-1), so the reuse window spans
        // about 2^c * (2^c - 1) * 2^(l-1) * 4 bytes of the sweep
        int count = levels - l >= R.levels_per_pass ? R.levels_per_pass : levels - l;
        const int64_t h = int64_t(1) << (l - 1);
        while (count > 1 && (int64_t(1) << count) * ((int64_t(1) << count) - 1) * h * 4 > kL2ReuseBytes) --count;
        int blocks = int(ceil_div(ld / 4, R.block));
        if (blocks > grid_cap) blocks = grid_cap;
        if (blocks < 1) blocks = 1;
        PhaseTimer pt(IS_MAX ? "rmq.level_max" : "rmq.level_min", s);
        launch(k_levels<IS_MAX>, blocks, R.block, 0, s, table, ld, l, count);
        note_launch();
        etl_status st = last_launch();
        if (st) return st;
        l += count;
    }
    return last_launch();
}

template etl_status sparse_table_build<false>(int32_t *, int64_t, int, cudaStream_t);
template etl_status sparse_table_build<true>(int32_t *, int64_t, int, cudaStream_t);

}  // namespace etl
