// Stable LSD radix sort of (key, value) int32 pairs, 8 bits per pass.
//
// Used to group the arcs of a tree by their source node: children by parent
// for a parent array, half-edges by tail for a spanning forest. This replaces
// the lexicographic sort of array A into B in the DCEL construction of
// Sec. 2.1: only the grouping by source is needed, and a stable sort keeps
// each group in ascending value order.
//
// One pass = per-tile digit histograms -> exclusive scan over (digit, tile) ->
// stable scatter. Inside a tile each warp ranks its 32-element rounds (peers
// with the same digit by __match_any_sync or by eight ballots) with per-warp
// smem counters, so the order of equal digits is preserved without any atomics
// on global memory; the ranked tile is staged in shared memory in digit order
// and written out in runs.
#include "etl_internal.cuh"

namespace etl {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / kWarp;
constexpr int kRadix = 256;
static_assert(kThreads == kRadix, "the scatter handles one digit per thread");
// R = 32-element rounds per warp: a tile of 8 warps holds 256 * R elements (R = 8 or 16, chosen by
// the SORT_ROUNDS tuning knob; larger tiles give longer runs per digit in the scatter)

__device__ __forceinline__ int64_t count_of(const int32_t *d_count, int64_t n_cap) {
    if (!d_count) return n_cap;
    int64_t c = *d_count;
    return c < 0 ? 0 : (c < n_cap ? c : n_cap);
}

// keys of the input: a plain array (first pass) or the .x of (key, value) pairs (later passes)
__device__ __forceinline__ int32_t key_at(const int32_t *keys, const int2 *kv, int64_t i) {
    return kv ? kv[i].x : keys[i];
}

template <int R>
__global__ void __launch_bounds__(kThreads)
    k_hist(const int32_t *__restrict__ keys, const int2 *__restrict__ kv, const int32_t *d_count, int64_t n_cap,
           int shift, int32_t key_limit, int32_t *__restrict__ ghist, int nblocks) {
    pdl_prologue();
    constexpr int kRounds = R, kWarpTile = kWarp * R, kTile = kWarps * kWarpTile;
    __shared__ int32_t h[kRadix];
    const int64_t count = count_of(d_count, n_cap);
    if (int64_t(blockIdx.x) * kTile >= count) {  // tile past the data: an all-zero histogram
        for (int d = threadIdx.x; d < kRadix; d += kThreads) ghist[int64_t(d) * nblocks + blockIdx.x] = 0;
        return;
    }
    for (int d = threadIdx.x; d < kRadix; d += kThreads) h[d] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kTile + warp * kWarpTile;
    int32_t key[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {  // loads first, all in flight together
        const int64_t idx = base + r * kWarp + lane;
        key[r] = idx < count ? key_at(keys, kv, idx) : -1;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int32_t k = key[r];
        if (k >= 0 && k < key_limit) atomicAdd(&h[(k >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kThreads) ghist[int64_t(d) * nblocks + blockIdx.x] = h[d];
}

// lanes of the warp whose 8-bit digit equals this lane's, among the valid lanes (an invalid lane
// matches itself only): __match_any_sync, or eight ballots on the digit's bits
template <bool BALLOT>
__device__ __forceinline__ unsigned digit_peers(int d, bool valid, int lane) {
    if (!BALLOT) return __match_any_sync(kFull, valid ? d : kRadix + lane);
    unsigned peers = __ballot_sync(kFull, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1;
        const unsigned m = __ballot_sync(kFull, bit);
        peers &= bit ? m : ~m;
    }
    return valid ? peers : (1u << lane);
}

// The tile's elements are first placed in shared memory in digit order (stable: by digit, then by
// position in the tile), then written out by consecutive threads: equal digits form one run of the
// output, so a warp's store touches a few runs instead of one segment per lane.
template <int R, bool BALLOT>
__global__ void __launch_bounds__(kThreads)
    k_scatter(const int32_t *__restrict__ keys, const int32_t *__restrict__ vals, const int2 *__restrict__ kv,
              const int32_t *d_count, int64_t n_cap, int shift, int32_t key_limit, const int32_t *__restrict__ goff,
              int nblocks, int2 *__restrict__ kv_out) {
    pdl_prologue();
    constexpr int kRounds = R, kWarpTile = kWarp * R, kTile = kWarps * kWarpTile;
    __shared__ int32_t wcnt[kWarps][kRadix];
    __shared__ int32_t gbase[kRadix];
    __shared__ int32_t dstart[kRadix];  // first tile position of each digit (digit order)
    __shared__ int32_t wtot[kWarps];
    __shared__ int2 stage[kTile];
    const int64_t count = count_of(d_count, n_cap);
    if (int64_t(blockIdx.x) * kTile >= count) return;  // nothing of this tile to place
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kTile + warp * kWarpTile;
    int32_t key[kRounds], val[kRounds], dig[kRounds], lrank[kRounds];
    // all loads of the tile first, so that they are in flight together (the ranking rounds below
    // are ordered by __syncwarp and would otherwise wait for one load each)
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int64_t idx = base + r * kWarp + lane;
        key[r] = -1;
        val[r] = 0;
        if (idx < count) {
            if (kv) {
                const int2 x = __ldcs(kv + idx);
                key[r] = x.x;
                val[r] = x.y;
            } else {
                key[r] = __ldcs(keys + idx);
                val[r] = vals ? __ldcs(vals + idx) : int32_t(idx);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const int32_t k = key[r];
        const bool valid = k >= 0 && k < key_limit;  // also false past the end (k = -1)
        const int d = valid ? ((k >> shift) & (kRadix - 1)) : 0;
        const unsigned peers = digit_peers<BALLOT>(d, valid, lane);
        int pre = 0;
        if (valid) pre = wcnt[warp][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = pre + __popc(peers);
        __syncwarp();
        dig[r] = valid ? d : -1;
        lrank[r] = pre + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // per digit (one per thread): counts of the warps -> exclusive offsets across warps, and the
    // digit's total; then the digits' totals -> exclusive offsets across digits (block scan)
    const int d = threadIdx.x;  // kThreads == kRadix
    int32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const int32_t t = wcnt[w][d];
        wcnt[w][d] = run;
        run += t;
    }
    gbase[d] = goff[int64_t(d) * nblocks + blockIdx.x];
    int32_t inc = run;  // inclusive scan of the digits' totals: warp scan, then the warps' sums
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == kWarp - 1) wtot[warp] = inc;
    __syncthreads();
    int32_t wofs = 0;
    for (int w = 0; w < warp; ++w) wofs += wtot[w];
    dstart[d] = wofs + inc - run;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r)
        if (dig[r] >= 0) stage[dstart[dig[r]] + wcnt[warp][dig[r]] + lrank[r]] = make_int2(key[r], val[r]);
    __syncthreads();
    int32_t placed = 0;  // elements of the tile with a valid key
#pragma unroll
    for (int w = 0; w < kWarps; ++w) placed += wtot[w];
    for (int i = threadIdx.x; i < placed; i += kThreads) {
        const int2 x = stage[i];
        const int dd = (x.x >> shift) & (kRadix - 1);
        kv_out[gbase[dd] + (i - dstart[dd])] = x;
    }
}

template <int R>
etl_status radix_sort_impl(const int32_t *keys_in, const int32_t *vals_in, const int32_t *d_count, int64_t n_cap,
                           int key_bits, int32_t key_limit, Workspace &ws, SortResult *out) {
    constexpr int kTile = kWarps * kWarp * R;
    cudaStream_t s = ws.stream();
    const int64_t cap = n_cap > 0 ? n_cap : 1;
    const int nblocks = int(ceil_div(cap, kTile));
    const int passes = key_bits <= 8 ? 1 : (key_bits + 7) / 8;
    if (key_bits < 31 && key_limit > (int32_t(1) << key_bits)) key_limit = int32_t(1) << key_bits;
    int2 *buf[2] = {ws.get<int2>(cap), ws.get<int2>(cap)};
    int32_t *ghist = ws.get<int32_t>(int64_t(kRadix) * nblocks);
    if (!ws.ok()) return ETL_ENOMEM;
    const int2 *kvin = nullptr;
    const int32_t *cnt = d_count;
    for (int p = 0; p < passes; ++p) {
        int32_t *goff = ws.get<int32_t>(int64_t(kRadix) * nblocks + 1);
        if (!ws.ok()) return ETL_ENOMEM;
        const int shift = 8 * p;
        etl_status st;
        {
            PhaseTimer pt("sort.hist", s);
            launch(k_hist<R>, nblocks, kThreads, 0, s, keys_in, kvin, cnt, cap, shift, key_limit, ghist, nblocks);
            note_launch();
            st = last_launch();
        }
        if (st) return st;
        st = scan_exclusive_i32(ghist, goff, int64_t(kRadix) * nblocks, ws);
        if (st) return st;
        int2 *out_kv = buf[p & 1];
        {
            PhaseTimer pt("sort.scatter", s);
            if (sort_params().ballot)
                launch(k_scatter<R, true>, nblocks, kThreads, 0, s, keys_in, vals_in, kvin, cnt, cap, shift, key_limit,
                       goff, nblocks, out_kv);
            else
                launch(k_scatter<R, false>, nblocks, kThreads, 0, s, keys_in, vals_in, kvin, cnt, cap, shift, key_limit,
                       goff, nblocks, out_kv);
            note_launch();
            st = last_launch();
        }
        if (st) return st;
        kvin = out_kv;
        cnt = goff + int64_t(kRadix) * nblocks;  // number of kept elements
    }
    out->kv = kvin;
    out->d_total = cnt;
    return ETL_OK;
}

}  // namespace

SortParams &sort_params() {
    static SortParams p;
    return p;
}

etl_status radix_sort_pairs(const int32_t *keys_in, const int32_t *vals_in, const int32_t *d_count, int64_t n_cap,
                            int key_bits, int32_t key_limit, Workspace &ws, SortResult *out) {
    if (sort_params().rounds == 16)
        return radix_sort_impl<16>(keys_in, vals_in, d_count, n_cap, key_bits, key_limit, ws, out);
    return radix_sort_impl<8>(keys_in, vals_in, d_count, n_cap, key_bits, key_limit, ws, out);
}

}  // namespace etl
