// Device-wide exclusive prefix sums (reduce-then-scan), used for CSR offsets,
// stream compaction and radix-sort digit offsets. Loads are warp-striped, so
// every warp-wide load touches one contiguous 128-byte line.
#include "etl_internal.cuh"

namespace etl {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096 elements per block
constexpr int kWarps = kThreads / kWarp;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t x, int lane) {
#pragma unroll
    for (int d = 1; d < kWarp; d <<= 1) {
        int32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

template <class T>
__device__ __forceinline__ int64_t eff_len(int64_t n, const int32_t *d_n) {
    if (!d_n) return n;
    int64_t m = *d_n;
    return m < n ? (m < 0 ? 0 : m) : n;
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_reduce(const T *__restrict__ in, int64_t n, const int32_t *d_n,
                                                     int32_t *__restrict__ partial) {
    pdl_prologue();
    __shared__ int32_t wsum[kWarps];
    const int64_t nn = eff_len<T>(n, d_n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kTile + warp * (kWarp * kItems);
    int32_t s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int64_t idx = base + j * kWarp + lane;
        if (idx < nn) s += int32_t(in[idx]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
    if (lane == 0) wsum[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < kWarps; ++w) t += wsum[w];
        partial[blockIdx.x] = t;
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads)
    k_scan_tile(const T *__restrict__ in, int32_t *__restrict__ out, int64_t n, const int32_t *d_n,
                const int32_t *__restrict__ offs, int64_t nblocks) {
    pdl_prologue();
    __shared__ int32_t wsum[kWarps];
    const int64_t nn = eff_len<T>(n, d_n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = int64_t(blockIdx.x) * kTile + warp * (kWarp * kItems);
    int32_t vals[kItems];
    int32_t running = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int64_t idx = base + j * kWarp + lane;
        int32_t x = idx < nn ? int32_t(in[idx]) : 0;
        int32_t inc = warp_incl_scan(x, lane);
        vals[j] = running + inc - x;
        running += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) wsum[warp] = running;
    __syncthreads();
    int32_t woff = offs ? offs[blockIdx.x] : 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int64_t idx = base + j * kWarp + lane;
        if (idx < n) out[idx] = vals[j] + woff;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // total into out[n]
        int32_t total = 0;
        if (offs) {
            total = offs[nblocks];
        } else {
            for (int w = 0; w < kWarps; ++w) total += wsum[w];
        }
        out[n] = total;
    }
}

// A short input (one tile of 16384 entries at most) is scanned by one block of 1024 threads: one
// launch instead of reduce + scan of the partials + scan of the tiles, three launches that each cost a
// few microseconds the work itself does not need (the digit offsets of a radix pass over up to 2^19
// elements, for instance). Longer inputs keep the three launches: a block walking several tiles one
// after another measured slower than them.
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / kWarp;
constexpr int64_t kSmallMax = int64_t(kSmallThreads) * kItems;
static_assert(kSmallWarps == kWarp, "the warp totals are scanned by one warp");

template <class T>
__global__ void __launch_bounds__(kSmallThreads)
    k_scan_small(const T *__restrict__ in, int32_t *__restrict__ out, int64_t n, const int32_t *d_n) {
    pdl_prologue();
    __shared__ int32_t wsum[kSmallWarps], wpre[kSmallWarps];
    __shared__ int32_t total;
    const int64_t nn = eff_len<T>(n, d_n);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = warp * (kWarp * kItems);
    int32_t vals[kItems];
    int32_t running = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + j * kWarp + lane;
        const int32_t x = idx < nn ? int32_t(in[idx]) : 0;
        const int32_t inc = warp_incl_scan(x, lane);
        vals[j] = running + inc - x;
        running += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) wsum[warp] = running;
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the warps' totals (kSmallWarps == 32)
        const int32_t w = wsum[lane];
        const int32_t inc = warp_incl_scan(w, lane);
        wpre[lane] = inc - w;
        if (lane == kWarp - 1) total = inc;
    }
    __syncthreads();
    const int32_t woff = wpre[warp];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + j * kWarp + lane;
        if (idx < n) out[idx] = vals[j] + woff;
    }
    if (threadIdx.x == 0) out[n] = total;
}

template <class T>
etl_status scan_impl(const T *in, int32_t *out, int64_t n, const int32_t *d_n, Workspace &ws) {
    cudaStream_t s = ws.stream();
    if (n <= 0) {
        memset_async(out, 0, sizeof(int32_t), s);
        return last_launch();
    }
    int64_t nb = ceil_div(n, kTile);
    if (nb == 1) {
        launch(k_scan_tile<T>, 1, kThreads, 0, s, in, out, n, d_n, nullptr, 1);
        note_launch();
        return last_launch();
    }
    if (n <= kSmallMax) {
        launch(k_scan_small<T>, 1, kSmallThreads, 0, s, in, out, n, d_n);
        note_launch();
        return last_launch();
    }
    int32_t *partial = ws.get<int32_t>(nb);
    int32_t *pscan = ws.get<int32_t>(nb + 1);
    if (!ws.ok()) return ETL_ENOMEM;
    launch(k_reduce<T>, unsigned(nb), kThreads, 0, s, in, n, d_n, partial);
    note_launch();
    etl_status st = last_launch();
    if (st) return st;
    st = scan_impl<int32_t>(partial, pscan, nb, nullptr, ws);
    if (st) return st;
    launch(k_scan_tile<T>, unsigned(nb), kThreads, 0, s, in, out, n, d_n, pscan, nb);
    note_launch();
    return last_launch();
}

}  // namespace

etl_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, Workspace &ws) {
    PhaseTimer pt("scan", ws.stream());
    return scan_impl<int32_t>(in, out, n, nullptr, ws);
}

etl_status scan_exclusive_u8(const uint8_t *in, int32_t *out, int64_t n, Workspace &ws) {
    PhaseTimer pt("scan", ws.stream());
    return scan_impl<uint8_t>(in, out, n, nullptr, ws);
}

}  // namespace etl
