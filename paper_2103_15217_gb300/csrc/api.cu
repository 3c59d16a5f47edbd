// Shared host helpers and the generic list-ranking entry point.
#include <atomic>
#include <mutex>

#include "etl_internal.cuh"

namespace etl {

bool &pdl_enabled() {
    static bool on = true;
    return on;
}

int num_sms() {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> g(mu);
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cached[dev] = v;
    }
    return cached[dev];
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {nullptr};
std::atomic<int64_t> g_allocs{0};
thread_local Arena *t_arena = nullptr;
// placeholder addresses handed out while measuring: never dereferenced (the kernels are only captured)
constexpr uintptr_t kMeasureBase = uintptr_t(1) << 40;

cudaError_t arena_take(Arena *a, void **p, size_t bytes) {
    const uintptr_t base = a->measure ? kMeasureBase : reinterpret_cast<uintptr_t>(a->base);
    const uintptr_t at = (base + a->used + 255) & ~uintptr_t(255);
    const size_t end = size_t(at - base) + bytes;
    if (!a->measure && end > a->cap) return cudaErrorMemoryAllocation;
    a->used = end;
    *p = reinterpret_cast<void *>(at);
    return cudaSuccess;
}
}  // namespace

Arena *current_arena() { return t_arena; }
ArenaScope::ArenaScope(Arena *a) : prev_(t_arena) { t_arena = a; }
ArenaScope::~ArenaScope() { t_arena = prev_; }

cudaError_t memset_async(void *p, int value, size_t bytes, cudaStream_t s) {
    if (measuring()) return cudaSuccess;
    return cudaMemsetAsync(p, value, bytes, s);
}

cudaError_t copy_d2d_async(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (measuring()) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    if (Arena *a = t_arena) return arena_take(a, p, bytes);
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return cudaMallocAsync(p, bytes, s);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> g(g_pool_mu);
        if (!g_pool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t np = nullptr;
            if (cudaMemPoolCreate(&np, &props) != cudaSuccess) return cudaMallocAsync(p, bytes, s);
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
            // never make a stream wait on another one to reuse a block freed there: independent
            // calls on different streams must not be serialised by the allocator
            int no = 0;
            cudaMemPoolSetAttribute(np, cudaMemPoolReuseAllowInternalDependencies, &no);
            g_pool[dev] = np;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

}  // namespace etl

using namespace etl;

extern "C" etl_status etl_pool_stats(int64_t *reserved, int64_t *used) {
    if (!reserved || !used) return ETL_EINVAL;
    *reserved = *used = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ETL_ECUDA;
    std::lock_guard<std::mutex> g(g_pool_mu);
    if (!g_pool[dev]) return ETL_OK;
    uint64_t r = 0, u = 0;
    if (cudaMemPoolGetAttribute(g_pool[dev], cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess ||
        cudaMemPoolGetAttribute(g_pool[dev], cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess)
        return ETL_ECUDA;
    *reserved = int64_t(r);
    *used = int64_t(u);
    return ETL_OK;
}

extern "C" etl_status etl_alloc_count(int64_t *count) {
    if (!count) return ETL_EINVAL;
    *count = g_allocs.load(std::memory_order_relaxed);
    return ETL_OK;
}

extern "C" etl_status etl_trim(void) {
    std::lock_guard<std::mutex> g(g_pool_mu);
    for (cudaMemPool_t p : g_pool)
        if (p && cudaMemPoolTrimTo(p, 0) != cudaSuccess) return ETL_ECUDA;
    return ETL_OK;
}

extern "C" const char *etl_status_string(int32_t status) {
    switch (status) {
        case ETL_OK: return "ETL_OK";
        case ETL_EINVAL: return "ETL_EINVAL";
        case ETL_ENOMEM: return "ETL_ENOMEM";
        case ETL_ECUDA: return "ETL_ECUDA";
        case ETL_EBADTREE: return "ETL_EBADTREE";
        case ETL_EBADQUERY: return "ETL_EBADQUERY";
        case ETL_EBADGRAPH: return "ETL_EBADGRAPH";
        case ETL_ETIMEOUT: return "ETL_ETIMEOUT";
        default: return "ETL_UNKNOWN";
    }
}

extern "C" etl_status etl_list_rank(const int32_t *succ, int64_t len, int32_t head, int32_t *rank, int32_t *status,
                                    void *stream) {
    if (!succ || !rank || len < 1 || len > int64_t(INT32_MAX) - 1 || head < 0 || head >= len) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    int32_t *d_head = ws.get<int32_t>(1);
    int32_t *st = status ? status : ws.get<int32_t>(1);
    if (!ws.ok()) return ETL_ENOMEM;
    etl_status rc = set_device_i32(d_head, head, s);
    RankResult rr{};
    if (!rc) rc = list_rank(succ, len, nullptr, d_head, false, len, st, ws, &rr);
    if (!rc) rc = final_rank(rr, len, rank, s);
    return rc;
}

extern "C" etl_status etl_tune_set(int32_t key, int32_t value) {
    RankParams &P = rank_params();
    switch (key) {
        case ETL_TUNE_RANK_K0_LOG2:
            if (value < 1 || value > 8) return ETL_EINVAL;
            P.k0_log2 = value;
            return ETL_OK;
        case ETL_TUNE_RANK_K_LOG2:
            if (value < 1 || value > 8) return ETL_EINVAL;
            P.k_log2 = value;
            return ETL_OK;
        case ETL_TUNE_RANK_BLOCK:
            if (value != 64 && value != 128 && value != 256 && value != 512 && value != 1024) return ETL_EINVAL;
            if (value * P.blocks_per_sm > 2048) P.blocks_per_sm = 2048 / value;
            P.block = value;
            return ETL_OK;
        case ETL_TUNE_RANK_BLOCKS_PER_SM:
            if (value < 1 || value * P.block > 2048) return ETL_EINVAL;
            P.blocks_per_sm = value;
            return ETL_OK;
        case ETL_TUNE_RMQ_LEVELS_PER_PASS:
            if (value < 1 || value > 3) return ETL_EINVAL;
            rmq_params().levels_per_pass = value;
            return ETL_OK;
        case ETL_TUNE_RMQ_BLOCK:
            if (value != 128 && value != 256 && value != 512 && value != 1024) return ETL_EINVAL;
            rmq_params().block = value;
            return ETL_OK;
        case ETL_TUNE_CC_FIRST_SLICE:
            if (value < 1 || value > 64) return ETL_EINVAL;
            cc_params().first_slice_quarters = value;
            return ETL_OK;
        case ETL_TUNE_RMQ_BLOCKED:
            if (value != 0 && value != 1) return ETL_EINVAL;
            rmq_params().blocked = value != 0;
            return ETL_OK;
        case ETL_TUNE_SORT_ROUNDS:
            if (value != 8 && value != 16) return ETL_EINVAL;
            sort_params().rounds = value;
            return ETL_OK;
        case ETL_TUNE_CC_DOUBLING:
            if (value != 0 && value != 1) return ETL_EINVAL;
            cc_params().doubling = value != 0;
            return ETL_OK;
        case ETL_TUNE_CC_GIANT:
            if (value != 0 && value != 1) return ETL_EINVAL;
            cc_params().giant = value != 0;
            return ETL_OK;
        case ETL_TUNE_SORT_BALLOT:
            if (value != 0 && value != 1) return ETL_EINVAL;
            sort_params().ballot = value != 0;
            return ETL_OK;
        case ETL_TUNE_PDL:
            if (value != 0 && value != 1) return ETL_EINVAL;
            pdl_enabled() = value != 0;
            return ETL_OK;
        default:
            return ETL_EINVAL;
    }
}

extern "C" etl_status etl_tune_get(int32_t key, int32_t *value) {
    if (!value) return ETL_EINVAL;
    const RankParams &P = rank_params();
    switch (key) {
        case ETL_TUNE_RANK_K0_LOG2: *value = P.k0_log2; return ETL_OK;
        case ETL_TUNE_RANK_K_LOG2: *value = P.k_log2; return ETL_OK;
        case ETL_TUNE_RANK_BLOCK: *value = P.block; return ETL_OK;
        case ETL_TUNE_RANK_BLOCKS_PER_SM: *value = P.blocks_per_sm; return ETL_OK;
        case ETL_TUNE_RMQ_LEVELS_PER_PASS: *value = rmq_params().levels_per_pass; return ETL_OK;
        case ETL_TUNE_RMQ_BLOCK: *value = rmq_params().block; return ETL_OK;
        case ETL_TUNE_CC_FIRST_SLICE: *value = cc_params().first_slice_quarters; return ETL_OK;
        case ETL_TUNE_RMQ_BLOCKED: *value = rmq_params().blocked ? 1 : 0; return ETL_OK;
        case ETL_TUNE_SORT_ROUNDS: *value = sort_params().rounds; return ETL_OK;
        case ETL_TUNE_CC_DOUBLING: *value = cc_params().doubling ? 1 : 0; return ETL_OK;
        case ETL_TUNE_CC_GIANT: *value = cc_params().giant ? 1 : 0; return ETL_OK;
        case ETL_TUNE_SORT_BALLOT: *value = sort_params().ballot ? 1 : 0; return ETL_OK;
        case ETL_TUNE_PDL: *value = pdl_enabled() ? 1 : 0; return ETL_OK;
        default: return ETL_EINVAL;
    }
}
