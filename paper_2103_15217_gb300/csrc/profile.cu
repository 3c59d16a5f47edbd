// Opt-in phase timers: when enabled, every launch group of the library is
// bracketed by two CUDA events on the stream it runs on, so a caller can read
// per-phase device time of a live run (used by the benchmark's roofline).
// Disabled by default; skipped while a stream is being captured.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "etl_internal.cuh"

namespace etl {
namespace {

struct Rec {
    std::string name;
    cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
struct Agg {
    double ms = 0;
    int64_t launches = 0;
};
std::map<std::string, Agg> g_agg;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_locked() {
    for (Rec &r : g_recs) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            Agg &g = g_agg[r.name];
            g.ms += ms;
            g.launches += 1;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}

}  // namespace

PhaseTimer::PhaseTimer(const char *name, cudaStream_t s) : name_(name), s_(s) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    a_ = take_event();
    b_ = take_event();
    if (a_ && b_) cudaEventRecord(static_cast<cudaEvent_t>(a_), s);
}

PhaseTimer::~PhaseTimer() {
    if (!a_ || !b_) return;
    std::lock_guard<std::mutex> g(g_mu);
    cudaEventRecord(static_cast<cudaEvent_t>(b_), s_);
    g_recs.push_back(Rec{name_, static_cast<cudaEvent_t>(a_), static_cast<cudaEvent_t>(b_)});
}

// Measurement aid: the access pattern of one step of the ranking walk (read the successor of a
// random element, write an 8-byte record at the same random index) without the walk's chain of
// dependent loads: element i of a random permutation is visited by thread i, so every gather is
// independent and the memory system sees as many as it can take. Its rate is the ceiling of any
// walk over a list in random order. Indices outside [0, n) are skipped.
__global__ void k_probe_gather_scatter(const int32_t *__restrict__ order, const int32_t *__restrict__ succ,
                                       int64_t n, uint2 *__restrict__ out) {
    pdl_prologue();
    constexpr int kIlp = 4;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t base = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; base < n; base += stride * kIlp) {
        int32_t j[kIlp], x[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const int64_t i = base + k * stride;
            j[k] = i < n ? __ldcs(order + i) : -1;
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) x[k] = (j[k] >= 0 && j[k] < n) ? __ldg(succ + j[k]) : 0;
#pragma unroll
        for (int k = 0; k < kIlp; ++k)
            if (j[k] >= 0 && j[k] < n) out[j[k]] = make_uint2(uint32_t(x[k]), uint32_t(base + k * stride));
    }
}

std::atomic<int64_t> g_launches{0};
void note_launch() {
    if (!measuring()) g_launches.fetch_add(1, std::memory_order_relaxed);
}

}  // namespace etl

using namespace etl;

extern "C" etl_status etl_probe_gather_scatter(const int32_t *order, const int32_t *succ, int64_t n, void *out,
                                                void *stream) {
    if (!order || !succ || !out || n < 1 || n > int64_t(INT32_MAX)) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t blocks = ceil_div(ceil_div(n, 4), 256);
    const int64_t cap = int64_t(num_sms()) * 8 * 4;  // four waves of full occupancy
    if (blocks > cap) blocks = cap;
    launch(k_probe_gather_scatter, int(blocks), 256, 0, s, order, succ, n, static_cast<uint2 *>(out));
    note_launch();
    return last_launch();
}

extern "C" etl_status etl_launch_count(int64_t *count) {
    if (!count) return ETL_EINVAL;
    *count = g_launches.load();
    return ETL_OK;
}

extern "C" etl_status etl_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> g(g_mu);
    g_on = on != 0;
    return ETL_OK;
}

extern "C" etl_status etl_profile_reset(void) {
    std::lock_guard<std::mutex> g(g_mu);
    drain_locked();
    g_agg.clear();
    return ETL_OK;
}

extern "C" etl_status etl_profile_count(int32_t *count) {
    if (!count) return ETL_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    drain_locked();
    *count = int32_t(g_agg.size());
    return ETL_OK;
}

extern "C" etl_status etl_profile_get(int32_t i, char *name, int32_t name_len, double *total_ms, int64_t *launches) {
    if (!name || name_len < 1 || !total_ms || !launches) return ETL_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    drain_locked();
    if (i < 0 || i >= int32_t(g_agg.size())) return ETL_EINVAL;
    auto it = g_agg.begin();
    std::advance(it, i);
    std::strncpy(name, it->first.c_str(), size_t(name_len) - 1);
    name[name_len - 1] = '\0';
    *total_ms = it->second.ms;
    *launches = it->second.launches;
    return ETL_OK;
}
