// Caller-owned workspaces: the size query and the _ws entry points.
//
// A _ws call runs the ordinary entry point with an Arena active on the calling
// thread, so that every device allocation it would have made (scratch, status
// words, an LCA handle's tables) is carved from the caller's buffer instead;
// the allocator is never called. etl_workspace_size finds the number of bytes
// by running the same entry point once more with a measuring arena on a
// private stream that is being captured: the arena hands out placeholder
// addresses, the kernels that receive them are only recorded into a graph
// that is destroyed without ever being launched, and the memset / copy helpers
// skip their work. So the size is exact for the same sizes and tuning
// parameters, and it cannot drift from the code that uses the memory.
#include "etl_internal.cuh"

namespace etl {
namespace {

// placeholder for the caller's arrays while measuring (never dereferenced)
template <class T>
T *placeholder() {
    return reinterpret_cast<T *>(uintptr_t(1) << 41);
}

template <class F>
etl_status measure(F &&call, size_t *bytes) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return ETL_ECUDA;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(s);
        return ETL_ECUDA;
    }
    Arena a;
    a.measure = true;
    etl_status rc;
    {
        ArenaScope scope(&a);
        rc = call(s);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(s);
    cudaGetLastError();  // a failed capture leaves nothing behind for the caller's next check
    if (rc) return rc;
    if (e != cudaSuccess) return ETL_ECUDA;
    *bytes = a.used ? a.used + 256 : 0;  // + room to align a caller's base that is not 256-byte aligned
    return ETL_OK;
}

template <class F>
etl_status in_workspace(void *ws, size_t ws_bytes, F &&call) {
    if (!ws) return ETL_EINVAL;
    Arena a;
    a.base = static_cast<char *>(ws);
    a.cap = ws_bytes;
    ArenaScope scope(&a);
    return call();
}

}  // namespace
}  // namespace etl

using namespace etl;

extern "C" etl_status etl_workspace_size(int32_t kind, int64_t n, int64_t m_or_q, size_t *bytes) {
    if (!bytes) return ETL_EINVAL;
    *bytes = 0;
    switch (kind) {
        case ETL_WS_LIST_RANK:
            if (n < 1 || n > int64_t(INT32_MAX) - 1) return ETL_EINVAL;
            return measure([&](cudaStream_t s) {
                return etl_list_rank(placeholder<const int32_t>(), n, 0, placeholder<int32_t>(), nullptr, s);
            }, bytes);
        case ETL_WS_LCA_PREPROCESS:
            if (n < 1 || n > (1 << 30) - 1) return ETL_EINVAL;
            return measure([&](cudaStream_t s) {
                etl_lca_t h = nullptr;
                etl_status rc = lca_preprocess(placeholder<const int32_t>(), int32_t(n), s, &h);
                if (h) lca_free(h);
                return rc;
            }, bytes);
        case ETL_WS_LCA_QUERY:  // queries read the handle's tables and need no scratch
            if (n < 1 || n > (1 << 30) - 1 || m_or_q < 0 || m_or_q > (int64_t(1) << 40)) return ETL_EINVAL;
            return ETL_OK;
        case ETL_WS_FIND_BRIDGES:
            if (n < 1 || n > (1 << 30) - 1 || m_or_q < 0 || m_or_q > int64_t(INT32_MAX) - 1) return ETL_EINVAL;
            return measure([&](cudaStream_t s) {
                return find_bridges(placeholder<const int32_t>(), m_or_q, int32_t(n), placeholder<uint8_t>(),
                                    nullptr, s);
            }, bytes);
        default:
            return ETL_EINVAL;
    }
}

extern "C" etl_status etl_workspace_size_batch(int32_t kind, int32_t k, int64_t total_n, int64_t max_n_or_total_m,
                                               size_t *bytes) {
    if (!bytes) return ETL_EINVAL;
    *bytes = 0;
    if (k < 1 || total_n < k || total_n > (1 << 30) - 1) return ETL_EINVAL;
    switch (kind) {
        case ETL_WS_LCA_PREPROCESS:
            if (max_n_or_total_m < 1 || max_n_or_total_m > total_n) return ETL_EINVAL;
            return measure([&](cudaStream_t s) {
                etl_lca_t h = nullptr;
                etl_status rc = lca_preprocess_batch(placeholder<const int32_t>(), placeholder<const int32_t>(), k,
                                                     int32_t(total_n), int32_t(max_n_or_total_m), s, &h);
                if (h) lca_free(h);
                return rc;
            }, bytes);
        case ETL_WS_LCA_QUERY:
            return ETL_OK;
        case ETL_WS_FIND_BRIDGES:
            if (max_n_or_total_m < 0 || max_n_or_total_m > int64_t(INT32_MAX) - 1) return ETL_EINVAL;
            return measure([&](cudaStream_t s) {
                return find_bridges_batch(placeholder<const int32_t>(), placeholder<const int32_t>(),
                                          placeholder<const int32_t>(), k, max_n_or_total_m, int32_t(total_n),
                                          placeholder<uint8_t>(), nullptr, s);
            }, bytes);
        default:
            return ETL_EINVAL;
    }
}

extern "C" etl_status etl_list_rank_ws(const int32_t *succ, int64_t len, int32_t head, int32_t *rank,
                                       int32_t *status, void *ws, size_t ws_bytes, void *stream) {
    return in_workspace(ws, ws_bytes, [&] { return etl_list_rank(succ, len, head, rank, status, stream); });
}

extern "C" etl_status lca_preprocess_ws(const int32_t *parent, int32_t n, void *ws, size_t ws_bytes, void *stream,
                                        etl_lca_t *out) {
    if (out) *out = nullptr;
    return in_workspace(ws, ws_bytes, [&] { return lca_preprocess(parent, n, stream, out); });
}

extern "C" etl_status lca_preprocess_batch_ws(const int32_t *parent, const int32_t *node_off, int32_t k,
                                              int32_t total_n, int32_t max_n, void *ws, size_t ws_bytes,
                                              void *stream, etl_lca_t *out) {
    if (out) *out = nullptr;
    return in_workspace(ws, ws_bytes,
                        [&] { return lca_preprocess_batch(parent, node_off, k, total_n, max_n, stream, out); });
}

extern "C" etl_status find_bridges_ws(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge,
                                      int32_t *status, void *ws, size_t ws_bytes, void *stream) {
    return in_workspace(ws, ws_bytes, [&] { return find_bridges(edges, m, n, is_bridge, status, stream); });
}

extern "C" etl_status find_bridges_batch_ws(const int32_t *edges, const int32_t *edge_off, const int32_t *node_off,
                                            int32_t k, int64_t total_m, int32_t total_n, uint8_t *is_bridge,
                                            int32_t *status, void *ws, size_t ws_bytes, void *stream) {
    return in_workspace(ws, ws_bytes, [&] {
        return find_bridges_batch(edges, edge_off, node_off, k, total_m, total_n, is_bridge, status, stream);
    });
}

extern "C" etl_status etl_status_get(void *stream, const int32_t *d_status, int32_t *h_status) {
    if (!d_status || !h_status) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t v = -1;
    if (cudaMemcpyAsync(&v, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ETL_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ETL_ECUDA;
    *h_status = v;
    return ETL_OK;
}
