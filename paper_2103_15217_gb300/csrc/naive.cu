// The naive GPU LCA of Martins et al. that the paper compares against
// (Sec. 3.1, "The Naive Algorithm"):
//
//  * Preprocessing computes every node's level by pointer jumping: each node
//    keeps an ancestor pointer (initially its parent) and the distance to it;
//    pointers double until they reach a node whose level is known, and the
//    level is then that node's level plus the distance. As in the paper, each
//    launch performs five jumps per node before the next global
//    synchronisation. The (ancestor, distance) pair is one 64-bit word read and
//    written atomically, so nodes can jump asynchronously inside a launch and
//    the pair always names an ancestor and its true distance.
//  * A query climbs from both ends: the deeper end up to the other's level,
//    then both together until they meet -- one thread per query, work
//    proportional to the distance between the ends.
//
// Records are (parent, level) pairs so every climbing step is one 8-byte load.
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

__device__ __forceinline__ int64_t gtid() { return blockIdx.x * int64_t(blockDim.x) + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

constexpr int kJumpsPerLaunch = 5;

__device__ __forceinline__ unsigned long long pack(int32_t anc, int32_t dist) {
    return (unsigned long long)(uint32_t(anc)) | ((unsigned long long)(uint32_t(dist)) << 32);
}

__global__ void k_naive_init(const int32_t *__restrict__ parent, int32_t n, unsigned long long *__restrict__ ad,
                             int32_t *__restrict__ level, int32_t *__restrict__ roots, int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int32_t p = parent[v];
        if (p == -1) {
            level[v] = 0;
            atomicAdd(roots, 1);
        } else {
            if (p < 0 || p >= n || p == v) set_status(status, ETL_EBADTREE);
            level[v] = -1;
        }
        ad[v] = pack(p >= 0 && p < n ? p : int32_t(v), 1);
    }
}

__global__ void k_naive_jump(int32_t n, unsigned long long *__restrict__ ad, int32_t *__restrict__ level,
                             int32_t *__restrict__ pending) {
    pdl_prologue();
    for (int64_t v = gtid(); v < n; v += gstride()) {
        if (__ldcg(level + v) >= 0) continue;
        bool done = false;
        for (int j = 0; j < kJumpsPerLaunch && !done; ++j) {
            const unsigned long long mine = __ldcg(ad + v);  // aligned 8-byte load: a consistent pair
            const int32_t a = int32_t(uint32_t(mine)), d = int32_t(uint32_t(mine >> 32));
            const int32_t la = __ldcg(level + a);
            if (la >= 0) {
                level[v] = la + d;
                done = true;
            } else {
                const unsigned long long up = __ldcg(ad + a);
                const int32_t aa = int32_t(uint32_t(up)), dd = int32_t(uint32_t(up >> 32));
                __stcg(ad + v, pack(aa, d + dd));  // aligned 8-byte store: written as one pair
            }
        }
        if (!done) atomicAdd(pending, 1);
    }
}

__global__ void k_naive_records(const int32_t *__restrict__ parent, const int32_t *__restrict__ level, int32_t n,
                                const int32_t *__restrict__ roots, int2 *__restrict__ rec,
                                int32_t *__restrict__ status) {
    pdl_prologue();
    if (gtid() == 0 && *roots != 1) set_status(status, ETL_EBADTREE);
    for (int64_t v = gtid(); v < n; v += gstride()) {
        const int32_t l = level[v];
        if (l < 0) set_status(status, ETL_EBADTREE);  // never reached the root: a cycle
        rec[v] = make_int2(parent[v], l);
    }
}

__global__ void __launch_bounds__(256)
    k_naive_query(const int2 *__restrict__ rec, int32_t n, const int32_t *__restrict__ u,
                  const int32_t *__restrict__ v, int64_t q, int32_t *__restrict__ out, int32_t *__restrict__ status) {
    pdl_prologue();
    for (int64_t i = gtid(); i < q; i += gstride()) {
        int32_t a = __ldcs(u + i), b = __ldcs(v + i);
        int32_t res = -1;
        if (a < 0 || a >= n || b < 0 || b >= n) {
            set_status(status, ETL_EBADQUERY);
        } else {
            int2 ra = __ldg(rec + a), rb = __ldg(rec + b);
            int64_t steps = 0;
            bool ok = ra.y >= 0 && rb.y >= 0;
            while (ok && ra.y > rb.y && steps++ < n) {
                a = ra.x;
                ok = a >= 0 && a < n;
                if (ok) ra = __ldg(rec + a);
            }
            while (ok && rb.y > ra.y && steps++ < n) {
                b = rb.x;
                ok = b >= 0 && b < n;
                if (ok) rb = __ldg(rec + b);
            }
            while (ok && a != b && steps++ < 2 * int64_t(n)) {
                a = ra.x;
                b = rb.x;
                ok = a >= 0 && a < n && b >= 0 && b < n;
                if (ok) {
                    ra = __ldg(rec + a);
                    rb = __ldg(rec + b);
                }
            }
            if (ok && a == b) res = a;
            else set_status(status, ETL_ETIMEOUT);
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

extern "C" etl_status lca_naive_preprocess(const int32_t *parent, int32_t n, int32_t *rec, int32_t *status,
                                           void *stream) {
    if (!parent || !rec || n < 1 || n > (1 << 30)) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws(s);
    unsigned long long *ad = ws.get<unsigned long long>(n);
    int32_t *level = ws.get<int32_t>(n);
    int32_t *cnt = ws.get<int32_t>(2);  // [0] roots, [1] nodes still pending after the last launch
    int32_t *st = status ? status : ws.get<int32_t>(1);
    if (!ws.ok()) return ETL_ENOMEM;
    memset_async(st, 0, sizeof(int32_t), s);
    memset_async(cnt, 0, 2 * sizeof(int32_t), s);
    const int g = grid_for(n, 256);
    PhaseTimer pt("naive.levels", s);
    launch(k_naive_init, g, 256, 0, s, parent, n, ad, level, cnt, st);
    note_launch();
    // every jump adds at least the distance the ancestor covered at the end of the previous launch,
    // so launch r covers >= 6^r levels even with asynchronous jumps: ceil(log6 n) + 1 launches suffice
    int launches = 1;
    for (double c = 1; c < double(n); c *= (kJumpsPerLaunch + 1)) ++launches;
    for (int r = 0; r < launches; ++r) {
        if (r == launches - 1) memset_async(cnt + 1, 0, sizeof(int32_t), s);
        launch(k_naive_jump, g, 256, 0, s, n, ad, level, cnt + 1);
        note_launch();
    }
    launch(k_naive_records, g, 256, 0, s, parent, level, n, cnt, reinterpret_cast<int2 *>(rec), st);
    note_launch();
    return last_launch();
}

extern "C" etl_status lca_naive_query(const int32_t *rec, int32_t n, const int32_t *u, const int32_t *v, int64_t q,
                                      int32_t *out, int32_t *status, void *stream) {
    if (!rec || n < 1 || q < 0 || q > (int64_t(1) << 40)) return ETL_EINVAL;
    if (q == 0) return ETL_OK;
    if (!u || !v || !out) return ETL_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PhaseTimer pt("naive.query", s);
    launch(k_naive_query, grid_for(q, 256), 256, 0, s, reinterpret_cast<const int2 *>(rec), n, u, v, q, out, status);
    note_launch();
    return last_launch();
}
