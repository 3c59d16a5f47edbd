// Sparse tables for range-minimum / range-maximum queries (Sec. 3.1 reduces
// LCA to RMQ; Sec. 4.1 aggregates low / high over subtrees by RMQ). Level l
// is built from level l-1 by one coalesced streaming pass:
//     T_l[i] = op(T_{l-1}[i], T_{l-1}[i + 2^(l-1)]).
// The second operand trails the first by 2^(l-1) entries, which the 129 MB L2
// still holds for every level of the sizes used here, so each level costs
// about one DRAM read and one DRAM write per entry.
#include <climits>

#include "etl_internal.cuh"

namespace etl {
namespace {

template <bool IS_MAX>
__device__ __forceinline__ int32_t op(int32_t a, int32_t b) {
    return IS_MAX ? max(a, b) : min(a, b);
}

template <bool IS_MAX>
__global__ void k_level_vec4(int32_t *__restrict__ table, int64_t n, int l) {
    // n % 4 == 0 and 2^(l-1) % 4 == 0: whole int4 vectors
    const int32_t ident = IS_MAX ? INT_MIN : INT_MAX;
    const int4 *prev = reinterpret_cast<const int4 *>(table + int64_t(l - 1) * n);
    int4 *cur = reinterpret_cast<int4 *>(table + int64_t(l) * n);
    const int64_t nv = n >> 2, hv = (int64_t(1) << (l - 1)) >> 2;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < nv; i += int64_t(gridDim.x) * blockDim.x) {
        int4 a = prev[i];
        int4 b = i + hv < nv ? prev[i + hv] : make_int4(ident, ident, ident, ident);
        cur[i] = make_int4(op<IS_MAX>(a.x, b.x), op<IS_MAX>(a.y, b.y), op<IS_MAX>(a.z, b.z), op<IS_MAX>(a.w, b.w));
    }
}

template <bool IS_MAX>
__global__ void k_level(int32_t *__restrict__ table, int64_t n, int l) {
    const int32_t ident = IS_MAX ? INT_MIN : INT_MAX;
    const int32_t *prev = table + int64_t(l - 1) * n;
    int32_t *cur = table + int64_t(l) * n;
    const int64_t h = int64_t(1) << (l - 1);
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int32_t a = prev[i];
        int32_t b = i + h < n ? prev[i + h] : ident;
        cur[i] = op<IS_MAX>(a, b);
    }
}

}  // namespace

int sparse_levels(int64_t max_len) {
    int L = 1;
    while ((int64_t(1) << L) <= max_len) ++L;
    return L;
}

template <bool IS_MAX>
etl_status sparse_table_build(int32_t *table, int64_t n, int levels, cudaStream_t s) {
    const int grid_cap = num_sms() * 8;
    for (int l = 1; l < levels; ++l) {
        const bool vec = (n % 4 == 0) && l >= 3;
        const int64_t work = vec ? n / 4 : n;
        int blocks = int(ceil_div(work, 256));
        if (blocks > grid_cap) blocks = grid_cap;
        if (blocks < 1) blocks = 1;
        PhaseTimer pt(IS_MAX ? "rmq.level_max" : "rmq.level_min", s);
        if (vec)
            k_level_vec4<IS_MAX><<<blocks, 256, 0, s>>>(table, n, l);
        else
            k_level<IS_MAX><<<blocks, 256, 0, s>>>(table, n, l);
        note_launch();
        etl_status st = last_launch();
        if (st) return st;
    }
    return ETL_OK;
}

template etl_status sparse_table_build<false>(int32_t *, int64_t, int, cudaStream_t);
template etl_status sparse_table_build<true>(int32_t *, int64_t, int, cudaStream_t);

}  // namespace etl
