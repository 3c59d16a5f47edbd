// Internal declarations of the Euler-tour library (sm_103a). Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "etl.h"

#define ETL_END (-1)

namespace etl {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// ----------------------------------------------------------------- host helpers

// Number of SMs of the current device (cached per device).
int num_sms();

// Caller-owned device memory. While an ArenaScope is active on the calling
// thread, every device allocation the library makes (dev_alloc, and so
// Workspace::get and the tables of an LCA handle) is carved from the arena
// instead of the allocator: 256-byte aligned, never freed, never reused within
// the call. A measuring arena has no memory behind it: it hands out placeholder
// addresses and only counts bytes; it is used with a stream under capture, so
// the kernels that receive those addresses are recorded and never run, and the
// async memset / copy helpers below skip their work.
struct Arena {
    char *base = nullptr;  // caller's memory (null while measuring)
    size_t cap = 0;        // bytes available from base
    size_t used = 0;       // bytes handed out so far (alignment included)
    bool measure = false;
};
Arena *current_arena();
class ArenaScope {
  public:
    explicit ArenaScope(Arena *a);
    ~ArenaScope();
    ArenaScope(const ArenaScope &) = delete;
    ArenaScope &operator=(const ArenaScope &) = delete;

  private:
    Arena *prev_;
};
inline bool measuring() {
    const Arena *a = current_arena();
    return a && a->measure;
}

// Stream-ordered device allocation from the library's own per-device memory
// pool, which keeps freed memory reserved (release threshold = max) so that
// repeated calls do not pay for re-mapping, and never reuses a block freed on
// another stream by making this stream wait for that one; while the stream is
// being captured into a graph the default pool is used (graph memory nodes).
// Freed with cudaFreeAsync. Inside an ArenaScope the memory comes from the
// arena instead (and must not be freed). Returns cudaSuccess or the
// allocator's error (cudaErrorMemoryAllocation when the arena is too small).
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s);

// cudaMemsetAsync / device-to-device cudaMemcpyAsync, skipped while measuring
cudaError_t memset_async(void *p, int value, size_t bytes, cudaStream_t s);
cudaError_t copy_d2d_async(void *dst, const void *src, size_t bytes, cudaStream_t s);

// Stream-ordered scratch: every buffer taken here is released with
// cudaFreeAsync on the same stream when the Workspace goes out of scope.
class Workspace {
  public:
    explicit Workspace(cudaStream_t s) : s_(s), arena_(current_arena() != nullptr) {}
    ~Workspace() { release(); }
    Workspace(const Workspace &) = delete;
    Workspace &operator=(const Workspace &) = delete;
    template <class T>
    T *get(size_t count) {
        void *p = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (dev_alloc(&p, bytes, s_) != cudaSuccess) {
            ok_ = false;
            return nullptr;
        }
        bufs_.push_back(p);
        return static_cast<T *>(p);
    }
    bool ok() const { return ok_; }
    void release() {
        if (!arena_)
            for (void *p : bufs_) cudaFreeAsync(p, s_);
        bufs_.clear();
    }
    cudaStream_t stream() const { return s_; }

  private:
    cudaStream_t s_;
    std::vector<void *> bufs_;
    bool ok_ = true;
    bool arena_;  // buffers come from a caller-owned arena: nothing to free
};

// Brackets a launch group with CUDA events when phase timing is enabled
// (etl_profile_enable); a no-op otherwise and while the stream is captured.
class PhaseTimer {
  public:
    PhaseTimer(const char *name, cudaStream_t s);
    ~PhaseTimer();
    PhaseTimer(const PhaseTimer &) = delete;
    PhaseTimer &operator=(const PhaseTimer &) = delete;

  private:
    const char *name_;
    cudaStream_t s_;
    void *a_ = nullptr, *b_ = nullptr;
};

// Host-side count of kernel launches issued by the library (for reporting).
void note_launch();

inline etl_status last_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ETL_OK : ETL_ECUDA;
}

// Programmatic dependent launch (ETL_TUNE_PDL). Every kernel of the library starts with
// pdl_prologue(): it waits until the grid launched before it on the stream has finished and its
// writes are visible (a no-op when the kernel was not launched as a dependent), then allows the
// next grid on the stream to be scheduled. launch() issues a kernel with the attribute when the knob
// is on, so the next kernel's launch overlaps the end of the current one instead of following it.
bool &pdl_enabled();

__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int ceil_log2(uint64_t x) {  // smallest b with 2^b >= x (x >= 1)
    int b = 0;
    while ((uint64_t(1) << b) < x) ++b;
    return b;
}

// ----------------------------------------------------------------- device helpers

__device__ __forceinline__ void set_status(int32_t *st, int32_t code) {
    if (st) atomicCAS(st, 0, code);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ----------------------------------------------------------------- primitives

// Exclusive scan of in[0..n) into out[0..n], out[n] = total. If d_n is not
// null, only in[0..*d_n) is read (the rest counts as 0); n is the capacity.
etl_status scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, Workspace &ws);
etl_status scan_exclusive_u8(const uint8_t *in, int32_t *out, int64_t n, Workspace &ws);

// Stable LSD radix sort of (key, value) pairs by key, keys in [0, key_limit)
// with key_limit <= 2^key_bits. Elements are in[0..count) where count =
// *d_count if d_count != null else n_cap. With vals_in == null the value of
// element i is i. Elements whose key is outside [0, key_limit) are dropped
// (they do not appear in the output). On return kv points at the sorted
// (key, value) pairs (inside the workspace) and *d_total (device) holds the
// number of elements kept.
struct SortResult {
    const int2 *kv;
    const int32_t *d_total;
};
etl_status radix_sort_pairs(const int32_t *keys_in, const int32_t *vals_in, const int32_t *d_count, int64_t n_cap,
                            int key_bits, int32_t key_limit, Workspace &ws, SortResult *out);

// ----------------------------------------------------------------- list ranking

// Result of ranking one list: element e lies in sublist sid = packed[e].x at
// local offset (packed[e].y & 0xffff) with (packed[e].y >> 16) even-indexed
// elements before it inside the sublist; R[sid] / O[sid] are the number of
// elements / of even-indexed elements before that sublist's first element.
// So rank(e) = R[sid] + lr and evens_before(e) = O[sid] + lo.
struct RankResult {
    const uint2 *packed;
    const int32_t *R;
    const int32_t *O;
    int64_t rcap;  // entries of R / O; a packed sublist id >= rcap marks an element off the list
};

struct RankParams {
    int k0_log2 = 5;     // level-0 splitter density: one in 2^k0_log2 elements
    int k_log2 = 3;      // density at the upper levels (1 in 8: 1-4% faster than 1 in 16 on trees of 2^15 .. 2^22)
    int block = 128;     // threads per block of the walk kernels
    int blocks_per_sm = 4;  // 512 walkers per SM: more of them measured slower (DRAM contention)
};
RankParams &rank_params();

struct SortParams {
    int rounds = 8;       // 32-element rounds per warp in the radix passes: tiles of 256 * rounds elements
    bool ballot = true;   // rank equal digits in a warp by ballots instead of __match_any_sync
};
SortParams &sort_params();

struct CcParams {
    int first_slice_quarters = 2;  // edges hooked before the first compression, in units of n/4
    bool doubling = false;         // later slices double in size, each after a compression
    bool giant = true;             // after a compression, the most frequent root ranks above all
};
CcParams &cc_params();

struct RmqParams {
    int levels_per_pass = 3;  // 1..3 levels built by one streaming pass
    int block = 256;          // threads per block of the level kernel
    bool blocked = true;      // two-level (blocked) tables instead of full sparse tables
};
RmqParams &rmq_params();

// succ[0..n_cap) with elements >= *d_len (if d_len) inert; head = *d_head.
// dual: also count even-indexed elements (the opening brackets of a tour).
etl_status list_rank(const int32_t *succ, int64_t n_cap, const int32_t *d_len, const int32_t *d_head, bool dual,
                     int64_t expect_len, int32_t *status, Workspace &ws, RankResult *out);

// rank[e] for e in [0, len) (plain output of the generic list-ranking entry point)
etl_status final_rank(const RankResult &r, int64_t len, int32_t *rank, cudaStream_t s);
// *p = v on the stream (a kernel, so no host buffer has to outlive the call)
etl_status set_device_i32(int32_t *p, int32_t v, cudaStream_t s);

__device__ __forceinline__ int32_t rank_of(const RankResult &r, uint2 p) { return r.R[p.x] + int32_t(p.y & 0xffffu); }
__device__ __forceinline__ int32_t evens_before(const RankResult &r, uint2 p) {
    return r.O[p.x] + int32_t(p.y >> 16);
}

// ----------------------------------------------------------------- sparse tables

// Full sparse table over x[0..n): level l holds min (or max) of x[i .. i+2^l)
// (entries past the end are folded with the identity). levels =
// floor(log2(max_len)) + 1 where max_len is the longest range ever queried.
// Level 0 must already be in table[0..n); rows are sparse_ld(n) apart and the
// build pads each row's tail with the identity.
int sparse_levels(int64_t max_len);
// row length (entries) of a table over n entries: n rounded up to a multiple of 4
int64_t sparse_ld(int64_t n);
template <bool IS_MAX>
etl_status sparse_table_build(int32_t *table, int64_t n, int levels, cudaStream_t s);

template <bool IS_MAX>
__device__ __forceinline__ int32_t sparse_query(const int32_t *__restrict__ table, int64_t ld, int32_t lo,
                                                int32_t hi) {  // inclusive range, lo <= hi; ld = row length
    int len = hi - lo + 1;
    int l = 31 - __clz(len);
    const int32_t *t = table + int64_t(l) * ld;
    int32_t a = __ldg(t + lo), b = __ldg(t + hi - (1 << l) + 1);
    return IS_MAX ? max(a, b) : min(a, b);
}

// ----------------------------------------------------------------- blocked range-min / max tables
//
// Two levels over x[0..n): x is cut into blocks of 32 entries; pm[i] / sm[i]
// hold op over x from the start of i's block to i / from i to the end of its
// block, and `top` is a full sparse table over the nblk block results. A range
// [lo, hi] inside one block is answered from x directly (at most 32 entries of
// one 128-byte line); otherwise it is op(sm[lo], pm[hi]) plus, when whole
// blocks lie between, one query of `top`. The build reads x once and writes
// 2n + O(n / 32 * log n) entries; `top` (n / 32 entries per level) stays in L2.
// Layout of one allocation of element type T: x, pm, sm (nblk * 32 entries
// each, x padded with the identity by the build) then tlevels rows of `top`,
// nblk entries apart.

struct OpMin {
    using T = int32_t;
    __device__ static __forceinline__ T id() { return INT32_MAX; }
    __device__ static __forceinline__ T f(T a, T b) { return min(a, b); }
};
struct OpMax {
    using T = int32_t;
    __device__ static __forceinline__ T id() { return INT32_MIN; }
    __device__ static __forceinline__ T f(T a, T b) { return max(a, b); }
};
struct OpMinKey {  // 64-bit keys: a value in the high half, a payload it carries in the low half
    using T = long long;
    __device__ static __forceinline__ T id() { return INT64_MAX; }
    __device__ static __forceinline__ T f(T a, T b) { return min(a, b); }
};
struct OpMinMax {  // x = min of the first component, y = max of the second
    using T = int2;
    __device__ static __forceinline__ T id() { return make_int2(INT32_MAX, INT32_MIN); }
    __device__ static __forceinline__ T f(T a, T b) { return make_int2(min(a.x, b.x), max(a.y, b.y)); }
};

constexpr int kRmqBlockLog2 = 5;
constexpr int kRmqBlock = 1 << kRmqBlockLog2;

struct BlockedLayout {
    int64_t nblk;  // blocks of 32 entries
    int tlevels;   // levels of the top table
    int64_t elems() const { return 3 * nblk * kRmqBlock + nblk * tlevels; }
};
// a table over n entries answering ranges of up to max_len entries
BlockedLayout blocked_layout(int64_t n, int64_t max_len);
// x (first n entries of base) must be filled; builds pad, pm, sm and top. pairs (int32 entries only):
// pm and sm interleaved as (pm[i], sm[i]) pairs in the 2N entries after x (then blocked_query, which
// reads them as separate arrays, must not be used on the table; x and top are unchanged)
template <class Op>
etl_status blocked_build(typename Op::T *base, int64_t n, const BlockedLayout &L, cudaStream_t s,
                         bool pairs = false);

template <class Op>
struct BlockedView {
    const typename Op::T *x, *pm, *sm, *top;
    int64_t nblk;
    int tlevels;
};
template <class Op>
inline BlockedView<Op> blocked_view(const typename Op::T *base, const BlockedLayout &L) {
    const int64_t N = L.nblk * kRmqBlock;
    return BlockedView<Op>{base, base + N, base + 2 * N, base + 3 * N, L.nblk, L.tlevels};
}
// longest range a layout answers (a range of len entries spans at most (len - 1) / 32 whole blocks)
inline int64_t blocked_max_len(const BlockedLayout &L) { return (int64_t(kRmqBlock) << L.tlevels) - 1; }

template <class Op>
__device__ __forceinline__ typename Op::T blocked_query(const BlockedView<Op> &t, int32_t lo,
                                                        int32_t hi) {  // inclusive, lo <= hi
    using T = typename Op::T;
    const int32_t bl = lo >> kRmqBlockLog2, bh = hi >> kRmqBlockLog2;
    if (bl == bh) {
        T m = __ldg(t.x + lo);
        for (int32_t j = lo + 1; j <= hi; ++j) m = Op::f(m, __ldg(t.x + j));
        return m;
    }
    T m = Op::f(__ldg(t.sm + lo), __ldg(t.pm + hi));
    if (bh - bl > 1) {
        const int32_t a = bl + 1, b = bh - 1;
        const int l = 31 - __clz(b - a + 1);
        const T *row = t.top + int64_t(l) * t.nblk;
        m = Op::f(m, Op::f(__ldg(row + a), __ldg(row + b - (1 << l) + 1)));
    }
    return m;
}

}  // namespace etl

// ----------------------------------------------------------------- the LCA handle
struct etl_lca_s {
    int32_t n = 0;       // nodes (all instances of a batch together)
    int32_t k = 1;       // trees in the handle
    int32_t *node_off = nullptr;  // batch only: k+1 instance offsets (device)
    int levels = 0;
    cudaStream_t stream = nullptr;
    int32_t *pre = nullptr, *depth = nullptr, *size = nullptr, *order = nullptr;
    int64_t ld = 0;             // row length of the sparse table
    int32_t *table = nullptr;   // levels * ld (full sparse table) or the blocked table's allocation
    bool blocked = false;       // table is a blocked two-level table (layout `bl`)
    void *nrec = nullptr;       // blocked table: per node (pre, pm[pre], sm[pre + 1], 0), int4[n]
    etl::BlockedLayout bl{};
    int32_t *status = nullptr;  // device status word
    bool has_table = false;     // RMQ sparse table built (lca_query available)
    void *inrec = nullptr;      // Inlabel: per node (inlabel, ascendant, depth, parent), int4[n]
    void *inpath = nullptr;     // Inlabel: per inlabel value (parent of the path head, its depth), int2[n+1]
    void *tour_table = nullptr;  // Euler-tour RMQ: blocked table of (depth << 32 | node) keys over 2n positions
    int32_t *tpos = nullptr;     // Euler-tour RMQ: tour position of each node's opening bracket
    etl::BlockedLayout tbl{};
    bool arena = false;          // device arrays live in a caller-owned workspace: lca_free frees none of them
};
