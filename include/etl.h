/*
 * etl.h -- C ABI of the GB300 (sm_103a) Euler-tour library.
 *
 * The library computes, on one GPU, the Euler tour technique of "Euler Meets
 * GPU: Practical Graph Algorithms with Theoretical Guarantees" (Polak,
 * Siwiec, Stobierski; arXiv 2103.15217) and its two applications:
 * lowest common ancestors by range-minimum queries over the tour, and bridges
 * by the Tarjan-Vishkin method.
 *
 * Common rules for every entry point below:
 *  - Array arguments are DEVICE pointers (cudaMalloc / torch CUDA memory) in
 *    the caller's current CUDA context, unless a comment says otherwise; all
 *    integers are little-endian int32 unless stated. Inputs are read-only;
 *    outputs are written completely. The caller owns every array it passes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Every call only enqueues work on that stream and returns; it
 *    never synchronises unless its comment says so. Device memory the call
 *    needs for itself is taken from the library's own stream-ordered memory
 *    pool (cudaMallocFromPoolAsync / cudaFreeAsync on that same stream; the
 *    pool keeps freed memory reserved until etl_trim, and never makes one
 *    stream wait on another to reuse it); while the stream is being captured
 *    into a CUDA graph, the default pool's graph allocations are used. The
 *    _ws variants (end of this header) take that memory from a caller-owned
 *    buffer instead and allocate nothing.
 *  - The return value reports what the host can see at call time: ETL_EINVAL
 *    for bad sizes or null pointers (nothing is enqueued then), ETL_ENOMEM /
 *    ETL_ECUDA for a failed allocation or launch. Errors in the DATA (a parent
 *    array that is not one tree, an id out of range, an exhausted iteration
 *    cap) are only known on the device: they are written as an etl_status code
 *    into a device int32 "status word" (first error wins; 0 = ok) and the
 *    affected outputs are set to -1 (LCA) or 0 (bridge mask). Every device loop
 *    whose trip count depends on the data has a cap, so no input makes a
 *    kernel spin.
 *  - Concurrency: calls on different streams may overlap; a preprocessed LCA
 *    handle is read-only for queries, so queries on several streams may run
 *    at once.
 */
#ifndef ETL_H
#define ETL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum etl_status {
    ETL_OK = 0,
    ETL_EINVAL = 1,     /* bad argument seen on the host; nothing enqueued */
    ETL_ENOMEM = 2,     /* device allocation failed */
    ETL_ECUDA = 3,      /* a CUDA call or launch failed */
    ETL_EBADTREE = 4,   /* parent array is not exactly one rooted tree on all n nodes */
    ETL_EBADQUERY = 5,  /* a query id outside [0, n) */
    ETL_EBADGRAPH = 6,  /* an edge endpoint outside [0, n) */
    ETL_ETIMEOUT = 7    /* a capped device loop ran out (malformed or adversarial input) */
} etl_status;

/* Human-readable name of a status code (static string). */
const char *etl_status_string(int32_t status);

/* ------------------------------------------------------------------ list ranking
 * List ranking (Sec. 2.2, "Using an Euler Tour on GPU"): for a singly linked
 * list stored as succ[0..len) (succ[e] = next element, -1 at the tail) that
 * starts at element `head`, writes rank[e] = distance of e from the head
 * (rank[head] = 0). All len elements must lie on the one list; otherwise
 * `status` (device int32, may be NULL) receives ETL_EBADTREE and the ranks of
 * the unreachable elements are unspecified. This is the ruling-set ranker
 * that the tree and bridge paths use internally, exposed for reuse.
 * len in [1, 2^31 - 2]; head in [0, len).
 */
etl_status etl_list_rank(const int32_t *succ, int64_t len, int32_t head, int32_t *rank, int32_t *status,
                         void *stream);

/*
 * etl_list_rank_static: the same result as etl_list_rank for lists of at most
 * 262,144 (2^18) elements, computed WITHOUT allocating any device memory.
 * The paper has no counterpart: this entry point serves callers that cannot
 * allocate at the point of the call -- code running under a memory manager
 * that owns the whole device, code that must not wait on the allocator, code
 * with a fixed memory plan. The caller still passes succ, rank and (optional)
 * status. All scratch lives in one fixed 3 MiB __device__ array inside the
 * library, which every GPU that loads the library holds until the process
 * exits. Rules:
 *  - len > 2^18 returns ETL_EINVAL and enqueues nothing;
 *  - every call shares that array and it keeps the last call's contents (the
 *    call clears what must start at zero); calls whose work overlaps on the
 *    GPU (other streams, other host threads) race and produce wrong ranks, so
 *    serialise them;
 *  - the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it, so make
 *    that first call before any stream capture on the device. The cache also
 *    holds the id of the CUDA context the address belongs to: after a
 *    cudaDeviceReset the next call looks the address up again (make it, too,
 *    outside any stream capture).
 */
etl_status etl_list_rank_static(const int32_t *succ, int64_t len, int32_t head, int32_t *rank, int32_t *status,
                                void *stream);

/* ------------------------------------------------------------------ LCA
 * Lowest common ancestors (Sec. 3): preprocessing builds the Euler tour of the
 * tree (Sec. 2.1, successor = next(twin)), ranks it once (Sec. 2.2), derives
 * preorder, depth and subtree size from the ranks, and builds a range-minimum
 * table over the preorder sequence (the RMQ reduction of Sec. 3.1): a blocked
 * two-level table by default, else a full sparse table (ETL_TUNE_RMQ_BLOCKED).
 * A query is then answered in O(1) with a few table reads.
 *
 * Opaque handle; it owns the device arrays of one preprocessed tree.
 */
typedef struct etl_lca_s *etl_lca_t;

/*
 * lca_preprocess: parent[0..n) with parent[root] = -1 and every other entry in
 * [0, n) describes one rooted tree (the input format of Sec. 3.2). n in
 * [1, 2^30 - 1]. On success *out receives a new handle (host memory, owned by the
 * caller until lca_free). The handle's tables are being built asynchronously
 * on `stream`; queries enqueued on the same stream see them, queries on
 * another stream must wait for it (event or synchronisation). Data errors go
 * to the handle's status word (see lca_status). Children are visited in
 * ascending label order, so the preorder numbering is unique.
 */
etl_status lca_preprocess(const int32_t *parent, int32_t n, void *stream, etl_lca_t *out);

/*
 * lca_preprocess_ex: as lca_preprocess, choosing which query structures to
 * build: ETL_LCA_RMQ (the range-minimum table, for lca_query) and/or
 * ETL_LCA_INLABEL (the Inlabel records, for lca_query_inlabel; the paper's
 * GPU method, O(n) memory) and/or ETL_LCA_TOUR_RMQ (range minimum over the
 * depth-annotated Euler tour, the classical LCA-to-RMQ reduction of Sec. 3.1,
 * for lca_query_tour: a blocked table of 64-bit keys over 2n tour positions).
 * Unknown bits or no bit: ETL_EINVAL.
 */
enum { ETL_LCA_RMQ = 1, ETL_LCA_INLABEL = 2, ETL_LCA_TOUR_RMQ = 4 };
etl_status lca_preprocess_ex(const int32_t *parent, int32_t n, int32_t flags, void *stream, etl_lca_t *out);

/*
 * lca_query: out[i] = LCA(u[i], v[i]) for i in [0, q), for the tree of h
 * (built with the RMQ structure: lca_preprocess, or lca_preprocess_ex with
 * ETL_LCA_RMQ)
 * (Sec. 3, problem statement: the deepest node that is an ancestor of both,
 * a node being its own ancestor). Ids outside [0, n) give out[i] = -1 and
 * ETL_EBADQUERY in *status (device int32, may be NULL; written only on error,
 * never cleared, so several query calls may share it). If the handle holds a
 * malformed tree every answer is -1. q in [0, 2^40]; u, v, out may not alias.
 */
etl_status lca_query(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                     int32_t *status, void *stream);

/*
 * lca_preprocess_batch: k independent trees preprocessed together (one
 * launch sequence for all of them). parent[0..total_n) is the concatenation of
 * the trees' parent arrays in LOCAL ids: tree i owns entries node_off[i] ..
 * node_off[i+1]-1, its nodes are numbered 0 .. size-1 and its root has -1.
 * node_off is a DEVICE int32[k+1] array with node_off[0] = 0, node_off[k] =
 * total_n and every tree non-empty (else ETL_EINVAL in the status word).
 * max_n (host) must be >= the largest tree's size; it sizes the range-minimum table.
 * The trees' Euler tours are chained into one list and ranked once; tree i
 * then occupies preorder positions node_off[i] .. node_off[i+1]-1, so
 * lca_arrays / lca_export return GLOBAL preorder numbers (pre - node_off[i]
 * is the preorder inside tree i; depth and size are per tree). k >= 1,
 * total_n in [k, 2^30 - 1].
 */
etl_status lca_preprocess_batch(const int32_t *parent, const int32_t *node_off, int32_t k, int32_t total_n,
                                int32_t max_n, void *stream, etl_lca_t *out);

/*
 * lca_query_batch: for a handle from lca_preprocess_batch, out[i] =
 * LCA(u[i], v[i]) in tree inst[i], with u, v and the answer in that tree's
 * LOCAL ids. inst, u, v, out are device int32[q]; queries of different trees
 * may be mixed in any order. A tree index outside [0, k) or an id outside the
 * tree gives -1 and ETL_EBADQUERY in *status (device, may be NULL, never
 * cleared). lca_query on a batch handle (and this call on a single-tree
 * handle) returns ETL_EINVAL.
 */
etl_status lca_query_batch(etl_lca_t h, const int32_t *inst, const int32_t *u, const int32_t *v, int64_t q,
                           int32_t *out, int32_t *status, void *stream);

/*
 * lca_build_inlabel: adds the Inlabel (Schieber-Vishkin) structures to a
 * single-tree handle -- the paper's GPU LCA method (Sec. 3.1, "The Inlabel
 * Algorithm") -- from the handle's preorder, size and depth and the same
 * parent array the handle was built from (device, int32[n]; must still hold
 * the same values). O(n) extra memory (24 bytes per node). ETL_EINVAL for a
 * batch handle.
 * lca_query_inlabel: out[i] = LCA(u[i], v[i]) by the Inlabel method (same
 * results and error rules as lca_query); needs lca_build_inlabel first.
 */
etl_status lca_build_inlabel(etl_lca_t h, const int32_t *parent, void *stream);
etl_status lca_query_inlabel(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                             int32_t *status, void *stream);

/*
 * lca_query_tour: out[i] = LCA(u[i], v[i]) by range minimum over the Euler
 * tour (Sec. 3.1): entry r of the tour holds depth << 32 | node of the node
 * the tour is at after bracket r, and the minimum over the positions of the
 * two opening brackets names the LCA. Same results and error rules as
 * lca_query; the handle must come from lca_preprocess_ex with
 * ETL_LCA_TOUR_RMQ (ETL_EINVAL otherwise, and for batch handles). Arrays are
 * device pointers owned by the caller, enqueued on `stream`.
 */
etl_status lca_query_tour(etl_lca_t h, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                          int32_t *status, void *stream);

/*
 * The naive GPU LCA the paper compares against (Sec. 3.1, "The Naive
 * Algorithm"; Martins et al.). lca_naive_preprocess computes every node's
 * level by pointer jumping (five jumps per global synchronisation) and writes
 * rec[2v] = parent(v), rec[2v+1] = level(v) (device int32[2n], caller-owned).
 * lca_naive_query answers each query by climbing: the deeper end up to the
 * other's level, then both ends together -- O(distance) work per query, so
 * slow on deep trees (that is the point of the comparison). Parent arrays
 * that are not one tree give ETL_EBADTREE in *status (device, may be NULL;
 * preprocessing zeroes it first when given); a climb longer than 2n steps
 * gives ETL_ETIMEOUT and -1. Same id rules as lca_query.
 */
etl_status lca_naive_preprocess(const int32_t *parent, int32_t n, int32_t *rec, int32_t *status, void *stream);
etl_status lca_naive_query(const int32_t *rec, int32_t n, const int32_t *u, const int32_t *v, int64_t q,
                           int32_t *out, int32_t *status, void *stream);

/*
 * lca_status: waits for the stream the handle was built on, then writes the
 * handle's data status (an etl_status code, 0 = the tree was valid) to the
 * HOST int32 *status. Synchronising.
 */
etl_status lca_status(etl_lca_t h, int32_t *status);

/*
 * lca_arrays: device pointers (owned by the handle, valid until lca_free) to
 * the per-node results of preprocessing, each int32[n]: pre (preorder number,
 * root 0, children in ascending label order), depth (root 0), size (nodes in
 * the subtree), order (order[pre[v]] = v). Any output pointer may be NULL.
 */
etl_status lca_arrays(etl_lca_t h, const int32_t **pre, const int32_t **depth, const int32_t **size,
                      const int32_t **order);

/*
 * lca_export: copies (device to device, on `stream`, ordered after the
 * handle's own stream only if it is the same stream) the per-node arrays of
 * lca_arrays into caller-owned int32[n] device arrays; any may be NULL.
 */
etl_status lca_export(etl_lca_t h, int32_t *pre, int32_t *depth, int32_t *size, int32_t *order, void *stream);

/* lca_free: releases the handle and its device memory (stream-ordered on the
 * handle's stream, which must still exist). NULL is accepted. */
etl_status lca_free(etl_lca_t h);

/* ------------------------------------------------------------------ bridges
 * find_bridges: Tarjan-Vishkin bridge finding (Sec. 4.1). edges[0..2m) holds
 * m undirected edges as (u0, v0, u1, v1, ...), ids in [0, n); self-loops and
 * parallel edges are allowed and the graph may be disconnected. Writes
 * is_bridge[e] = 1 if deleting edge e increases the number of connected
 * components, else 0. Phases: a spanning forest from a hook-and-compress
 * connected-components pass (an edge whose hook succeeds is a forest edge),
 * the Euler tour of that forest, per-vertex minimum / maximum over non-forest
 * neighbours, subtree low / high by range-minimum / -maximum queries over the
 * tour, and the test: forest edge {u, parent(u)} is a bridge iff no
 * non-forest edge leaves the subtree of u. Endpoints out of range give
 * ETL_EBADGRAPH in *status (device int32, may be NULL; the call first sets it
 * to 0) and an all-zero mask.
 * n in [1, 2^30 - 1] (the forest tour of 2(n - 1) half-edges plus a head stays within
 * the list ranker's 2^31 - 2 elements), m in [0, 2^31 - 2].
 */
etl_status find_bridges(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge, int32_t *status,
                        void *stream);

/* ------------------------------------------------------------------ tuning knobs
 * Launch parameters that do not change any result, exposed for the autotuner
 * (paper_2103_15217_gb300/tune.py). Process-wide; set them between calls,
 * not while calls are being enqueued from another thread.
 *   ETL_TUNE_RANK_K0_LOG2   level-0 splitter density of the list ranker: one
 *                           splitter per 2^k elements, k in [1, 8] (default 5),
 *                           for lists of more than 2^22 elements; shorter
 *                           lists (bound by the latency of their longest
 *                           sublist) take one in 4 up to 2^15 elements, one in
 *                           8 up to 2^20, one in 16 up to 2^22, or this value
 *                           where it is denser
 *   ETL_TUNE_RANK_K_LOG2    density at the upper ranking levels, [1, 8] (3)
 *   ETL_TUNE_RANK_BLOCK     threads per block of the walk kernels, one of
 *                           64, 128, 256, 512, 1024 (128)
 *   ETL_TUNE_RANK_BLOCKS_PER_SM  resident walk blocks per SM, block * value
 *                           <= 2048 (4)
 *   ETL_TUNE_RMQ_LEVELS_PER_PASS sparse-table levels built per streaming
 *                           pass, 1..3 (3)
 *   ETL_TUNE_RMQ_BLOCK      threads per block of the sparse-table build,
 *                           128, 256, 512 or 1024 (256)
 *   ETL_TUNE_CC_FIRST_SLICE edges hooked before the first compression of the
 *                           connected-components pass, in units of n/4,
 *                           1..64 (2, i.e. n/2 edges: a random sample of that
 *                           size is still below the giant-component threshold)
 *   ETL_TUNE_RMQ_BLOCKED    1: range-min / max tables are blocked two-level
 *                           tables (prefix / suffix results inside blocks of
 *                           32 entries plus a sparse table over the blocks,
 *                           O(n) memory); 0: full sparse tables (n log n
 *                           entries). Both answer every query exactly. (1)
 *                           Read when a handle or a bridge call is built.
 *   ETL_TUNE_SORT_ROUNDS    32-element rounds per warp in the radix-sort
 *                           passes that group children by parent: tiles of
 *                           256 * value elements, value 8 or 16 (8)
 *   ETL_TUNE_CC_DOUBLING    1: after the first slice the connected-components
 *                           pass hooks the edges in slices that double in
 *                           size, compressing the forest before each; 0: the
 *                           rest in one launch (0)
 *   ETL_TUNE_CC_GIANT       1: after each compression the most frequent root
 *                           of a sample (the giant component's) outranks all
 *                           others when roots are hooked, so it never moves;
 *                           0: plain smaller-id order (1)
 *   ETL_TUNE_SORT_BALLOT    1: the radix scatter finds the lanes holding the
 *                           same digit with eight warp ballots; 0: with
 *                           __match_any_sync (1)
 *   ETL_TUNE_PDL            1: the library's kernels are launched with
 *                           programmatic dependent launch, so each one is
 *                           scheduled while the kernel before it on the
 *                           stream finishes, and waits for its results on the
 *                           device (CUDA-graph captures keep the overlap); 0:
 *                           plain stream order (1)
 * Unknown keys or out-of-range values return ETL_EINVAL.
 */
enum {
    ETL_TUNE_RANK_K0_LOG2 = 1,
    ETL_TUNE_RANK_K_LOG2 = 2,
    ETL_TUNE_RANK_BLOCK = 3,
    ETL_TUNE_RANK_BLOCKS_PER_SM = 4,
    ETL_TUNE_RMQ_LEVELS_PER_PASS = 5,
    ETL_TUNE_RMQ_BLOCK = 6,
    ETL_TUNE_CC_FIRST_SLICE = 7,
    ETL_TUNE_RMQ_BLOCKED = 8,
    ETL_TUNE_SORT_ROUNDS = 9,
    ETL_TUNE_CC_DOUBLING = 10,
    ETL_TUNE_CC_GIANT = 11,
    ETL_TUNE_SORT_BALLOT = 12,
    ETL_TUNE_PDL = 13
};
etl_status etl_tune_set(int32_t key, int32_t value);
etl_status etl_tune_get(int32_t key, int32_t *value);

/* ------------------------------------------------------------------ phase timers
 * Opt-in device timing of the library's own launch groups (not part of the
 * method; used by the benchmark). When enabled, each launch group is
 * bracketed by two CUDA events on its stream (skipped while the stream is
 * being captured into a graph). etl_profile_count / etl_profile_get wait for
 * the recorded events and aggregate per phase name: total milliseconds and
 * number of launches. Process-wide; thread-safe.
 */
etl_status etl_profile_enable(int32_t on);
etl_status etl_profile_reset(void);
etl_status etl_profile_count(int32_t *count);
etl_status etl_profile_get(int32_t i, char *name, int32_t name_len, double *total_ms, int64_t *launches);
/* Release the device memory the library keeps reserved in its own stream-ordered memory pools
 * (freed buffers stay reserved for reuse until this call). Synchronous with respect to the pools. */
etl_status etl_trim(void);
/* Bytes the library's memory pool of the current device holds reserved (mapped) and in use; 0 and
 * 0 before its first allocation. ETL_EINVAL for null pointers. */
etl_status etl_pool_stats(int64_t *reserved, int64_t *used);
/* Number of kernels this process has launched through the library so far (host-side counter). */
etl_status etl_launch_count(int64_t *count);
/*
 * Measurement aid (not part of the method): the memory access pattern of one
 * step of the list-ranking walk of Sec. 2.2 -- read succ[j] at a random index
 * j, write an 8-byte record out[j] = (succ[j], i) at the same index -- for
 * j = order[i], i in [0, n), with every gather independent (no chain of
 * dependent loads). order is a DEVICE int32[n] permutation of [0, n) (entries
 * outside it are skipped), succ DEVICE int32[n], out DEVICE 8-byte records[n].
 * Its rate is the ceiling of a walk over a list in random order, against which
 * the benchmark reports the walk. n in [1, 2^31 - 1].
 */
etl_status etl_probe_gather_scatter(const int32_t *order, const int32_t *succ, int64_t n, void *out, void *stream);

/*
 * find_bridges_batch: k independent graphs in one launch sequence.
 * edges[0..2*total_m) is the concatenation of the graphs' edge lists in LOCAL
 * node ids; graph i owns edges edge_off[i] .. edge_off[i+1]-1 and nodes
 * 0 .. node_off[i+1]-node_off[i]-1. edge_off and node_off are DEVICE
 * int32[k+1] arrays, non-decreasing from 0 to total_m / total_n, every graph
 * with at least one node (else ETL_EINVAL in the status word). Writes
 * is_bridge[e] for every edge of every graph, the same as find_bridges on
 * that graph alone. The disjoint union is processed as one graph: bridges of
 * a disjoint union are the bridges of its parts. total_n in [k, 2^30 - 1],
 * total_m in [0, 2^31 - 2].
 */
etl_status find_bridges_batch(const int32_t *edges, const int32_t *edge_off, const int32_t *node_off, int32_t k,
                              int64_t total_m, int32_t total_n, uint8_t *is_bridge, int32_t *status, void *stream);

/*
 * find_bridges_hybrid: the hybrid the paper proposes (Sec. 4.3): the same
 * connected-components spanning forest and Euler tour as find_bridges, used
 * only for parents and levels, followed by Chaitanya-Kothapalli marking --
 * every non-tree edge walks both ends up to their LCA and marks the tree
 * edges it passes; tree edges left unmarked are bridges. Same results and
 * rules as find_bridges; work grows with the tree distance between the ends
 * of each non-tree edge (a walk longer than 2n steps sets ETL_ETIMEOUT).
 */
etl_status find_bridges_hybrid(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge, int32_t *status,
                               void *stream);

/*
 * two_edge_cc: 2-edge-connected components, by the decomposition Sec. 4
 * describes: find all bridges (find_bridges), delete them, and take the
 * connected components of the rest (the same hook-and-compress pass).
 * label[v] (device int32[n]) = the smallest vertex of v's component.
 * Same input rules as find_bridges; on a data error every label is -1 and
 * *status (device, may be NULL; zeroed first) holds the code.
 */
etl_status two_edge_cc(const int32_t *edges, int64_t m, int32_t n, int32_t *label, int32_t *status, void *stream);

/* ------------------------------------------------------------------ caller-owned workspaces
 * The problem statements of Sec. 3 (LCA: preprocess a tree, then answer
 * queries) and Sec. 4.1 (bridges of a graph) need scratch memory on the way:
 * the tour's successor array, the ranking's sublist records, sort buffers and
 * so on. The plain entry points take it from the library's memory pool. The
 * _ws variants below take ALL of it from one device buffer the caller owns
 * and allocate nothing, so a caller with a fixed memory plan, or one that
 * captures the calls into a CUDA graph and wants no graph memory nodes, can
 * size and place every byte itself.
 *
 * etl_workspace_size: *bytes = the size of the buffer a _ws call of this kind
 * and these sizes needs, for the tuning parameters in force (query it again
 * after etl_tune_set). It is exact: the library runs the same entry point once
 * with a counting arena on a private stream whose work is captured into a CUDA
 * graph and discarded unlaunched (nothing runs on the device and nothing is
 * allocated on it). Call it outside any stream capture on this thread.
 *   kind                      n            m_or_q
 *   ETL_WS_LIST_RANK          len          (unused)
 *   ETL_WS_LCA_PREPROCESS     n            (unused)   includes the handle's tables
 *   ETL_WS_LCA_QUERY          n            q          always 0: lca_query,
 *                                                     lca_query_batch need no scratch
 *   ETL_WS_FIND_BRIDGES       n            m
 * etl_workspace_size_batch: the same for lca_preprocess_batch_ws
 * (ETL_WS_LCA_PREPROCESS: third argument = max_n) and find_bridges_batch_ws
 * (ETL_WS_FIND_BRIDGES: third argument = total_m), k instances, total_n nodes.
 * Sizes outside an entry point's limits, or an unknown kind: ETL_EINVAL.
 */
enum { ETL_WS_LIST_RANK = 1, ETL_WS_LCA_PREPROCESS = 2, ETL_WS_LCA_QUERY = 3, ETL_WS_FIND_BRIDGES = 4 };
etl_status etl_workspace_size(int32_t kind, int64_t n, int64_t m_or_q, size_t *bytes);
etl_status etl_workspace_size_batch(int32_t kind, int32_t k, int64_t total_n, int64_t max_n_or_total_m,
                                    size_t *bytes);

/*
 * The _ws variants: the same arguments, results and error rules as the entry
 * point without the suffix, plus ws (DEVICE memory owned by the caller, any
 * alignment) and ws_bytes. They call no allocator (cudaMalloc*, memory pools,
 * graph memory nodes): every byte the call needs comes from ws, so they can be
 * captured into a CUDA graph without adding memory nodes to it.
 *  - ws_bytes >= etl_workspace_size(...) for the same sizes; a smaller buffer
 *    returns ETL_ENOMEM, possibly after part of the work was enqueued into ws
 *    (the outputs are then unspecified). ws == NULL: ETL_EINVAL.
 *  - ws belongs to the call until its work on `stream` has finished; the
 *    caller may then reuse it -- except for lca_preprocess_ws /
 *    lca_preprocess_batch_ws, whose handle keeps its tables inside ws: keep ws
 *    alive and unmodified until lca_free(h) (which then frees only the host
 *    side of the handle). Such a handle takes no further structures
 *    (lca_build_inlabel returns ETL_EINVAL).
 *  - Two calls that use the same ws at the same time on the GPU race.
 */
etl_status etl_list_rank_ws(const int32_t *succ, int64_t len, int32_t head, int32_t *rank, int32_t *status,
                            void *ws, size_t ws_bytes, void *stream);
etl_status lca_preprocess_ws(const int32_t *parent, int32_t n, void *ws, size_t ws_bytes, void *stream,
                             etl_lca_t *out);
etl_status lca_preprocess_batch_ws(const int32_t *parent, const int32_t *node_off, int32_t k, int32_t total_n,
                                   int32_t max_n, void *ws, size_t ws_bytes, void *stream, etl_lca_t *out);
etl_status find_bridges_ws(const int32_t *edges, int64_t m, int32_t n, uint8_t *is_bridge, int32_t *status,
                           void *ws, size_t ws_bytes, void *stream);
etl_status find_bridges_batch_ws(const int32_t *edges, const int32_t *edge_off, const int32_t *node_off, int32_t k,
                                 int64_t total_m, int32_t total_n, uint8_t *is_bridge, int32_t *status, void *ws,
                                 size_t ws_bytes, void *stream);

/*
 * etl_status_get: waits for `stream`, then copies the device status word
 * *d_status (the data-error word a call on that stream wrote: 0 or an
 * etl_status code) to the HOST int32 *h_status. Synchronising; not for use
 * while `stream` is being captured.
 */
etl_status etl_status_get(void *stream, const int32_t *d_status, int32_t *h_status);

/* Number of device allocations the library has requested so far in this
 * process (pool or graph allocations; carving from a caller's workspace does
 * not count). Host-side counter. */
etl_status etl_alloc_count(int64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* ETL_H */
