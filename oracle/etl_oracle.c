/*
 * CPU oracle for the Euler-tour path of "Euler Meets GPU" (arXiv 2103.15217).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library calls this file; only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every routine is a plain, single-threaded restatement of a definition or of
 * a classical sequential algorithm, written for readability, not speed:
 *
 *   oracle_tree_tour     Euler tour of a rooted tree by iterative DFS, and the
 *                        preorder / depth / subtree size it defines (Sec. 2).
 *   oracle_dcel_tour     the paper's DCEL construction from an edge list:
 *                        arrays A and B, first[], next, twin, succ = next(twin),
 *                        list split at an arc leaving the root (Sec. 2.1).
 *   oracle_lca_climb     LCA by lifting the deeper node, then both (Sec. 3.1,
 *                        "The Naive Algorithm"), which is the LCA definition.
 *   oracle_lca_offline   Tarjan's offline union-find LCA (classical, exact).
 *   oracle_bridges_dfs   sequential bridge finding with a DFS tree and the low
 *                        function: bridge iff low(u) >= pre(u) (Sec. 4.1).
 *   oracle_bridges_tv    Tarjan-Vishkin criterion with an arbitrary spanning
 *                        forest: low and high over each subtree (Sec. 4.1).
 *   oracle_two_edge_cc   2-edge-connected components: delete the bridges,
 *                        take connected components (Sec. 4).
 *
 * Conventions: parent[root] = -1; node ids in [0, n); arcs of a rooted tree are
 * numbered 2v (the arc entering v from its parent, "down", an opening bracket)
 * and 2v+1 (the arc leaving v back to its parent, "up", a closing bracket);
 * the root gets a virtual opening and closing bracket at the two ends of the
 * tour, so the tour has 2n entries. Children are visited in ascending label
 * order. Return value 0 = ok, otherwise an error code (see etl_oracle_status).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EBADTREE = 4, OR_EBADQUERY = 5, OR_EBADGRAPH = 6 };

/* children of every node, ascending by label (counting sort by parent, stable) */
static int children_csr(int32_t n, const int32_t *parent, int32_t *root_out, int64_t **off_out,
                        int32_t **kids_out) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *kids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n - 1 : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!off || !kids || !fill) { free(off); free(kids); free(fill); return OR_ENOMEM; }
    int32_t root = -1, roots = 0;
    for (int32_t v = 0; v < n; ++v) {
        int32_t p = parent[v];
        if (p == -1) { root = v; ++roots; continue; }
        if (p < 0 || p >= n || p == v) { free(off); free(kids); free(fill); return OR_EBADTREE; }
        off[p + 1]++;
    }
    if (roots != 1) { free(off); free(kids); free(fill); return OR_EBADTREE; }
    for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    for (int32_t v = 0; v < n; ++v) fill[v] = off[v];
    for (int32_t c = 0; c < n; ++c)
        if (parent[c] >= 0) kids[fill[parent[c]]++] = c;
    free(fill);
    *root_out = root;
    *off_out = off;
    *kids_out = kids;
    return OR_OK;
}

/*
 * Euler tour of the rooted tree given by parent[] (Sec. 2): the list of
 * directed half-edges in DFS order. pre = order of first visit, depth =
 * distance from the root, size = number of nodes in the subtree. tour (may be
 * NULL) receives the 2n bracket ids in tour order. Fails with OR_EBADTREE if
 * parent[] is not one rooted tree on all n nodes.
 */
int oracle_tree_tour(int32_t n, const int32_t *parent, int32_t *pre, int32_t *depth, int32_t *size,
                     int32_t *tour) {
    if (n < 1 || !parent || !pre || !depth || !size) return OR_EINVAL;
    int32_t root;
    int64_t *off;
    int32_t *kids;
    int rc = children_csr(n, parent, &root, &off, &kids);
    if (rc) return rc;
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!stack || !cursor) { free(off); free(kids); free(stack); free(cursor); return OR_ENOMEM; }
    for (int32_t v = 0; v < n; ++v) { pre[v] = -1; cursor[v] = off[v]; }
    int64_t sp = 0, pos = 0;
    int32_t visited = 0;
    stack[sp++] = root;
    pre[root] = visited++;
    depth[root] = 0;
    if (tour) tour[pos++] = 2 * root;
    while (sp > 0) {
        int32_t v = stack[sp - 1];
        if (cursor[v] < off[v + 1]) {
            int32_t c = kids[cursor[v]++];
            pre[c] = visited++;
            depth[c] = depth[v] + 1;
            if (tour) tour[pos++] = 2 * c;
            stack[sp++] = c;
        } else {
            --sp;
            size[v] = visited - pre[v];
            if (tour) tour[pos++] = 2 * v + 1;
        }
    }
    free(stack); free(cursor); free(off); free(kids);
    return visited == n ? OR_OK : OR_EBADTREE; /* a cycle leaves nodes unreached */
}

/*
 * The paper's DCEL construction (Sec. 2.1, Fig. 2) for a tree given as k
 * undirected edges. A holds the half-edges of edge i at 2i = (x,y) and
 * 2i+1 = (y,x), so twin(a) = a xor 1. B is A sorted lexicographically, with
 * posB[a] the position of half-edge a in B. next(a) is the following entry of
 * B if it starts at the same node, else the first entry of B starting there
 * (first[x]). succ(a) = next(twin(a)). The cyclic list is cut in front of
 * first[root], which becomes the head. Outputs succ[2k] (head's predecessor
 * gets -1) and the tour as half-edge ids in list order (2k entries).
 */
static const int32_t *g_arcs; /* qsort comparator context (single-threaded oracle) */
static int cmp_arc(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    int32_t ax = g_arcs[2 * a], ay = g_arcs[2 * a + 1], bx = g_arcs[2 * b], by = g_arcs[2 * b + 1];
    if (ax != bx) return ax < bx ? -1 : 1;
    if (ay != by) return ay < by ? -1 : 1;
    return a < b ? -1 : (a > b);
}

int oracle_dcel_tour(int32_t n, int64_t k, const int32_t *edges, int32_t root, int32_t *succ, int32_t *tour,
                     int32_t *B_out /* 2k, may be NULL */) {
    if (n < 1 || k < 0 || (k > 0 && (!edges || !succ || !tour)) || root < 0 || root >= n) return OR_EINVAL;
    if (k == 0) return OR_OK;
    int64_t na = 2 * k;
    int32_t *arcs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * na)); /* (src, dst) per half-edge */
    int64_t *B = (int64_t *)malloc(sizeof(int64_t) * (size_t)na);
    int64_t *posB = (int64_t *)malloc(sizeof(int64_t) * (size_t)na);
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!arcs || !B || !posB || !first) { free(arcs); free(B); free(posB); free(first); return OR_ENOMEM; }
    for (int64_t i = 0; i < k; ++i) {
        int32_t x = edges[2 * i], y = edges[2 * i + 1];
        if (x < 0 || x >= n || y < 0 || y >= n) { free(arcs); free(B); free(posB); free(first); return OR_EBADGRAPH; }
        arcs[4 * i + 0] = x; arcs[4 * i + 1] = y;     /* A[2i]   = (x, y) */
        arcs[4 * i + 2] = y; arcs[4 * i + 3] = x;     /* A[2i+1] = (y, x) */
    }
    for (int64_t a = 0; a < na; ++a) B[a] = a;
    g_arcs = arcs;
    qsort(B, (size_t)na, sizeof(int64_t), cmp_arc);
    for (int32_t x = 0; x < n; ++x) first[x] = -1;
    for (int64_t i = 0; i < na; ++i) {
        posB[B[i]] = i;
        int32_t x = arcs[2 * B[i]];
        if (first[x] < 0) first[x] = i;
        if (B_out) B_out[i] = (int32_t)B[i];
    }
    for (int64_t a = 0; a < na; ++a) {
        int64_t t = a ^ 1;                 /* twin(a) */
        int64_t i = posB[t];               /* next(t): following entry of B, or wrap to first[src] */
        int32_t x = arcs[2 * t];
        int64_t nx = (i + 1 < na && arcs[2 * B[i + 1]] == x) ? B[i + 1] : B[first[x]];
        succ[a] = (int32_t)nx;
    }
    if (first[root] < 0) { free(arcs); free(B); free(posB); free(first); return OR_EBADTREE; }
    int64_t head = B[first[root]];
    for (int64_t a = 0; a < na; ++a)
        if (succ[a] == head) succ[a] = -1; /* cut the cyclic list in front of the head */
    int64_t pos = 0;
    for (int64_t a = head; a >= 0 && pos < na; a = succ[a]) tour[pos++] = (int32_t)a;
    free(arcs); free(B); free(posB); free(first);
    return pos == na ? OR_OK : OR_EBADTREE;
}

/*
 * LCA by climbing (Sec. 3.1): lift the deeper endpoint until both are at the
 * same depth, then lift both until they meet. depth[] must be the true depths
 * (e.g. from oracle_tree_tour). Out-of-range queries give -1 and OR_EBADQUERY.
 */
int oracle_lca_climb(int32_t n, const int32_t *parent, const int32_t *depth, int64_t q, const int32_t *u,
                     const int32_t *v, int32_t *out) {
    if (n < 1 || q < 0 || !parent || !depth || (q > 0 && (!u || !v || !out))) return OR_EINVAL;
    int rc = OR_OK;
    for (int64_t i = 0; i < q; ++i) {
        int32_t a = u[i], b = v[i];
        if (a < 0 || a >= n || b < 0 || b >= n) { out[i] = -1; rc = OR_EBADQUERY; continue; }
        while (depth[a] > depth[b]) a = parent[a];
        while (depth[b] > depth[a]) b = parent[b];
        while (a != b) { a = parent[a]; b = parent[b]; }
        out[i] = a;
    }
    return rc;
}

/* union-find with path compression and union by size, for the offline LCA */
static int32_t uf_find(int32_t *uf, int32_t x) {
    int32_t r = x;
    while (uf[r] != r) r = uf[r];
    while (uf[x] != r) { int32_t nx = uf[x]; uf[x] = r; x = nx; }
    return r;
}

/*
 * Tarjan's offline LCA: a DFS that, when it finishes node x, answers every
 * query (x, y) whose other end y is already finished with the current
 * "ancestor" label of y's union-find set. Exact for any tree; O((n+q) alpha).
 */
int oracle_lca_offline(int32_t n, const int32_t *parent, int64_t q, const int32_t *u, const int32_t *v,
                       int32_t *out) {
    if (n < 1 || q < 0 || !parent || (q > 0 && (!u || !v || !out))) return OR_EINVAL;
    int32_t root;
    int64_t *off;
    int32_t *kids;
    int rc = children_csr(n, parent, &root, &off, &kids);
    if (rc) return rc;
    int64_t *qoff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *qlist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * q + 1));
    int64_t *qfill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *uf = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sz = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!qoff || !qlist || !qfill || !uf || !sz || !anc || !done || !stack || !cursor) { rc = OR_ENOMEM; goto out; }
    for (int64_t i = 0; i < q; ++i) {
        int32_t a = u[i], b = v[i];
        if (a < 0 || a >= n || b < 0 || b >= n) { out[i] = -1; rc = OR_EBADQUERY; continue; }
        qoff[a + 1]++;
        if (b != a) qoff[b + 1]++;
    }
    for (int32_t x = 0; x < n; ++x) qoff[x + 1] += qoff[x];
    for (int32_t x = 0; x < n; ++x) qfill[x] = qoff[x];
    for (int64_t i = 0; i < q; ++i) {
        int32_t a = u[i], b = v[i];
        if (a < 0 || a >= n || b < 0 || b >= n) continue;
        qlist[qfill[a]++] = i;
        if (b != a) qlist[qfill[b]++] = i;
    }
    for (int32_t x = 0; x < n; ++x) { uf[x] = x; sz[x] = 1; anc[x] = x; cursor[x] = off[x]; }
    int64_t sp = 0;
    stack[sp++] = root;
    int32_t finished = 0;
    while (sp > 0) {
        int32_t x = stack[sp - 1];
        if (cursor[x] < off[x + 1]) {
            stack[sp++] = kids[cursor[x]++];
            continue;
        }
        --sp; /* x is finished: answer its queries, then merge it into its parent */
        done[x] = 1;
        ++finished;
        for (int64_t j = qoff[x]; j < qoff[x + 1]; ++j) {
            int64_t i = qlist[j];
            int32_t y = (u[i] == x) ? v[i] : u[i];
            if (done[y]) out[i] = anc[uf_find(uf, y)];
        }
        if (sp > 0) {
            int32_t p = stack[sp - 1];
            int32_t rp = uf_find(uf, p), rx = uf_find(uf, x);
            if (sz[rp] < sz[rx]) { int32_t t = rp; rp = rx; rx = t; }
            uf[rx] = rp;
            sz[rp] += sz[rx];
            anc[rp] = p;
        }
    }
    if (finished != n && rc == OR_OK) rc = OR_EBADTREE;
out:
    free(off); free(kids); free(qoff); free(qlist); free(qfill); free(uf); free(sz); free(anc); free(done);
    free(stack); free(cursor);
    return rc;
}

/* adjacency lists of an undirected multigraph: entry = (neighbour, edge id) */
static int adjacency(int32_t n, int64_t m, const int32_t *edges, int64_t **off_out, int32_t **nbr_out,
                     int64_t **eid_out) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!off || !nbr || !eid || !fill) { free(off); free(nbr); free(eid); free(fill); return OR_ENOMEM; }
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(off); free(nbr); free(eid); free(fill); return OR_EBADGRAPH; }
        off[a + 1]++;
        off[b + 1]++;
    }
    for (int32_t x = 0; x < n; ++x) off[x + 1] += off[x];
    for (int32_t x = 0; x < n; ++x) fill[x] = off[x];
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        nbr[fill[a]] = b; eid[fill[a]++] = e;
        nbr[fill[b]] = a; eid[fill[b]++] = e;
    }
    free(fill);
    *off_out = off; *nbr_out = nbr; *eid_out = eid;
    return OR_OK;
}

/*
 * Sequential bridge finding (Sec. 4.1): a DFS spanning forest (roots taken in
 * ascending label order), preorder numbers pre(), and
 *   low(v) = min( pre(v), pre(w) for every non-tree edge (x, w) with x in the
 *                 subtree of v ),
 * which the DFS accumulates bottom-up. For a DFS tree the tree edge
 * {u, parent(u)} is a bridge iff low(u) >= pre(u); non-tree edges never are.
 * The edge a node was entered by is skipped by its id only, so a parallel copy
 * of a tree edge counts as a non-tree edge.
 */
int oracle_bridges_dfs(int32_t n, int64_t m, const int32_t *edges, uint8_t *is_bridge) {
    if (n < 1 || m < 0 || (m > 0 && (!edges || !is_bridge))) return OR_EINVAL;
    int64_t *off, *eid;
    int32_t *nbr;
    int rc = adjacency(n, m, edges, &off, &nbr, &eid);
    if (rc) return rc;
    int32_t *pre = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *low = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *in_edge = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!pre || !low || !in_edge || !cursor || !stack) { rc = OR_ENOMEM; goto out; }
    for (int64_t e = 0; e < m; ++e) is_bridge[e] = 0;
    for (int32_t x = 0; x < n; ++x) { pre[x] = -1; cursor[x] = off[x]; in_edge[x] = -1; }
    int32_t counter = 0;
    for (int32_t s = 0; s < n; ++s) {
        if (pre[s] >= 0) continue;
        int64_t sp = 0;
        stack[sp++] = s;
        pre[s] = low[s] = counter++;
        while (sp > 0) {
            int32_t x = stack[sp - 1];
            if (cursor[x] < off[x + 1]) {
                int64_t j = cursor[x]++;
                int32_t w = nbr[j];
                if (eid[j] == in_edge[x]) continue; /* the tree edge x was entered by */
                if (pre[w] < 0) {                   /* tree edge: descend */
                    in_edge[w] = eid[j];
                    pre[w] = low[w] = counter++;
                    stack[sp++] = w;
                } else if (pre[w] < low[x]) {       /* non-tree edge */
                    low[x] = pre[w];
                }
                continue;
            }
            --sp; /* x finished */
            if (sp > 0) {
                int32_t p = stack[sp - 1];
                if (low[x] < low[p]) low[p] = low[x];
                is_bridge[in_edge[x]] = (uint8_t)(low[x] >= pre[x]);
            }
        }
    }
out:
    free(off); free(nbr); free(eid); free(pre); free(low); free(in_edge); free(cursor); free(stack);
    return rc;
}

/*
 * Tarjan-Vishkin bridge criterion with an arbitrary spanning forest (Sec. 4.1).
 * tree[e] != 0 marks the forest edges (if tree is NULL the forest is taken by
 * Kruskal over the edges in input order). Each component is rooted at its
 * smallest vertex; pre() and size() come from a DFS over forest edges only.
 * For every vertex x, nlo(x) / nhi(x) are the min / max of pre(x) and of
 * pre(w) over non-forest edges (x, w); low(u) / high(u) are the min / max of
 * nlo / nhi over the subtree of u. The forest edge {u, parent(u)} is a bridge
 * iff low(u) >= pre(u) and high(u) < pre(u) + size(u), i.e. no non-forest edge
 * leaves the subtree interval [pre(u), pre(u) + size(u)). Fails with
 * OR_EBADGRAPH if the marked edges are not a spanning forest.
 */
int oracle_bridges_tv(int32_t n, int64_t m, const int32_t *edges, const uint8_t *tree, uint8_t *is_bridge) {
    if (n < 1 || m < 0 || (m > 0 && (!edges || !is_bridge))) return OR_EINVAL;
    int rc = OR_OK;
    uint8_t *intree = (uint8_t *)calloc((size_t)(m + 1), 1);
    int32_t *uf = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sz = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *tedges = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * n));
    int64_t *tid = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *off = NULL, *eid = NULL;
    int32_t *nbr = NULL;
    int32_t *pre = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *size = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nlo = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nhi = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *in_edge = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!intree || !uf || !sz || !tedges || !tid || !pre || !size || !nlo || !nhi || !in_edge || !cursor || !stack) {
        rc = OR_ENOMEM; goto out;
    }
    for (int32_t x = 0; x < n; ++x) { uf[x] = x; sz[x] = 1; }
    int64_t k = 0; /* forest edges, checked to be acyclic */
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || a >= n || b < 0 || b >= n) { rc = OR_EBADGRAPH; goto out; }
        int want = tree ? (tree[e] != 0) : 1;
        if (!want) continue;
        int32_t ra = uf_find(uf, a), rb = uf_find(uf, b);
        if (ra == rb) {
            if (tree) { rc = OR_EBADGRAPH; goto out; } /* marked edges contain a cycle */
            continue;
        }
        if (sz[ra] < sz[rb]) { int32_t t = ra; ra = rb; rb = t; }
        uf[rb] = ra; sz[ra] += sz[rb];
        intree[e] = 1;
        tedges[2 * k] = a; tedges[2 * k + 1] = b; tid[k] = e;
        ++k;
    }
    for (int64_t e = 0; e < m; ++e) { /* spanning: every edge's ends lie in one forest tree */
        if (uf_find(uf, edges[2 * e]) != uf_find(uf, edges[2 * e + 1])) { rc = OR_EBADGRAPH; goto out; }
    }
    rc = adjacency(n, k, tedges, &off, &nbr, &eid);
    if (rc) goto out;
    for (int32_t x = 0; x < n; ++x) { pre[x] = -1; cursor[x] = off[x]; in_edge[x] = -1; }
    int32_t counter = 0;
    for (int32_t s = 0; s < n; ++s) { /* roots in ascending order = smallest vertex of each component */
        if (pre[s] >= 0) continue;
        int64_t sp = 0;
        stack[sp++] = s;
        pre[s] = counter++;
        while (sp > 0) {
            int32_t x = stack[sp - 1];
            if (cursor[x] < off[x + 1]) {
                int64_t j = cursor[x]++;
                int32_t w = nbr[j];
                if (eid[j] == in_edge[x]) continue;
                in_edge[w] = eid[j];
                pre[w] = counter++;
                stack[sp++] = w;
                continue;
            }
            --sp;
            size[x] = counter - pre[x];
        }
    }
    for (int32_t x = 0; x < n; ++x) nlo[x] = nhi[x] = pre[x];
    for (int64_t e = 0; e < m; ++e) {
        if (intree[e]) continue;
        int32_t a = edges[2 * e], b = edges[2 * e + 1];
        if (pre[b] < nlo[a]) nlo[a] = pre[b];
        if (pre[b] > nhi[a]) nhi[a] = pre[b];
        if (pre[a] < nlo[b]) nlo[b] = pre[a];
        if (pre[a] > nhi[b]) nhi[b] = pre[a];
    }
    /* subtree aggregation: children have larger preorder numbers than their parent */
    {
        int32_t *byPre = stack; /* reuse: node at each preorder position */
        for (int32_t x = 0; x < n; ++x) byPre[pre[x]] = x;
        for (int32_t i = n - 1; i >= 0; --i) {
            int32_t x = byPre[i];
            if (in_edge[x] < 0) continue;
            int64_t te = in_edge[x];
            int32_t p = tedges[2 * te] == x ? tedges[2 * te + 1] : tedges[2 * te];
            if (nlo[x] < nlo[p]) nlo[p] = nlo[x];
            if (nhi[x] > nhi[p]) nhi[p] = nhi[x];
        }
    }
    for (int64_t e = 0; e < m; ++e) is_bridge[e] = 0;
    for (int32_t x = 0; x < n; ++x) {
        if (in_edge[x] < 0) continue; /* component root */
        int32_t lo = nlo[x], hi = nhi[x]; /* now low(x), high(x) */
        is_bridge[tid[in_edge[x]]] = (uint8_t)(lo >= pre[x] && hi < pre[x] + size[x]);
    }
out:
    free(intree); free(uf); free(sz); free(tedges); free(tid); free(off); free(nbr); free(eid); free(pre);
    free(size); free(nlo); free(nhi); free(in_edge); free(cursor); free(stack);
    return rc;
}

/*
 * 2-edge-connected components (Sec. 4, the decomposition the paper describes:
 * find all bridges, delete them, take connected components of what is left).
 * label[v] = the smallest vertex of v's component. Bridges from the DFS
 * method above; components by union-find over the remaining edges.
 */
int oracle_two_edge_cc(int32_t n, int64_t m, const int32_t *edges, int32_t *label) {
    if (n < 1 || m < 0 || !label || (m > 0 && !edges)) return OR_EINVAL;
    uint8_t *br = (uint8_t *)malloc((size_t)(m + 1));
    int32_t *uf = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!br || !uf) { free(br); free(uf); return OR_ENOMEM; }
    int rc = m > 0 ? oracle_bridges_dfs(n, m, edges, br) : OR_OK;
    if (rc) { free(br); free(uf); return rc; }
    for (int32_t x = 0; x < n; ++x) uf[x] = x;
    for (int64_t e = 0; e < m; ++e) {
        if (br[e]) continue;
        int32_t a = uf_find(uf, edges[2 * e]), b = uf_find(uf, edges[2 * e + 1]);
        if (a == b) continue;
        if (a < b) uf[b] = a; else uf[a] = b;  /* the smaller vertex stays the representative */
    }
    for (int32_t x = 0; x < n; ++x) label[x] = uf_find(uf, x);
    free(br); free(uf);
    return OR_OK;
}
