/*
 * CPU oracle for prime paths (PPs) and test paths (TPs).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against; it is compiled and called only by the tests, by the smoke
 * check and by the benchmark's CPU-baseline leg.  It shares no code, header
 * or table with the CUDA library.
 *
 * Definitions followed (paper Sec. 2 and Def. 1, related-work Sec. 7.2):
 *  - A path is a vertex sequence v1..vk (k >= 1) with (vi, vi+1) in E.
 *  - It is SIMPLE iff v1..v(k-1) are pairwise distinct and v2..vk are
 *    pairwise distinct: the only repeat allowed is v1 = vk (a simple cycle;
 *    a self-loop <v, v> is one).
 *  - A PP is a simple path that is not a proper subpath (contiguous proper
 *    subsequence) of any simple path (Def. 1: a maximal simple path).
 *
 * Method (a plain single-threaded enumeration, not the paper's kernel):
 *  1. For every root r in ascending order, a depth-first search over
 *     successors in ascending id order visits every simple path starting at
 *     r exactly once.  A path that closes a cycle is visited and not
 *     extended.
 *  2. A visited path p is a PP iff no one-vertex extension w.p or p.w is a
 *     simple path.  (If p is a proper subpath of a simple q, the window of q
 *     one vertex longer than p that contains p is a contiguous proper window
 *     of a simple sequence, hence simple, and it is such an extension; the
 *     converse is immediate.)
 *  3. The PPs are put in canonical order: lexicographic on int32 sequences,
 *     a proper prefix first.
 *  4. TPs (Problem 1 output; the Ammann-Offutt touring of Sec. 7.3): from a
 *     breadth-first search out of every source a, P[a][x] is the lowest id
 *     u with (u, x) in E and d(a, u) = d(a, x) - 1.  path(a -> b) is read
 *     backwards from b through P[a][.].  TP(p) = path(entry -> first p),
 *     then p, then path(last p -> exit), joined at the shared endpoints; the
 *     TP set is the sorted, duplicate-free set of TP(p) over all PPs p.
 *  5. A smaller TP set by longest-first touring (Ammann and Offutt's method
 *     as Sec. 7.3 describes it): take the longest PP that no chosen TP
 *     covers yet, extend it to the entry and the exit (its TP(p) of step 4),
 *     and repeat until every PP is covered.  A PP is covered when it is a
 *     contiguous subpath (Sec. 2) of a chosen TP.  Readings: "longest" counts
 *     vertices; equal lengths go in canonical order; the result is put in
 *     canonical order.  orc_test_paths_greedy.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ENOMEM (-4)
#define ORC_ELIMIT (-3)
#define ORC_EUNREACH (-2)
#define ORC_EINVAL (-1)

typedef struct {
    int64_t n;         /* number of sequences */
    int64_t cap;
    int64_t *off;      /* [n+1] */
    int64_t nv, capv;
    int32_t *v;        /* [off[n]] */
} seqlist;

typedef struct orc_result {
    int n;
    seqlist pp, tp;
    seqlist gtp;            /* longest-first touring (step 5) */
    int64_t n_simple;       /* simple paths visited, cycles included */
    int64_t *len_counts;    /* [n+2] simple paths by vertex count */
    int64_t *pp_len_counts; /* [n+2] PPs by vertex count */
    int64_t *root_paths;    /* [n] simple paths per first vertex */
    int64_t *root_pp_ints;  /* [n] total PP vertices per first vertex */
    int64_t *root_pps;      /* [n] PPs per first vertex */
    int32_t *bfs_dist;      /* [n*n] or NULL */
    int32_t *bfs_pred;      /* [n*n] or NULL */
    int err;
} orc_result;

void orc_free(orc_result *r);
int orc_bfs_tables(int n, const int32_t *row_ptr, const int32_t *col, int32_t *dist, int32_t *pred);
orc_result *orc_prime_paths_range(int n, const int32_t *row_ptr, const int32_t *col,
                                  int want_paths, int64_t limit, int root_lo, int root_hi);

static int sl_init(seqlist *s) {
    s->n = 0; s->cap = 1024; s->nv = 0; s->capv = 8192;
    s->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->cap + 1));
    s->v = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->capv);
    if (!s->off || !s->v) return ORC_ENOMEM;
    s->off[0] = 0;
    return ORC_OK;
}

static void sl_free(seqlist *s) {
    free(s->off); free(s->v);
    s->off = NULL; s->v = NULL; s->n = s->nv = 0;
}

static int sl_push(seqlist *s, const int32_t *seq, int len, int extra) {
    /* append seq[0..len) followed by `extra` if extra >= 0 */
    int total = len + (extra >= 0 ? 1 : 0);
    if (s->n + 1 > s->cap) {
        int64_t nc = s->cap * 2;
        int64_t *no = (int64_t *)realloc(s->off, sizeof(int64_t) * (size_t)(nc + 1));
        if (!no) return ORC_ENOMEM;
        s->off = no; s->cap = nc;
    }
    if (s->nv + total > s->capv) {
        int64_t nc = s->capv * 2;
        while (nc < s->nv + total) nc *= 2;
        int32_t *nv = (int32_t *)realloc(s->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return ORC_ENOMEM;
        s->v = nv; s->capv = nc;
    }
    memcpy(s->v + s->nv, seq, sizeof(int32_t) * (size_t)len);
    if (extra >= 0) s->v[s->nv + len] = extra;
    s->nv += total;
    s->n += 1;
    s->off[s->n] = s->nv;
    return ORC_OK;
}

/* lexicographic comparison, a proper prefix sorts first */
static int seq_cmp(const int32_t *a, int64_t la, const int32_t *b, int64_t lb) {
    int64_t l = la < lb ? la : lb;
    for (int64_t i = 0; i < l; i++) {
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    }
    if (la == lb) return 0;
    return la < lb ? -1 : 1;
}

/* Definition of a simple path, written out: v1..v(k-1) pairwise distinct
 * and v2..vk pairwise distinct.  `mark` is a scratch array of n zeros. */
static int is_simple(const int32_t *s, int k, int32_t *mark) {
    int ok = 1;
    for (int i = 0; i + 1 < k && ok; i++) { if (mark[s[i]]) ok = 0; mark[s[i]] = 1; }
    for (int i = 0; i + 1 < k; i++) mark[s[i]] = 0;
    for (int i = 1; i < k && ok; i++) { if (mark[s[i]]) ok = 0; mark[s[i]] = 1; }
    for (int i = 1; i < k; i++) mark[s[i]] = 0;
    return ok;
}

typedef struct {
    int n;
    const int32_t *rp, *col;
    int32_t *prp, *pcol;     /* predecessor CSR */
} graph;

static int build_pred(graph *g) {
    int n = g->n;
    int64_t m = g->rp[n];
    g->prp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    g->pcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!g->prp || !g->pcol) return ORC_ENOMEM;
    for (int64_t e = 0; e < m; e++) g->prp[g->col[e] + 1]++;
    for (int v = 0; v < n; v++) g->prp[v + 1] += g->prp[v];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!fill) return ORC_ENOMEM;
    memcpy(fill, g->prp, sizeof(int32_t) * (size_t)(n + 1));
    for (int u = 0; u < n; u++)
        for (int32_t e = g->rp[u]; e < g->rp[u + 1]; e++) g->pcol[fill[g->col[e]]++] = u;
    free(fill);
    return ORC_OK;
}

static const seqlist *g_sort_list;
static int cmp_idx(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    const seqlist *s = g_sort_list;
    return seq_cmp(s->v + s->off[a], s->off[a + 1] - s->off[a],
                   s->v + s->off[b], s->off[b + 1] - s->off[b]);
}

/* Canonical order + exact dedup of a sequence list (in place). */
static int sort_unique(seqlist *s, int dedup) {
    int64_t n = s->n;
    int sorted = 1;
    for (int64_t i = 1; i < n && sorted; i++) {
        int c = seq_cmp(s->v + s->off[i - 1], s->off[i] - s->off[i - 1],
                        s->v + s->off[i], s->off[i + 1] - s->off[i]);
        if (c > 0 || (dedup && c == 0)) sorted = 0;
    }
    if (sorted) return ORC_OK;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!idx) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    g_sort_list = s;
    qsort(idx, (size_t)n, sizeof(int64_t), cmp_idx);
    seqlist out;
    if (sl_init(&out)) { free(idx); return ORC_ENOMEM; }
    for (int64_t j = 0; j < n; j++) {
        int64_t i = idx[j];
        if (dedup && out.n > 0) {
            int64_t p = out.n - 1;
            if (seq_cmp(out.v + out.off[p], out.off[p + 1] - out.off[p],
                        s->v + s->off[i], s->off[i + 1] - s->off[i]) == 0) continue;
        }
        if (sl_push(&out, s->v + s->off[i], (int)(s->off[i + 1] - s->off[i]), -1)) {
            free(idx); sl_free(&out); return ORC_ENOMEM;
        }
    }
    free(idx);
    sl_free(s);
    *s = out;
    return ORC_OK;
}

/*
 * Enumerate every simple path (step 1) and keep the PPs (step 2).
 * want_paths = 0 only counts.  limit > 0 aborts with ORC_ELIMIT once more
 * than `limit` simple paths have been visited.
 */
orc_result *orc_prime_paths_range(int n, const int32_t *row_ptr, const int32_t *col,
                                  int want_paths, int64_t limit, int root_lo, int root_hi) {
    orc_result *r = (orc_result *)calloc(1, sizeof(orc_result));
    if (!r) return NULL;
    r->n = n;
    if (n < 1) { r->err = ORC_EINVAL; return r; }
    graph g = {n, row_ptr, col, NULL, NULL};
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 3));
    int32_t *it = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 2));
    int32_t *onpath = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *mark = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *ext = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 3));
    r->len_counts = (int64_t *)calloc((size_t)n + 3, sizeof(int64_t));
    r->pp_len_counts = (int64_t *)calloc((size_t)n + 3, sizeof(int64_t));
    r->root_paths = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    r->root_pp_ints = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    r->root_pps = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!path || !it || !onpath || !mark || !ext || !r->len_counts || !r->pp_len_counts ||
        !r->root_paths || !r->root_pp_ints || !r->root_pps || build_pred(&g) || sl_init(&r->pp)) {
        r->err = ORC_ENOMEM;
        goto done;
    }
    if (root_lo < 0) root_lo = 0;
    if (root_hi > n) root_hi = n;
    for (int root = root_lo; root < root_hi && !r->err; root++) {
        int len = 1;
        path[0] = root;
        onpath[root] = 1;
        it[0] = row_ptr[root];
        int visit = 1;              /* the current top path is new */
        while (len > 0) {
            if (visit) {
                visit = 0;
                /* acyclic simple path path[0..len) */
                r->n_simple++;
                r->len_counts[len]++;
                r->root_paths[root]++;
                if (limit > 0 && r->n_simple > limit) { r->err = ORC_ELIMIT; break; }
                int last = path[len - 1], first = path[0];
                int extendable = 0;
                /* p.w is simple iff w is not among path[1..len) */
                for (int32_t e = row_ptr[last]; e < row_ptr[last + 1] && !extendable; e++) {
                    int w = col[e];
                    if (!onpath[w] || (w == first)) extendable = 1;
                }
                /* u.p is simple iff u is not among path[0..len-1) */
                for (int32_t e = g.prp[first]; e < g.prp[first + 1] && !extendable; e++) {
                    int u = g.pcol[e];
                    if (!onpath[u] || (u == last)) extendable = 1;
                }
                if (!extendable) {
                    r->pp_len_counts[len]++;
                    r->root_pps[root]++;
                    r->root_pp_ints[root] += len;
                    if (want_paths && sl_push(&r->pp, path, len, -1)) { r->err = ORC_ENOMEM; break; }
                }
            }
            int v = path[len - 1];
            if (it[len - 1] < row_ptr[v + 1]) {
                int w = col[it[len - 1]++];
                if (w == path[0]) {
                    /* closes a simple cycle path[0..len) . w; it is visited,
                     * not extended; it is a PP iff no one-vertex extension
                     * is simple (tested with the definition itself). */
                    r->n_simple++;
                    r->len_counts[len + 1]++;
                    r->root_paths[root]++;
                    if (limit > 0 && r->n_simple > limit) { r->err = ORC_ELIMIT; break; }
                    path[len] = w;
                    int extendable = 0;
                    for (int32_t e = row_ptr[w]; e < row_ptr[w + 1] && !extendable; e++) {
                        path[len + 1] = col[e];
                        if (is_simple(path, len + 2, mark)) extendable = 1;
                    }
                    for (int32_t e = g.prp[path[0]]; e < g.prp[path[0] + 1] && !extendable; e++) {
                        /* u . cycle, built in the scratch buffer */
                        ext[0] = g.pcol[e];
                        memcpy(ext + 1, path, sizeof(int32_t) * (size_t)(len + 1));
                        if (is_simple(ext, len + 2, mark)) extendable = 1;
                    }
                    if (!extendable) {
                        r->pp_len_counts[len + 1]++;
                        r->root_pps[root]++;
                        r->root_pp_ints[root] += len + 1;
                        if (want_paths && sl_push(&r->pp, path, len, w)) { r->err = ORC_ENOMEM; break; }
                    }
                } else if (!onpath[w]) {
                    path[len] = w;
                    onpath[w] = 1;
                    it[len] = row_ptr[w];
                    len++;
                    visit = 1;
                }
                /* else: w is on the path and is not its first vertex, so
                 * p.w repeats a vertex: not simple, not visited. */
            } else {
                onpath[v] = 0;
                len--;
            }
        }
        for (int i = 0; i < len; i++) onpath[path[i]] = 0;
    }
    if (!r->err && want_paths) r->err = sort_unique(&r->pp, 0);
done:
    free(path); free(it); free(onpath); free(mark); free(ext);
    free(g.prp); free(g.pcol);
    return r;
}

/* Every root (step 1 over all of V). */
orc_result *orc_prime_paths(int n, const int32_t *row_ptr, const int32_t *col,
                            int want_paths, int64_t limit) {
    return orc_prime_paths_range(n, row_ptr, col, want_paths, limit, 0, n);
}

/* All-pairs BFS with the lowest-id predecessor tie-break (step 4). */
int orc_bfs_tables(int n, const int32_t *row_ptr, const int32_t *col,
                   int32_t *dist, int32_t *pred) {
    graph g = {n, row_ptr, col, NULL, NULL};
    if (build_pred(&g)) return ORC_ENOMEM;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) { free(g.prp); free(g.pcol); return ORC_ENOMEM; }
    for (int a = 0; a < n; a++) {
        int32_t *d = dist + (int64_t)a * n;
        int32_t *p = pred + (int64_t)a * n;
        for (int x = 0; x < n; x++) { d[x] = -1; p[x] = -1; }
        int qh = 0, qt = 0;
        d[a] = 0;
        queue[qt++] = a;
        while (qh < qt) {
            int u = queue[qh++];
            for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                int w = col[e];
                if (d[w] < 0) { d[w] = d[u] + 1; queue[qt++] = w; }
            }
        }
        for (int x = 0; x < n; x++) {
            if (x == a || d[x] < 0) continue;
            int best = -1;
            for (int32_t e = g.prp[x]; e < g.prp[x + 1]; e++) {
                int u = g.pcol[e];
                if (d[u] >= 0 && d[u] == d[x] - 1 && (best < 0 || u < best)) best = u;
            }
            p[x] = best;
        }
    }
    free(queue); free(g.prp); free(g.pcol);
    return ORC_OK;
}

/* path(a -> b) written backwards from b through P[a][.]; returns its vertex
 * count (0 if b is unreachable from a). */
static int bfs_path(int n, const int32_t *dist, const int32_t *pred, int a, int b, int32_t *out) {
    const int32_t *d = dist + (int64_t)a * n;
    const int32_t *p = pred + (int64_t)a * n;
    if (d[b] < 0) return 0;
    int len = d[b] + 1;
    int x = b;
    for (int i = len - 1; i >= 0; i--) { out[i] = x; x = (i > 0) ? p[x] : x; }
    return len;
}

/* TP(p) for the PPs i0..i1-1 of r (in that order) appended to `out`. */
static int tp_build_range(const orc_result *r, const int32_t *dist, const int32_t *pred,
                          int entry, int exitv, int64_t i0, int64_t i1, seqlist *out) {
    int n = r->n;
    int32_t *pre = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *suf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * n + 4));
    if (!pre || !suf || !buf) { free(pre); free(suf); free(buf); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int64_t i = i0; i < i1 && rc == ORC_OK; i++) {
        const int32_t *p = r->pp.v + r->pp.off[i];
        int len = (int)(r->pp.off[i + 1] - r->pp.off[i]);
        int lp = bfs_path(n, dist, pred, entry, p[0], pre);
        int ls = bfs_path(n, dist, pred, p[len - 1], exitv, suf);
        if (lp == 0 || ls == 0) { rc = ORC_EUNREACH; break; }
        int k = 0;
        for (int j = 0; j + 1 < lp; j++) buf[k++] = pre[j];   /* pre ends at p[0] */
        for (int j = 0; j < len; j++) buf[k++] = p[j];
        for (int j = 1; j < ls; j++) buf[k++] = suf[j];       /* suf starts at last */
        if (sl_push(out, buf, k, -1)) rc = ORC_ENOMEM;
    }
    free(pre); free(suf); free(buf);
    return rc;
}

int orc_test_paths(orc_result *r, const int32_t *row_ptr, const int32_t *col,
                   int entry, int exitv) {
    int n = r->n;
    if (r->err) return r->err;
    if (entry < 0 || entry >= n || exitv < 0 || exitv >= n) return ORC_EINVAL;
    r->bfs_dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
    r->bfs_pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
    if (!r->bfs_dist || !r->bfs_pred) return ORC_ENOMEM;
    if (orc_bfs_tables(n, row_ptr, col, r->bfs_dist, r->bfs_pred)) return ORC_ENOMEM;
    if (sl_init(&r->tp)) return ORC_ENOMEM;
    int rc = tp_build_range(r, r->bfs_dist, r->bfs_pred, entry, exitv, 0, r->pp.n, &r->tp);
    if (rc == ORC_OK) rc = sort_unique(&r->tp, 1);
    return rc;
}

/* ---- step 5: longest-first touring ---- */

/* 64-bit FNV-1a over a vertex sequence (never 0: 0 marks an empty slot) */
static uint64_t seq_hash(const int32_t *s, int64_t k) {
    uint64_t h = 1469598103934665603ull;
    for (int64_t i = 0; i < k; i++) {
        uint32_t x = (uint32_t)s[i];
        for (int b = 0; b < 4; b++) { h ^= (x >> (8 * b)) & 0xffu; h *= 1099511628211ull; }
    }
    return h ? h : 1;
}

/* An open-addressing set of the PP list: slot -> PP index + 1 (0 = empty). */
typedef struct {
    int64_t mask;
    int64_t *slot;
    uint64_t *key;
} pp_set;

static int pp_set_build(pp_set *t, const seqlist *pp) {
    int64_t size = 16;
    while (size < 2 * pp->n) size *= 2;
    t->mask = size - 1;
    t->slot = (int64_t *)calloc((size_t)size, sizeof(int64_t));
    t->key = (uint64_t *)calloc((size_t)size, sizeof(uint64_t));
    if (!t->slot || !t->key) return ORC_ENOMEM;
    for (int64_t i = 0; i < pp->n; i++) {
        uint64_t h = seq_hash(pp->v + pp->off[i], pp->off[i + 1] - pp->off[i]);
        int64_t j = (int64_t)(h & (uint64_t)t->mask);
        while (t->slot[j]) j = (j + 1) & t->mask;
        t->slot[j] = i + 1;
        t->key[j] = h;
    }
    return ORC_OK;
}

/* index of the PP equal to s[0..k), or -1 */
static int64_t pp_set_find(const pp_set *t, const seqlist *pp, const int32_t *s, int64_t k) {
    uint64_t h = seq_hash(s, k);
    for (int64_t j = (int64_t)(h & (uint64_t)t->mask); t->slot[j]; j = (j + 1) & t->mask) {
        int64_t i = t->slot[j] - 1;
        if (t->key[j] == h && seq_cmp(pp->v + pp->off[i], pp->off[i + 1] - pp->off[i], s, k) == 0) return i;
    }
    return -1;
}

static const seqlist *g_len_list;
/* longest first; equal lengths in list (canonical) order */
static int cmp_len_desc(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    const seqlist *s = g_len_list;
    int64_t la = s->off[a + 1] - s->off[a], lb = s->off[b + 1] - s->off[b];
    if (la != lb) return la > lb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_test_paths_greedy(orc_result *r, const int32_t *row_ptr, const int32_t *col,
                          int entry, int exitv) {
    int n = r->n;
    if (r->err) return r->err;
    if (entry < 0 || entry >= n || exitv < 0 || exitv >= n) return ORC_EINVAL;
    if (!r->bfs_dist) {
        r->bfs_dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
        r->bfs_pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
        if (!r->bfs_dist || !r->bfs_pred) return ORC_ENOMEM;
        if (orc_bfs_tables(n, row_ptr, col, r->bfs_dist, r->bfs_pred)) return ORC_ENOMEM;
    }
    sl_free(&r->gtp);
    if (sl_init(&r->gtp)) return ORC_ENOMEM;
    const seqlist *pp = &r->pp;
    const int64_t P = pp->n;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
    char *covered = (char *)calloc((size_t)(P > 0 ? P : 1), 1);
    int32_t *mark = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    seqlist one = {0, 0, NULL, 0, 0, NULL};
    pp_set set = {0, NULL, NULL};
    int rc = (order && covered && mark && sl_init(&one) == ORC_OK) ? pp_set_build(&set, pp) : ORC_ENOMEM;
    if (rc == ORC_OK) {
        for (int64_t i = 0; i < P; i++) order[i] = i;
        g_len_list = pp;
        qsort(order, (size_t)P, sizeof(int64_t), cmp_len_desc);
    }
    for (int64_t oi = 0; oi < P && rc == ORC_OK; oi++) {
        const int64_t p = order[oi];
        if (covered[p]) continue;
        /* TP(p), step 4 */
        one.n = 0; one.nv = 0;
        rc = tp_build_range(r, r->bfs_dist, r->bfs_pred, entry, exitv, p, p + 1, &one);
        if (rc) break;
        const int32_t *t = one.v;
        const int64_t L = one.nv;
        if (sl_push(&r->gtp, t, (int)L, -1)) { rc = ORC_ENOMEM; break; }
        /* every window t[i..j] that is a simple path, looked up among the PPs
         * (a window that is not simple cannot be a PP) */
        for (int64_t i = 0; i < L; i++) {
            int64_t j = i;
            for (; j < L; j++) {
                if (j > i && t[j] == t[i]) {           /* closes a simple cycle */
                    int64_t q = pp_set_find(&set, pp, t + i, j - i + 1);
                    if (q >= 0) covered[q] = 1;
                    break;
                }
                if (mark[t[j]]) break;                 /* a repeat inside: not simple */
                mark[t[j]] = 1;
                int64_t q = pp_set_find(&set, pp, t + i, j - i + 1);
                if (q >= 0) covered[q] = 1;
            }
            for (int64_t x = i; x < j && x < L; x++) mark[t[x]] = 0;
        }
        if (!covered[p]) { rc = ORC_EINVAL; break; }   /* TP(p) contains p */
    }
    if (rc == ORC_OK) rc = sort_unique(&r->gtp, 1);
    free(order); free(covered); free(mark); free(set.slot); free(set.key);
    if (one.off) sl_free(&one);
    return rc;
}

/*
 * Root-parallel driver, for the all-core CPU baseline.
 *
 * Every PP has exactly one first vertex, and the depth-first enumeration
 * from one root never looks at another root's paths (simplicity and
 * maximality, Sec. 2 and Def. 1, are properties of the path alone), so the
 * roots are independent: `nthreads` threads take roots one at a time from a
 * shared counter and run the enumeration above on each (step 1 restricted
 * to one root).  The per-root lists are concatenated in root order and put
 * in canonical order by the same sort (step 3).  TPs are built by the same
 * construction (step 4) over contiguous ranges of the PP list, one range
 * per thread, concatenated in order, then sorted and deduplicated.  The
 * arithmetic is the serial oracle's; only the order of the work changes.
 */
typedef struct {
    int n;
    const int32_t *rp, *col;
    int want_paths;
    atomic_int next;
    orc_result **per_root;
} root_job;

static void *root_worker(void *arg) {
    root_job *j = (root_job *)arg;
    for (;;) {
        int r = atomic_fetch_add(&j->next, 1);
        if (r >= j->n) break;
        j->per_root[r] = orc_prime_paths_range(j->n, j->rp, j->col, j->want_paths, 0, r, r + 1);
    }
    return NULL;
}

typedef struct {
    const orc_result *r;
    int entry, exitv;
    int64_t i0, i1;
    seqlist out;
    int rc;
} tp_job;

static void *tp_worker(void *arg) {
    tp_job *j = (tp_job *)arg;
    j->rc = sl_init(&j->out);
    if (j->rc == ORC_OK)
        j->rc = tp_build_range(j->r, j->r->bfs_dist, j->r->bfs_pred, j->entry, j->exitv, j->i0, j->i1, &j->out);
    return NULL;
}

/* run fn(arg_t) on nthreads jobs: threads 1.. on new threads, job 0 here */
static void run_jobs(void *(*fn)(void *), void *jobs, size_t stride, int njobs) {
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)(njobs > 0 ? njobs : 1));
    int *ok = (int *)calloc((size_t)(njobs > 0 ? njobs : 1), sizeof(int));
    for (int t = 1; t < njobs; t++)
        ok[t] = th && ok && pthread_create(&th[t], NULL, fn, (char *)jobs + stride * (size_t)t) == 0;
    fn(jobs);
    for (int t = 1; t < njobs; t++) {
        if (ok && ok[t]) pthread_join(th[t], NULL);
        else fn((char *)jobs + stride * (size_t)t);  /* no thread: run it here */
    }
    free(th); free(ok);
}

orc_result *orc_run_parallel(int n, const int32_t *row_ptr, const int32_t *col, int entry,
                             int exitv, int want_paths, int want_tp, int nthreads) {
    if (want_tp) want_paths = 1;
    if (n < 1) return orc_prime_paths_range(n, row_ptr, col, want_paths, 0, 0, 0);
    if (nthreads < 1) nthreads = 1;
    orc_result *out = (orc_result *)calloc(1, sizeof(orc_result));
    orc_result **parts = (orc_result **)calloc((size_t)n, sizeof(orc_result *));
    if (!out || !parts) { free(out); free(parts); return NULL; }
    out->n = n;
    root_job job;
    job.n = n; job.rp = row_ptr; job.col = col; job.want_paths = want_paths;
    atomic_init(&job.next, 0);
    job.per_root = parts;
    root_job *jobs = &job;
    /* every thread shares the one job (the counter hands out the roots) */
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int t = 1; th && t < nthreads; t++)
        if (pthread_create(&th[started], NULL, root_worker, jobs) == 0) started++;
    root_worker(jobs);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
    /* merge in root order */
    out->len_counts = (int64_t *)calloc((size_t)n + 3, sizeof(int64_t));
    out->pp_len_counts = (int64_t *)calloc((size_t)n + 3, sizeof(int64_t));
    out->root_paths = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    out->root_pp_ints = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    out->root_pps = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!out->len_counts || !out->pp_len_counts || !out->root_paths || !out->root_pp_ints ||
        !out->root_pps || sl_init(&out->pp))
        out->err = ORC_ENOMEM;
    for (int r = 0; r < n; r++) {
        orc_result *q = parts[r];
        if (!out->err) {
            if (!q) out->err = ORC_ENOMEM;
            else if (q->err) out->err = q->err;
        }
        if (!out->err) {
            out->n_simple += q->n_simple;
            for (int k = 0; k < n + 3; k++) {
                out->len_counts[k] += q->len_counts[k];
                out->pp_len_counts[k] += q->pp_len_counts[k];
            }
            out->root_paths[r] = q->root_paths[r];
            out->root_pp_ints[r] = q->root_pp_ints[r];
            out->root_pps[r] = q->root_pps[r];
            for (int64_t i = 0; i < q->pp.n && !out->err; i++)
                if (sl_push(&out->pp, q->pp.v + q->pp.off[i], (int)(q->pp.off[i + 1] - q->pp.off[i]), -1))
                    out->err = ORC_ENOMEM;
        }
        orc_free(q);
    }
    free(parts);
    if (!out->err && want_paths) out->err = sort_unique(&out->pp, 0);
    if (out->err || !want_tp) return out;
    /* TPs over PP ranges */
    if (entry < 0 || entry >= n || exitv < 0 || exitv >= n) { out->err = ORC_EINVAL; return out; }
    out->bfs_dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
    out->bfs_pred = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
    if (!out->bfs_dist || !out->bfs_pred ||
        orc_bfs_tables(n, row_ptr, col, out->bfs_dist, out->bfs_pred) || sl_init(&out->tp)) {
        out->err = ORC_ENOMEM;
        return out;
    }
    tp_job *tj = (tp_job *)calloc((size_t)nthreads, sizeof(tp_job));
    if (!tj) { out->err = ORC_ENOMEM; return out; }
    int64_t P = out->pp.n;
    for (int t = 0; t < nthreads; t++) {
        tj[t].r = out; tj[t].entry = entry; tj[t].exitv = exitv;
        tj[t].i0 = P * t / nthreads; tj[t].i1 = P * (t + 1) / nthreads;
    }
    run_jobs(tp_worker, tj, sizeof(tp_job), nthreads);
    for (int t = 0; t < nthreads; t++) {
        if (!out->err && tj[t].rc) out->err = tj[t].rc;
        for (int64_t i = 0; i < tj[t].out.n && !out->err; i++)
            if (sl_push(&out->tp, tj[t].out.v + tj[t].out.off[i],
                        (int)(tj[t].out.off[i + 1] - tj[t].out.off[i]), -1))
                out->err = ORC_ENOMEM;
        sl_free(&tj[t].out);
    }
    free(tj);
    if (!out->err) out->err = sort_unique(&out->tp, 1);
    return out;
}

/* accessors for the ctypes wrapper */
int orc_error(const orc_result *r) { return r ? r->err : ORC_ENOMEM; }
int64_t orc_n_simple(const orc_result *r) { return r->n_simple; }
int64_t orc_pp_count(const orc_result *r) { return r->pp.n; }
int64_t orc_pp_total(const orc_result *r) { return r->pp.nv; }
const int64_t *orc_pp_offsets(const orc_result *r) { return r->pp.off; }
const int32_t *orc_pp_vertices(const orc_result *r) { return r->pp.v; }
int64_t orc_gtp_count(const orc_result *r) { return r->gtp.n; }
int64_t orc_gtp_total(const orc_result *r) { return r->gtp.nv; }
const int64_t *orc_gtp_offsets(const orc_result *r) { return r->gtp.off; }
const int32_t *orc_gtp_vertices(const orc_result *r) { return r->gtp.v; }
int64_t orc_tp_count(const orc_result *r) { return r->tp.n; }
int64_t orc_tp_total(const orc_result *r) { return r->tp.nv; }
const int64_t *orc_tp_offsets(const orc_result *r) { return r->tp.off; }
const int32_t *orc_tp_vertices(const orc_result *r) { return r->tp.v; }
const int64_t *orc_len_counts(const orc_result *r) { return r->len_counts; }
const int64_t *orc_pp_len_counts(const orc_result *r) { return r->pp_len_counts; }
const int64_t *orc_root_paths(const orc_result *r) { return r->root_paths; }
const int64_t *orc_root_pp_ints(const orc_result *r) { return r->root_pp_ints; }
const int64_t *orc_root_pps(const orc_result *r) { return r->root_pps; }

void orc_free(orc_result *r) {
    if (!r) return;
    sl_free(&r->pp);
    sl_free(&r->tp);
    sl_free(&r->gtp);
    free(r->len_counts); free(r->pp_len_counts);
    free(r->root_paths); free(r->root_pp_ints); free(r->root_pps);
    free(r->bfs_dist); free(r->bfs_pred);
    free(r);
}
