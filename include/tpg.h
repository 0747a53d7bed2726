/*
 * tpg.h -- C ABI of the GB300 prime-path / test-path library (libtpg.so).
 *
 * The library computes, for a control-flow graph G = (V, E) with a start
 * vertex s and an end vertex e, the output of Problem 1 of the TPGen paper
 * (Sec. 3): every prime path (PP) of G -- a maximal simple path, Def. 1,
 * where a simple path may repeat only its first vertex as its last (Sec. 2)
 * -- and a set of test paths (TPs), entry-to-exit paths that tour every PP.
 *
 * All compute runs in hand-written sm_103a CUDA kernels.  Entry points take
 * plain host or device pointers and sizes; no C++ or framework type crosses
 * this boundary.
 *
 * Conventions
 *  - Vertex ids are 0..n-1.  A graph is given as int32 CSR of successor
 *    lists: row_ptr[n+1] (row_ptr[0] = 0, non-decreasing) and col[m]
 *    (col[row_ptr[u] .. row_ptr[u+1]) = successors of u, strictly ascending,
 *    each in 0..n-1).  This is the CSR the paper stores on the device
 *    (Sec. 4.1); the library derives the predecessor lists itself.
 *  - Out-degree is not limited to 2 (the paper's restriction, Sec. 3, is a
 *    convenience of its kernel, not of the problem).
 *  - Canonical order of a path list: lexicographic on the int32 vertex
 *    sequences, a proper prefix first.  A simple cycle is written with its
 *    first vertex repeated at the end (<2,3,4,8,2> in Def. 1).  Rotations of
 *    one cycle are distinct PPs.
 *  - Every function returns TPG_OK (0) or a negative TPG_E* code; on error
 *    an output handle pointer is set to NULL.  tpg_strerror() names a code.
 *  - A handle is not to be used from two host threads at once.  Work is
 *    issued on the handle's CUDA stream (tpg_set_stream); calls return only
 *    after their results are complete.
 *
 * Typical use
 *     tpg_cfg *g;
 *     tpg_paths *pp, *tp;
 *     if (tpg_load_cfg(n, row_ptr, col, entry, exit, &g) != TPG_OK) ...;
 *     tpg_prime_paths(g, &pp);   // pp->offsets[0..P], pp->vertices[0..offsets[P])
 *     tpg_test_paths(g, &tp);    // same layout; may share pp's storage
 *     ...
 *     tpg_free(tp); tpg_free(pp); tpg_free(g);
 * Many graphs at once: tpg_load_cfg_batch (results grouped by graph through
 * graph_path_ptr), and for repeated batches of one shape tpg_graph_capture /
 * tpg_graph_launch, which replay the whole pipeline as one CUDA graph.
 */
#ifndef TPG_H
#define TPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPG_OK 0
#define TPG_EINVAL (-1)    /* malformed input (see tpg_load_cfg) */
#define TPG_EUNREACH (-2)  /* a PP vertex is unreachable from entry or cannot reach exit */
#define TPG_ETOOBIG (-3)   /* n above TPG_MAX_N, or a level beyond int32 indexing */
#define TPG_ENOMEM (-4)    /* device or pinned host allocation failed */
#define TPG_ECUDA (-5)     /* a CUDA runtime call failed */
#define TPG_ETIMEOUT (-6)  /* a bounded device-side wait ran out */
#define TPG_EHANDLE (-7)   /* NULL or foreign handle */

#define TPG_MAX_N 4096     /* vertices per graph (bitset of 128 words) */

/* where tpg_paths arrays live */
#define TPG_RESULT_HOST 0   /* page-locked host memory (default) */
#define TPG_RESULT_DEVICE 1 /* device memory of the handle's GPU */

typedef struct tpg_cfg tpg_cfg; /* opaque: device copy of the graph(s) + tables */

/* A path list owned by the library; release it with tpg_free(). */
typedef struct tpg_paths {
    uint32_t magic;                 /* internal tag */
    int32_t num_graphs;             /* 1 for tpg_load_cfg handles */
    int64_t num_paths;              /* P */
    const int64_t *graph_path_ptr;  /* [num_graphs+1]: paths of graph g are
                                       [graph_path_ptr[g], graph_path_ptr[g+1]) */
    const int64_t *offsets;         /* [P+1], offsets[0] = 0 */
    const int32_t *vertices;        /* [offsets[P]], graph-local vertex ids, canonical order per graph */
    /* fields after the six above (which every caller may rely on) */
    int64_t num_vertices;           /* offsets[P], so that no read of a device array is needed */
    int32_t location;               /* TPG_RESULT_HOST or TPG_RESULT_DEVICE */
    int32_t reserved;
} tpg_paths;

/* Statistics of the last tpg_prime_paths call on a handle. */
typedef struct tpg_stats {
    int64_t simple_paths;       /* frontier nodes enumerated (simple paths incl. closed cycles) */
    int64_t prime_paths;        /* P */
    int64_t pp_vertices;        /* total vertex ids in the PP list */
    int32_t levels;             /* frontier levels processed */
    int32_t pp_levels;          /* levels that held at least one PP */
    int64_t peak_level_nodes;   /* largest frontier level */
    int64_t arena_bytes_used;   /* persistent path arena bytes written */
    int64_t arena_bytes_alloc;  /* path arena bytes allocated */
    int64_t frontier_bytes_alloc; /* ping-pong frontier bytes allocated */
    int32_t attempts;           /* 1 + overflow retries */
    int32_t bitset_words;       /* W: 32-bit words of the visited bitset */
    int64_t test_paths;         /* TPs after dedup (last tpg_test_paths) */
    int64_t tp_vertices;
    float t_enumerate_ms;       /* device time of the frontier launch (CUDA events) */
    float t_order_ms;           /* device time of ordering + materialisation */
    float t_test_paths_ms;      /* device time of the last tpg_test_paths pipeline */
    int32_t enumerate_grid;     /* blocks of the persistent frontier launch */
    int32_t tile_block;         /* threads per block of the frontier launch */
    int32_t tile_items;         /* paths per thread (tile = block * items paths) */
    float t_graph_ms;           /* device time of the last tpg_graph_launch replay */
    int32_t graph_launches;     /* tpg_graph_launch calls on this handle */
    int32_t graph_fallbacks;    /* of them, replays whose capacities were too small */
    int32_t graph_flags;        /* status word of the last replay (0 = complete) */
    int32_t graph_enum_error;   /* frontier-launch error word of the last replay */
    float t_result_copy_ms;     /* device time of the device-to-host copies of the last host result
                                   (0 when it shared an earlier copy or lives on the device) */
    int64_t result_copy_bytes;  /* bytes those copies moved */
    float t_touring_ms;         /* device time of the last tpg_test_paths_greedy after its one-per-PP
                                   TP list: PP hash table, cover edges, decision sweeps, gather */
    int32_t touring_sweeps;     /* decision sweeps it took */
    int64_t touring_test_paths; /* TPs it chose */
    int64_t touring_edges;      /* cover edges (TP(p) holds q, q after p in the order) */
    float t_pervertex_ms;       /* device time of the last tpg_prime_paths_pervertex */
    int64_t pervertex_paths;    /* simple paths it copied into the vertex lists */
    int64_t pervertex_bytes;    /* bytes of those lists (vertices, flags, per-vertex pointers) */
    float t_scc_ms;             /* device time of the last tpg_scc_internal_pps */
    int64_t scc_pps;            /* PPs of the SCC subgraphs it found */
    int64_t scc_internal_pps;   /* of them, SccInternalPPs */
    float t_compositional_ms;   /* device time of the last tpg_prime_paths_compositional */
    int64_t comp_entry_exit_paths; /* its SccEntryExitPaths (Def. 6), all SCCs */
    int64_t comp_exit_paths;       /* its SccExitPaths (Def. 7) */
    int64_t comp_entry_paths;      /* its SccEntryPaths (Def. 8) */
    int64_t comp_crossing_pps;     /* PPs it joined across SCCs */
} tpg_stats;

/*
 * tpg_load_cfg -- validate one CFG and copy it to the device.
 *
 * Problem 1 input (Sec. 3): G, start vertex `entry`, end vertex `exit`.
 * row_ptr[n+1] and col[row_ptr[n]] are HOST pointers; the caller keeps them.
 * The call builds, on the device, the predecessor CSR and the all-pairs BFS
 * tables (distance and lowest-id predecessor) used by tpg_test_paths.
 *
 * TPG_EINVAL if: n < 1; row_ptr[0] != 0 or row_ptr decreasing; a col entry
 * outside 0..n-1; a successor list not strictly ascending (duplicate arc);
 * entry or exit outside 0..n-1 or entry == exit; in-degree(entry) != 0 or
 * out-degree(exit) != 0 (Sec. 3).  TPG_ETOOBIG if n > TPG_MAX_N.
 * Self-loops are accepted.  On success *out owns device memory until
 * tpg_free(*out).
 */
int tpg_load_cfg(int32_t n, const int32_t *row_ptr, const int32_t *col,
                 int32_t entry, int32_t exit, tpg_cfg **out);

/*
 * tpg_load_cfg_device -- as tpg_load_cfg, but row_ptr and col are DEVICE
 * pointers (read on the handle's stream, copied into the handle) and the
 * validation runs in a kernel.  `m` is the arc count (col length); `stream`
 * is a cudaStream_t (NULL = legacy default stream) that also becomes the
 * handle's stream.
 */
int tpg_load_cfg_device(int32_t n, int32_t m, const int32_t *row_ptr_dev,
                        const int32_t *col_dev, int32_t entry, int32_t exit,
                        void *stream, tpg_cfg **out);

/*
 * tpg_load_cfg_batch -- many independent CFGs in one handle.
 *
 * Graph g has n_per_graph[g] vertices with LOCAL ids; its CSR is
 * row_ptr_cat[R_g .. R_g + n_g] (local arc offsets starting at 0) and
 * col_cat[C_g .. C_g + m_g) with R_g = sum_{h<g} (n_h + 1) and
 * C_g = sum_{h<g} m_h.  entries[g], exits[g] are local ids.  All HOST
 * pointers.  Each graph is validated as in tpg_load_cfg (the first failing
 * graph's error is returned).  Results of tpg_prime_paths / tpg_test_paths
 * on a batch handle carry graph_path_ptr[G+1] and graph-local vertex ids.
 */
int tpg_load_cfg_batch(int32_t num_graphs, const int32_t *n_per_graph,
                       const int32_t *row_ptr_cat, const int32_t *col_cat,
                       const int32_t *entries, const int32_t *exits,
                       tpg_cfg **out);

/*
 * tpg_prime_paths -- every PP of the graph(s) in canonical order.
 *
 * Def. 1 (maximal simple path).  The method: level-synchronous extension of
 * all simple paths from every vertex (the paper's Alg. 2 seeds v.list = {v}
 * for every v), primality by the can't-extend-at-either-end rule (Alg. 3
 * prune step), cycle closing as in Alg. 4, then a canonical ordering.
 * *out is allocated by the library (location per tpg_set_result_location)
 * and released with tpg_free.  May retry internally with a larger path
 * arena when the arena overflows; results never depend on the arena size.
 */
int tpg_prime_paths(tpg_cfg *g, tpg_paths **out);

/*
 * tpg_test_paths -- the TP set touring every PP (Problem 1 output).
 *
 * TP(p) = path(entry -> first p), then p, then path(last p -> exit), joined
 * at shared endpoints, where path(a -> b) is read backwards from b through
 * the BFS table P[a][x] = lowest-id u with (u, x) in E and
 * d(a, u) = d(a, x) - 1.  The TP set is the canonical-order, duplicate-free
 * set {TP(p)}.  Runs tpg_prime_paths internally if needed.
 * TPG_EUNREACH if some PP cannot be toured.
 */
int tpg_test_paths(tpg_cfg *g, tpg_paths **out);

/*
 * tpg_test_paths_greedy -- a smaller TP set by longest-first touring: the
 * construction Sec. 7.3 credits to Ammann and Offutt (take the longest PP,
 * extend it to the entry and the exit, repeat with the longest PP that no
 * chosen TP covers yet).  Here the extension of p is TP(p) as in
 * tpg_test_paths, a PP is covered when it is a contiguous subpath of a
 * chosen TP, PPs of equal length are taken in canonical order, and the
 * chosen TPs are returned in canonical order: a subset of tpg_test_paths's
 * list that still tours every PP.  Graphs of a batch are toured
 * independently (num_graphs and graph_path_ptr as for tpg_test_paths).
 * Runs tpg_prime_paths and the one-per-PP TP pipeline internally.
 * TPG_EUNREACH if some PP cannot be toured; TPG_ETOOBIG if the PP or TP
 * list holds 2^31 paths or more.
 */
int tpg_test_paths_greedy(tpg_cfg *g, tpg_paths **out);

/*
 * tpg_prime_paths_pervertex -- a baseline in the paper's own design
 * (Sec. 4 and 5, Alg. 1-4), for comparison with tpg_prime_paths: one thread
 * per vertex, each vertex keeping the simple paths that end at it as whole
 * copied vertex sequences with the paper's per-path flags (extended, read by
 * the left / right successor, cyclic); one launch pair per path length
 * instead of the paper's self-stabilising loop (threads of different blocks
 * cannot wait on one another), then each vertex prunes its own list (a path
 * extended by a successor, or a proper suffix of a longer path of the same
 * list, is not a PP).  The result holds the same PPs as tpg_prime_paths,
 * grouped by END VERTEX as Problem 1 states the output: num_graphs = n and
 * graph_path_ptr[v] .. graph_path_ptr[v+1]-1 are the PPs finished at v (by
 * length, then in creation order).  Single-graph handles only, every vertex
 * of out-degree at most 2 (binarise switches first, Sec. 3): else
 * TPG_EINVAL.  Its memory grows with the total length of all simple paths.
 */
int tpg_prime_paths_pervertex(tpg_cfg *g, tpg_paths **out);

/*
 * The per-SCC step of the compositional route (Sec. 2.1, Defs. 3, 5, 9).
 *
 * tpg_scc_ids           comp_host[v] (n values) = the smallest vertex of
 *                       v's strongly connected component (v and u share one
 *                       iff each reaches the other), from the handle's BFS
 *                       tables.
 * tpg_scc_internal_pps  the SccInternalPPs of every SCC, canonical order:
 *                       the PPs of the SCC's own subgraph (the graph
 *                       restricted to arcs inside one SCC, run through the
 *                       regular frontier path) that are cycles, or that
 *                       neither start at an SccEntryVertex (a predecessor in
 *                       another SCC) nor end at an SccExitVertex (a
 *                       successor in another SCC).  On the worked example
 *                       of Sec. 2.1 these are the 11 internal PPs it lists.
 * Single-graph handles only (else TPG_EINVAL).
 */
int tpg_scc_ids(tpg_cfg *g, int32_t *comp_host);
int tpg_scc_internal_pps(tpg_cfg *g, tpg_paths **out);

/*
 * tpg_prime_paths_compositional -- the PPs by the compositional route of
 * Sec. 2.1 instead of the direct enumeration: the SccInternalPPs (above),
 * plus every PP that crosses SCCs, joined from an SccExitPath (Def. 7: an
 * acyclic path to an SccExitVertex whose first vertex has every predecessor
 * on it), SccEntryExitPaths (Def. 6) of the SCCs it passes and an
 * SccEntryPath (Def. 8: from an SccEntryVertex, every successor of its last
 * vertex on it), consecutive parts linked by arcs between SCCs.  Same result
 * as tpg_prime_paths, canonical order.  Single-graph handles (TPG_EINVAL)
 * of at most 256 vertices (TPG_ETOOBIG).
 */
int tpg_prime_paths_compositional(tpg_cfg *g, tpg_paths **out);

/* Release a tpg_cfg*, tpg_paths* or tpg_sizer* (tag-checked).  NULL is a no-op. */
void tpg_free(void *handle);

/* Issue the handle's work on `stream` (a cudaStream_t; NULL = default). */
int tpg_set_stream(tpg_cfg *g, void *stream);

/* TPG_RESULT_HOST (default) or TPG_RESULT_DEVICE for later results. */
int tpg_set_result_location(tpg_cfg *g, int32_t location);

/*
 * Device allocator used for all device buffers of all handles created
 * after the call (NULL, NULL restores cudaMallocAsync/cudaFreeAsync on the
 * handle stream).  alloc(bytes, stream, ctx) returns a device pointer or
 * NULL; release(ptr, stream, ctx) frees it.
 */
typedef void *(*tpg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*tpg_release_fn)(void *ptr, void *stream, void *ctx);
int tpg_set_allocator(tpg_alloc_fn alloc, tpg_release_fn release, void *ctx);

/*
 * Device blocks the library releases (handle scratch, freed results) are
 * kept, up to 32 GiB, for reuse by later calls with the same allocator on
 * the same stream and of the same size class (4 KiB steps up to 1 MiB, 2 MiB
 * steps above), so a repeated call sequence stops allocating after its
 * first round.  This hands every kept block back to its allocator (it is
 * also done by tpg_set_allocator).  Blocks still owned by handles or
 * results are not affected.  Always TPG_OK.
 */
int tpg_release_cached_memory(void);

/*
 * Tile shape of the frontier kernel for this handle: `block` threads per
 * block, `items` paths per thread.  Supported: block 256 with items 1, 2
 * or 4, block 512 with items 1 or 2, block 1024 with items 1 (bitsets of
 * <= 8 words); block 256 items 1 for wider bitsets.  TPG_EINVAL otherwise.  Results never depend
 * on the shape; the autotuner uses this.
 */
int tpg_set_tile_shape(tpg_cfg *g, int32_t block, int32_t items);

/*
 * Work units per chunk of the frontier kernel for this handle (1..4,
 * default 1): each chunk of a level is cut into `split` parts that go to
 * different warps, which balances levels whose chunk costs vary a lot (a
 * part's offsets are found by summing the count words of the chunk's
 * earlier parts).  TPG_EINVAL outside 1..4.  Results never depend on it;
 * the autotuner uses it.
 */
int tpg_set_work_split(tpg_cfg *g, int32_t split);

/*
 * Limit, in nanoseconds, of every wait at a grid-wide barrier of the
 * handle's frontier launches (default 4 s; ns < 0 restores it).  The
 * frontier kernel is one persistent launch whose blocks meet at a barrier
 * after each level; a block that waits longer than this stops, the launch
 * ends with its error flag set, and the call returns TPG_ETIMEOUT with the
 * handle still usable.  A watchdog for callers that must never wait on a
 * stalled GPU; with ns = 0 any wait at all times out, which is how the
 * error path is tested.  Results never depend on it otherwise.
 */
int tpg_set_wait_limit(tpg_cfg *g, int64_t ns);

/*
 * Initial capacities of the handle's path arena: total simple paths,
 * simple paths of one level, and prime paths.  When one is exceeded, the
 * frontier launch stops after the exact size of the level that did not fit
 * is known; the library adds an arena segment (or a larger frontier or PP
 * list) and relaunches at that level, so finished levels are kept and
 * results never depend on these values.  Capacities whose buffers the
 * allocator cannot give are halved until they fit.  A pre-sizing policy
 * (e.g. the learned sizer) sets them.
 */
int tpg_set_capacity(tpg_cfg *g, int64_t nodes, int64_t level_nodes, int64_t prime_paths);

/*
 * Graph mode (batched persistent launch captured in a CUDA graph).
 *
 * tpg_graph_capture records the whole hot path of the handle -- the
 * persistent frontier launch over every graph of the handle, the PP ordering
 * and materialisation, TP assembly, sort and dedup -- as one CUDA graph whose
 * kernels read every size from device memory, with fixed buffer capacities:
 * those set by tpg_set_capacity / tpg_set_output_capacity, else the exact
 * sizes of the handle's last tpg_prime_paths + tpg_test_paths (run once
 * first if there was none).  The capture is tied to the handle's stream
 * (a private stream if it is the legacy default stream).
 *
 * tpg_graph_launch replays it and returns the PP and TP lists in *pp and
 * *tp (result location as set).  Device results of a replay alias the
 * capture's output buffers: they stay valid until the next replay on this
 * handle.  If a capacity proved too small, the call computes the exact
 * result with the host-driven path instead, counts a fallback in the stats
 * and re-captures on the next launch; results are identical either way.
 *
 * tpg_set_output_capacity sets the output capacities used by the next
 * capture: PPs, PP vertices, TP vertices before dedup, TP vertices.
 */
int tpg_graph_capture(tpg_cfg *g);
int tpg_graph_launch(tpg_cfg *g, tpg_paths **pp, tpg_paths **tp);
int tpg_set_output_capacity(tpg_cfg *g, int64_t prime_paths, int64_t pp_vertices,
                            int64_t tp_vertices_raw, int64_t tp_vertices);

/*
 * tpg_root_counts -- exact per-root volumes of the enumeration.
 *
 * counts_host[3*v + 0..2] (v a global vertex id; for a batch, graph g's
 * vertices follow each other in graph order) receive, over the simple paths
 * whose first vertex is v: their number (closed cycles included), the
 * number of those that are prime, and the total vertices of those prime
 * paths.  These are the training labels of the learned sizer.  Runs the
 * frontier kernel in counting mode (no ordering, no outputs).
 */
int tpg_root_counts(tpg_cfg *g, int64_t *counts_host);

/*
 * Learned sizer (no counterpart in the paper; it addresses the storage cost
 * the paper attributes to copying predecessor paths, Sec. 4.3).
 *
 * A message-passing network over the CFG (8 vertex features, three layers
 * of width 64, BF16 weights and activations, FP32 accumulation and FP32
 * master weights trained with Adam) predicts for every vertex r the log1p
 * of three enumeration volumes rooted at r: simple paths, prime paths and
 * prime-path vertices.  Summed over a handle, they pre-size its graph-mode
 * capture (tpg_sizer_presize), so a new batch can be captured and replayed
 * without an exact sizing run; a replay whose capacities prove too small
 * falls back to the exact path, so results never depend on the network.
 *
 * tpg_sizer_create      new network, weights initialised from `seed`.
 * tpg_sizer_add_batch   keep a training batch: the handle's graph, its
 *                       features and exact per-root labels (tpg_root_counts)
 *                       and its whole-batch volumes; volumes_out (optional,
 *                       6 values): simple paths, peak level, PPs, PP
 *                       vertices, TP vertices before and after dedup.
 * tpg_sizer_train       `epochs` passes over the kept batches (one Adam step
 *                       per batch, rate cosine-decayed from lr to lr/10);
 *                       loss_per_epoch (optional) receives the mean loss.
 *                       Afterwards each target's predicted batch total is
 *                       calibrated: the largest exact/predicted ratio over
 *                       the kept batches scales later pre-sizing.
 * tpg_sizer_predict     per-vertex predictions pred_host[3*N] (optional) and
 *                       their expm1 sums totals_host[3] (optional).
 * tpg_sizer_presize     capacities of the handle's next graph capture from
 *                       the calibrated predicted totals times `margin` (>= 1),
 *                       scaled down so that the capture's buffers take at
 *                       most half of the free device memory, each list below
 *                       2^31 entries; caps_out (optional, 7 values) receives
 *                       them.
 * tpg_sizer_features    the 8 features of every vertex (x_host[8*N]).
 * tpg_sizer_get_params / tpg_sizer_set_params   FP32 master weights
 *                       (tpg_sizer_num_params() floats).
 * tpg_sizer_loss_grad   loss and gradient on kept batch `batch` at the
 *                       current weights, without an update.
 * tpg_sizer_batch_targets  the labels of kept batch `batch` (targets[3*N]).
 * tpg_sizer_save / tpg_sizer_load   weights, volume ratios and calibration
 *                       to a file.
 * A tpg_sizer* is released with tpg_free.
 */
typedef struct tpg_sizer tpg_sizer;
int tpg_sizer_num_params(void);
int tpg_sizer_create(uint64_t seed, tpg_sizer **out);
int tpg_sizer_add_batch(tpg_sizer *z, tpg_cfg *g, int64_t *volumes_out);
int tpg_sizer_train(tpg_sizer *z, int32_t epochs, float lr, float *loss_per_epoch);
int tpg_sizer_predict(tpg_sizer *z, tpg_cfg *g, float *pred_host, double *totals_host);
int tpg_sizer_presize(tpg_sizer *z, tpg_cfg *g, double margin, int64_t *caps_out);
int tpg_sizer_features(tpg_cfg *g, float *x_host);
int tpg_sizer_get_params(const tpg_sizer *z, float *host);
int tpg_sizer_set_params(tpg_sizer *z, const float *host);
int tpg_sizer_loss_grad(tpg_sizer *z, int32_t batch, double *loss, float *grad_host);
int tpg_sizer_batch_targets(tpg_sizer *z, int32_t batch, float *targets_host);
int tpg_sizer_save(const tpg_sizer *z, const char *path);
int tpg_sizer_load(tpg_sizer *z, const char *path);

/* Statistics of the handle's last calls. */
int tpg_get_stats(const tpg_cfg *g, tpg_stats *out);

/*
 * Per-level trace of the frontier launch (a profiling aid; the paper has no
 * counterpart).  With tracing on, each tpg_prime_paths call records for
 * every level k of the enumeration (paths of k vertices) four int64 values,
 * out[4k .. 4k+3]: the level's start (the earliest block to start it) and
 * the end of its last warp, in nanoseconds from the first level's start;
 * the summed busy time of the warps that had work in the level; and the
 * number of those warps.  tpg_get_level_trace copies up to max_levels
 * levels of the last call's trace and sets *levels_out to the number of
 * levels recorded (values -1 where a level recorded nothing).  Tracing adds
 * a few atomics per warp and level; results never depend on it.
 */
int tpg_set_level_trace(tpg_cfg *g, int32_t on);
int tpg_get_level_trace(const tpg_cfg *g, int64_t *out, int32_t max_levels, int32_t *levels_out);

/*
 * tpg_prime_paths_noalloc -- prime paths of one small graph, allocating
 * nothing.  (The paper has no counterpart; this is a convenience of the
 * library.)
 *
 * For callers that cannot allocate memory when they need the result: code
 * working inside a device-memory budget fixed in advance (where a
 * cudaMalloc in mid-run could fail or break the budget), and hosts whose
 * framework owns every allocation and hands the library only the buffers
 * it reads and writes.  The call runs the same kernels as tpg_load_cfg +
 * tpg_prime_paths, keeps every
 * temporary in one fixed-size device array built into the library (about
 * 33 MB, held by every GPU that loads the library until the process exits),
 * and writes into buffers the caller owns.  It calls no cudaMalloc,
 * cudaFree, cudaHostAlloc or other allocating routine.
 *
 * n, m: vertices and arcs; row_ptr_dev[n+1], col_dev[m]: DEVICE int32 CSR
 * (ascending successor lists, ids 0..n-1).  No entry/exit rule applies: PPs
 * are defined on any digraph.  offsets_dev[cap_paths+1] (int64) and
 * vertices_dev[cap_vertices] (int32) are DEVICE buffers of the caller;
 * on TPG_OK they hold the canonical PP list, exactly as tpg_prime_paths
 * returns it, and *num_paths / *num_vertices its sizes.  `stream` is a
 * cudaStream_t (NULL = legacy default stream); the call returns after the
 * results are complete.
 *
 * Limits: n <= 128, m <= 16384, at most 2^20 simple paths in all, 2^18 in
 * one level and 2^18 PPs; beyond them the call returns TPG_ETOOBIG.  If the
 * caller's buffers are too small it returns TPG_ETOOBIG with *num_paths and
 * *num_vertices set to the sizes needed.  TPG_EINVAL for a malformed CSR.
 *
 * The first call on a device looks up the array's device address (with
 * that device current) and caches it.  The call waits on `stream` between
 * its steps (it reads level sizes back to choose the next launches).
 * Every call reuses the same array and clears what must start at zero;
 * calls whose GPU work overlaps (e.g. on two streams at once) race on it.
 */
int tpg_prime_paths_noalloc(int32_t n, int32_t m, const int32_t *row_ptr_dev,
                            const int32_t *col_dev, int64_t *offsets_dev,
                            int64_t cap_paths, int32_t *vertices_dev,
                            int64_t cap_vertices, void *stream,
                            int64_t *num_paths, int64_t *num_vertices);

/* Number of CUDA kernels this library has launched in this process. */
int64_t tpg_kernel_launches(void);

/* Static text for an error code. */
const char *tpg_strerror(int code);

/* Library version string. */
const char *tpg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TPG_H */
