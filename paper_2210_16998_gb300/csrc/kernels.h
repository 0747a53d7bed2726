// Internal kernel entry points of libtpg (host-callable launchers).
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "common.cuh"

namespace tpg {

// kernels launched by this library in this process (tpg_kernel_launches)
extern std::atomic<long long> g_kernel_launches;
inline void note_launch(int n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// per-chunk level counts of the frontier launch: a level is cut into
// ENUM_UPW chunks per warp of the launch (CPG = ENUM_UPW x warps per block
// chunks per block); 3 rotating slots of {children, PPs} per chunk and per
// block.  enum_agg_words(grid, CPG) int64 values hold them for one launch;
// enum_agg_words_max(num_sms) for any tile shape on that GPU (at most 64
// warps and 8 blocks per SM).
#ifndef TPG_ENUM_UPW
#define TPG_ENUM_UPW 4
#endif
constexpr int ENUM_UPW = TPG_ENUM_UPW;
constexpr long long enum_agg_words(long long grid, long long cpg) { return 3 * (2 * cpg * grid + 2 * grid) + 4; }
constexpr long long enum_agg_words_max(long long num_sms) {
    return 3 * (2 * ENUM_UPW * 64 * num_sms + 2 * 8 * num_sms) + 4;
}
// frontier count word of a path: bits 0-12 are the mask of the successors of
// its last vertex that extend it (successor list position s -> bit s; lists
// of at most CNT_MASK_DEG successors), or, with CNT_WIDE set, the number of
// such successors (at most TPG_MAX_N); CNT_PP flags a prime path
constexpr unsigned CNT_BITS = 0x1fffu;
constexpr unsigned CNT_WIDE = 0x4000u;
constexpr unsigned CNT_PP = 0x8000u;
constexpr int CNT_MASK_DEG = 13;
__host__ __device__ inline int cnt_children(unsigned cw) {
#ifdef __CUDA_ARCH__
    return (cw & CNT_WIDE) ? (int)(cw & CNT_BITS) : __popc(cw & CNT_BITS);
#else
    return (cw & CNT_WIDE) ? (int)(cw & CNT_BITS) : __builtin_popcount(cw & CNT_BITS);
#endif
}
// control block of a launch (err, stop_level, ...); the frontier's grid
// barrier lives at CTL_BAR_OFFSET, the PP ranking's at CTL_RANK_BAR_OFFSET,
// other cooperative kernels use offset 128
constexpr int CTL_BYTES = 1024;
constexpr int CTL_BAR_OFFSET = 256;
constexpr int CTL_RANK_BAR_OFFSET = 512;  // grid barrier of the PP ranking
constexpr int CTL_HANDOFF_OFFSET = 64;    // level a frontier launch's single-block start hands to the grid

struct EnumArgs {
    GraphDev g;
    int2 *seg;               // current arena segment (nodes {last, parent})
    long long seg_cap;
    int2 *next_nodes;        // where level start_level+1 starts (null: right after level start_level)
    int *pp_seg;             // current PP-reference segment
    long long pp_seg_cap;
    int2 *tfl[2];            // ping-pong {first, last}
    unsigned *tvis[2];       // ping-pong bitsets, W word-arrays of lvl_cap each
    unsigned short *tcnt[2]; // ping-pong count words (children | PP flag)
    long long lvl_cap;
    LevelRec *levels;        // [max_levels]
    int max_levels;
    int start_level;         // first level processed by this launch
    int seed_level1;         // 1 on a fresh run: level 1 is written first (never on a resume)
    int split;               // work units per chunk in the per-warp levels (1..4; results never depend on it)
    long long *agg;          // per-block level counts (no initialisation needed)
    long long agg_cap;       // int64 values in agg (enum_agg_words(grid, chunks per block) at least)
    int *err;                // error flags (zeroed)
    int *stop_level;         // level whose next level did not fit (written with the flags)
    unsigned *bar;           // grid barrier: bar[0] is its arrival counter (zeroed)
    unsigned long long *root_counts;  // optional [3*N]: per first vertex, simple paths, PPs, PP vertices
    unsigned long long spin_ns;       // limit of every grid-barrier wait (SPIN_LIMIT_NS unless set)
    unsigned long long *trace;        // optional [LEVEL_TRACE_WORDS * max_levels] per-level timing
    int *handoff;            // optional: on a fresh run, block 0 walks the small first levels alone and
                             // leaves here the level the grid starts at (null: the grid does every level)
};
// per-level trace of a frontier launch, 4 words per level: ~(earliest block
// start), latest warp end, summed busy time of the warps with work, number
// of those warps (globaltimer nanoseconds; zeroed before the launch)
constexpr int LEVEL_TRACE_WORDS = 4;

// enumerate.cu
struct EnumShape {
    int block;  // threads per block
    int items;  // paths per thread; a tile is block * items consecutive paths
};
int bitset_words_supported(int maxn);
bool enum_shape_supported(int W, EnumShape shape);
EnumShape default_enum_shape(int W);
// level capacity of the ping-pong frontier: a multiple of 2048 paths (tiles
// and bulk copies stay 16-byte aligned), at least x, below 2^31 - 1
long long round_frontier_cap(long long x);
cudaError_t launch_enumerate(const EnumArgs &args, EnumShape shape, int num_sms, cudaStream_t s, int *grid_out);
// level 1 of a fresh run (one path per vertex)
cudaError_t launch_seed_level1(const EnumArgs &args, cudaStream_t s);
// copy the first `count` frontier records to buffers of another capacity
cudaError_t relayout_frontier(const int2 *fl_old, const unsigned *vis_old, long long cap_old, int2 *fl_new,
                              unsigned *vis_new, long long cap_new, long long count, int W, cudaStream_t s);

// scan.cu: exclusive scan of int64 (in may equal out); tmp must hold
// scan_tmp_elems(n) int64 values.  out[n] receives the total.
size_t scan_tmp_elems(long long n);
cudaError_t scan_i64(const long long *in, long long *out, long long n, long long *tmp, cudaStream_t s);
// scan_i64 in two halves: the total first (at tmp[scan_total_index(n)]),
// the prefix array only when it is needed
cudaError_t scan_i64_sums(const long long *in, long long n, long long *tmp, cudaStream_t s);
long long scan_total_index(long long n);
cudaError_t scan_i64_finish(const long long *in, long long *out, long long n, const long long *tmp, cudaStream_t s);
// exclusive scan of int32 inputs into int64 outputs (out[n] = total)
cudaError_t scan_i32_to_i64(const int *in, long long *out, long long n, long long *tmp, cudaStream_t s);

// order.cu
// canonical ordering of PP references across levels (ancestor-index merge)
cudaError_t order_init_run(const int *pp_refs_level, int level, long long n, int *keys,
                           long long *refs, cudaStream_t s);
cudaError_t order_ascend(int *keys, long long n, const LevelRec *levels, int from_level, int to_level,
                         cudaStream_t s);
cudaError_t order_merge(const int *ka, const long long *ra, long long na, const int *kb, int level_b,
                        long long nb, int *kc, long long *rc, const LevelRec *levels, int from_level,
                        cudaStream_t s);
cudaError_t pp_lengths(const long long *refs, long long n, long long *len_out, cudaStream_t s);
cudaError_t pp_offsets_single_level(long long *off, long long n, int level, cudaStream_t s);
// out_graph and out_ends (optional) receive each PP's graph id and its
// (first, last) local vertex.
cudaError_t pp_materialize(const long long *refs, const int *single_refs, int single_level, long long n,
                           const long long *offsets, const LevelRec *levels, int max_levels, const GraphDev &g,
                           int *out_vertices, int *out_graph, cudaStream_t s, int2 *out_ends = nullptr);
cudaError_t graph_ptr_from_ids(const int *ids, long long n, int G, long long *ptr, cudaStream_t s);

// canonical PP order by pre-order rank in the arena's prefix tree (one
// cooperative launch; all level sizes are read from the device level table)
struct RankArgs {
    const LevelRec *levels;
    int max_levels;
    int *cnt;             // [cnt_cap] >= all simple paths: per-node PP counts
    long long cnt_cap;
    int *pre[2];          // [pre_cap] each >= the largest level: ranks of two consecutive levels
    long long pre_cap;
    long long *noff;      // [max_levels + 8]: node offset of each level, then totals
    long long *bsum;      // [grid]
    long long *refs;      // [refs_cap]: the sorted PP references (level << 32 | index)
    long long refs_cap;
    unsigned *bar;        // grid barrier: bar[0] is its arrival counter (zeroed)
    int *err;             // ERR_INVAL (a capacity too small), ERR_TIMEOUT
    const int *skip;      // optional: nothing is done when (*skip & skip_mask)
    int skip_mask;
    int cnt_zeroed;       // 1: cnt[0 .. all simple paths) is zero at launch (else the launch zeroes it)
};
// scratch of rank_pps beyond cnt/pre: noff [max_levels + 8], bsum [rank_pps_grid(num_sms)]
int rank_pps_grid(int num_sms);
cudaError_t rank_pps(const RankArgs &a, int num_sms, cudaStream_t s);

// graphmode.cu: the device-driven pipeline captured into a CUDA graph
enum : int {
    GM_ENUM_FAILED = 1,  // the frontier launch stopped (capacity) or failed
    GM_OVF_PP = 2,       // more PPs than P_cap
    GM_OVF_PPV = 4,      // more PP vertices than V_cap
    GM_UNREACH = 8,      // a PP cannot be toured
    GM_TIMEOUT = ERR_TIMEOUT,  // a bounded grid barrier ran out (the barrier ORs this bit)
    GM_OVF_TPV0 = 32,    // more TP vertices (before dedup) than TV0_cap
    GM_OVF_TPV = 64,     // more TP vertices (after dedup) than TV_cap
};
static_assert(GM_TIMEOUT == 16, "flag bits must stay distinct");
struct GmCounts {
    long long P, V, TV0, R, T, TV;
    int flags;
    int pp_buf;  // which keys/refs buffer holds the ordered PPs
};
struct GmArgs {
    GraphDev g;
    const LevelRec *levels;
    int max_levels;
    const int *enum_err;
    long long P_cap, V_cap, TV0_cap, TV_cap;
    int num_sms, tp_rounds;
    unsigned *bar;          // grid barrier of the ordering kernel (zeroed)
    long long *lvl_pp_off;  // [max_levels+1]
    int *keys[2];
    long long *refs[2];
    long long *len;         // [P_cap]
    long long *scan_tmp;    // gm_scan_tmp_elems(P_cap)
    long long *pp_off;      // [P_cap+1]
    int *pp_vert;           // [V_cap]
    int *pp_graph;          // [P_cap] (batches)
    long long *pp_gptr;     // [G+1]
    long long *tp_len;      // [P_cap]
    int *run_start;         // [P_cap]
    long long *run_rank;    // [P_cap+1]
    int *tp_graph0;         // [P_cap]
    long long *run_base, *nruns;  // [G]
    long long *bounds0;     // [P_cap+1]
    long long *tp_off0;     // [P_cap+1]
    int *tp_vert0;          // unused: TPs are assembled from their parts in sorted order
    long long *key_off;     // [P_cap+1] word offsets of the packed TP keys
    unsigned long long *key;  // [K_cap] packed TP keys
    long long K_cap;
    int key_bits;           // 8 (graphs of <= 255 vertices) or 16
    long long *perm[2];     // [P_cap]
    int *keep;              // [P_cap]
    long long *keep_off, *keep_rank;  // [P_cap+1]
    long long *tp_off;      // [P_cap+1]
    int *tp_vert;           // [TV_cap]
    int *tp_graph;          // [P_cap]
    long long *tp_gptr;     // [G+1]
    GmCounts *counts;
    // PP ranking scratch (rank_pps)
    int *rank_cnt;
    long long rank_cnt_cap;
    int *rank_pre[2];
    long long rank_pre_cap;
    long long *rank_noff, *rank_bsum;
    unsigned *rank_bar;
};
int gm_tp_rounds(int maxn);
size_t gm_scan_tmp_elems(long long n_cap);
cudaError_t gm_enqueue_pp(const GmArgs &a, cudaStream_t s);
cudaError_t gm_enqueue_tp(const GmArgs &a, cudaStream_t s);

// sizer.cu: the learned sizer's network
struct SizerNet;
struct SzGraph {
    long long N;
    const int *rp, *col, *prp, *pcol;  // successor / predecessor CSR (global ids)
    const float *X;                    // [N][8] features
    const float *T;                    // [N][3] targets (training only)
};
int sz_param_count();
int sz_features_per_vertex();
int sz_targets();
SizerNet *sz_create(unsigned long long seed, cudaStream_t s, int num_sms);
void sz_destroy(SizerNet *n);
cudaError_t sz_set_params(SizerNet *n, const float *host);
cudaError_t sz_get_params(SizerNet *n, float *host);
cudaError_t sz_get_grads(SizerNet *n, float *host);
cudaError_t sz_features(const GraphDev &g, float *X, cudaStream_t s, int num_sms);
cudaError_t sz_labels(const unsigned long long *counts, long long N, float *T, cudaStream_t s, int num_sms);
cudaError_t sz_forward(SizerNet *n, const SzGraph &b);
cudaError_t sz_loss_backward(SizerNet *n, const SzGraph &b, double *loss_host);
cudaError_t sz_adam_step(SizerNet *n, float lr);
cudaError_t sz_predict(SizerNet *n, const SzGraph &b, float *Y_host, double *totals_host);
cudaError_t sz_log_totals(SizerNet *n, const float *Y, long long N, double *totals_host);
// device allocator of the library (api.cu)
void *lib_dev_alloc(size_t bytes, cudaStream_t s);
void lib_dev_free(void *p, cudaStream_t s);

// preprocess.cu
cudaError_t build_union_csr(const int *unused, const long long *rp_base_dev,
                            const long long *arc_base_dev, const int *rp_cat, const int *col_cat,
                            int G, int N, long long M, int *rp, int *col, int *vgraph, int *vbase_out,
                            cudaStream_t s);
cudaError_t validate_csr_device(const int *rp, const int *col, int n, long long m, int entry, int exit,
                                int *err, cudaStream_t s);
cudaError_t build_pred_csr(const GraphDev &g, int *prp, int *pcol, int *indeg_tmp, long long *scan_tmp,
                           long long *scan_buf, cudaStream_t s);
// gate (optional): a device flag; the BFS does nothing when it is nonzero.
// max_arcs: arcs of the graph with the most arcs (sizes the shared-memory
// copy of the predecessor lists).
cudaError_t bfs_all_pairs(const GraphDev &g, cudaStream_t s, const int *gate, long long max_arcs);
// One graph of at most PREP_SMALL_N vertices: optional CSR validation (sets
// ERR_INVAL in *err, which must be zero on entry, and skips the rest), the
// predecessor CSR, tbl_base, the BFS tables and the tour tables in three
// launches; g.pre_seq / g.suf_seq must hold N(N+1)/2 entries each.
constexpr int PREP_SMALL_N = 1024;
cudaError_t preprocess_small(const GraphDev &g, int *prp, int *pcol, long long *tbl_base, bool validate, int entry,
                             int exit, int *err, cudaStream_t s, unsigned *smask = nullptr, unsigned *pmask = nullptr);
// successor / predecessor bitsets of every vertex (GraphDev::smask, pmask),
// W <= MASK_MAX_W; nothing is done while *gate is nonzero (gate optional)
cudaError_t build_vertex_masks(const GraphDev &g, unsigned *smask, unsigned *pmask, const int *gate, cudaStream_t s);
cudaError_t tour_lengths(const GraphDev &g, long long *scan_tmp, cudaStream_t s);
cudaError_t tour_fill(const GraphDev &g, cudaStream_t s);

// testpaths.cu
cudaError_t tp_lengths(const long long *pp_off, const int2 *pp_ends, const int *pp_graph, long long P,
                       const GraphDev &g, long long *tp_len, int *run_start, int *tp_graph, int *err,
                       cudaStream_t s);
cudaError_t tp_write(const long long *pp_off, const int *pp_vert, const int *pp_graph, long long P,
                     const GraphDev &g, const long long *tp_off, int *tp_vert, cudaStream_t s);
cudaError_t tp_run_bounds(const int *run_start, const long long *run_rank, long long P, long long R,
                          long long *bounds, cudaStream_t s);
cudaError_t tp_iota(long long *perm, long long P, cudaStream_t s);
cudaError_t tp_gather(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                      const long long *tp_off, const int *tp_vert, const int *tp_graph,
                      const long long *keep_off, long long *final_off, int *out_vert, int *out_graph,
                      cudaStream_t s);

}  // namespace tpg
