// Canonical order of the prime paths (kernel (e) for PPs) and their
// materialisation as vertex sequences.
//
// Every level of the path arena is in lexicographic order, and the prime
// paths form an antichain of the prefix tree (a PP is never a proper prefix
// of a simple path, Def. 1).  So for two PPs x (k vertices) and y (>= k
// vertices), x < y exactly when x's index in level k is below the index of
// y's level-k ancestor.  The canonical list is built from the deepest level
// upward: the run accumulated so far is keyed by each element's ancestor
// index at the current level (one parent-link step per level), and merged
// with that level's own PPs by key.  Keys of the two inputs never tie.
#include "common.cuh"
#include "kernels.h"
#include "paths_dev.cuh"

namespace tpg {

__global__ void order_init_run_kernel(const int *pp, int level, long long n, int *keys, long long *refs) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = pp[i];
        keys[i] = r;
        refs[i] = ((long long)level << 32) | (unsigned)r;
    }
}

cudaError_t order_init_run(const int *pp_refs_level, int level, long long n, int *keys, long long *refs,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8);
    order_init_run_kernel<<<grid, 256, 0, s>>>(pp_refs_level, level, n, keys, refs);
    note_launch();
    return cudaGetLastError();
}

__global__ void order_ascend_kernel(int *keys, long long n, const LevelRec *levels, int from_level, int to_level) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int key = keys[i];
        for (int j = from_level; j > to_level; --j) key = levels[j].nodes[key].y;
        keys[i] = key;
    }
}

cudaError_t order_ascend(int *keys, long long n, const LevelRec *levels, int from_level, int to_level,
                         cudaStream_t s) {
    if (n <= 0 || from_level <= to_level) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    order_ascend_kernel<<<(unsigned)(blocks < 1 << 20 ? blocks : 1 << 20), 256, 0, s>>>(
        keys, n, levels, from_level, to_level);
    note_launch();
    return cudaGetLastError();
}

constexpr int MERGE_ITEMS = 8;

// Merge path: thread t produces outputs [t*ITEMS, t*ITEMS + ITEMS).  The
// keys of run A are stored at level from_level and lifted to level
// to_level (the level of run B) on the fly.  On equal keys A goes first
// (cannot happen between A and B here, but keeps the merge stable).
__global__ void order_merge_kernel(const int *ka, const long long *ra, long long na, const int *kb,
                                   int level_b, long long nb, int *kc, long long *rc, const LevelRec *levels,
                                   int from_level) {
    const long long total = na + nb;
    const long long diag = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * MERGE_ITEMS;
    if (diag >= total) return;
    auto lift = [&](long long i) {
        int key = ka[i];
        for (int j = from_level; j > level_b; --j) key = levels[j].nodes[key].y;
        return key;
    };
    long long lo = diag > nb ? diag - nb : 0;
    long long hi = diag < na ? diag : na;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (lift(mid) <= kb[diag - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    long long i = lo, j = diag - lo;
    int ki = (i < na) ? lift(i) : 0;
    for (int t = 0; t < MERGE_ITEMS && diag + t < total; ++t) {
        if (i < na && (j >= nb || ki <= kb[j])) {
            kc[diag + t] = ki;
            rc[diag + t] = ra[i];
            ++i;
            if (i < na) ki = lift(i);
        } else {
            const int r = kb[j];
            kc[diag + t] = r;
            rc[diag + t] = ((long long)level_b << 32) | (unsigned)r;
            ++j;
        }
    }
}

cudaError_t order_merge(const int *ka, const long long *ra, long long na, const int *kb, int level_b, long long nb,
                        int *kc, long long *rc, const LevelRec *levels, int from_level, cudaStream_t s) {
    const long long total = na + nb;
    if (total <= 0) return cudaSuccess;
    const long long threads = (total + MERGE_ITEMS - 1) / MERGE_ITEMS;
    order_merge_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(ka, ra, na, kb, level_b, nb, kc, rc, levels,
                                                                        from_level);
    note_launch();
    return cudaGetLastError();
}

__global__ void pp_lengths_kernel(const long long *refs, long long n, long long *len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        len[i] = refs[i] >> 32;
}

cudaError_t pp_lengths(const long long *refs, long long n, long long *len_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    pp_lengths_kernel<<<(unsigned)(blocks < 1 << 20 ? blocks : 1 << 20), 256, 0, s>>>(refs, n, len_out);
    note_launch();
    return cudaGetLastError();
}

__global__ void pp_offsets_single_kernel(long long *off, long long n, int level) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= n;
         i += (long long)gridDim.x * blockDim.x)
        off[i] = i * level;
}

cudaError_t pp_offsets_single_level(long long *off, long long n, int level, cudaStream_t s) {
    const long long blocks = (n + 1 + 255) / 256;
    pp_offsets_single_kernel<<<(unsigned)(blocks < 1 << 20 ? blocks : 1 << 20), 256, 0, s>>>(off, n, level);
    note_launch();
    return cudaGetLastError();
}

constexpr int MAT_WARPS = 8;

__global__ void __launch_bounds__(MAT_WARPS * 32, 8)
    pp_materialize_kernel(const long long *refs, const int *single_refs, int single_level, long long n,
                          const long long *offsets, const LevelRec *levels, int max_levels, GraphDev g,
                          int *out, int *out_graph) {
    __shared__ unsigned short buf[MAT_WARPS][MAT_BUF];
    __shared__ int2 *s_nodes[MAT_MAX_LV];
    int2 *const *lv = cache_level_nodes(levels, max_levels, s_nodes);
    materialize_warps(refs, single_refs, single_level, n, offsets, levels, g, out, out_graph, buf, lv);
}

cudaError_t pp_materialize(const long long *refs, const int *single_refs, int single_level, long long n,
                           const long long *offsets, const LevelRec *levels, int max_levels, const GraphDev &g,
                           int *out_vertices, int *out_graph, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long warps = (n + 31) / 32;
    long long blocks = (warps + MAT_WARPS - 1) / MAT_WARPS;
    if (blocks > 152 * 64) blocks = 152 * 64;
    pp_materialize_kernel<<<(unsigned)blocks, MAT_WARPS * 32, 0, s>>>(refs, single_refs, single_level, n, offsets,
                                                                     levels, max_levels, g, out_vertices, out_graph);
    note_launch();
    return cudaGetLastError();
}

// graph_path_ptr[g] = first path index whose graph id is >= g (ids sorted).
__global__ void graph_ptr_kernel(const int *ids, long long n, int G, long long *ptr) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= n;
         i += (long long)gridDim.x * blockDim.x) {
        const int cur = (i < n) ? ids[i] : G;
        const int prev = (i > 0) ? ids[i - 1] : -1;
        for (int gg = prev + 1; gg <= cur; ++gg) ptr[gg] = i;
    }
}

cudaError_t graph_ptr_from_ids(const int *ids, long long n, int G, long long *ptr, cudaStream_t s) {
    const long long blocks = (n + 1 + 255) / 256;
    graph_ptr_kernel<<<(unsigned)(blocks < 1 << 20 ? blocks : 1 << 20), 256, 0, s>>>(ids, n, G, ptr);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
