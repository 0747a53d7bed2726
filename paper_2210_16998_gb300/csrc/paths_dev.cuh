// Device helpers shared by the host-driven and the graph-captured pipelines.
#pragma once
#include "common.cuh"

namespace tpg {

// Packed comparison keys of vertex sequences: vertex v is stored as v + 1
// in `bits` (8 or 16) bits, most significant first, vpw = 64 / bits vertices
// per 64-bit word, the last word zero-padded.  Comparing word by word (a
// missing word reads as 0) orders the sequences lexicographically with a
// proper prefix first, and equal keys mean equal sequences.  This form
// compares two sequences of the same graph (no graph ids read); key_cmp
// orders by graph id first.
__device__ __forceinline__ int key_cmp_same_graph(long long a, long long b, const long long *koff,
                                                  const unsigned long long *key) {
    const long long a0 = koff[a], wa = koff[a + 1] - a0;
    const long long b0 = koff[b], wb = koff[b + 1] - b0;
    const long long w = wa > wb ? wa : wb;
    for (long long t = 0; t < w; ++t) {
        const unsigned long long x = t < wa ? key[a0 + t] : 0ull;
        const unsigned long long y = t < wb ? key[b0 + t] : 0ull;
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

__device__ __forceinline__ int key_cmp(long long a, long long b, const long long *koff,
                                       const unsigned long long *key, const int *graph) {
    const int ga = graph[a], gb = graph[b];
    if (ga != gb) return ga < gb ? -1 : 1;
    return key_cmp_same_graph(a, b, koff, key);
}

// Materialise PPs [0, n): one warp handles 32 consecutive PPs; each lane
// walks its path's parent links from the last vertex back to the first,
// writing into a per-warp shared-memory window that the warp then stores
// contiguously (lanes store directly when the window does not fit).  The
// window holds local ids as 16-bit values (a graph has at most TPG_MAX_N
// vertices), so more warps fit an SM: the walk is latency-bound and the
// number of walks in flight sets its speed.  A PP is
// refs[i] = (level << 32 | index in level), or, with refs == nullptr, index
// single_refs[i] in level single_level.  out_graph (optional) receives the
// graph id of each PP, out_ends (optional) its (first, last) local vertex.
static_assert(TPG_MAX_N <= 65536, "local vertex ids fit 16 bits");
constexpr int MAT_BUF = 1536;  // local vertex ids (uint16, < TPG_MAX_N) per warp: 32 PPs of up to 48 vertices
constexpr int MAT_MAX_LV = 256; // level-pointer table cached in shared memory up to this many levels
                                // (2 KB: with a 24 KB window per 8 warps, 8 blocks fit an SM)

// Copy the levels' node pointers to shared memory (one dependent load per
// parent-link step instead of two); returns nullptr when there are too many.
__device__ __forceinline__ int2 *const *cache_level_nodes(const LevelRec *levels, int max_levels,
                                                          int2 **s_nodes) {
    if (max_levels > MAT_MAX_LV) return nullptr;
    for (int k = threadIdx.x; k < max_levels; k += blockDim.x) s_nodes[k] = levels[k].nodes;
    __syncthreads();
    return s_nodes;
}

template <int NWARPS>
__device__ __forceinline__ void materialize_warps(const long long *refs, const int *single_refs, int single_level,
                                                  long long n, const long long *offsets, const LevelRec *levels,
                                                  const GraphDev &g, int *out, int *out_graph,
                                                  unsigned short (&buf)[NWARPS][MAT_BUF], int2 *const *lvl_nodes,
                                                  int2 *out_ends = nullptr) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long nwarps = (long long)gridDim.x * NWARPS;
    for (long long w0 = (blockIdx.x * (long long)NWARPS + wid) * 32; w0 < n; w0 += nwarps * 32) {
        const long long idx = w0 + lane;
        const bool valid = idx < n;
        int level = 0, rel = 0;
        if (valid) {
            if (refs) {
                const long long r = refs[idx];
                level = (int)(r >> 32);
                rel = (int)(r & 0xffffffffll);
            } else {
                level = single_level;
                rel = single_refs[idx];
            }
        }
        const long long w_end_idx = (w0 + 32 < n) ? w0 + 32 : n;
        const long long start = offsets[w0];
        const long long span = offsets[w_end_idx] - start;
        const long long off = valid ? offsets[idx] : 0;
        const bool staged = span <= MAT_BUF;
        int node = rel, root = 0, first_loc = 0, last_loc = 0;
        for (int j = level; j >= 1; --j) {
            const int2 rec = lvl_nodes ? lvl_nodes[j][node] : levels[j].nodes[node];
            const int v = rec.x;
            const int loc = g.vgraph ? v - g.vbase[g.vgraph[v]] : v;
            if (staged) buf[wid][off - start + (j - 1)] = (unsigned short)loc;
            else out[off + (j - 1)] = loc;
            if (j == level) last_loc = loc;
            first_loc = loc;
            root = v;
            node = rec.y;
        }
        if (valid && out_graph) out_graph[idx] = g.vgraph ? g.vgraph[root] : 0;
        if (valid && out_ends) out_ends[idx] = make_int2(first_loc, last_loc);
        if (staged) {
            __syncwarp();
            for (long long t = lane; t < span; t += 32) out[start + t] = (int)buf[wid][t];
            __syncwarp();
        }
    }
}

}  // namespace tpg
