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

// Materialise PPs [0, n): one warp handles 32 * CH consecutive PPs, CH per
// lane (lane l takes PPs l, l + 32, ...); each lane walks its paths' parent
// links from the last vertex back to the first, the CH walks interleaved so
// that CH dependent loads are in flight per lane, writing into a per-warp
// shared-memory window that the warp then stores contiguously (lanes store
// directly when the window does not fit).  The window holds local ids as T
// (8-bit for graphs of at most 256 vertices, else 16-bit: a graph has at most
// TPG_MAX_N vertices), so more warps fit an SM: the walk is latency-bound and
// the number of walks in flight sets its speed.  A PP is
// refs[i] = (level << 32 | index in level), or, with refs == nullptr, index
// single_refs[i] in level single_level.  out_graph (optional) receives the
// graph id of each PP, out_ends (optional) its (first, last) local vertex.
static_assert(TPG_MAX_N <= 65536, "local vertex ids fit 16 bits");
constexpr int MAT_BUF = 1536;  // window entries per warp and per walk of a lane: 32 PPs of up to 48 vertices
constexpr int MAT_MAX_LV = 256; // level-pointer table cached in shared memory up to this many levels
                                // (2 KB: with a 24 KB window per 8 warps, 8 blocks fit an SM)
constexpr int MAT_SMALL_N = 256;  // graphs up to this size use 8-bit windows and two walks per lane

// Copy the levels' node pointers to shared memory (one dependent load per
// parent-link step instead of two); returns nullptr when there are too many.
__device__ __forceinline__ int2 *const *cache_level_nodes(const LevelRec *levels, int max_levels,
                                                          int2 **s_nodes) {
    if (max_levels > MAT_MAX_LV) return nullptr;
    for (int k = threadIdx.x; k < max_levels; k += blockDim.x) s_nodes[k] = levels[k].nodes;
    __syncthreads();
    return s_nodes;
}

template <int NWARPS, int CH, typename T>
__device__ __forceinline__ void materialize_warps(const long long *refs, const int *single_refs, int single_level,
                                                  long long n, const long long *offsets, const LevelRec *levels,
                                                  const GraphDev &g, int *out, int *out_graph,
                                                  T (&buf)[NWARPS][MAT_BUF * CH], int2 *const *lvl_nodes,
                                                  int2 *out_ends = nullptr) {
    constexpr int TILE = 32 * CH;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long nwarps = (long long)gridDim.x * NWARPS;
    for (long long w0 = (blockIdx.x * (long long)NWARPS + wid) * TILE; w0 < n; w0 += nwarps * TILE) {
        int level[CH], node[CH], vb[CH], root[CH], first_loc[CH], last_loc[CH];
        long long off[CH];
        int jmax = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const long long idx = w0 + c * 32 + lane;
            level[c] = 0;
            node[c] = 0;
            if (idx < n) {
                if (refs) {
                    const long long r = refs[idx];
                    level[c] = (int)(r >> 32);
                    node[c] = (int)(r & 0xffffffffll);
                } else {
                    level[c] = single_level;
                    node[c] = single_refs[idx];
                }
            }
            off[c] = idx < n ? offsets[idx] : 0;
            vb[c] = root[c] = first_loc[c] = last_loc[c] = 0;
            jmax = level[c] > jmax ? level[c] : jmax;
        }
        jmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)jmax);
        const long long w_end_idx = (w0 + TILE < n) ? w0 + TILE : n;
        const long long start = offsets[w0];
        const long long span = offsets[w_end_idx] - start;
        const bool staged = span <= MAT_BUF * CH;
        for (int j = jmax; j >= 1; --j) {
            int2 rec[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (j <= level[c]) rec[c] = lvl_nodes ? lvl_nodes[j][node[c]] : levels[j].nodes[node[c]];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (j > level[c]) continue;
                const int v = rec[c].x;
                if (j == level[c] && g.vgraph) vb[c] = g.vbase[g.vgraph[v]];  // one graph per path
                const int loc = v - vb[c];
                if (staged) buf[wid][off[c] - start + (j - 1)] = (T)loc;
                else out[off[c] + (j - 1)] = loc;
                if (j == level[c]) last_loc[c] = loc;
                first_loc[c] = loc;
                root[c] = v;
                node[c] = rec[c].y;
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const long long idx = w0 + c * 32 + lane;
            if (idx < n && out_graph) out_graph[idx] = g.vgraph ? g.vgraph[root[c]] : 0;
            if (idx < n && out_ends) out_ends[idx] = make_int2(first_loc[c], last_loc[c]);
        }
        if (staged) {
            __syncwarp();
            for (long long t = lane; t < span; t += 32) out[start + t] = (int)buf[wid][t];
            __syncwarp();
        }
    }
}

}  // namespace tpg
