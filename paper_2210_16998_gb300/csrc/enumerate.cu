// Level-synchronous frontier of simple paths (kernels (a), (b), (c)).
//
// Method: the paper's host seeds every vertex with the one-vertex path
// (Alg. 2, v.list = {v}); a vertex extends the paths of its predecessors by
// itself when the result stays simple or closes a cycle on the path's first
// vertex (Alg. 3 extension step, Alg. 4 ExtendPath); a path that no
// successor extends and that is not contained in a longer simple path is
// kept as a prime path (Alg. 3 prune step, Def. 1).
//
// GB300 design: instead of one thread per vertex with per-vertex path lists
// (TPAM, Sec. 4.3), every level F_k of all simple paths with k vertices is a
// flat array; one persistent cooperative launch walks the levels with a
// bounded grid barrier between them.  Per level, each thread takes one path,
// holds its visited bitset in registers, counts its children (simple
// one-vertex extensions, closing arcs included), decides primality, and the
// block writes the children of its tile into the next level at offsets from
// a block scan plus a decoupled look-back across tiles.  Children are written
// in (parent order, ascending successor id), so every level stays in
// lexicographic order.  A closed cycle becomes a node of the next level and
// is reported there as a PP.
//
// Path arena (persistent, level-major): node = {last vertex (global id),
// index of the parent in the previous level}.  Frontier (ping-pong, two
// buffers): node = {first, last} (int2) and the visited bitset stored as W
// separate word arrays (word j of node i at j * lvl_cap + i).
#include "common.cuh"
#include "kernels.h"

namespace tpg {

template <int W>
__device__ __forceinline__ bool test_bit(const unsigned (&v)[W], int b) {
    if constexpr (W <= 8) {
        const int wi = b >> 5;
        unsigned word = 0;
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (j == wi) word = v[j];
        return (word >> (b & 31)) & 1u;
    } else {
        return (v[b >> 5] >> (b & 31)) & 1u;
    }
}

// Level 1: one path <v> per vertex (Alg. 2 initialisation).
template <int W>
__global__ void init_level1_kernel(EnumArgs a) {
    const GraphDev &g = a.g;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)i;
        a.nodes[i] = make_int2(v, -1);
        a.tfl[1][i] = make_int2(v, v);
        const int loc = g.vgraph ? v - g.vbase[g.vgraph[v]] : v;
#pragma unroll
        for (int j = 0; j < W; ++j)
            a.tvis[1][j * a.lvl_cap + i] = (j == (loc >> 5)) ? (1u << (loc & 31)) : 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LevelRec r = {};
        r.node_base = 0;
        r.count = g.N;
        r.pp_base = 0;
        r.status_base = 0;
        a.levels[1] = r;
    }
}

template <int W, int BLOCK>
__global__ void __launch_bounds__(BLOCK) enumerate_kernel(EnumArgs a) {
    __shared__ long long s_tile;
    __shared__ unsigned long long s_pa, s_pb;
    const GraphDev &g = a.g;
    const int tid = threadIdx.x;

    for (int k = 1; k + 1 < a.max_levels; ++k) {
        if (__ldcg(a.err) & (ERR_OVERFLOW_MASK | ERR_TIMEOUT | ERR_OVF_LEVELS | ERR_OVF_COUNT)) break;
        const LevelRec *Lp = a.levels + k;
        const long long count = __ldcg(&Lp->count);
        if (count <= 0) break;
        const long long node_base = __ldcg(&Lp->node_base);
        const long long pp_base = __ldcg(&Lp->pp_base);
        const long long status_base = __ldcg(&Lp->status_base);
        const long long next_base = node_base + count;
        const long long ntiles = (count + BLOCK - 1) / BLOCK;
        const int2 *in_fl = a.tfl[k & 1];
        const unsigned *in_vis = a.tvis[k & 1];
        int2 *out_fl = a.tfl[(k + 1) & 1];
        unsigned *out_vis = a.tvis[(k + 1) & 1];
        unsigned long long *status = a.status + status_base;

        while (true) {
            if (tid == 0) s_tile = atomicAdd(a.tile_ctr + k, 1);
            __syncthreads();
            const long long tile = s_tile;
            if (tile >= ntiles) break;

            const long long i = tile * BLOCK + tid;
            const bool valid = i < count;
            int first = 0, last = 0, vb = 0, nch = 0;
            bool pp = false;
            unsigned vis[W];
#pragma unroll
            for (int j = 0; j < W; ++j) vis[j] = 0u;
            int e0 = 0, e1 = 0;
            if (valid) {
                const int2 fl = __ldcg(in_fl + i);
                first = fl.x;
                last = fl.y;
                if (k >= 2 && first == last) {
                    pp = true;  // closed simple cycle: never extended, always prime
                } else {
                    vb = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + first)) : 0;
#pragma unroll
                    for (int j = 0; j < W; ++j) vis[j] = __ldcg(in_vis + j * a.lvl_cap + i);
                    e0 = __ldg(g.rp + last);
                    e1 = __ldg(g.rp + last + 1);
                    for (int e = e0; e < e1; ++e) {
                        const int w = __ldg(g.col + e);
                        if (w == first || !test_bit<W>(vis, w - vb)) ++nch;
                    }
                    if (nch == 0) {
                        // right-maximal; left-maximal iff every predecessor u of
                        // the first vertex is on the path and is not its last
                        // vertex (u.p would otherwise be simple)
                        bool lm = true;
                        const int p0 = __ldg(g.prp + first), p1 = __ldg(g.prp + first + 1);
                        for (int e = p0; e < p1; ++e) {
                            const int u = __ldg(g.pcol + e);
                            if (u == last || !test_bit<W>(vis, u - vb)) {
                                lm = false;
                                break;
                            }
                        }
                        pp = lm;
                    }
                }
            }
            unsigned long long total;
            const unsigned long long ex = block_excl_scan_u64<BLOCK>(
                ((unsigned long long)nch << 32) | (pp ? 1ull : 0ull), total);
            const unsigned long long agg_c = total >> 32, agg_p = total & 0xffffffffull;
            if (tid < 32) {
                unsigned long long pa, pb;
                lookback_pair(status, tile, agg_c, agg_p, pa, pb, a.err);
                if (tid == 0) {
                    s_pa = pa;
                    s_pb = pb;
                }
            }
            __syncthreads();
            long long cpos = (long long)s_pa + (long long)(ex >> 32);
            const long long ppos = (long long)s_pb + (long long)(ex & 0xffffffffull);
            if (nch > 0) {
                for (int e = e0; e < e1; ++e) {
                    const int w = __ldg(g.col + e);
                    const bool closes = (w == first);
                    if (closes || !test_bit<W>(vis, w - vb)) {
                        const long long gi = next_base + cpos;
                        if (cpos < a.lvl_cap && gi < a.node_cap) {
                            a.nodes[gi] = make_int2(w, (int)i);
                            out_fl[cpos] = make_int2(first, w);
                            if (!closes) {
                                const int b = w - vb;
#pragma unroll
                                for (int j = 0; j < W; ++j)
                                    out_vis[j * a.lvl_cap + cpos] =
                                        vis[j] | ((j == (b >> 5)) ? (1u << (b & 31)) : 0u);
                            }
                        }
                        ++cpos;
                    }
                }
            }
            if (pp) {
                const long long q = pp_base + ppos;
                if (q < a.pp_cap) a.pp_refs[q] = (int)i;
            }
            if (tile == ntiles - 1 && tid == 0) {
                const long long C = (long long)s_pa + (long long)agg_c;
                const long long P = (long long)s_pb + (long long)agg_p;
                int e = 0;
                if (C >= (long long)MAX31 || P >= (long long)MAX31) e |= ERR_OVF_COUNT;
                if (next_base + C > a.node_cap) e |= ERR_OVF_NODES;
                if (C > a.lvl_cap) e |= ERR_OVF_LEVEL;
                if (pp_base + P > a.pp_cap) e |= ERR_OVF_PP;
                const long long nt_next = (C + BLOCK - 1) / BLOCK;
                if (status_base + ntiles + nt_next > a.status_cap) e |= ERR_OVF_STATUS;
                if (k + 2 >= a.max_levels && C > 0) e |= ERR_OVF_LEVELS;
                a.levels[k].pp_count = P;
                a.levels[k].children = C;
                LevelRec r = {};
                r.node_base = next_base;
                r.count = C;
                r.pp_base = pp_base + P;
                r.status_base = status_base + ntiles;
                a.levels[k + 1] = r;
                if (e) atomicOr(a.err, e);
            }
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.err)) break;
    }
}

// ---------------------------------------------------------------------------
// host-side launch
// ---------------------------------------------------------------------------
template <int W, int BLOCK>
static cudaError_t launch_w(const EnumArgs &args, int num_sms, cudaStream_t s, int *grid_out) {
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks_per_sm, enumerate_kernel<W, BLOCK>, BLOCK, 0);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int grid = num_sms * blocks_per_sm;
    *grid_out = grid;
    init_level1_kernel<W><<<(args.g.N + 255) / 256, 256, 0, s>>>(args);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    EnumArgs a = args;
    void *params[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)enumerate_kernel<W, BLOCK>, dim3(grid), dim3(BLOCK),
                                    params, 0, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

int bitset_words_supported(int maxn) {
    const int w = (maxn + 31) / 32;
    const int sizes[] = {1, 2, 3, 4, 5, 6, 8, 16, 32, 64, 128};
    for (int s : sizes)
        if (w <= s) return s;
    return -1;
}

cudaError_t launch_enumerate(const EnumArgs &args, int num_sms, cudaStream_t s, int *grid_out) {
    constexpr int B = ENUM_BLOCK;
    switch (args.g.W) {
        case 1: return launch_w<1, B>(args, num_sms, s, grid_out);
        case 2: return launch_w<2, B>(args, num_sms, s, grid_out);
        case 3: return launch_w<3, B>(args, num_sms, s, grid_out);
        case 4: return launch_w<4, B>(args, num_sms, s, grid_out);
        case 5: return launch_w<5, B>(args, num_sms, s, grid_out);
        case 6: return launch_w<6, B>(args, num_sms, s, grid_out);
        case 8: return launch_w<8, B>(args, num_sms, s, grid_out);
        case 16: return launch_w<16, B>(args, num_sms, s, grid_out);
        case 32: return launch_w<32, B>(args, num_sms, s, grid_out);
        case 64: return launch_w<64, B>(args, num_sms, s, grid_out);
        case 128: return launch_w<128, B>(args, num_sms, s, grid_out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tpg
