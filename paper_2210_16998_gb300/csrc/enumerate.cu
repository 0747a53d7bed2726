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
// Path arena: a chain of segments; each level lies inside one segment and is
// addressed by a pointer in its level record; node = {last vertex (global
// id), index of the parent in the previous level}.  When the next level does
// not fit in the current segment (or the frontier or the PP list is full),
// the launch stops after recording the exact size that was needed; the host
// supplies a larger segment or buffer and relaunches AT THAT LEVEL, so no
// finished level is ever recomputed or copied.  Frontier (ping-pong, two
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
        a.seg[i] = make_int2(v, -1);
        a.tfl[1][i] = make_int2(v, v);
        const int loc = g.vgraph ? v - g.vbase[g.vgraph[v]] : v;
#pragma unroll
        for (int j = 0; j < W; ++j)
            a.tvis[1][j * a.lvl_cap + i] = (j == (loc >> 5)) ? (1u << (loc & 31)) : 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        LevelRec r = {};
        r.nodes = a.seg;
        r.count = g.N;
        r.pp = a.pp_seg;
        r.status_base = 0;
        a.levels[1] = r;
    }
}

// Per level, a block claims tiles of TILE = BLOCK * ITEMS consecutive paths;
// thread t owns paths tile*TILE + j*BLOCK + t (j < ITEMS), so every load is
// coalesced.  The per-path counts (children, PP flag) are scanned in path
// order through shared memory (striped -> blocked -> striped), and the tile's
// offset in the next level comes from the decoupled look-back.
template <int W, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) enumerate_kernel(EnumArgs a) {
    constexpr int TILE = BLOCK * ITEMS;
    __shared__ unsigned long long s_cnt[TILE];
    __shared__ long long s_tile;
    __shared__ unsigned long long s_pa, s_pb;
    const GraphDev &g = a.g;
    const int tid = threadIdx.x;

    for (int k = a.start_level; k + 1 < a.max_levels; ++k) {
        if (__ldcg(a.err) & (ERR_OVERFLOW_MASK | ERR_TIMEOUT | ERR_OVF_LEVELS | ERR_OVF_COUNT)) break;
        const LevelRec *Lp = a.levels + k;
        const long long count = __ldcg(&Lp->count);
        if (count <= 0) break;
        int2 *const lnodes = (int2 *)__ldcg((const unsigned long long *)&Lp->nodes);
        int *const lpp = (int *)__ldcg((const unsigned long long *)&Lp->pp);
        const long long status_base = __ldcg(&Lp->status_base);
        int2 *const next = (k == a.start_level && a.next_nodes) ? a.next_nodes : lnodes + count;
        const long long next_off = next - a.seg;     // offset of the next level in the segment
        const long long pp_off = lpp - a.pp_seg;     // offset of this level's PPs in their segment
        const long long ntiles = (count + TILE - 1) / TILE;
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

            int first[ITEMS], last[ITEMS], vb[ITEMS], nch[ITEMS], e0[ITEMS], e1[ITEMS];
            bool pp[ITEMS];
            unsigned vis[ITEMS][W];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                first[j] = last[j] = vb[j] = nch[j] = e0[j] = e1[j] = 0;
                pp[j] = false;
#pragma unroll
                for (int w = 0; w < W; ++w) vis[j][w] = 0u;
            }
            // loads first (all ITEMS in flight), then the per-path work
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const long long i = tile * TILE + (long long)j * BLOCK + tid;
                if (i < count) {
                    const int2 fl = __ldcg(in_fl + i);
                    first[j] = fl.x;
                    last[j] = fl.y;
#pragma unroll
                    for (int w = 0; w < W; ++w) vis[j][w] = __ldcg(in_vis + w * a.lvl_cap + i);
                } else {
                    first[j] = -1;
                }
            }
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if (first[j] < 0) continue;
                if (k >= 2 && first[j] == last[j]) {
                    pp[j] = true;  // closed simple cycle: never extended, always prime
                    continue;
                }
                vb[j] = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + first[j])) : 0;
                e0[j] = __ldg(g.rp + last[j]);
                e1[j] = __ldg(g.rp + last[j] + 1);
                int c = 0;
                for (int e = e0[j]; e < e1[j]; ++e) {
                    const int w = __ldg(g.col + e);
                    if (w == first[j] || !test_bit<W>(vis[j], w - vb[j])) ++c;
                }
                nch[j] = c;
                if (c == 0) {
                    // right-maximal; left-maximal iff every predecessor u of
                    // the first vertex is on the path and is not its last
                    // vertex (u.p would otherwise be simple)
                    bool lm = true;
                    const int p0 = __ldg(g.prp + first[j]), p1 = __ldg(g.prp + first[j] + 1);
                    for (int e = p0; e < p1; ++e) {
                        const int u = __ldg(g.pcol + e);
                        if (u == last[j] || !test_bit<W>(vis[j], u - vb[j])) {
                            lm = false;
                            break;
                        }
                    }
                    pp[j] = lm;
                }
            }
            if (a.root_counts) {
                // per-root totals: paths arrive sorted by first vertex, so a
                // warp's lanes mostly share one root; one atomic per group
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const unsigned grp = __match_any_sync(0xffffffffu, first[j]);
                    const unsigned one = first[j] >= 0 ? 1u : 0u;
                    const unsigned isp = (first[j] >= 0 && pp[j]) ? 1u : 0u;
                    const unsigned c0 = __reduce_add_sync(grp, one);
                    const unsigned c1 = __reduce_add_sync(grp, isp);
                    const unsigned c2 = __reduce_add_sync(grp, isp * (unsigned)k);
                    if (first[j] >= 0 && (threadIdx.x & 31) == __ffs(grp) - 1) {
                        unsigned long long *rc = a.root_counts + 3ll * first[j];
                        atomicAdd(rc, (unsigned long long)c0);
                        if (c1) atomicAdd(rc + 1, (unsigned long long)c1);
                        if (c2) atomicAdd(rc + 2, (unsigned long long)c2);
                    }
                }
            }
            // exclusive scan of (children, PP) in path order
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                s_cnt[j * BLOCK + tid] = ((unsigned long long)nch[j] << 32) | (pp[j] ? 1ull : 0ull);
            __syncthreads();
            unsigned long long run = 0;
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) run += s_cnt[tid * ITEMS + q];
            unsigned long long total;
            unsigned long long base = block_excl_scan_u64<BLOCK>(run, total);
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const unsigned long long v = s_cnt[tid * ITEMS + q];
                s_cnt[tid * ITEMS + q] = base;
                base += v;
            }
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
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const unsigned long long ex = s_cnt[j * BLOCK + tid];
                const long long i = tile * TILE + (long long)j * BLOCK + tid;
                if (nch[j] > 0) {
                    long long cpos = (long long)s_pa + (long long)(ex >> 32);
                    for (int e = e0[j]; e < e1[j]; ++e) {
                        const int w = __ldg(g.col + e);
                        const bool closes = (w == first[j]);
                        if (closes || !test_bit<W>(vis[j], w - vb[j])) {
                            if (cpos < a.lvl_cap && next_off + cpos < a.seg_cap) {
                                next[cpos] = make_int2(w, (int)i);
                                out_fl[cpos] = make_int2(first[j], w);
                                if (!closes) {
                                    const int b = w - vb[j];
#pragma unroll
                                    for (int ww = 0; ww < W; ++ww)
                                        out_vis[ww * a.lvl_cap + cpos] =
                                            vis[j][ww] | ((ww == (b >> 5)) ? (1u << (b & 31)) : 0u);
                                }
                            }
                            ++cpos;
                        }
                    }
                }
                if (pp[j]) {
                    const long long q = (long long)s_pb + (long long)(ex & 0xffffffffull);
                    if (pp_off + q < a.pp_seg_cap) lpp[q] = (int)i;
                }
            }
            if (tile == ntiles - 1 && tid == 0) {
                const long long C = (long long)s_pa + (long long)agg_c;
                const long long P = (long long)s_pb + (long long)agg_p;
                int e = 0;
                if (C >= (long long)MAX31 || P >= (long long)MAX31) e |= ERR_OVF_COUNT;
                if (next_off + C > a.seg_cap) e |= ERR_OVF_NODES;
                if (C > a.lvl_cap) e |= ERR_OVF_LEVEL;
                if (pp_off + P > a.pp_seg_cap) e |= ERR_OVF_PP;
                const long long nt_next = (C + TILE - 1) / TILE;
                if (status_base + ntiles + nt_next > a.status_cap) e |= ERR_OVF_STATUS;
                if (k + 2 >= a.max_levels && C > 0) e |= ERR_OVF_LEVELS;
                a.levels[k].pp_count = P;
                a.levels[k].children = C;
                if (e) {
                    *a.stop_level = k;
                    atomicOr(a.err, e);
                } else {
                    LevelRec r = {};
                    r.nodes = next;
                    r.count = C;
                    r.pp = lpp + P;
                    r.status_base = status_base + ntiles;
                    a.levels[k + 1] = r;
                }
            }
            __syncthreads();
        }
        if (!grid_barrier(a.bar, a.err)) break;
    }
}

// ---------------------------------------------------------------------------
// host-side launch
// ---------------------------------------------------------------------------
template <int W, int BLOCK, int ITEMS>
static cudaError_t launch_wbi(const EnumArgs &args, int num_sms, cudaStream_t s, int *grid_out) {
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks_per_sm, enumerate_kernel<W, BLOCK, ITEMS>, BLOCK, 0);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int grid = num_sms * blocks_per_sm;
    *grid_out = grid;
    cudaError_t e;
    if (args.seed_level1) {
        init_level1_kernel<W><<<(args.g.N + 255) / 256, 256, 0, s>>>(args);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    EnumArgs a = args;
    void *params[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)enumerate_kernel<W, BLOCK, ITEMS>, dim3(grid), dim3(BLOCK),
                                    params, 0, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

// tile shapes available per bitset width (the autotuner picks among them)
template <int W>
static cudaError_t launch_w(const EnumArgs &args, EnumShape shape, int num_sms, cudaStream_t s, int *grid_out) {
    if constexpr (W <= 8) {
        if (shape.block == 128) {
            if (shape.items == 1) return launch_wbi<W, 128, 1>(args, num_sms, s, grid_out);
            if (shape.items == 2) return launch_wbi<W, 128, 2>(args, num_sms, s, grid_out);
            if (shape.items == 4) return launch_wbi<W, 128, 4>(args, num_sms, s, grid_out);
        } else if (shape.block == 256) {
            if (shape.items == 1) return launch_wbi<W, 256, 1>(args, num_sms, s, grid_out);
            if (shape.items == 2) return launch_wbi<W, 256, 2>(args, num_sms, s, grid_out);
            if (shape.items == 4) return launch_wbi<W, 256, 4>(args, num_sms, s, grid_out);
        } else if (shape.block == 512) {
            if (shape.items == 1) return launch_wbi<W, 512, 1>(args, num_sms, s, grid_out);
            if (shape.items == 2) return launch_wbi<W, 512, 2>(args, num_sms, s, grid_out);
        }
        return cudaErrorInvalidValue;
    } else {
        return launch_wbi<W, 256, 1>(args, num_sms, s, grid_out);
    }
}

__global__ void relayout_kernel(const int2 *fl_old, const unsigned *vis_old, long long cap_old, int2 *fl_new,
                                unsigned *vis_new, long long cap_new, long long count, int W) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        fl_new[i] = fl_old[i];
        for (int w = 0; w < W; ++w) vis_new[w * cap_new + i] = vis_old[w * cap_old + i];
    }
}

cudaError_t relayout_frontier(const int2 *fl_old, const unsigned *vis_old, long long cap_old, int2 *fl_new,
                              unsigned *vis_new, long long cap_new, long long count, int W, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    long long blocks = (count + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    relayout_kernel<<<(unsigned)blocks, 256, 0, s>>>(fl_old, vis_old, cap_old, fl_new, vis_new, cap_new, count, W);
    note_launch();
    return cudaGetLastError();
}

bool enum_shape_supported(int W, EnumShape shape) {
    if (W > 8) return shape.block == 256 && shape.items == 1;
    if (shape.block == 128 || shape.block == 256) return shape.items == 1 || shape.items == 2 || shape.items == 4;
    if (shape.block == 512) return shape.items == 1 || shape.items == 2;
    return false;
}

EnumShape default_enum_shape(int W) {
    if (W > 8) return EnumShape{256, 1};
    return EnumShape{256, 4};
}

int bitset_words_supported(int maxn) {
    const int w = (maxn + 31) / 32;
    const int sizes[] = {1, 2, 3, 4, 5, 6, 8, 16, 32, 64, 128};
    for (int s : sizes)
        if (w <= s) return s;
    return -1;
}

cudaError_t launch_enumerate(const EnumArgs &args, EnumShape shape, int num_sms, cudaStream_t s, int *grid_out) {
    if (!enum_shape_supported(args.g.W, shape)) return cudaErrorInvalidValue;
    switch (args.g.W) {
        case 1: return launch_w<1>(args, shape, num_sms, s, grid_out);
        case 2: return launch_w<2>(args, shape, num_sms, s, grid_out);
        case 3: return launch_w<3>(args, shape, num_sms, s, grid_out);
        case 4: return launch_w<4>(args, shape, num_sms, s, grid_out);
        case 5: return launch_w<5>(args, shape, num_sms, s, grid_out);
        case 6: return launch_w<6>(args, shape, num_sms, s, grid_out);
        case 8: return launch_w<8>(args, shape, num_sms, s, grid_out);
        case 16: return launch_w<16>(args, shape, num_sms, s, grid_out);
        case 32: return launch_w<32>(args, shape, num_sms, s, grid_out);
        case 64: return launch_w<64>(args, shape, num_sms, s, grid_out);
        case 128: return launch_w<128>(args, shape, num_sms, s, grid_out);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tpg
