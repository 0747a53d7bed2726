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
// flat array; one persistent cooperative launch walks the levels with one
// bounded grid barrier per level.  Per level, each thread takes one path,
// holds its visited bitset in registers, counts its children (simple
// one-vertex extensions, closing arcs included), decides primality, and the
// block writes the children of its chunk of the level at offsets known
// before the level starts (see enumerate_kernel).  Children are written in
// (parent order, ascending successor id), so every level stays in
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
        a.levels[1] = r;
    }
}

// What a path of level k does next (Alg. 3 extension and prune steps): its
// number of children (simple one-vertex extensions, closing arcs included)
// and whether it is prime, packed as a count word (CNT_MASK | CNT_PP).  A
// closed cycle (k >= 2, first == last) is never extended and always prime.
// `extra` is a vertex on the path that is not in `vis` (-1 for none): a child
// is evaluated as its parent's bitset plus the child's last vertex.
template <int W>
__device__ __forceinline__ unsigned eval_path(const GraphDev &g, int k, int first, int last, int vb,
                                              const unsigned (&vis)[W], int extra) {
    if (k >= 2 && first == last) return CNT_PP;
    const int e0 = __ldg(g.rp + last), e1 = __ldg(g.rp + last + 1);
    unsigned c = 0;
    for (int e = e0; e < e1; ++e) {
        const int w = __ldg(g.col + e);
        if (w == first || (w != extra && !test_bit<W>(vis, w - vb))) ++c;
    }
    if (c) return c;
    // right-maximal; left-maximal iff every predecessor u of the first vertex
    // is on the path and is not its last vertex (u.p would otherwise be simple)
    const int p0 = __ldg(g.prp + first), p1 = __ldg(g.prp + first + 1);
    for (int e = p0; e < p1; ++e) {
        const int u = __ldg(g.pcol + e);
        if (u == last || (u != extra && !test_bit<W>(vis, u - vb))) return 0u;
    }
    return CNT_PP;
}

// paths per warp of a level of `count` paths: ceil(count / GW) rounded up to
// a multiple of 32; warp w owns [w * chunk, (w + 1) * chunk) clipped to count
__device__ __forceinline__ int warp_chunk(long long count, int GW) {
    const long long q = (count + GW - 1) / GW;
    return (int)((q + 31) & ~31ll);
}

template <int BLOCK>
__device__ __forceinline__ void block_sum4(long long (&v)[4]) {
    __shared__ long long s_part[4][BLOCK / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        if (lane == 0) s_part[i][wid] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < BLOCK / 32; ++w) t += s_part[i][w];
        v[i] = t;
    }
    __syncthreads();
}

// Per-chunk counts of one level: slot s holds, for every warp chunk and for
// every block (the sum of its warps' chunks), the children and the PPs the
// chunk produces.
struct AggSlots {
    long long *base;
    int GW, G;
    __device__ long long *wc(int s) const { return base + s * (2ll * GW + 2ll * G); }
    __device__ long long *wp(int s) const { return wc(s) + GW; }
    __device__ long long *bc(int s) const { return wc(s) + 2ll * GW; }
    __device__ long long *bp(int s) const { return wc(s) + 2ll * GW + G; }
};

// Add (c, p) to warp chunk `own` of slot s (and to its block).  Lanes with
// nothing to add pass own = -1.  One set of atomics per warp when all lanes
// share one owner (the usual case), per lane otherwise.
template <int NW>
__device__ __forceinline__ void flush_counts(const AggSlots &A, int s, int own, unsigned long long c,
                                             unsigned long long p) {
    const unsigned have = __ballot_sync(0xffffffffu, own >= 0 && (c | p));
    if (!have) return;
    const int own0 = __shfl_sync(0xffffffffu, own, __ffs(have) - 1);
    const bool mine = own >= 0 && (c | p);
    if (__all_sync(0xffffffffu, !mine || own == own0)) {
        if (!mine) c = p = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            p += __shfl_xor_sync(0xffffffffu, p, o);
        }
        if ((threadIdx.x & 31) == 0) {
            if (c) {
                atomicAdd((unsigned long long *)A.wc(s) + own0, c);
                atomicAdd((unsigned long long *)A.bc(s) + own0 / NW, c);
            }
            if (p) {
                atomicAdd((unsigned long long *)A.wp(s) + own0, p);
                atomicAdd((unsigned long long *)A.bp(s) + own0 / NW, p);
            }
        }
    } else if (mine) {
        if (c) {
            atomicAdd((unsigned long long *)A.wc(s) + own, c);
            atomicAdd((unsigned long long *)A.bc(s) + own / NW, c);
        }
        if (p) {
            atomicAdd((unsigned long long *)A.wp(s) + own, p);
            atomicAdd((unsigned long long *)A.bp(s) + own / NW, p);
        }
    }
}

// One persistent cooperative launch walks the levels.  Level k is split into
// GW equal contiguous chunks, one per warp.  Before a warp touches level k it
// knows how many children and PPs every chunk produces: the count word of
// each path of level k (tcnt) was computed when that path was written, and
// the writers added it to the entry of the chunk that owns the path.  After
// one grid barrier per level, a block sums the block entries before its own
// and a warp the warp entries before its own in the block: that is the
// warp's exact offset in level k+1 and in the PP list.  The warp then walks
// its chunk in tiles of 32 * ITEMS paths (lane l owns paths j*32 + l, so
// every load is coalesced) with warp-level scans only -- no block-wide
// synchronisation inside a level -- and writes every child together with
// the child's own count word.  Each path is read once and written once.
//
// Slots rotate: level k reads slot k%3, accumulates into slot (k+1)%3, and
// each warp / block clears its own entries of slot (k+2)%3, which nobody
// reads or accumulates until after the next barrier.  The first level of a
// launch (level 1 of a fresh run, or the level a resume starts at) is
// counted by a separate pass.
template <int W, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK, W <= 8 ? 1024 / BLOCK : 1) enumerate_kernel(EnumArgs a) {
    constexpr int NW = BLOCK / 32;
    constexpr int WT = 32 * ITEMS;  // paths per warp tile
    __shared__ long long s_wsum[NW][2];
    __shared__ long long s_lvl[4];
    const GraphDev &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x, GW = G * NW, gw = b * NW + wid;
    const unsigned lt_mask = (1u << lane) - 1u;
    const AggSlots A{a.agg, GW, G};

    // ---- counting pass over the first level of this launch ----
    {
        const int k = a.start_level;
        const long long count = __ldcg(&a.levels[k].count);
        const int chunk = warp_chunk(count, GW);
        const int lo = (int)min((long long)gw * chunk, count), hi = (int)min((long long)lo + chunk, count);
        const int2 *in_fl = a.tfl[k & 1];
        const unsigned *in_vis = a.tvis[k & 1];
        unsigned short *cnt = a.tcnt[k & 1];
        long long c_sum = 0, p_sum = 0;
        for (int i = lo + lane; i < hi; i += 32) {
            const int2 fl = __ldcg(in_fl + i);
            unsigned vis[W];
#pragma unroll
            for (int w = 0; w < W; ++w) vis[w] = __ldcg(in_vis + w * a.lvl_cap + i);
            const int vb = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + fl.x)) : 0;
            const unsigned cw = eval_path<W>(g, k, fl.x, fl.y, vb, vis, -1);
            cnt[i] = (unsigned short)cw;
            c_sum += cw & CNT_MASK;
            p_sum += cw >> 15;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c_sum += __shfl_xor_sync(0xffffffffu, c_sum, o);
            p_sum += __shfl_xor_sync(0xffffffffu, p_sum, o);
        }
        if (lane == 0) {
            A.wc(k % 3)[gw] = c_sum;
            A.wp(k % 3)[gw] = p_sum;
            A.wc((k + 1) % 3)[gw] = A.wp((k + 1) % 3)[gw] = 0;
            A.wc((k + 2) % 3)[gw] = A.wp((k + 2) % 3)[gw] = 0;
            s_wsum[wid][0] = c_sum;
            s_wsum[wid][1] = p_sum;
        }
        __syncthreads();
        if (tid == 0) {
            long long c = 0, p = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                c += s_wsum[w][0];
                p += s_wsum[w][1];
            }
            A.bc(k % 3)[b] = c;
            A.bp(k % 3)[b] = p;
            A.bc((k + 1) % 3)[b] = A.bp((k + 1) % 3)[b] = 0;
            A.bc((k + 2) % 3)[b] = A.bp((k + 2) % 3)[b] = 0;
        }
        if (!grid_barrier_tree(a.bar, a.err)) return;
    }

    for (int k = a.start_level; k + 1 < a.max_levels; ++k) {
        if (__ldcg(a.err) & (ERR_OVERFLOW_MASK | ERR_TIMEOUT | ERR_OVF_LEVELS | ERR_OVF_COUNT | ERR_INVAL)) break;
        const LevelRec *Lp = a.levels + k;
        const long long count = __ldcg(&Lp->count);
        if (count <= 0) break;
        int2 *const lnodes = (int2 *)__ldcg((const unsigned long long *)&Lp->nodes);
        int *const lpp = (int *)__ldcg((const unsigned long long *)&Lp->pp);
        int2 *const next = (k == a.start_level && a.next_nodes) ? a.next_nodes : lnodes + count;
        const long long next_off = next - a.seg;  // offset of the next level in the segment
        const long long pp_off = lpp - a.pp_seg;  // offset of this level's PPs in their segment
        const int2 *in_fl = a.tfl[k & 1];
        const unsigned *in_vis = a.tvis[k & 1];
        const unsigned short *in_cnt = a.tcnt[k & 1];
        int2 *out_fl = a.tfl[(k + 1) & 1];
        unsigned *out_vis = a.tvis[(k + 1) & 1];
        unsigned short *out_cnt = a.tcnt[(k + 1) & 1];
        const int s0 = k % 3, s1 = (k + 1) % 3, s2 = (k + 2) % 3;

        // level totals and this block's offsets: sums over the block entries
        {
            long long v[4] = {0, 0, 0, 0};
            for (int j = tid; j < G; j += BLOCK) {
                const long long c = __ldcg(A.bc(s0) + j), p = __ldcg(A.bp(s0) + j);
                v[0] += c;
                v[1] += p;
                if (j < b) {
                    v[2] += c;
                    v[3] += p;
                }
            }
            block_sum4<BLOCK>(v);
            if (tid == 0) {
                s_lvl[0] = v[0];
                s_lvl[1] = v[1];
                s_lvl[2] = v[2];
                s_lvl[3] = v[3];
                A.bc(s2)[b] = A.bp(s2)[b] = 0;
            }
            __syncthreads();
        }
        const long long C = s_lvl[0], P = s_lvl[1];
        // this warp's offsets: the block's plus the warp entries before it
        long long wc = 0, wpv = 0;
        if (lane < NW) {
            wc = __ldcg(A.wc(s0) + b * NW + lane);
            wpv = __ldcg(A.wp(s0) + b * NW + lane);
        }
        const long long own_c = __shfl_sync(0xffffffffu, wc, wid), own_p = __shfl_sync(0xffffffffu, wpv, wid);
        long long xc = lane < wid ? wc : 0, xp = lane < wid ? wpv : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            xc += __shfl_xor_sync(0xffffffffu, xc, o);
            xp += __shfl_xor_sync(0xffffffffu, xp, o);
        }
        if (lane == 0) A.wc(s2)[gw] = A.wp(s2)[gw] = 0;

        // every block takes the same decision from the same counts
        int e = 0;
        if (C >= (long long)MAX31 || P >= (long long)MAX31) e |= ERR_OVF_COUNT;
        if (next_off + C > a.seg_cap) e |= ERR_OVF_NODES;
        if (C > a.lvl_cap) e |= ERR_OVF_LEVEL;
        if (pp_off + P > a.pp_seg_cap) e |= ERR_OVF_PP;
        if (k + 2 >= a.max_levels && C > 0) e |= ERR_OVF_LEVELS;
        if (b == 0 && tid == 0) {
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
                a.levels[k + 1] = r;
            }
        }
        if (e) break;

        // all positions below fit in int32 (C, P < 2^31 - 1)
        const int chunk = warp_chunk(count, GW);
        const int lo = (int)min((long long)gw * chunk, count), hi = (int)min((long long)lo + chunk, count);
        const int chunk_n = C > 0 ? warp_chunk(C, GW) : 1;  // the next level's chunk
        const int pa = (int)(s_lvl[2] + xc), pb = (int)(s_lvl[3] + xp);
        int pos_c = pa, pos_p = pb;
        // next-level counts of the children this lane wrote, per owner chunk
        int cur_own = -1;
        unsigned bound = 0;  // first position of the chunk after cur_own
        unsigned long long acc_c = 0, acc_p = 0;

        for (int t0 = lo; t0 < hi; t0 += WT) {
            int first[ITEMS], last[ITEMS];
            unsigned cw[ITEMS];
            unsigned vis[ITEMS][W];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int i = t0 + j * 32 + lane;
                if (i < hi) {
                    const int2 fl = __ldcg(in_fl + i);
                    first[j] = fl.x;
                    last[j] = fl.y;
                    cw[j] = __ldcg(in_cnt + i);
#pragma unroll
                    for (int w = 0; w < W; ++w) vis[j][w] = __ldcg(in_vis + w * a.lvl_cap + i);
                } else {
                    first[j] = -1;
                    last[j] = 0;
                    cw[j] = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) vis[j][w] = 0u;
                }
            }
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int i = t0 + j * 32 + lane;
                const int nch = (int)(cw[j] & CNT_MASK);
                const bool pp = (cw[j] & CNT_PP) != 0;
                int x = nch;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const int tot = __shfl_sync(0xffffffffu, x, 31);
                const unsigned ppm = __ballot_sync(0xffffffffu, pp);
                if (a.root_counts) {
                    // per-root totals: paths arrive sorted by first vertex, so
                    // a warp's lanes mostly share one root; one atomic per group
                    const unsigned grp = __match_any_sync(0xffffffffu, first[j]);
                    const unsigned c0 = __reduce_add_sync(grp, first[j] >= 0 ? 1u : 0u);
                    const unsigned c1 = __reduce_add_sync(grp, pp ? 1u : 0u);
                    const unsigned c2 = __reduce_add_sync(grp, pp ? (unsigned)k : 0u);
                    if (first[j] >= 0 && lane == __ffs(grp) - 1) {
                        unsigned long long *rc = a.root_counts + 3ll * first[j];
                        atomicAdd(rc, (unsigned long long)c0);
                        if (c1) atomicAdd(rc + 1, (unsigned long long)c1);
                        if (c2) atomicAdd(rc + 2, (unsigned long long)c2);
                    }
                }
                if (nch > 0) {
                    const int vb = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + first[j])) : 0;
                    int cpos = pos_c + x - nch;
                    const int e0 = __ldg(g.rp + last[j]), e1 = __ldg(g.rp + last[j] + 1);
                    for (int e = e0; e < e1; ++e) {
                        const int w = __ldg(g.col + e);
                        const bool closes = (w == first[j]);
                        if (!closes && test_bit<W>(vis[j], w - vb)) continue;
                        const unsigned c2w = eval_path<W>(g, k + 1, first[j], w, vb, vis[j], w);
                        if (cpos < C && next_off + cpos < a.seg_cap) {  // holds when the counts agree
                            next[cpos] = make_int2(w, i);
                            out_fl[cpos] = make_int2(first[j], w);
                            out_cnt[cpos] = (unsigned short)c2w;
                            if (!closes) {
                                const int bb = w - vb;
#pragma unroll
                                for (int ww = 0; ww < W; ++ww)
                                    out_vis[ww * a.lvl_cap + cpos] =
                                        vis[j][ww] | ((ww == (bb >> 5)) ? (1u << (bb & 31)) : 0u);
                            }
                            if ((unsigned)cpos >= bound) {
                                // the child belongs to a later chunk: hand over
                                // the finished owner's counts
                                if (cur_own >= 0 && (acc_c | acc_p)) {
                                    atomicAdd((unsigned long long *)A.wc(s1) + cur_own, acc_c);
                                    atomicAdd((unsigned long long *)A.bc(s1) + cur_own / NW, acc_c);
                                    if (acc_p) {
                                        atomicAdd((unsigned long long *)A.wp(s1) + cur_own, acc_p);
                                        atomicAdd((unsigned long long *)A.bp(s1) + cur_own / NW, acc_p);
                                    }
                                }
                                cur_own = cpos / chunk_n;
                                bound = (unsigned)(cur_own + 1) * (unsigned)chunk_n;
                                acc_c = acc_p = 0;
                            }
                            acc_c += c2w & CNT_MASK;
                            acc_p += c2w >> 15;
                        }
                        ++cpos;
                    }
                }
                if (pp) {
                    const int q = pos_p + __popc(ppm & lt_mask);
                    if (pp_off + q < a.pp_seg_cap) lpp[q] = i;
                }
                pos_c += tot;
                pos_p += __popc(ppm);
            }
        }
        flush_counts<NW>(A, s1, cur_own, acc_c, acc_p);
        // the chunk must have produced exactly what its count promised
        if (lane == 0 && (pos_c - pa != own_c || pos_p - pb != own_p)) atomicOr(a.err, ERR_INVAL);
        if (!grid_barrier_tree(a.bar, a.err)) break;
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
    if (args.agg_cap < 3 * (2ll * grid * (BLOCK / 32) + 2ll * grid)) return cudaErrorInvalidValue;
    cudaError_t e;
    if (args.seed_level1) {
        if ((e = launch_seed_level1(args, s)) != cudaSuccess) return e;
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
    return EnumShape{256, 2};
}

int bitset_words_supported(int maxn) {
    const int w = (maxn + 31) / 32;
    const int sizes[] = {1, 2, 3, 4, 5, 6, 8, 16, 32, 64, 128};
    for (int s : sizes)
        if (w <= s) return s;
    return -1;
}

long long round_frontier_cap(long long x) {
    const long long q = 2048, top = ((long long)MAX31 - 1) / q * q;
    const long long r = (x + q - 1) / q * q;
    return r < q ? q : (r > top ? top : r);
}

template <int W>
static cudaError_t seed_w(const EnumArgs &args, cudaStream_t s) {
    init_level1_kernel<W><<<(args.g.N + 255) / 256, 256, 0, s>>>(args);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_seed_level1(const EnumArgs &args, cudaStream_t s) {
    switch (args.g.W) {
        case 1: return seed_w<1>(args, s);
        case 2: return seed_w<2>(args, s);
        case 3: return seed_w<3>(args, s);
        case 4: return seed_w<4>(args, s);
        case 5: return seed_w<5>(args, s);
        case 6: return seed_w<6>(args, s);
        case 8: return seed_w<8>(args, s);
        case 16: return seed_w<16>(args, s);
        case 32: return seed_w<32>(args, s);
        case 64: return seed_w<64>(args, s);
        case 128: return seed_w<128>(args, s);
        default: return cudaErrorInvalidValue;
    }
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
