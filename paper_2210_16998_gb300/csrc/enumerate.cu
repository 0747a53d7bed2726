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
#include <mutex>

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

// What a path of level k does next (Alg. 3 extension and prune steps): which
// successors of its last vertex extend it (simple one-vertex extensions,
// closing arcs included) and whether it is prime, packed as a count word
// (see CNT_BITS).  A closed cycle (k >= 2, first == last) is never extended
// and always prime.  `extra` is a vertex on the path that is not in `vis`
// (-1 for none): a child is evaluated as its parent's bitset plus the
// child's last vertex.
template <int W>
__device__ __forceinline__ unsigned eval_path(const GraphDev &g, int k, int first, int last, int vb,
                                              const unsigned (&vis)[W], int extra) {
    if (k >= 2 && first == last) return CNT_PP;
    const int e0 = __ldg(g.rp + last), e1 = __ldg(g.rp + last + 1);
    if (e1 - e0 <= CNT_MASK_DEG) {
        unsigned m = 0;
        for (int e = e0; e < e1; ++e) {
            const int w = __ldg(g.col + e);
            if (w == first || (w != extra && !test_bit<W>(vis, w - vb))) m |= 1u << (e - e0);
        }
        if (m) return m;
    } else {
        unsigned c = 0;
        for (int e = e0; e < e1; ++e) {
            const int w = __ldg(g.col + e);
            if (w == first || (w != extra && !test_bit<W>(vis, w - vb))) ++c;
        }
        if (c) return CNT_WIDE | c;
    }
    // right-maximal; left-maximal iff every predecessor u of the first vertex
    // is on the path and is not its last vertex (u.p would otherwise be simple)
    const int p0 = __ldg(g.prp + first), p1 = __ldg(g.prp + first + 1);
    for (int e = p0; e < p1; ++e) {
        const int u = __ldg(g.pcol + e);
        if (u == last || (u != extra && !test_bit<W>(vis, u - vb))) return 0u;
    }
    return CNT_PP;
}

// With the vertex bitsets (bitsets of at most MASK_MAX_W words): the
// successors of `last` that extend the path as a W-word bitset of local ids
// (the successors not on the path, plus the first vertex when the arc to it
// closes a cycle).  Ascending bit order is ascending successor id.
template <int W>
__device__ __forceinline__ void ext_mask(const GraphDev &g, int first, int last, int vb, const unsigned (&vis)[W],
                                         unsigned (&m)[W]) {
    const unsigned *sm = g.smask + (long long)last * W;
    const int fb = first - vb;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const unsigned sj = __ldg(sm + j);
        m[j] = (sj & ~vis[j]) | ((j == (fb >> 5)) ? (sj & (1u << (fb & 31))) : 0u);
    }
}

// eval_path with the vertex bitsets, for a path whose visited set is `vis`
// (last vertex included): the count word holds the number of extending
// successors (CNT_WIDE form); with none, the path is prime iff every
// predecessor of its first vertex is on it (the last vertex is never one
// here: an arc last -> first would be an extension).
template <int W>
__device__ __forceinline__ unsigned eval_mask(const GraphDev &g, int k, int first, int last, int vb,
                                              const unsigned (&vis)[W]) {
    if (k >= 2 && first == last) return CNT_PP;
    unsigned m[W];
    ext_mask<W>(g, first, last, vb, vis, m);
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) c += __popc(m[j]);
    if (c) return CNT_WIDE | c;
    const unsigned *pm = g.pmask + (long long)first * W;
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (__ldg(pm + j) & ~vis[j]) return 0u;
    return CNT_PP;
}

// position of the (r+1)-th set bit of m (r = 0: the lowest); m has more than r set bits
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
    for (; r > 0; --r) m &= m - 1;
    return __ffs(m) - 1;
}


#ifndef TPG_ENUM_TREE_BARRIER
#define TPG_ENUM_TREE_BARRIER 0  // grid barrier: 0 = one growing counter, 1 = two-level tree
#endif
#ifndef TPG_ENUM_MASK
#define TPG_ENUM_MASK 1  // evaluate paths with the vertex bitsets where they exist
#endif
#ifndef TPG_ENUM_PREFETCH
#define TPG_ENUM_PREFETCH 1  // load a warp's next tile of records while it processes the current one
#endif
#ifndef TPG_ENUM_LANEWISE
#define TPG_ENUM_LANEWISE 1  // lane-wise child writing when it needs no more rounds than dealing
#endif

#ifndef TPG_ENUM_PROLOGUE
#define TPG_ENUM_PROLOGUE 1  // a fresh run's small first levels run in block 0 alone
#endif

// The small first levels of a fresh run in one block.  A single graph's
// first levels hold few paths (one per vertex, then a few more per level),
// and with the whole grid each still costs a grid barrier and a prefix step
// for a few microseconds of work.  Block 0 walks them alone while a level
// holds at most BLOCK * PI paths: thread t takes a contiguous run of at most
// PI paths of the level, evaluates them (count word: extending successors,
// primality), one block scan places their children and PPs, the children
// are written in order (parent order, ascending successor id, as in the
// grid's levels), and __syncthreads separates the levels.  Every level makes
// the grid's capacity checks and stops the same way (the flags, the stop
// level, the level record).  Returns the level handed to the grid (the
// first one above the bound, or an empty one), 0 after a stop.
template <int W, int BLOCK, int PI, bool MASK>
__device__ __forceinline__ int enum_prologue(const EnumArgs &a) {
    const GraphDev &g = a.g;
    const int tid = threadIdx.x;
    int k = 1;
    long long count = __ldcg(&a.levels[1].count);
    int2 *lnodes = (int2 *)__ldcg((const unsigned long long *)&a.levels[1].nodes);
    int *lpp = (int *)__ldcg((const unsigned long long *)&a.levels[1].pp);
    while (count > 0 && count <= (long long)BLOCK * PI && k + 1 < a.max_levels) {
        const unsigned long long t_start = a.trace ? global_ns() : 0ull;
        int2 *const next = lnodes + count;
        const long long next_off = next - a.seg, pp_off = lpp - a.pp_seg;
        const int2 *in_fl = a.tfl[k & 1];
        const unsigned *in_vis = a.tvis[k & 1];
        int2 *out_fl = a.tfl[(k + 1) & 1];
        unsigned *out_vis = a.tvis[(k + 1) & 1];
        const int n = (int)count, q = (n + BLOCK - 1) / BLOCK;  // q <= PI
        const int lo = min(tid * q, n), hi = min(lo + q, n);
        int first[PI], last[PI], vb[PI];
        unsigned vis[PI][W], cw[PI];
#pragma unroll
        for (int j = 0; j < PI; ++j) {
            const int i = lo + j;
            first[j] = last[j] = vb[j] = 0;
            cw[j] = 0u;
#pragma unroll
            for (int w = 0; w < W; ++w) vis[j][w] = 0u;
            if (i < hi) {
                const int2 fl = __ldcg(in_fl + i);
                // clamped into range before any use as an index (as in the grid's levels)
                first[j] = (int)min((unsigned)fl.x, (unsigned)(g.N - 1));
                last[j] = (int)min((unsigned)fl.y, (unsigned)(g.N - 1));
#pragma unroll
                for (int w = 0; w < W; ++w) vis[j][w] = __ldcg(in_vis + w * a.lvl_cap + i);
            }
        }
        unsigned long long cp = 0;  // children << 32 | PPs of this thread's paths
#pragma unroll
        for (int j = 0; j < PI; ++j) {
            if (lo + j < hi) {
                vb[j] = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + first[j])) : 0;
                if constexpr (MASK) cw[j] = eval_mask<W>(g, k, first[j], last[j], vb[j], vis[j]);
                else cw[j] = eval_path<W>(g, k, first[j], last[j], vb[j], vis[j], -1);
                cp += ((unsigned long long)cnt_children(cw[j]) << 32) | (cw[j] >> 15);
            }
        }
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan_u64<BLOCK>(cp, tot);
        const long long C = (long long)(tot >> 32), P = (long long)(tot & 0xffffffffull);
        int e = 0;
        if (C >= (long long)MAX31 || P >= (long long)MAX31) e |= ERR_OVF_COUNT;
        if (next_off + C > a.seg_cap) e |= ERR_OVF_NODES;
        if (C > a.lvl_cap) e |= ERR_OVF_LEVEL;
        if (pp_off + P > a.pp_seg_cap) e |= ERR_OVF_PP;
        if (k + 2 >= a.max_levels && C > 0) e |= ERR_OVF_LEVELS;
        if (tid == 0) {
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
        if (e) return 0;
        int pos_c = (int)(ex >> 32), pos_p = (int)(ex & 0xffffffffull);
#pragma unroll
        for (int j = 0; j < PI; ++j) {
            const int i = lo + j;
            if (i >= hi) continue;
            if (cw[j] & CNT_PP) lpp[pos_p++] = i;
            if (cnt_children(cw[j]) == 0) continue;
            auto child = [&](int w) {
                const int bb = w - vb[j];
                next[pos_c] = make_int2(w, i);
                out_fl[pos_c] = make_int2(first[j], w);
                if (w != first[j]) {
#pragma unroll
                    for (int ww = 0; ww < W; ++ww)
                        out_vis[ww * a.lvl_cap + pos_c] = vis[j][ww] | ((ww == (bb >> 5)) ? (1u << (bb & 31)) : 0u);
                }
                ++pos_c;
            };
            if constexpr (MASK) {
                unsigned m[W];
                ext_mask<W>(g, first[j], last[j], vb[j], vis[j], m);
#pragma unroll
                for (int ww = 0; ww < W; ++ww)
                    for (unsigned x = m[ww]; x; x &= x - 1) child(vb[j] + 32 * ww + __ffs(x) - 1);
            } else {
                const int e0 = __ldg(g.rp + last[j]), e1 = __ldg(g.rp + last[j] + 1);
                for (int ed = e0; ed < e1; ++ed) {
                    const int w = __ldg(g.col + ed);
                    if (w == first[j] || !test_bit<W>(vis[j], w - vb[j])) child(w);
                }
            }
        }
        if (a.trace && tid == 0) {
            unsigned long long *tr = a.trace + LEVEL_TRACE_WORDS * k;
            const unsigned long long t_end = global_ns();
            atomicMax(tr, ~t_start);
            atomicMax(tr + 1, t_end);
            atomicAdd(tr + 2, t_end - t_start);
            atomicAdd(tr + 3, 1ull);
        }
        __syncthreads();  // this level's records are read by other threads of the block next
        count = C;
        lnodes = next;
        lpp += P;
        ++k;
    }
    return k;
}

// paths per chunk of a level of `count` paths cut into nchk chunks:
// ceil(count / nchk) rounded up to a multiple of 32
__device__ __forceinline__ int level_chunk(long long count, int nchk) {
    const long long q = (count + nchk - 1) / nchk;
    return (int)((q + 31) & ~31ll);
}

// Per-chunk counts of one level.  Slot s holds, for every chunk and for every
// group of 2^lg consecutive chunks (one block's), the children and the PPs it
// produces.
struct AggSlots {
    long long *base;
    int NC, G;  // chunks, groups (= blocks)
    int lg;     // log2 of the chunks per group
    __device__ long long *cc(int s) const { return base + s * (2ll * NC + 2ll * G); }
    __device__ long long *cp(int s) const { return cc(s) + NC; }
    __device__ long long *gc(int s) const { return cc(s) + 2ll * NC; }
    __device__ long long *gp(int s) const { return cc(s) + 2ll * NC + G; }
};

__device__ __forceinline__ void add_counts(const AggSlots &A, int s, int own, unsigned long long c,
                                           unsigned long long p) {
    // (c, p) fit 32 bits for one lane; a warp sum is widened before it is added
    if (c) {
        atomicAdd((unsigned long long *)A.cc(s) + own, c);
        atomicAdd((unsigned long long *)A.gc(s) + (own >> A.lg), c);
    }
    if (p) {
        atomicAdd((unsigned long long *)A.cp(s) + own, p);
        atomicAdd((unsigned long long *)A.gp(s) + (own >> A.lg), p);
    }
}

// Add (c, p) to chunk `own` of slot s (and to its group).  Lanes with nothing
// to add pass own = -1.  Lanes are grouped by owner and each group's leader
// adds the group's sums, so a warp issues one set of atomics per distinct
// owner (usually one).
__device__ __forceinline__ void flush_counts(const AggSlots &A, int s, int own, unsigned c, unsigned p) {
    const bool mine = own >= 0 && (c | p);
    if (!__any_sync(0xffffffffu, mine)) return;
    const unsigned peers = __match_any_sync(0xffffffffu, mine ? own : -1);
    // (32-bit sums: one chunk holds < 2^31 / NC + 32 paths of < 2^13 children each)
    const unsigned sc = __reduce_add_sync(peers, mine ? c : 0u);
    const unsigned sp = __reduce_add_sync(peers, mine ? p : 0u);
    if (mine && (threadIdx.x & 31) == __ffs(peers) - 1) add_counts(A, s, own, sc, sp);
}

// One persistent cooperative launch walks the levels.  Level k is cut into
// NC = CPG * G equal contiguous chunks, and each chunk into `split` work
// units; warp w of block b takes units w * G + b, then every GW-th after it,
// so each warp's and each block's (SM's) work is spread over the whole level
// and a region of costly paths is shared by many warps and SMs.  Any chunk's
// offsets in level k+1 and in the PP list are known before the level starts:
// the count word of each path of level k (tcnt) was computed when that path
// was written, and the writer added it to the entry of the chunk that owns
// the path and to that chunk's group (CPG consecutive chunks).  After one
// grid barrier per level each block scans the G group totals into shared
// memory; a warp that claims chunk c adds the entries of the chunks before c
// in its group (and, for a later unit of the chunk, the children and PPs of
// the chunk's earlier units, summed from their count words).  The warp walks
// its unit in tiles of 32 * ITEMS paths (lane l owns paths j*32 + l, so
// every load is coalesced) with warp-level scans only, and writes every
// child together with the child's own count word.
// Each path is read once and written once.
//
// Slots rotate: level k reads slot k%3, accumulates into slot (k+1)%3, and
// each block clears its group's entries of slot (k+2)%3, which nobody reads
// or accumulates until after the next barrier.  The first level the grid
// walks (level 1 of a fresh run, the level a resume starts at, or the level
// handed over by the single-block start, enum_prologue) is counted by a
// separate pass with a static chunk assignment.
template <int W, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK, W <= 8 ? 1024 / BLOCK : 1) enumerate_kernel(EnumArgs a) {
    constexpr int NW = BLOCK / 32;
    constexpr int CPG = ENUM_UPW * NW;  // chunks per block: a level is cut into CPG * blocks chunks
    constexpr int LG = CPG >= 256 ? 8 : CPG >= 128 ? 7 : CPG >= 64 ? 6 : 5;
    constexpr int F = CPG / NW;      // chunks per warp in the counting pass
    constexpr bool MASK = TPG_ENUM_MASK && W <= MASK_MAX_W;  // successor / predecessor bitsets in g.smask, g.pmask
    constexpr int WT = 32 * ITEMS;  // paths per warp tile
    static_assert(CPG % NW == 0, "a block's warps split its chunks evenly");
    static_assert(CPG % 32 == 0 && CPG <= BLOCK, "lanes split a group's entries; threads clear them");
    static_assert(CPG == (1 << LG), "chunks per block: a power of two from 32 to 256");
    extern __shared__ long long s_gpre[];  // [2 * G]: exclusive group prefixes (children, PPs)
    __shared__ long long s_wsum[NW][2];
    __shared__ long long s_tot[2];
    __shared__ unsigned long long s_t0[NW];  // trace: start of each warp's work in the level
    __shared__ unsigned long long s_tr[3];   // trace: the block's latest end, summed busy time, busy warps
    __shared__ int s_next;                   // next of the block's units to claim in this level
    const GraphDev &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x, NC = CPG * G;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (tid < 3) s_tr[tid] = 0ull;  // (read after the first level's __syncthreads)
    const AggSlots A{a.agg, NC, G, LG};
    // the grid barrier between levels: one growing arrival counter, or the
    // two-level tree (TPG_ENUM_TREE_BARRIER)
    unsigned bar_target = 0;
    auto enum_barrier = [&](unsigned target, int stop) -> bool {
        if constexpr (TPG_ENUM_TREE_BARRIER) return grid_barrier_tree(a.bar, a.err, stop, a.spin_ns);
        else return grid_barrier_count(a.bar, target, a.err, stop, a.spin_ns);
    };

    // a fresh run's small first levels: block 0 alone, the grid waits once
    int k_first = a.start_level;
    if constexpr (TPG_ENUM_PROLOGUE) {
        if (a.handoff && a.seed_level1 && a.start_level == 1 && !a.root_counts) {
            constexpr int PI = (W <= 4 ? 4 : 2) * BLOCK <= 2048 ? (W <= 4 ? 4 : 2) : 2048 / BLOCK;
            if (b == 0) {
                const int k0 = enum_prologue<W, BLOCK, PI, MASK>(a);
                if (tid == 0) *a.handoff = k0;
            }
            bar_target += G;
            if (!enum_barrier(bar_target, ERR_TIMEOUT | ERR_OVERFLOW_MASK | ERR_OVF_COUNT | ERR_OVF_LEVELS)) return;
            k_first = __ldcg(a.handoff);
        }
    }

    // ---- counting pass over the first level of this launch ----
    {
        const int k = k_first;
        const long long count = __ldcg(&a.levels[k].count);
        const int chunk = level_chunk(count, NC);
        const int2 *in_fl = a.tfl[k & 1];
        const unsigned *in_vis = a.tvis[k & 1];
        unsigned short *cnt = a.tcnt[k & 1];
        long long wc_sum = 0, wp_sum = 0;
        for (int f = 0; f < F; ++f) {
            const int c = b * CPG + wid * F + f;
            const int lo = (int)min((long long)c * chunk, count), hi = (int)min((long long)lo + chunk, count);
            long long c_sum = 0, p_sum = 0;
            for (int i = lo + lane; i < hi; i += 32) {
                int2 fl = __ldcg(in_fl + i);
                // ids are clamped into range before any use as an index (a
                // record is a path whenever the level counts agree, which the
                // chunks check; this only keeps a broken count from faulting)
                fl.x = (int)min((unsigned)fl.x, (unsigned)(g.N - 1));
                fl.y = (int)min((unsigned)fl.y, (unsigned)(g.N - 1));
                unsigned vis[W];
#pragma unroll
                for (int w = 0; w < W; ++w) vis[w] = __ldcg(in_vis + w * a.lvl_cap + i);
                const int vb = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + fl.x)) : 0;
                unsigned cw;
                if constexpr (MASK) cw = eval_mask<W>(g, k, fl.x, fl.y, vb, vis);
                else cw = eval_path<W>(g, k, fl.x, fl.y, vb, vis, -1);
                cnt[i] = (unsigned short)cw;
                c_sum += cnt_children(cw);
                p_sum += cw >> 15;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c_sum += __shfl_xor_sync(0xffffffffu, c_sum, o);
                p_sum += __shfl_xor_sync(0xffffffffu, p_sum, o);
            }
            if (lane == 0) {
                A.cc(k % 3)[c] = c_sum;
                A.cp(k % 3)[c] = p_sum;
                A.cc((k + 1) % 3)[c] = A.cp((k + 1) % 3)[c] = 0;
                A.cc((k + 2) % 3)[c] = A.cp((k + 2) % 3)[c] = 0;
            }
            wc_sum += c_sum;
            wp_sum += p_sum;
        }
        if (lane == 0) {
            s_wsum[wid][0] = wc_sum;
            s_wsum[wid][1] = wp_sum;
        }
        __syncthreads();
        if (tid == 0) {
            long long c = 0, p = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                c += s_wsum[w][0];
                p += s_wsum[w][1];
            }
            A.gc(k % 3)[b] = c;
            A.gp(k % 3)[b] = p;
            A.gc((k + 1) % 3)[b] = A.gp((k + 1) % 3)[b] = 0;
            A.gc((k + 2) % 3)[b] = A.gp((k + 2) % 3)[b] = 0;
        }
        bar_target += G;
        if (!enum_barrier(bar_target, ERR_TIMEOUT)) return;
    }

    // the level being processed; after the first, every block derives the
    // next level's record from the totals it computed itself
    long long count = __ldcg(&a.levels[k_first].count);
    int2 *lnodes = (int2 *)__ldcg((const unsigned long long *)&a.levels[k_first].nodes);
    int *lpp = (int *)__ldcg((const unsigned long long *)&a.levels[k_first].pp);
    for (int k = k_first; k + 1 < a.max_levels && count > 0; ++k) {
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

        // exclusive prefixes of the group totals, and the level totals
        {
            const int per = (G + BLOCK - 1) / BLOCK, g0 = min(tid * per, G), g1 = min(g0 + per, G);
            long long sc = 0, sp = 0;
            for (int q = g0; q < g1; ++q) {
                sc += __ldcg(A.gc(s0) + q);
                sp += __ldcg(A.gp(s0) + q);
            }
            long long tc, tp;
            long long xc = block_excl_scan_i64<BLOCK>(sc, tc);
            long long xp = block_excl_scan_i64<BLOCK>(sp, tp);
            for (int q = g0; q < g1; ++q) {
                s_gpre[q] = xc;
                s_gpre[G + q] = xp;
                xc += __ldcg(A.gc(s0) + q);
                xp += __ldcg(A.gp(s0) + q);
            }
            if (tid == 0) {
                s_tot[0] = tc;
                s_tot[1] = tp;
                A.gc(s2)[b] = A.gp(s2)[b] = 0;
                s_next = NW;  // the block's units 0 .. NW-1 go to its warps in order
            }
            if (tid < CPG) A.cc(s2)[b * CPG + tid] = A.cp(s2)[b * CPG + tid] = 0;
            __syncthreads();
        }
        const long long C = s_tot[0], P = s_tot[1];
        if (a.trace && tid == 0) atomicMax(a.trace + LEVEL_TRACE_WORDS * k, ~global_ns());

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
        const int chunk = level_chunk(count, NC);
        const int nchk = (int)((count + chunk - 1) / chunk);  // chunks that hold paths
        const int chunk_n = C > 0 ? level_chunk(C, NC) : 1;  // the next level's chunk
        // next-level counts of the children this lane wrote, per owner chunk;
        // a finished owner's counts retire and are flushed by the whole warp
        // (32-bit sums: a chunk holds < 2^31 / NC + 32 positions of < 2^13 children)
        int cur_own = -1, ret_own = -1;
        unsigned bound = 0;  // first position of the chunk after cur_own
        unsigned acc_c = 0, acc_p = 0, ret_c = 0, ret_p = 0;

        // the entries of chunk c's group that precede c (r = c's place in
        // the group), summed per lane: lane l takes those at l, l + 32, ...
        auto load_entries = [&](int c, long long &sc, long long &sp) {
            sc = sp = 0;
            if (c < nchk) {
                const int grp = c / CPG, r = c - grp * CPG;
                const long long *ecc = A.cc(s0) + (long long)grp * CPG, *ecp = A.cp(s0) + (long long)grp * CPG;
#pragma unroll
                for (int t = 0; t < CPG / 32; ++t) {
                    const int q = t * 32 + lane;
                    if (q < r) {
                        sc += __ldcg(ecc + q);
                        sp += __ldcg(ecp + q);
                    }
                }
            }
        };
        // Work units: part s of chunk c (SPLIT parts of sub paths) is unit
        // c * SPLIT + s.  Block b owns units b, b + G, b + 2G, ...: every
        // block (one SM's share of the issue slots) samples the whole level,
        // so a costly region is spread over all SMs.  Its warps take its
        // first NW units in order and then claim the rest one at a time from
        // a shared-memory counter (claimed one unit ahead), so within the SM
        // a warp whose units were cheap takes more of them.  A part's offsets
        // are its chunk's plus the children and PPs of the chunk's earlier
        // parts, summed from their count words, whichever warp takes it.
        const int SPLIT = a.split < 1 ? 1 : (a.split > 4 ? 4 : a.split);
        const int nunit = nchk * SPLIT;
        const int sub = ((chunk + SPLIT - 1) / SPLIT + 31) & ~31;
        long long ec, ep;
        int u = b + G * wid;
        load_entries(SPLIT == 1 ? u : u / SPLIT, ec, ep);
        if (a.trace && lane == 0) s_t0[wid] = u < nunit ? global_ns() : 0ull;
        while (u < nunit) {
            const int c = SPLIT == 1 ? u : u / SPLIT, part = u - c * SPLIT;
            // the next unit is claimed, and its chunk entries load, while
            // this unit is processed
            int i_next = 0;
            if (lane == 0) i_next = atomicAdd(&s_next, 1);
            const int u_next = b + G * __shfl_sync(0xffffffffu, i_next, 0);
            long long ec_next, ep_next;
            load_entries(SPLIT == 1 ? u_next : u_next / SPLIT, ec_next, ep_next);
            // offsets of chunk c: its group's prefix plus the chunks before it
            // in the group; its own entry is checked when its last part is done
            const int grp = c / CPG;
            const bool last_part = part == SPLIT - 1;
            const long long own_c = last_part ? __ldcg(A.cc(s0) + c) : 0, own_p = last_part ? __ldcg(A.cp(s0) + c) : 0;
            long long xc = ec, xp = ep;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                xc += __shfl_xor_sync(0xffffffffu, xc, o);
                xp += __shfl_xor_sync(0xffffffffu, xp, o);
            }
            const int pa = (int)(s_gpre[grp] + xc), pb = (int)(s_gpre[G + grp] + xp);
            const int clo = (int)min((long long)c * chunk, count), chi = (int)min((long long)clo + chunk, count);
            const int lo = min(clo + part * sub, chi), hi = min(lo + sub, chi);
            int pos_c = pa, pos_p = pb;
            if (part > 0) {
                unsigned sc = 0, sp = 0;
#pragma unroll 4
                for (int i = clo + lane; i < lo; i += 32) {
                    const unsigned w = __ldcg(in_cnt + i);
                    sc += (unsigned)cnt_children(w);
                    sp += w >> 15;
                }
                pos_c += (int)__reduce_add_sync(0xffffffffu, sc);
                pos_p += (int)__reduce_add_sync(0xffffffffu, sp);
            }

#if TPG_ENUM_PREFETCH
            // the records of the next tile load while this one is processed
            int2 pfl[ITEMS];
            unsigned pcw[ITEMS], pvis[ITEMS][W];
            auto load_tile = [&](int t0) {
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const int i = t0 + j * 32 + lane;
                    if (i < hi) {
                        pfl[j] = __ldcg(in_fl + i);
                        pcw[j] = __ldcg(in_cnt + i);
#pragma unroll
                        for (int w = 0; w < W; ++w) pvis[j][w] = __ldcg(in_vis + w * a.lvl_cap + i);
                    }
                }
            };
            if (lo < hi) load_tile(lo);
#endif
            for (int t0 = lo; t0 < hi; t0 += WT) {
                int first[ITEMS], last[ITEMS];
                unsigned cw[ITEMS];
                unsigned vis[ITEMS][W];
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const int i = t0 + j * 32 + lane;
                    if (i < hi) {
#if TPG_ENUM_PREFETCH
                        const int2 fl = pfl[j];
                        cw[j] = pcw[j];
#pragma unroll
                        for (int w = 0; w < W; ++w) vis[j][w] = pvis[j][w];
#else
                        const int2 fl = __ldcg(in_fl + i);
                        cw[j] = __ldcg(in_cnt + i);
#pragma unroll
                        for (int w = 0; w < W; ++w) vis[j][w] = __ldcg(in_vis + w * a.lvl_cap + i);
#endif
                        // clamped into range before any use as an index (see
                        // the counting pass)
                        first[j] = (int)min((unsigned)fl.x, (unsigned)(g.N - 1));
                        last[j] = (int)min((unsigned)fl.y, (unsigned)(g.N - 1));
                    } else {
                        first[j] = -1;
                        last[j] = 0;
                        cw[j] = 0;
#pragma unroll
                        for (int w = 0; w < W; ++w) vis[j][w] = 0u;
                    }
                }
#if TPG_ENUM_PREFETCH
                if (t0 + WT < hi) load_tile(t0 + WT);
#endif
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    const int i = t0 + j * 32 + lane;
                    const int nch = cnt_children(cw[j]);
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
                        // per-root totals: paths arrive sorted by first vertex,
                        // so a warp's lanes mostly share one root
                        const unsigned grp2 = __match_any_sync(0xffffffffu, first[j]);
                        const unsigned c0 = __reduce_add_sync(grp2, first[j] >= 0 ? 1u : 0u);
                        const unsigned c1 = __reduce_add_sync(grp2, pp ? 1u : 0u);
                        const unsigned c2 = __reduce_add_sync(grp2, pp ? (unsigned)k : 0u);
                        if (first[j] >= 0 && lane == __ffs(grp2) - 1) {
                            unsigned long long *rc = a.root_counts + 3ll * first[j];
                            atomicAdd(rc, (unsigned long long)c0);
                            if (c1) atomicAdd(rc + 1, (unsigned long long)c1);
                            if (c2) atomicAdd(rc + 2, (unsigned long long)c2);
                        }
                    }
                    const int excl = x - nch;
                    int vb_l = 0, e0_l = 0;
                    if (nch > 0) {
                        vb_l = g.vgraph ? __ldg(g.vbase + __ldg(g.vgraph + first[j])) : 0;
                        if constexpr (!MASK) e0_l = __ldg(g.rp + last[j]);
                    }
                    // one child record: arena node, frontier record with the
                    // child's own count word (evaluated here), bitset, and its
                    // share of the next level's chunk counts
                    // fbm: the parent's first vertex as a W-word bitset (with
                    // the vertex bitsets; a successor equal to it closes a cycle)
                    auto emit = [&](int w, int cpos, int pf, int pvb, const unsigned (&pvis)[W], int pi,
                                    const unsigned (&fbm)[W]) {
                        const bool closes = (w == pf);
                        const int bb = w - pvb;
                        unsigned cvis[W];  // the child's visited set
#pragma unroll
                        for (int ww = 0; ww < W; ++ww) cvis[ww] = pvis[ww] | ((ww == (bb >> 5)) ? (1u << (bb & 31)) : 0u);
                        // the child's count word (eval_mask / eval_path), with its
                        // children and PP flag kept apart for the chunk counts
                        unsigned c2w, cc, cp;
                        if constexpr (MASK) {
                            if (closes) {
                                c2w = CNT_PP;
                                cc = 0u;
                                cp = 1u;
                            } else {
                                const unsigned *sm = g.smask + (long long)w * W;
                                unsigned c = 0u;
#pragma unroll
                                for (int ww = 0; ww < W; ++ww) c += __popc(__ldg(sm + ww) & (~cvis[ww] | fbm[ww]));
                                if (c) {
                                    c2w = CNT_WIDE | c;
                                    cc = c;
                                    cp = 0u;
                                } else {
                                    // prime iff every predecessor of the first vertex is on it
                                    const unsigned *pm = g.pmask + (long long)pf * W;
                                    unsigned off = 0u;
#pragma unroll
                                    for (int ww = 0; ww < W; ++ww) off |= __ldg(pm + ww) & ~cvis[ww];
                                    cp = off ? 0u : 1u;
                                    c2w = off ? 0u : CNT_PP;
                                    cc = 0u;
                                }
                            }
                        } else {
                            c2w = eval_path<W>(g, k + 1, pf, w, pvb, pvis, w);
                            cc = (unsigned)cnt_children(c2w);
                            cp = c2w >> 15;
                        }
                        if (cpos < C) {  // holds when the counts agree; C fits the segment and the frontier
                            next[cpos] = make_int2(w, pi);
                            out_fl[cpos] = make_int2(pf, w);
                            out_cnt[cpos] = (unsigned short)c2w;
                            if (!closes) {
#pragma unroll
                                for (int ww = 0; ww < W; ++ww) out_vis[ww * a.lvl_cap + cpos] = cvis[ww];
                            }
                            if ((unsigned)cpos >= bound) {
                                // the child belongs to a later chunk: the
                                // finished owner's counts retire
                                if (ret_own >= 0) add_counts(A, s1, ret_own, ret_c, ret_p);  // rare: 2nd in one item
                                ret_own = cur_own;
                                ret_c = acc_c;
                                ret_p = acc_p;
                                cur_own = cpos / chunk_n;
                                bound = (unsigned)(cur_own + 1) * (unsigned)chunk_n;
                                acc_c = acc_p = 0;
                            }
                            acc_c += cc;
                            acc_p += cp;
                        }
                    };
                    auto first_bits = [&](int pf, int pvb, unsigned (&fbm)[W]) {
                        const int fb = pf - pvb;
#pragma unroll
                        for (int ww = 0; ww < W; ++ww) fbm[ww] = (ww == (fb >> 5)) ? (1u << (fb & 31)) : 0u;
                    };
                    // Two ways to write the item's children.  Lane-wise: each
                    // lane writes its own path's children, one per round, for
                    // as many rounds as the busiest lane has children (no
                    // shuffles; chosen when that is at most about as many
                    // rounds as dealing needs).  Dealt: child q of the warp
                    // (0 <= q < tot, at position pos_c + q) goes to lane q % 32,
                    // which finds its parent lane (the last lane whose first
                    // child is at or before q) and reads the parent's path
                    // through shuffles, so a parent with many children costs
                    // the warp one round per 32 children and the child records
                    // are stored contiguously.
                    const int maxc = (int)__reduce_max_sync(0xffffffffu, (unsigned)nch);
                    // with the vertex bitsets, the extending successors as a
                    // bitset (none when the count word says so: a closed cycle)
                    unsigned xm[MASK ? W : 1];
                    unsigned fbm_l[W];  // this lane's parent's first vertex (lane-wise writing)
                    if constexpr (MASK) {
                        first_bits(first[j], vb_l, fbm_l);
                        if (nch > 0) {
                            const unsigned *sm = g.smask + (long long)last[j] * W;
#pragma unroll
                            for (int ww = 0; ww < W; ++ww) xm[ww] = __ldg(sm + ww) & (~vis[j][ww] | fbm_l[ww]);
                        } else {
#pragma unroll
                            for (int ww = 0; ww < W; ++ww) xm[ww] = 0u;
                        }
                    }
                    const bool lanewise = TPG_ENUM_LANEWISE &&
                                          (TPG_ENUM_LANEWISE == 1 ? 3 * maxc <= 4 * ((tot + 31) >> 5)
                                                                  : maxc <= ((tot + 31) >> 5)) &&
                                          (MASK || !__any_sync(0xffffffffu, (cw[j] & CNT_WIDE) != 0u));
                    if (lanewise) {
                        const int pi = t0 + j * 32 + lane;
                        if constexpr (MASK) {
                            for (int r = 0; r < maxc; ++r) {
                                // the next extending successor, ascending
                                int w = -1;
#pragma unroll
                                for (int ww = 0; ww < W; ++ww)
                                    if (w < 0 && xm[ww]) {
                                        w = vb_l + 32 * ww + __ffs(xm[ww]) - 1;
                                        xm[ww] &= xm[ww] - 1;
                                    }
                                if (w >= 0) emit(w, pos_c + excl + r, first[j], vb_l, vis[j], pi, fbm_l);
                            }
                        } else {
                            unsigned m = cw[j] & CNT_BITS;
                            for (int r = 0; r < maxc; ++r) {
                                if (m) {
                                    const int sidx = __ffs(m) - 1;
                                    m &= m - 1;
                                    // (clamped: a wrong count word must not index past the arcs)
                                    const int w = __ldg(g.col + min((unsigned)(e0_l + sidx), (unsigned)(g.M - 1)));
                                    emit(w, pos_c + excl + r, first[j], vb_l, vis[j], pi, fbm_l);
                                }
                            }
                        }
                    } else {
                        for (int q0 = 0; q0 < tot; q0 += 32) {
                            const int q = q0 + lane;
                            int p = 0;
#pragma unroll
                            for (int step = 16; step > 0; step >>= 1) {
                                const int cand = p + step;  // <= 31
                                if (__shfl_sync(0xffffffffu, excl, cand) <= q) p = cand;
                            }
                            const int pf = __shfl_sync(0xffffffffu, first[j], p);
                            const int pvb = __shfl_sync(0xffffffffu, vb_l, p);
                            const int rank = q - __shfl_sync(0xffffffffu, excl, p);
                            unsigned pvis[W];
#pragma unroll
                            for (int ww = 0; ww < W; ++ww) pvis[ww] = __shfl_sync(0xffffffffu, vis[j][ww], p);
                            const int pi = t0 + j * 32 + p;
                            if constexpr (MASK) {
                                unsigned pm[W];
#pragma unroll
                                for (int ww = 0; ww < W; ++ww) pm[ww] = __shfl_sync(0xffffffffu, xm[ww], p);
                                if (q >= tot) continue;
                                // the rank-th extending successor of the parent
                                int w = -1, rr = rank;
#pragma unroll
                                for (int ww = 0; ww < W; ++ww) {
                                    const int c = __popc(pm[ww]);
                                    if (w < 0) {
                                        if (rr < c) w = pvb + 32 * ww + nth_set_bit(pm[ww], rr);
                                        else rr -= c;
                                    }
                                }
                                unsigned fbm[W];
                                first_bits(pf, pvb, fbm);
                                if (w >= 0) emit(w, pos_c + q, pf, pvb, pvis, pi, fbm);
                                continue;
                            }
                            const int pl = __shfl_sync(0xffffffffu, last[j], p);
                            const int pe0 = __shfl_sync(0xffffffffu, e0_l, p);
                            const unsigned pcw = __shfl_sync(0xffffffffu, cw[j], p);
                            if (q >= tot) continue;
                            // the rank-th successor of the parent's last vertex that extends it
                            int w;
                            if (!(pcw & CNT_WIDE)) {
                                // (clamped: a wrong count word must not index past the arcs)
                                const unsigned ci = (unsigned)(pe0 + nth_set_bit(pcw & CNT_BITS, rank));
                                w = __ldg(g.col + min(ci, (unsigned)(g.M - 1)));
                            } else {
                                const int pe1 = __ldg(g.rp + pl + 1);
                                int left = rank, e = pe0;
                                for (; e < pe1; ++e) {
                                    const int v = __ldg(g.col + e);
                                    if (v == pf || !test_bit<W>(pvis, v - pvb)) {
                                        if (left == 0) break;
                                        --left;
                                    }
                                }
                                w = __ldg(g.col + (e < pe1 ? e : pe1 - 1));
                            }
                            emit(w, pos_c + q, pf, pvb, pvis, pi, fbm_l);
                        }
                    }
                    if (pp) {
                        const int q = pos_p + __popc(ppm & lt_mask);
                        if (pp_off + q < a.pp_seg_cap) lpp[q] = i;
                    }
                    pos_c += tot;
                    pos_p += __popc(ppm);
                    if (__any_sync(0xffffffffu, ret_own >= 0)) {
                        flush_counts(A, s1, ret_own, ret_c, ret_p);
                        ret_own = -1;
                    }
                }
            }
            // the chunk must have produced exactly what its count promised
            if (last_part && lane == 0 && (pos_c - pa != own_c || pos_p - pb != own_p)) atomicOr(a.err, ERR_INVAL);
            u = u_next;
            ec = ec_next;
            ep = ep_next;
        }
        flush_counts(A, s1, cur_own, acc_c, acc_p);
        if (a.trace) {
            // per block first (shared memory), then one set of atomics per block
            if (lane == 0 && s_t0[wid]) {
                const unsigned long long t_w1 = global_ns();
                atomicMax(&s_tr[0], t_w1);
                atomicAdd(&s_tr[1], t_w1 - s_t0[wid]);
                atomicAdd(&s_tr[2], 1ull);
            }
            __syncthreads();
            if (tid == 0) {
                unsigned long long *tr = a.trace + LEVEL_TRACE_WORDS * k;
                if (s_tr[2]) {
                    atomicMax(tr + 1, s_tr[0]);
                    atomicAdd(tr + 2, s_tr[1]);
                    atomicAdd(tr + 3, s_tr[2]);
                }
                s_tr[0] = s_tr[1] = s_tr[2] = 0ull;
            }
        }
        if (C == 0) break;  // nothing follows; the end of the launch orders the writes
        bar_target += G;
        if (!enum_barrier(bar_target, ERR_TIMEOUT | ERR_INVAL)) break;
        count = C;
        lnodes = next;
        lpp += P;
    }
}

// ---------------------------------------------------------------------------
// host-side launch
// ---------------------------------------------------------------------------
template <int W, int BLOCK, int ITEMS>
static cudaError_t launch_wbi(const EnumArgs &args, int num_sms, cudaStream_t s, int *grid_out) {
    // the group prefixes take 2 * grid int64 of shared memory; size it for
    // the largest grid this block size can have
    const size_t smem = sizeof(long long) * 2 * (size_t)num_sms * (2048 / BLOCK);
    // the shared-memory attribute and the occupancy are per device (and per
    // shared-memory size): cached for each device id
    constexpr int MAX_DEV = 64;
    static std::mutex mu;
    static size_t set_smem[MAX_DEV] = {};
    static int set_bps[MAX_DEV] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
    int blocks_per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (set_smem[dev] != smem) {
            e = cudaFuncSetAttribute(enumerate_kernel<W, BLOCK, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            int bps = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, enumerate_kernel<W, BLOCK, ITEMS>, BLOCK, smem);
            if (e != cudaSuccess) return e;
            if (bps < 1) return cudaErrorInvalidConfiguration;
            set_bps[dev] = bps > 2048 / BLOCK ? 2048 / BLOCK : bps;
            set_smem[dev] = smem;
        }
        blocks_per_sm = set_bps[dev];
    }
    const int grid = num_sms * blocks_per_sm;
    *grid_out = grid;
    if (args.agg_cap < enum_agg_words(grid, ENUM_UPW * (BLOCK / 32))) return cudaErrorInvalidValue;
    if (args.seed_level1) {
        if ((e = launch_seed_level1(args, s)) != cudaSuccess) return e;
    }
    EnumArgs a = args;
    void *params[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)enumerate_kernel<W, BLOCK, ITEMS>, dim3(grid), dim3(BLOCK),
                                    params, smem, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

// tile shapes available per bitset width (the autotuner picks among them)
template <int W>
static cudaError_t launch_w(const EnumArgs &args, EnumShape shape, int num_sms, cudaStream_t s, int *grid_out) {
    if constexpr (W <= 8) {
        if (shape.block == 256) {
            if (shape.items == 1) return launch_wbi<W, 256, 1>(args, num_sms, s, grid_out);
            if (shape.items == 2) return launch_wbi<W, 256, 2>(args, num_sms, s, grid_out);
            if (shape.items == 4) return launch_wbi<W, 256, 4>(args, num_sms, s, grid_out);
        } else if (shape.block == 512) {
            if (shape.items == 1) return launch_wbi<W, 512, 1>(args, num_sms, s, grid_out);
            if (shape.items == 2) return launch_wbi<W, 512, 2>(args, num_sms, s, grid_out);
        } else if (shape.block == 1024) {
            if (shape.items == 1) return launch_wbi<W, 1024, 1>(args, num_sms, s, grid_out);
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
    if (shape.block == 256) return shape.items == 1 || shape.items == 2 || shape.items == 4;
    if (shape.block == 512) return shape.items == 1 || shape.items == 2;
    if (shape.block == 1024) return shape.items == 1;
    return false;
}

EnumShape default_enum_shape(int W) {
    if (W > 8) return EnumShape{256, 1};
    return EnumShape{512, 1};
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
