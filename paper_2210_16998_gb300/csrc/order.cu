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
#include <atomic>
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

template <int CH, typename T>
__global__ void __launch_bounds__(MAT_WARPS * 32, 8)
    pp_materialize_kernel(const long long *refs, const int *single_refs, int single_level, long long n,
                          const long long *offsets, const LevelRec *levels, int max_levels, GraphDev g,
                          int *out, int *out_graph, int2 *out_ends) {
    __shared__ T buf[MAT_WARPS][MAT_BUF * CH];
    __shared__ int2 *s_nodes[MAT_MAX_LV];
    int2 *const *lv = cache_level_nodes(levels, max_levels, s_nodes);
    materialize_warps<MAT_WARPS, CH, T>(refs, single_refs, single_level, n, offsets, levels, g, out, out_graph, buf,
                                        lv, out_ends);
}

cudaError_t pp_materialize(const long long *refs, const int *single_refs, int single_level, long long n,
                           const long long *offsets, const LevelRec *levels, int max_levels, const GraphDev &g,
                           int *out_vertices, int *out_graph, cudaStream_t s, int2 *out_ends) {
    if (n <= 0) return cudaSuccess;
    const bool small = g.maxn <= MAT_SMALL_N;
    const long long warps = (n + (small ? 63 : 31)) / (small ? 64 : 32);
    long long blocks = (warps + MAT_WARPS - 1) / MAT_WARPS;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (small)
        pp_materialize_kernel<2, unsigned char><<<(unsigned)blocks, MAT_WARPS * 32, 0, s>>>(
            refs, single_refs, single_level, n, offsets, levels, max_levels, g, out_vertices, out_graph, out_ends);
    else
        pp_materialize_kernel<1, unsigned short><<<(unsigned)blocks, MAT_WARPS * 32, 0, s>>>(
            refs, single_refs, single_level, n, offsets, levels, max_levels, g, out_vertices, out_graph, out_ends);
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


// ---------------------------------------------------------------------------
// PP order by pre-order rank (Def. 1 makes the PPs leaves of the prefix tree)
// ---------------------------------------------------------------------------
// The arena is the prefix tree of all simple paths: level k holds the paths
// of k vertices in lexicographic order, every node points at its parent, and
// the children of a node are consecutive and ordered by their last vertex.
// Lexicographic order with a proper prefix first is the tree's pre-order,
// and a PP has no descendant in the tree (it is never a proper prefix of a
// simple path), so the canonical PP list is the pre-order list of the PP
// nodes.  Its rank is computed in two sweeps over the levels:
//   bottom-up  cnt(v) = [v is a PP] + sum of cnt over v's children;
//   top-down   rank(v) = rank(parent) + sum of cnt over v's earlier
//              siblings (rank of level-1 nodes: the prefix sum of cnt),
// and every PP is written to position rank as soon as its rank is known (a
// PP node's count carries a flag bit, so no separate placement pass is
// needed).  The work is one read and one write of a 4-byte count per arena
// node in each sweep, whatever the number of levels; one cooperative launch
// with a grid barrier between levels.  Levels of at most RANK_SMALL nodes at
// either end of the tree (the deepest ones, and the first ones when level 1
// is small) are walked by block 0 alone with __syncthreads between them
// while the other blocks wait at one grid barrier (or have left).
constexpr int RANK_BLOCK = 512;  // 3 blocks per SM: few blocks arrive at each grid barrier
constexpr unsigned RANK_PP = 0x80000000u;   // count flag: the node is a PP (a leaf, count 1)
constexpr unsigned RANK_CNT = 0x7fffffffu;  // count bits (at most P < 2^31)
constexpr long long RANK_SMALL = 2048;      // a level this small is walked by one block

__device__ __forceinline__ const int2 *level_nodes(const LevelRec *levels, int k) {
    return (const int2 *)__ldcg((const unsigned long long *)&levels[k].nodes);
}

__global__ void __launch_bounds__(RANK_BLOCK, 3) rank_pps_kernel(RankArgs a) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int G = gridDim.x, b = blockIdx.x;
    const long long T = (long long)G * RANK_BLOCK, gtid = (long long)b * RANK_BLOCK + tid;
    const unsigned full = 0xffffffffu;
    const int ml = a.max_levels;
    unsigned *const cnt = (unsigned *)a.cnt;
    if (a.skip && (*a.skip & a.skip_mask)) return;  // the same on every block
    // grid barrier on one growing arrival counter (a.bar[0], zero at launch)
    unsigned bar_target = 0;
    auto bar = [&](int stop) -> bool {
        bar_target += (unsigned)G;
        return grid_barrier_count(a.bar, bar_target, a.err, stop);
    };
    long long *meta = a.noff + ml + 1;  // L, total nodes, P, largest level, deepest big level, first big level >= 2

    // node offsets of the levels and the totals (block 0), then everyone reads them
    if (b == 0) {
        long long carry = 0, pcarry = 0, peak = 0;
        int L = 0, khi = 0, klo = 0x7fffffff;
        bool live = true;
        for (int base = 1; base < ml; base += RANK_BLOCK) {
            const int k = base + tid;
            long long c = 0, pc = 0;
            if (k < ml) {
                c = a.levels[k].count;
                pc = a.levels[k].pp_count;
            }
            // levels end at the first empty one
            const unsigned dead = __syncthreads_or(k < ml && c <= 0) ? 1u : 0u;
            __shared__ int s_first_dead;
            if (tid == 0) s_first_dead = RANK_BLOCK;
            __syncthreads();
            if (k < ml && c <= 0) atomicMin(&s_first_dead, tid);
            __syncthreads();
            const int fd = s_first_dead;
            if (!live || tid >= fd) c = pc = 0;
            long long tot, ptot;
            const long long ex = block_excl_scan_i64<RANK_BLOCK>(c, tot);
            block_excl_scan_i64<RANK_BLOCK>(pc, ptot);
            long long mx = c;
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(full, mx, o));
            __shared__ long long s_mx[RANK_BLOCK / 32];
            if (lane == 0) s_mx[tid >> 5] = mx;
            __syncthreads();
            if (tid == 0)
                for (int w = 0; w < RANK_BLOCK / 32; ++w) peak = max(peak, s_mx[w]);
            if (live && k < ml && tid < fd) a.noff[k] = carry + ex;
            if (live && k < ml && tid < fd && c > 0) L = max(L, k);
            if (live && k < ml && tid < fd && c > RANK_SMALL) {
                khi = max(khi, k);
                if (k >= 2) klo = min(klo, k);
            }
            carry += tot;
            pcarry += ptot;
            if (dead) live = false;
            __syncthreads();
        }
        // L = the largest level index with paths; the big levels' range (block extrema)
        __shared__ int s_L, s_khi, s_klo;
        if (tid == 0) {
            s_L = 0;
            s_khi = 0;
            s_klo = 0x7fffffff;
        }
        __syncthreads();
        atomicMax(&s_L, L);
        atomicMax(&s_khi, khi);
        atomicMin(&s_klo, klo);
        __syncthreads();
        if (tid == 0) {
            a.noff[s_L + 1] = carry;
            meta[0] = s_L;
            meta[1] = carry;
            meta[2] = pcarry;
            meta[3] = peak;
            meta[4] = s_khi;
            meta[5] = s_klo;
            if (carry > a.cnt_cap || peak > a.pre_cap || pcarry > a.refs_cap) atomicOr(a.err, ERR_INVAL);
        }
    }
    if (!bar(ERR_TIMEOUT | ERR_INVAL)) return;
    const int L = (int)__ldcg(meta + 0);
    const long long total = __ldcg(meta + 1);
    if (L < 1) return;
    const int khi = (int)__ldcg(meta + 4);  // deepest level above RANK_SMALL nodes (0: none)
    const long long n1 = __ldcg(a.noff + 2) - __ldcg(a.noff + 1);
    const bool top_small = n1 <= RANK_SMALL;  // level 1 and the levels before the first big one: block 0
    const int klo = top_small ? (int)min(__ldcg(meta + 5), (long long)L + 1) : 2;  // first level the grid ranks
    auto noff = [&](int k) { return __ldcg(a.noff + k); };

    // ---- per-level steps, for the whole grid (t = gtid, TT = T) or block 0 (t = tid, TT = RANK_BLOCK) ----
    // bottom-up at level k: add each node's count to its parent (consecutive
    // nodes mostly share a parent: one atomic per group of lanes)
    auto bottom = [&](int k, long long t, long long TT) {
        const long long o = noff(k), n = noff(k + 1) - o, op = noff(k - 1);
        const int2 *nodes = level_nodes(a.levels, k);
        constexpr int U = 4;  // chunks in flight per warp
        for (long long i0 = t - lane; i0 < n; i0 += TT * U) {
            unsigned v[U];
            int p[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long i = i0 + u * TT + lane;
                v[u] = i < n ? (__ldcg(cnt + o + i) & RANK_CNT) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long i = i0 + u * TT + lane;
                p[u] = v[u] ? __ldcg(&nodes[i].y) : -1;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned grp = __match_any_sync(full, p[u]);
                const unsigned sum = __reduce_add_sync(grp, v[u]);
                if (p[u] >= 0 && lane == __ffs(grp) - 1) atomicAdd(cnt + op + p[u], sum);
            }
        }
    };
    // top-down at level k over nwarps warps (this one is wg): rank(v) =
    // rank(parent) + counts of earlier siblings; a PP goes to its rank.  Each
    // warp walks a contiguous range of the level, carrying the sibling run
    // that crosses from one 32-node chunk into the next.
    auto top = [&](int k, long long wg, long long nwarps) {
        const long long o = noff(k), n = noff(k + 1) - o;
        const int *rp = a.pre[(k - 1) & 1];
        int *rk = a.pre[k & 1];
        const int2 *nodes = level_nodes(a.levels, k);
        const long long per = (((n + nwarps - 1) / nwarps) + 31) & ~31ll;
        const long long lo = min(wg * per, n), hi = min(lo + per, n);
        int run_p = -2;
        unsigned run_sum = 0;  // parent and count sum of the open run
        if (lo < hi && lo > 0) {
            unsigned sum = 0;
            int p0 = 0;
            if (lane == 0) {
                p0 = __ldcg(&nodes[lo].y);
                for (long long s2 = lo - 1; s2 >= 0 && __ldcg(&nodes[s2].y) == p0; --s2)
                    sum += __ldcg(cnt + o + s2) & RANK_CNT;
            }
            run_p = __shfl_sync(full, p0, 0);
            run_sum = __shfl_sync(full, sum, 0);
        }
        // the next chunk's count and parent load while this one is ranked
        unsigned raw_next = (lo + lane < hi) ? __ldcg(cnt + o + lo + lane) : 0u;
        int p_next = (lo + lane < hi) ? __ldcg(&nodes[lo + lane].y) : -1;
        for (long long i0 = lo; i0 < hi; i0 += 32) {
            const long long i = i0 + lane;
            const bool in = i < hi;
            const unsigned raw = raw_next, v = raw & RANK_CNT;
            const int p = p_next;
            const long long inx = i + 32;
            raw_next = inx < hi ? __ldcg(cnt + o + inx) : 0u;
            p_next = inx < hi ? __ldcg(&nodes[inx].y) : -1;
            int pprev = __shfl_up_sync(full, p, 1);
            if (lane == 0) pprev = run_p;
            const bool head = !in || p != pprev;
            // warp prefix of v, restarted at every head
            unsigned x = v;
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const unsigned y = __shfl_up_sync(full, x, o2);
                if (lane >= o2) x += y;
            }
            const unsigned hm = __ballot_sync(full, head) & (lane == 31 ? full : ((2u << lane) - 1u));
            const int start = hm ? 31 - __clz(hm) : 0;  // first lane of this lane's sibling run
            const unsigned before = __shfl_sync(full, x, start > 0 ? start - 1 : 0);
            unsigned sib = x - v - (start > 0 ? before : 0u);
            if (start == 0 && !(hm & 1u)) sib += run_sum;  // the run began in an earlier chunk
            if (in) {
                const int r = v ? __ldcg(rp + p) + (int)sib : -1;
                rk[i] = r;
                if ((raw & RANK_PP) && r >= 0 && r < a.refs_cap) a.refs[r] = ((long long)k << 32) | (unsigned)i;
            }
            const int lastl = (int)min(31ll, hi - i0 - 1);
            run_p = __shfl_sync(full, p, lastl);
            run_sum = __shfl_sync(full, sib + v, lastl);
        }
    };
    // level 1 by block 0: rank = exclusive prefix sum of the counts
    auto level1_block = [&]() {
        const long long o = noff(1);
        long long run = 0;
        for (long long t0 = 0; t0 < n1; t0 += RANK_BLOCK) {
            const long long i = t0 + tid;
            const unsigned raw = i < n1 ? __ldcg(cnt + o + i) : 0u;
            long long ttot;
            const long long ex = block_excl_scan_i64<RANK_BLOCK>((long long)(raw & RANK_CNT), ttot);
            if (i < n1) {
                const long long r = run + ex;
                a.pre[1][i] = (int)r;
                if ((raw & RANK_PP) && r < a.refs_cap) a.refs[r] = (1ll << 32) | (unsigned)i;
            }
            run += ttot;
        }
    };
    const int NWB = RANK_BLOCK / 32;

    // no level above RANK_SMALL nodes: block 0 does everything
    if (khi == 0) {
        if (b != 0) return;
        if (!a.cnt_zeroed)
            for (long long i = tid; i < total; i += RANK_BLOCK) cnt[i] = 0u;
        __syncthreads();
        for (int k = 1; k <= L; ++k) {
            const long long np = __ldcg(&a.levels[k].pp_count), o = noff(k);
            const int *pp = (const int *)__ldcg((const unsigned long long *)&a.levels[k].pp);
            for (long long i = tid; i < np; i += RANK_BLOCK) cnt[o + pp[i]] = 1u | RANK_PP;
        }
        __syncthreads();
        for (int k = L; k >= 2; --k) {
            bottom(k, tid, RANK_BLOCK);
            __syncthreads();
        }
        level1_block();
        __syncthreads();
        for (int k = 2; k <= L; ++k) {
            top(k, tid >> 5, NWB);
            __syncthreads();
        }
        return;
    }

    // counts: 0 (unless the caller zeroed them), then 1 and the flag at every PP
    if (!a.cnt_zeroed) {
        for (long long i = gtid; i < total; i += T) cnt[i] = 0u;
        if (!bar(ERR_TIMEOUT)) return;
    }
    for (int k = 1; k <= L; ++k) {
        const long long np = __ldcg(&a.levels[k].pp_count), o = noff(k);
        const int *pp = (const int *)__ldcg((const unsigned long long *)&a.levels[k].pp);
        for (long long i = gtid; i < np; i += T) cnt[o + pp[i]] = 1u | RANK_PP;
    }
    if (!bar(ERR_TIMEOUT)) return;

    // bottom-up: the small deepest levels (block 0), the grid's levels, the
    // small first levels (block 0)
    if (L > khi) {
        if (b == 0) {
            for (int k = L; k > khi; --k) {
                bottom(k, tid, RANK_BLOCK);
                __syncthreads();
            }
        }
        if (!bar(ERR_TIMEOUT)) return;
    }
    for (int k = khi; k >= klo && k >= 2; --k) {
        bottom(k, gtid, T);
        if (!bar(ERR_TIMEOUT)) return;
    }
    if (top_small) {
        // levels klo-1 .. 2 up, level 1, then levels 2 .. klo-1 down, in block 0
        if (b == 0) {
            for (int k = klo - 1; k >= 2; --k) {
                bottom(k, tid, RANK_BLOCK);
                __syncthreads();
            }
            level1_block();
            __syncthreads();
            for (int k = 2; k < klo; ++k) {
                top(k, tid >> 5, NWB);
                __syncthreads();
            }
        }
        if (!bar(ERR_TIMEOUT)) return;
    } else {
        // level 1: rank = exclusive prefix sum of cnt (two passes over blocks)
        const long long o = noff(1);
        const long long per = (n1 + G - 1) / G, lo = min((long long)b * per, n1), hi = min(lo + per, n1);
        long long sum = 0;
        for (long long i = lo + tid; i < hi; i += RANK_BLOCK) sum += __ldcg(cnt + o + i) & RANK_CNT;
        long long tot;
        block_excl_scan_i64<RANK_BLOCK>(sum, tot);
        if (tid == 0) a.bsum[b] = tot;
        if (!bar(ERR_TIMEOUT)) return;
        long long off = 0;
        for (int j = tid; j < b; j += RANK_BLOCK) off += __ldcg(a.bsum + j);
        long long offt;
        block_excl_scan_i64<RANK_BLOCK>(off, offt);
        long long run = offt;
        for (long long t0 = lo; t0 < hi; t0 += RANK_BLOCK) {
            const long long i = t0 + tid;
            const unsigned raw = i < hi ? __ldcg(cnt + o + i) : 0u;
            long long ttot;
            const long long ex = block_excl_scan_i64<RANK_BLOCK>((long long)(raw & RANK_CNT), ttot);
            if (i < hi) {
                const long long r = run + ex;
                a.pre[1][i] = (int)r;
                if ((raw & RANK_PP) && r < a.refs_cap) a.refs[r] = (1ll << 32) | (unsigned)i;
            }
            run += ttot;
        }
        if (!bar(ERR_TIMEOUT)) return;
    }

    // top-down: the grid's levels, then the small deepest levels (block 0)
    for (int k = klo; k <= khi; ++k) {
        top(k, gtid / 32, T / 32);
        if (!bar(ERR_TIMEOUT)) return;
    }
    if (b == 0)
        for (int k = khi + 1; k <= L; ++k) {
            top(k, tid >> 5, NWB);
            __syncthreads();
        }
}

#ifndef TPG_RANK_PER_SM
#define TPG_RANK_PER_SM 8  // most blocks per SM of the ranking launch (fewer arrive at each grid barrier)
#endif

int rank_pps_grid(int num_sms) { return num_sms * 8; }

cudaError_t rank_pps(const RankArgs &args, int num_sms, cudaStream_t s) {
    // occupancy per device id (0 = not yet asked)
    static std::atomic<int> per_sm_dev[64];
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int per_sm = per_sm_dev[dev].load();
    if (per_sm <= 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rank_pps_kernel, RANK_BLOCK, 0);
        if (e != cudaSuccess) return e;
        per_sm = per_sm < 1 ? 1 : (per_sm > TPG_RANK_PER_SM ? TPG_RANK_PER_SM : per_sm);
        per_sm_dev[dev].store(per_sm);
    }
    RankArgs a = args;
    void *params[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)rank_pps_kernel, dim3(num_sms * per_sm),
                                                dim3(RANK_BLOCK), params, 0, s);
    if (e == cudaSuccess) note_launch();
    return e;
}

}  // namespace tpg
