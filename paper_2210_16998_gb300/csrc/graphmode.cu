// Graph-captured pipeline: everything after the frontier launch, with every
// size read from device memory, so that the whole hot path of a handle (one
// graph or a batch of thousands) is a fixed sequence of launches that can be
// captured once into a CUDA graph and replayed.
//
// Prime-path order (kernel (e) for PPs): the PPs of each frontier level form
// a sorted run (levels are lexicographically ordered and PPs form an
// antichain of the prefix tree).  One cooperative persistent kernel walks
// the levels from the deepest up: the run accumulated so far is keyed by
// each element's ancestor index at the current level and merged with that
// level's PPs (whose keys are their own indices; the two never tie), with a
// bounded grid barrier between the steps.
//
// Test-path order: the TPs of one graph that share a first vertex form a
// sorted run; runs are merged pairwise inside each graph in
// ceil(log2(max vertices + 1)) fixed rounds, comparing whole sequences.
#include "common.cuh"
#include "kernels.h"
#include "paths_dev.cuh"

namespace tpg {

namespace {

constexpr int GMB = 256;      // threads per block of the streaming kernels
constexpr int GM_ITEMS = 4;   // outputs per thread of the PP merge
#ifndef TPG_TPM_ITEMS
#define TPG_TPM_ITEMS 4  // outputs per thread of a TP merge round
#endif
constexpr int TPM_ITEMS = TPG_TPM_ITEMS;  // outputs per thread of the TP run merge
constexpr int GM_SCAN_ITEMS = 8;
constexpr long long GM_SCAN_TILE = (long long)GMB * GM_SCAN_ITEMS;

__device__ __forceinline__ long long clampc(long long v, long long cap) { return v < 0 ? 0 : (v > cap ? cap : v); }

// largest k in [0, n] with a[k] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ int slot_of(const long long *a, int n, long long x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ long long slot_of64(const long long *a, long long lo, long long hi, long long x) {
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// device-count scans
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(GMB) gm_scan_reduce(const T *in, const long long *n_dev, long long n_cap,
                                                      long long *tile_sums) {
    const long long n = clampc(*n_dev, n_cap);
    const long long ntiles = (n + GM_SCAN_TILE - 1) / GM_SCAN_TILE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        long long s = 0;
        for (int j = 0; j < GM_SCAN_ITEMS; ++j) {
            const long long i = t * GM_SCAN_TILE + (long long)j * GMB + threadIdx.x;
            if (i < n) s += (long long)in[i];
        }
        long long total;
        block_excl_scan_i64<GMB>(s, total);
        if (threadIdx.x == 0) tile_sums[t] = total;
    }
}

__global__ void __launch_bounds__(GMB) gm_scan_tiles(long long *tile_sums, const long long *n_dev, long long n_cap,
                                                     long long *total_out) {
    const long long n = clampc(*n_dev, n_cap);
    const long long ntiles = (n + GM_SCAN_TILE - 1) / GM_SCAN_TILE;
    long long carry = 0;
    for (long long base = 0; base < ntiles; base += GMB) {
        const long long i = base + threadIdx.x;
        const long long v = (i < ntiles) ? tile_sums[i] : 0;
        long long total;
        const long long ex = block_excl_scan_i64<GMB>(v, total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        tile_sums[ntiles] = carry;
        if (total_out) *total_out = carry;
    }
}

template <typename T>
__global__ void __launch_bounds__(GMB) gm_scan_down(const T *in, long long *out, const long long *n_dev,
                                                    long long n_cap, const long long *tile_sums) {
    const long long n = clampc(*n_dev, n_cap);
    const long long ntiles = (n + GM_SCAN_TILE - 1) / GM_SCAN_TILE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long base = t * GM_SCAN_TILE + (long long)threadIdx.x * GM_SCAN_ITEMS;
        long long v[GM_SCAN_ITEMS];
        long long s = 0;
#pragma unroll
        for (int j = 0; j < GM_SCAN_ITEMS; ++j) {
            const long long i = base + j;
            v[j] = (i < n) ? (long long)in[i] : 0;
            s += v[j];
        }
        long long total;
        long long run = block_excl_scan_i64<GMB>(s, total) + tile_sums[t];
#pragma unroll
        for (int j = 0; j < GM_SCAN_ITEMS; ++j) {
            const long long i = base + j;
            if (i < n) out[i] = run;
            run += v[j];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_sums[ntiles];
}

// ---------------------------------------------------------------------------
// PP ordering
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GMB) gm_level_summary(GmArgs a) {
    const int ml = a.max_levels;
    const bool ok = (*a.enum_err == 0);
    long long carry = 0, vcarry = 0;
    for (int base = 0; base < ml; base += GMB) {
        const int k = base + threadIdx.x;
        long long v = 0;
        if (ok && k >= 1 && k < ml) v = a.levels[k].count > 0 ? a.levels[k].pp_count : 0;
        long long total, vtotal;
        const long long ex = block_excl_scan_i64<GMB>(v, total);
        block_excl_scan_i64<GMB>(v * k, vtotal);
        if (k < ml) a.lvl_pp_off[k] = carry + ex;
        carry += total;
        vcarry += vtotal;
    }
    if (threadIdx.x == 0) {
        a.lvl_pp_off[ml] = carry;
        GmCounts *c = a.counts;
        c->P = carry;
        c->V = vcarry;
        int f = ok ? 0 : GM_ENUM_FAILED;
        if (carry > a.P_cap) f |= GM_OVF_PP;
        if (vcarry > a.V_cap) f |= GM_OVF_PPV;
        c->flags = f;
    }
}

__device__ __forceinline__ long long gm_P(const GmArgs &a) {
    const GmCounts *c = a.counts;
    if (c->flags & (GM_ENUM_FAILED | GM_OVF_PP | GM_OVF_PPV)) return 0;
    return clampc(c->P, a.P_cap);
}

__global__ void __launch_bounds__(GMB) gm_pp_lengths(GmArgs a) {
    const long long P = gm_P(a);
    const long long *refs = a.refs[a.counts->pp_buf];
    for (long long i = blockIdx.x * (long long)GMB + threadIdx.x; i < P; i += (long long)gridDim.x * GMB)
        a.len[i] = refs[i] >> 32;
}

constexpr int GM_MAT_WARPS = 8;

template <int CH, typename T>
__global__ void __launch_bounds__(GM_MAT_WARPS * 32, 8) gm_materialize(GmArgs a) {
    __shared__ T sbuf[GM_MAT_WARPS][MAT_BUF * CH];
    __shared__ int2 *s_nodes[MAT_MAX_LV];
    int2 *const *lv = cache_level_nodes(a.levels, a.max_levels, s_nodes);
    const long long P = gm_P(a);
    materialize_warps<GM_MAT_WARPS, CH, T>(a.refs[a.counts->pp_buf], nullptr, 0, P, a.pp_off, a.levels, a.g,
                                           a.pp_vert, a.g.G > 1 ? a.pp_graph : nullptr, sbuf, lv);
}

// graph_path_ptr from sorted graph ids (ids == nullptr: one graph)
__global__ void __launch_bounds__(GMB) gm_graph_ptr(const int *ids, const long long *n_dev, long long n_cap, int G,
                                                    long long *ptr, const GmCounts *c, int fail_mask) {
    const long long n = (c->flags & fail_mask) ? 0 : clampc(*n_dev, n_cap);
    for (long long i = blockIdx.x * (long long)GMB + threadIdx.x; i <= n; i += (long long)gridDim.x * GMB) {
        const int cur = (i < n) ? (ids ? ids[i] : 0) : G;
        const int prev = (i > 0) ? (ids ? ids[i - 1] : 0) : -1;
        for (int gg = prev + 1; gg <= cur; ++gg) ptr[gg] = i;
    }
}

// ---------------------------------------------------------------------------
// TP assembly and ordering
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(GMB) gm_tp_len(GmArgs a) {
    const long long P = gm_P(a);
    const GraphDev &g = a.g;
    for (long long i = blockIdx.x * (long long)GMB + threadIdx.x; i < P; i += (long long)gridDim.x * GMB) {
        const long long o0 = a.pp_off[i], o1 = a.pp_off[i + 1];
        const int gid = g.G > 1 ? a.pp_graph[i] : 0;
        const int vb = g.vgraph ? g.vbase[gid] : 0;
        const int f = a.pp_vert[o0] + vb, l = a.pp_vert[o1 - 1] + vb;
        const int pl = g.pre_len[f], sl = g.suf_len[l];
        long long len = 0;
        if (pl == 0 || sl == 0) atomicOr(&a.counts->flags, GM_UNREACH);
        else len = (long long)(pl - 1) + (o1 - o0) + (sl - 1);
        a.tp_len[i] = len;
        const int vpw = 64 / a.key_bits;
        a.len[i] = (len + vpw - 1) / vpw;
        a.tp_graph0[i] = gid;
        int start = 1;
        if (i > 0) {
            const int gprev = g.G > 1 ? a.pp_graph[i - 1] : 0;
            start = (gprev != gid) || (a.pp_vert[a.pp_off[i - 1]] != a.pp_vert[o0]);
        }
        a.run_start[i] = start;
    }
}

__device__ __forceinline__ long long gm_P_tp(const GmArgs &a) {
    const GmCounts *c = a.counts;
    if (c->flags & (GM_ENUM_FAILED | GM_OVF_PP | GM_OVF_PPV | GM_UNREACH | GM_OVF_TPV0)) return 0;
    return clampc(c->P, a.P_cap);
}

__global__ void gm_tp_check(GmArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GmCounts *c = a.counts;
        c->TV0 = a.tp_off0[clampc(c->P, a.P_cap)];
        if (c->TV0 > a.TV0_cap || a.key_off[clampc(c->P, a.P_cap)] > a.K_cap) atomicOr(&c->flags, GM_OVF_TPV0);
        c->R = a.run_rank[clampc(c->P, a.P_cap)];
    }
}

__global__ void __launch_bounds__(GMB) gm_run_bases(GmArgs a) {
    const long long P = gm_P_tp(a);
    const int G = a.g.G;
    for (int g = blockIdx.x * GMB + threadIdx.x; g < G; g += gridDim.x * GMB) {
        const long long s0 = P ? a.pp_gptr[g] : 0, s1 = P ? a.pp_gptr[g + 1] : 0;
        a.run_base[g] = P ? a.run_rank[s0] : 0;
        a.nruns[g] = P ? a.run_rank[s1] - a.run_rank[s0] : 0;
    }
}

__global__ void __launch_bounds__(GMB) gm_bounds0(GmArgs a) {
    const long long P = gm_P_tp(a);
    for (long long i = blockIdx.x * (long long)GMB + threadIdx.x; i < P; i += (long long)gridDim.x * GMB) {
        if (a.run_start[i]) a.bounds0[a.run_rank[i]] = i;
        a.perm[0][i] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.bounds0[P ? a.counts->R : 0] = P;
}

// TP vertex at position p of TP i: prefix, PP, suffix
struct TpParts {
    const int *pre, *pp, *suf;
    long long pl, plen;
    __device__ __forceinline__ int at(long long p) const {
        if (p < pl) return pre[p];
        if (p < pl + plen) return pp[p - pl];
        return suf[p - pl - plen];
    }
};

constexpr int TP_LANES = 8;  // lanes per TP in the write and gather kernels

// The packed comparison keys of every TP, read from its parts (the TPs
// themselves are assembled once, in sorted order, by gm_tp_gather).
__global__ void __launch_bounds__(GMB) gm_tp_write(GmArgs a) {
    const long long P = gm_P_tp(a);
    const GraphDev &g = a.g;
    const int sub = threadIdx.x & (TP_LANES - 1);
    const long long ngroups = (long long)gridDim.x * (GMB / TP_LANES);
    const int bits = a.key_bits, vpw = 64 / bits;
    for (long long i = blockIdx.x * (long long)(GMB / TP_LANES) + (threadIdx.x / TP_LANES); i < P; i += ngroups) {
        const long long o0 = a.pp_off[i], o1 = a.pp_off[i + 1];
        const int gid = g.G > 1 ? a.pp_graph[i] : 0;
        const int vb = g.vgraph ? g.vbase[gid] : 0;
        const int f = a.pp_vert[o0] + vb, l = a.pp_vert[o1 - 1] + vb;
        TpParts t;
        t.pl = g.pre_len[f] - 1;
        t.plen = o1 - o0;
        t.pre = g.pre_seq + g.pre_off[f];
        t.pp = a.pp_vert + o0;
        t.suf = g.suf_seq + g.suf_off[l] + 1;
        const long long total = a.tp_off0[i + 1] - a.tp_off0[i];
        const long long k0 = a.key_off[i], nw = a.key_off[i + 1] - k0;
        for (long long w = sub; w < nw; w += TP_LANES) {
            unsigned long long word = 0;
            for (int q = 0; q < vpw; ++q) {
                const long long p = w * vpw + q;
                const unsigned long long v = p < total ? (unsigned long long)(t.at(p) + 1) : 0ull;
                word = (word << bits) | v;
            }
            a.key[k0 + w] = word;
        }
    }
}

// one round of pairwise run merging inside every graph (both runs of a merge
// belong to one graph, so the comparisons read no graph ids)
__global__ void __launch_bounds__(GMB) gm_tp_merge_round(GmArgs a, int r, int buf) {
    const long long P = gm_P_tp(a);
    const long long *pin = a.perm[buf];
    long long *pout = a.perm[buf ^ 1];
    const int G = a.g.G;
    const long long nthreads = (long long)gridDim.x * GMB;
    for (long long d0 = (blockIdx.x * (long long)GMB + threadIdx.x) * TPM_ITEMS; d0 < P; d0 += nthreads * TPM_ITEMS) {
        long long a_hi = 0, b_hi = -1, i = 0, j = 0;
        for (int t = 0; t < TPM_ITEMS; ++t) {
            const long long d = d0 + t;
            if (d >= P) break;
            if (d >= b_hi) {
                const int gg = G > 1 ? slot_of64(a.pp_gptr, 0, G, d) : 0;
                const long long rb = a.run_base[gg], nr = a.nruns[gg];
                const long long q0 = slot_of64(a.bounds0, rb, rb + nr - 1, d) - rb;
                const long long m = q0 >> (r + 1);
                const long long qa = m << (r + 1), qb = qa + (1ll << r), qe = (m + 1) << (r + 1);
                const long long a_lo = a.bounds0[rb + qa];
                a_hi = a.bounds0[rb + (qb < nr ? qb : nr)];
                b_hi = a.bounds0[rb + (qe < nr ? qe : nr)];
                const long long na = a_hi - a_lo, nb = b_hi - a_hi, diag = d - a_lo;
                long long lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
                while (lo < hi) {
                    const long long mid = (lo + hi) >> 1;
                    if (key_cmp_same_graph(pin[a_lo + mid], pin[a_hi + diag - mid - 1], a.key_off, a.key) <= 0)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                i = a_lo + lo;
                j = a_hi + (diag - lo);
            }
            bool take_a;
            if (i >= a_hi) take_a = false;
            else if (j >= b_hi) take_a = true;
            else take_a = key_cmp_same_graph(pin[i], pin[j], a.key_off, a.key) <= 0;
            pout[d] = take_a ? pin[i++] : pin[j++];
        }
    }
}

__global__ void __launch_bounds__(GMB) gm_tp_dedup(GmArgs a, int buf) {
    const long long P = gm_P_tp(a);
    const long long *perm = a.perm[buf];
    for (long long i = blockIdx.x * (long long)GMB + threadIdx.x; i < P; i += (long long)gridDim.x * GMB) {
        const long long x = perm[i];
        const int k = (i == 0) || key_cmp(perm[i - 1], x, a.key_off, a.key, a.tp_graph0) != 0;
        a.keep[i] = k;
        a.tp_len[i] = k ? a.tp_off0[x + 1] - a.tp_off0[x] : 0;
    }
}

__global__ void gm_tp_totals(GmArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GmCounts *c = a.counts;
        const long long P = gm_P_tp(a);
        c->T = P ? a.keep_rank[P] : 0;
        c->TV = P ? a.keep_off[P] : 0;
        if (c->TV > a.TV_cap) atomicOr(&c->flags, GM_OVF_TPV);
    }
}

__device__ __forceinline__ long long gm_P_final(const GmArgs &a) {
    if (a.counts->flags & GM_OVF_TPV) return 0;
    return gm_P_tp(a);
}

// The kept TPs in sorted order, each assembled from its parts (prefix path,
// PP, suffix path) straight into its final place: the TP list is never
// written in PP order.
__global__ void __launch_bounds__(GMB) gm_tp_gather(GmArgs a, int buf) {
    const long long P = gm_P_final(a);
    const long long *perm = a.perm[buf];
    const GraphDev &g = a.g;
    const int sub = threadIdx.x & (TP_LANES - 1);
    const long long ngroups = (long long)gridDim.x * (GMB / TP_LANES);
    for (long long i = blockIdx.x * (long long)(GMB / TP_LANES) + (threadIdx.x / TP_LANES); i < P; i += ngroups) {
        if (!a.keep[i]) continue;
        const long long x = perm[i], rk = a.keep_rank[i];
        const long long o0 = a.pp_off[x], o1 = a.pp_off[x + 1];
        const int gid = g.G > 1 ? a.pp_graph[x] : 0;
        const int vb = g.vgraph ? g.vbase[gid] : 0;
        const int f = a.pp_vert[o0] + vb, l = a.pp_vert[o1 - 1] + vb;
        TpParts t;
        t.pl = g.pre_len[f] - 1;
        t.plen = o1 - o0;
        t.pre = g.pre_seq + g.pre_off[f];
        t.pp = a.pp_vert + o0;
        t.suf = g.suf_seq + g.suf_off[l] + 1;
        const long long len = a.tp_off0[x + 1] - a.tp_off0[x], d0 = a.keep_off[i];
        for (long long p = sub; p < len; p += TP_LANES) a.tp_vert[d0 + p] = t.at(p);
        if (sub == 0) {
            a.tp_graph[rk] = a.tp_graph0[x];
            a.tp_off[rk] = d0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const GmCounts *c = a.counts;
        a.tp_off[P ? c->T : 0] = P ? c->TV : 0;
    }
}

unsigned stream_grid(int num_sms) { return (unsigned)(num_sms * 8); }

template <typename T>
cudaError_t gm_scan(const T *in, long long *out, const long long *n_dev, long long n_cap, long long *tmp,
                    long long *total_out, int num_sms, cudaStream_t s) {
    const unsigned grid = stream_grid(num_sms);
    gm_scan_reduce<T><<<grid, GMB, 0, s>>>(in, n_dev, n_cap, tmp);
    gm_scan_tiles<<<1, GMB, 0, s>>>(tmp, n_dev, n_cap, total_out);
    gm_scan_down<T><<<grid, GMB, 0, s>>>(in, out, n_dev, n_cap, tmp);
    note_launch(3);
    return cudaGetLastError();
}

}  // namespace

int gm_tp_rounds(int maxn) {
    int r = 0;
    while ((1 << r) < maxn + 1) ++r;
    return r;
}

size_t gm_scan_tmp_elems(long long n_cap) { return (size_t)((n_cap + GM_SCAN_TILE - 1) / GM_SCAN_TILE) + 2; }

cudaError_t gm_enqueue_pp(const GmArgs &a, cudaStream_t s) {
    const unsigned grid = stream_grid(a.num_sms);
    gm_level_summary<<<1, GMB, 0, s>>>(a);
    note_launch();
    RankArgs r{};
    r.levels = a.levels;
    r.max_levels = a.max_levels;
    r.cnt = a.rank_cnt;
    r.cnt_cap = a.rank_cnt_cap;
    r.pre[0] = a.rank_pre[0];
    r.pre[1] = a.rank_pre[1];
    r.pre_cap = a.rank_pre_cap;
    r.noff = a.rank_noff;
    r.bsum = a.rank_bsum;
    r.refs = a.refs[0];  // counts->pp_buf stays 0
    r.refs_cap = a.P_cap;
    r.bar = a.rank_bar;
    r.err = &a.counts->flags;  // any flag sends the replay to the exact path
    r.skip = &a.counts->flags;
    r.skip_mask = GM_ENUM_FAILED | GM_OVF_PP | GM_OVF_PPV;
    cudaError_t e = rank_pps(r, a.num_sms, s);
    if (e != cudaSuccess) return e;
    gm_pp_lengths<<<grid, GMB, 0, s>>>(a);
    note_launch();
    e = gm_scan<long long>(a.len, a.pp_off, &a.counts->P, a.P_cap, a.scan_tmp, nullptr, a.num_sms, s);
    if (e != cudaSuccess) return e;
    if (a.g.maxn <= MAT_SMALL_N) gm_materialize<2, unsigned char><<<grid, GM_MAT_WARPS * 32, 0, s>>>(a);
    else gm_materialize<1, unsigned short><<<grid, GM_MAT_WARPS * 32, 0, s>>>(a);
    gm_graph_ptr<<<grid, GMB, 0, s>>>(a.g.G > 1 ? a.pp_graph : nullptr, &a.counts->P, a.P_cap, a.g.G, a.pp_gptr,
                                      a.counts, GM_ENUM_FAILED | GM_OVF_PP | GM_OVF_PPV);
    note_launch(2);
    return cudaGetLastError();
}

cudaError_t gm_enqueue_tp(const GmArgs &a, cudaStream_t s) {
    const unsigned grid = stream_grid(a.num_sms);
    gm_tp_len<<<grid, GMB, 0, s>>>(a);
    note_launch();
    cudaError_t e;
    if ((e = gm_scan<long long>(a.tp_len, a.tp_off0, &a.counts->P, a.P_cap, a.scan_tmp, nullptr, a.num_sms, s)))
        return e;
    if ((e = gm_scan<int>(a.run_start, a.run_rank, &a.counts->P, a.P_cap, a.scan_tmp, nullptr, a.num_sms, s)))
        return e;
    if ((e = gm_scan<long long>(a.len, a.key_off, &a.counts->P, a.P_cap, a.scan_tmp, nullptr, a.num_sms, s)))
        return e;
    gm_tp_check<<<1, 32, 0, s>>>(a);
    gm_run_bases<<<grid, GMB, 0, s>>>(a);
    gm_bounds0<<<grid, GMB, 0, s>>>(a);
    gm_tp_write<<<grid, GMB, 0, s>>>(a);
    note_launch(4);
    int buf = 0;
    for (int r = 0; r < a.tp_rounds; ++r) {
        gm_tp_merge_round<<<grid, GMB, 0, s>>>(a, r, buf);
        note_launch();
        buf ^= 1;
    }
    gm_tp_dedup<<<grid, GMB, 0, s>>>(a, buf);
    note_launch();
    if ((e = gm_scan<long long>(a.tp_len, a.keep_off, &a.counts->P, a.P_cap, a.scan_tmp, nullptr, a.num_sms, s)))
        return e;
    if ((e = gm_scan<int>(a.keep, a.keep_rank, &a.counts->P, a.P_cap, a.scan_tmp, nullptr, a.num_sms, s)))
        return e;
    gm_tp_totals<<<1, 32, 0, s>>>(a);
    gm_tp_gather<<<grid, GMB, 0, s>>>(a, buf);
    gm_graph_ptr<<<grid, GMB, 0, s>>>(a.tp_graph, &a.counts->T, a.P_cap, a.g.G, a.tp_gptr, a.counts,
                                      GM_ENUM_FAILED | GM_OVF_PP | GM_OVF_PPV | GM_UNREACH | GM_OVF_TPV0 | GM_OVF_TPV);
    note_launch(3);
    return cudaGetLastError();
}

}  // namespace tpg
