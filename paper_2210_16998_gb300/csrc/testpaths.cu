// Test-path assembly (kernel (d)) and canonical sort + dedup of the test
// paths (kernel (e) for TPs).
//
// TP(p) = path(entry -> first p), then p, then path(last p -> exit), joined
// at the shared endpoints (Problem 1 output; the touring of Sec. 7.3), with
// path(a -> b) read from the lowest-id BFS predecessor table.  Because the
// PPs arrive in canonical order, TPs of PPs that share a first vertex share
// their prefix and are already in order among themselves; so the TP list is
// a sequence of sorted runs (one per (graph, first vertex)).  The runs of
// each graph are merged pairwise (merge path) in ceil(log2(runs)) rounds,
// comparing packed keys (8 or 16 bits per vertex, 64-bit words), and exact
// duplicates (two PPs of different first vertices can yield the same TP)
// are dropped after the final round.
#include "common.cuh"
#include "kernels.h"
#include "paths_dev.cuh"
#include "testpaths.h"

namespace tpg {

static unsigned grid_for(long long n, int block = 256) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

// TP lengths and run starts from each PP's (first, last) local vertex, which
// the materialisation wrote beside the PP list (coalesced reads only).
__global__ void tp_len_kernel(const long long *__restrict__ pp_off, const int2 *__restrict__ pp_ends,
                              const int *__restrict__ pp_graph, long long P, GraphDev g, long long *tp_len,
                              int *run_start, int *tp_graph, int *err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const long long o0 = pp_off[i], o1 = pp_off[i + 1];
        const int gid = pp_graph ? pp_graph[i] : 0;
        const int vb = g.vgraph ? g.vbase[gid] : 0;
        const int2 e = pp_ends[i];
        const int f = e.x + vb, l = e.y + vb;
        const int pl = g.pre_len[f], sl = g.suf_len[l];
        long long len = 0;
        if (pl == 0 || sl == 0) atomicOr(err, ERR_UNREACH);
        else len = (long long)(pl - 1) + (o1 - o0) + (sl - 1);
        tp_len[i] = len;
        tp_graph[i] = gid;
        int start = 1;
        if (i > 0) {
            const int gprev = pp_graph ? pp_graph[i - 1] : 0;
            start = (gprev != gid) || (pp_ends[i - 1].x != e.x);
        }
        run_start[i] = start;
    }
}

cudaError_t tp_lengths(const long long *pp_off, const int2 *pp_ends, const int *pp_graph, long long P,
                       const GraphDev &g, long long *tp_len, int *run_start, int *tp_graph, int *err,
                       cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    tp_len_kernel<<<grid_for(P), 256, 0, s>>>(pp_off, pp_ends, pp_graph, P, g, tp_len, run_start, tp_graph, err);
    note_launch();
    return cudaGetLastError();
}

// One warp per 32 consecutive TPs.  Lane l first gathers the parts of TP
// i0 + l (prefix path entry -> first vertex, the PP, suffix path last vertex
// -> exit) in parallel with the other lanes; the warp then copies the TPs one
// after another with its lanes striding over positions (coalesced).  When
// every TP of the warp is its own PP (empty prefix and suffix), the 32 TPs
// are one contiguous copy of the 32 PPs.
__global__ void tp_write_kernel(const long long *__restrict__ pp_off, const int *__restrict__ pp_vert,
                                const int *__restrict__ pp_graph, long long P, GraphDev g,
                                const long long *__restrict__ tp_off, int *__restrict__ tp_vert) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i0 = (blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; i0 < P;
         i0 += nw * 32) {
        const long long i = i0 + lane;
        const bool valid = i < P;
        long long o0 = 0, plen = 0, d0 = 0, total = 0;
        int pl = 0;
        const int *pre = nullptr, *suf = nullptr;
        if (valid) {
            o0 = pp_off[i];
            plen = pp_off[i + 1] - o0;
            d0 = tp_off[i];
            total = tp_off[i + 1] - d0;
            const int gid = pp_graph ? pp_graph[i] : 0;
            const int vb = g.vgraph ? g.vbase[gid] : 0;
            const int f = pp_vert[o0] + vb, l = pp_vert[o0 + plen - 1] + vb;
            pl = g.pre_len[f] - 1;
            pre = g.pre_seq + g.pre_off[f];
            suf = g.suf_seq + g.suf_off[l] + 1;
        }
        const int last = (int)((P - i0 < 32 ? P - i0 : 32) - 1);
        if (__all_sync(0xffffffffu, !valid || (pl == 0 && total == plen))) {
            // TP == PP for all: one contiguous range
            const long long src0 = __shfl_sync(0xffffffffu, o0, 0), dst0 = __shfl_sync(0xffffffffu, d0, 0);
            const long long len = __shfl_sync(0xffffffffu, d0 + total, last) - dst0;
            const int *src = pp_vert + src0;
            int *dst = tp_vert + dst0;
            long long p = lane;
            for (; p + 96 < len; p += 128) {
                const int a = src[p], b = src[p + 32], c = src[p + 64], d = src[p + 96];
                dst[p] = a;
                dst[p + 32] = b;
                dst[p + 64] = c;
                dst[p + 96] = d;
            }
            for (; p < len; p += 32) dst[p] = src[p];
            continue;
        }
        for (int t = 0; t <= last; ++t) {
            const long long to0 = __shfl_sync(0xffffffffu, o0, t), td0 = __shfl_sync(0xffffffffu, d0, t);
            const long long tplen = __shfl_sync(0xffffffffu, plen, t), ttot = __shfl_sync(0xffffffffu, total, t);
            const int tpl = __shfl_sync(0xffffffffu, pl, t);
            const int *tpre = (const int *)__shfl_sync(0xffffffffu, (unsigned long long)pre, t);
            const int *tsuf = (const int *)__shfl_sync(0xffffffffu, (unsigned long long)suf, t);
            for (long long p = lane; p < ttot; p += 32) {
                int v;
                if (p < tpl) v = tpre[p];
                else if (p < tpl + tplen) v = pp_vert[to0 + (p - tpl)];
                else v = tsuf[p - tpl - tplen];
                tp_vert[td0 + p] = v;
            }
        }
    }
}

cudaError_t tp_write(const long long *pp_off, const int *pp_vert, const int *pp_graph, long long P,
                     const GraphDev &g, const long long *tp_off, int *tp_vert, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    long long blocks = (P + 255) / 256;  // 8 warps of 32 TPs
    if (blocks > 65535) blocks = 65535;
    tp_write_kernel<<<(unsigned)blocks, 256, 0, s>>>(pp_off, pp_vert, pp_graph, P, g, tp_off, tp_vert);
    note_launch();
    return cudaGetLastError();
}

__global__ void run_bounds_kernel(const int *run_start, const long long *run_rank, long long P, long long R,
                                  long long *bounds) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x)
        if (run_start[i]) bounds[run_rank[i]] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) bounds[R] = P;
}

cudaError_t tp_run_bounds(const int *run_start, const long long *run_rank, long long P, long long R,
                          long long *bounds, cudaStream_t s) {
    run_bounds_kernel<<<grid_for(P), 256, 0, s>>>(run_start, run_rank, P, R, bounds);
    note_launch();
    return cudaGetLastError();
}

__global__ void iota_kernel(long long *perm, long long P) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x)
        perm[i] = i;
}

cudaError_t tp_iota(long long *perm, long long P, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    iota_kernel<<<grid_for(P), 256, 0, s>>>(perm, P);
    note_launch();
    return cudaGetLastError();
}

#ifndef TPG_TPM_ITEMS
#define TPG_TPM_ITEMS 4  // outputs per thread of a TP merge round
#endif
constexpr int TPM_ITEMS = TPG_TPM_ITEMS;

// largest s in [lo, hi] with a[s] <= x (a nondecreasing, a[lo] <= x)
__device__ __forceinline__ long long tp_slot(const long long *a, long long lo, long long hi, long long x) {
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void run_bases_kernel(const long long *gptr, const long long *run_rank, int G, long long *run_base,
                                 long long *nruns) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        run_base[g] = run_rank[gptr[g]];
        nruns[g] = run_rank[gptr[g + 1]] - run_base[g];
    }
}

cudaError_t tp_run_bases(const long long *gptr, const long long *run_rank, int G, long long *run_base,
                         long long *nruns, cudaStream_t s) {
    run_bases_kernel<<<grid_for(G), 256, 0, s>>>(gptr, run_rank, G, run_base, nruns);
    note_launch();
    return cudaGetLastError();
}

int tp_merge_rounds(long long max_runs) {
    int r = 0;
    while ((1ll << r) < max_runs) ++r;
    return r;
}

// Thread t writes outputs [t*ITEMS, t*ITEMS + ITEMS) of round r: it finds
// the graph and run of each output, the two run groups merged there, and the
// merge-path split by binary search (A first on ties, so equal TPs stay
// adjacent).  Graphs without TPs own no outputs.  cmp(a, b) orders two TPs
// of one graph (here: their packed keys).
template <typename Cmp>
__global__ void tp_merge_graph_kernel(const long long *perm_in, long long *perm_out, const long long *bounds,
                                      const long long *run_base, const long long *nruns, const long long *gptr,
                                      int G, int r, long long P, Cmp cmp) {
    const long long d0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * TPM_ITEMS;
    if (d0 >= P) return;
    long long a_hi = 0, b_hi = -1, i = 0, j = 0;
    for (int t = 0; t < TPM_ITEMS; ++t) {
        const long long d = d0 + t;
        if (d >= P) break;
        if (d >= b_hi) {
            const int gg = G > 1 ? (int)tp_slot(gptr, 0, G, d) : 0;
            const long long rb = run_base[gg], nr = nruns[gg];
            const long long q0 = tp_slot(bounds, rb, rb + nr - 1, d) - rb;
            const long long m = q0 >> (r + 1);
            const long long qa = m << (r + 1), qb = qa + (1ll << r), qe = (m + 1) << (r + 1);
            const long long a_lo = bounds[rb + qa];
            a_hi = bounds[rb + (qb < nr ? qb : nr)];
            b_hi = bounds[rb + (qe < nr ? qe : nr)];
            const long long na = a_hi - a_lo, nb = b_hi - a_hi, diag = d - a_lo;
            long long lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (cmp(perm_in[a_lo + mid], perm_in[a_hi + diag - mid - 1]) <= 0) lo = mid + 1;
                else hi = mid;
            }
            i = a_lo + lo;
            j = a_hi + (diag - lo);
        }
        bool take_a;
        if (i >= a_hi) take_a = false;
        else if (j >= b_hi) take_a = true;
        else take_a = cmp(perm_in[i], perm_in[j]) <= 0;
        perm_out[d] = take_a ? perm_in[i++] : perm_in[j++];
    }
}

struct KeyCmp {  // packed keys of one graph
    const long long *koff;
    const unsigned long long *key;
    __device__ __forceinline__ int operator()(long long a, long long b) const {
        return key_cmp_same_graph(a, b, koff, key);
    }
};

cudaError_t tp_merge_graph_round_keys(const long long *perm_in, long long *perm_out, const long long *bounds,
                                      const long long *run_base, const long long *nruns, const long long *gptr,
                                      int G, int r, long long P, const long long *key_off,
                                      const unsigned long long *key, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const long long threads = (P + TPM_ITEMS - 1) / TPM_ITEMS;
    tp_merge_graph_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(perm_in, perm_out, bounds, run_base,
                                                                           nruns, gptr, G, r, P,
                                                                           KeyCmp{key_off, key});
    note_launch();
    return cudaGetLastError();
}

__global__ void key_len_kernel(const long long *tp_off, long long P, int vpw, long long *key_len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x)
        key_len[i] = (tp_off[i + 1] - tp_off[i] + vpw - 1) / vpw;
}

cudaError_t tp_key_lengths(const long long *tp_off, long long P, int bits, long long *key_len, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    key_len_kernel<<<grid_for(P), 256, 0, s>>>(tp_off, P, 64 / bits, key_len);
    note_launch();
    return cudaGetLastError();
}

// 8 lanes per TP, each packing 64 / bits consecutive vertices into a word
constexpr int KEY_LANES = 8;
__global__ void keys_kernel(const long long *tp_off, const int *tp_vert, long long P, int bits,
                            const long long *key_off, unsigned long long *key) {
    const int sub = threadIdx.x & (KEY_LANES - 1), vpw = 64 / bits;
    const long long groups = (long long)gridDim.x * (blockDim.x / KEY_LANES);
    for (long long i = blockIdx.x * (long long)(blockDim.x / KEY_LANES) + threadIdx.x / KEY_LANES; i < P;
         i += groups) {
        const long long t0 = tp_off[i], len = tp_off[i + 1] - t0, k0 = key_off[i], nw = key_off[i + 1] - k0;
        for (long long w = sub; w < nw; w += KEY_LANES) {
            unsigned long long word = 0;
            for (int q = 0; q < vpw; ++q) {
                const long long p = w * vpw + q;
                const unsigned long long v = p < len ? (unsigned long long)(tp_vert[t0 + p] + 1) : 0ull;
                word = (word << bits) | v;
            }
            key[k0 + w] = word;
        }
    }
}

cudaError_t tp_write_keys(const long long *tp_off, const int *tp_vert, long long P, int bits, const long long *key_off,
                          unsigned long long *key, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    long long blocks = (P + (256 / KEY_LANES) - 1) / (256 / KEY_LANES);
    if (blocks > (1 << 20)) blocks = 1 << 20;
    keys_kernel<<<(unsigned)blocks, 256, 0, s>>>(tp_off, tp_vert, P, bits, key_off, key);
    note_launch();
    return cudaGetLastError();
}

__global__ void dedup_keys_kernel(const long long *perm, long long P, const long long *tp_off, const long long *key_off,
                                  const unsigned long long *key, const int *graph, long long *keep_len, int *keep) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = perm[i];
        const int k = (i == 0) || key_cmp(perm[i - 1], a, key_off, key, graph) != 0;
        keep[i] = k;
        keep_len[i] = k ? tp_off[a + 1] - tp_off[a] : 0;
    }
}

cudaError_t tp_dedup_flags_keys(const long long *perm, long long P, const long long *tp_off, const long long *key_off,
                                const unsigned long long *key, const int *tp_graph, long long *keep_len, int *keep,
                                cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    dedup_keys_kernel<<<grid_for(P), 256, 0, s>>>(perm, P, tp_off, key_off, key, tp_graph, keep_len, keep);
    note_launch();
    return cudaGetLastError();
}

__global__ void index_map_kernel(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                                 int *map) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        if (!perm) map[i] = (int)i;
        else map[perm[i]] = (int)(keep[i] ? keep_rank[i] : keep_rank[i] - 1);
    }
}

cudaError_t tp_index_map(const long long *perm, const int *keep, const long long *keep_rank, long long P, int *map,
                         cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    index_map_kernel<<<grid_for(P), 256, 0, s>>>(perm, keep, keep_rank, P, map);
    note_launch();
    return cudaGetLastError();
}

// A TP as its three parts: path(entry -> first p) without its last vertex,
// the PP, path(last p -> exit) without its first vertex.
struct TpView {
    const int *pre, *pp, *suf;
    long long pl, plen;
    __device__ __forceinline__ int at(long long p) const {
        if (p < pl) return pre[p];
        if (p < pl + plen) return pp[p - pl];
        return suf[p - pl - plen];
    }
};

__device__ __forceinline__ TpView tp_view(const long long *pp_off, const int *pp_vert, const int *pp_graph, long long i,
                                          const GraphDev &g) {
    const long long o0 = pp_off[i], o1 = pp_off[i + 1];
    const int gid = pp_graph ? pp_graph[i] : 0;
    const int vb = g.vgraph ? g.vbase[gid] : 0;
    const int f = pp_vert[o0] + vb, l = pp_vert[o1 - 1] + vb;
    TpView t;
    t.pl = g.pre_len[f] - 1;
    t.plen = o1 - o0;
    t.pre = g.pre_seq + g.pre_off[f];
    t.pp = pp_vert + o0;
    t.suf = g.suf_seq + g.suf_off[l] + 1;
    return t;
}

constexpr int TPV_LANES = 8;  // lanes per TP in the key and assembly kernels

// packed keys of TP(p) for every PP p, read from the parts
__global__ void keys_parts_kernel(const long long *pp_off, const int *pp_vert, const int *pp_graph, long long P,
                                  GraphDev g, const long long *tp_off, int bits, const long long *key_off,
                                  unsigned long long *key) {
    const int sub = threadIdx.x & (TPV_LANES - 1), vpw = 64 / bits;
    const long long ngroups = (long long)gridDim.x * (blockDim.x / TPV_LANES);
    for (long long i = blockIdx.x * (long long)(blockDim.x / TPV_LANES) + (threadIdx.x / TPV_LANES); i < P;
         i += ngroups) {
        const TpView t = tp_view(pp_off, pp_vert, pp_graph, i, g);
        const long long total = tp_off[i + 1] - tp_off[i];
        const long long k0 = key_off[i], nw = key_off[i + 1] - k0;
        for (long long w = sub; w < nw; w += TPV_LANES) {
            unsigned long long word = 0;
            for (int q = 0; q < vpw; ++q) {
                const long long p = w * vpw + q;
                word = (word << bits) | (p < total ? (unsigned long long)(t.at(p) + 1) : 0ull);
            }
            key[k0 + w] = word;
        }
    }
}

cudaError_t tp_write_keys_parts(const long long *pp_off, const int *pp_vert, const int *pp_graph, long long P,
                                const GraphDev &g, const long long *tp_off, int bits, const long long *key_off,
                                unsigned long long *key, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    keys_parts_kernel<<<grid_for(P * TPV_LANES), 256, 0, s>>>(pp_off, pp_vert, pp_graph, P, g, tp_off, bits, key_off,
                                                              key);
    note_launch();
    return cudaGetLastError();
}

// the kept TPs in sorted order, each assembled from its parts straight into
// its final place (the TP list is never written in PP order)
__global__ void assemble_kernel(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                                const long long *pp_off, const int *pp_vert, const int *pp_graph, GraphDev g,
                                const long long *tp_off, const long long *keep_off, long long *final_off,
                                int *out_vert, int *out_graph) {
    const int sub = threadIdx.x & (TPV_LANES - 1);
    const long long ngroups = (long long)gridDim.x * (blockDim.x / TPV_LANES);
    for (long long i = blockIdx.x * (long long)(blockDim.x / TPV_LANES) + (threadIdx.x / TPV_LANES); i < P;
         i += ngroups) {
        if (!keep[i]) continue;
        const long long x = perm[i], r = keep_rank[i];
        const TpView t = tp_view(pp_off, pp_vert, pp_graph, x, g);
        const long long len = tp_off[x + 1] - tp_off[x], d0 = keep_off[i];
        for (long long p = sub; p < len; p += TPV_LANES) out_vert[d0 + p] = t.at(p);
        if (sub == 0) {
            out_graph[r] = pp_graph ? pp_graph[x] : 0;
            final_off[r] = d0;
        }
    }
}

cudaError_t tp_assemble(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                        const long long *pp_off, const int *pp_vert, const int *pp_graph, const GraphDev &g,
                        const long long *tp_off, const long long *keep_off, long long *final_off, int *out_vert,
                        int *out_graph, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    assemble_kernel<<<grid_for(P * TPV_LANES), 256, 0, s>>>(perm, keep, keep_rank, P, pp_off, pp_vert, pp_graph, g,
                                                            tp_off, keep_off, final_off, out_vert, out_graph);
    note_launch();
    return cudaGetLastError();
}

// one warp per kept TP: copy into its final slot
__global__ void tp_gather_kernel(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                                 const long long *off, const int *vert, const int *graph,
                                 const long long *keep_off, long long *final_off, int *out_vert,
                                 int *out_graph) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < P; i += nw) {
        if (!keep[i]) continue;
        const long long a = perm[i], r = keep_rank[i];
        const long long s0 = off[a], len = off[a + 1] - s0, d0 = keep_off[i];
        for (long long p = lane; p < len; p += 32) out_vert[d0 + p] = vert[s0 + p];
        if (lane == 0) {
            out_graph[r] = graph[a];
            final_off[r] = d0;
        }
    }
}

cudaError_t tp_gather(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                      const long long *tp_off, const int *tp_vert, const int *tp_graph, const long long *keep_off,
                      long long *final_off, int *out_vert, int *out_graph, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    long long blocks = (P + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    tp_gather_kernel<<<(unsigned)blocks, 256, 0, s>>>(perm, keep, keep_rank, P, tp_off, tp_vert, tp_graph, keep_off,
                                                     final_off, out_vert, out_graph);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
