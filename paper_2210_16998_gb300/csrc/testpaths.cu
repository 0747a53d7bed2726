// Test-path assembly (kernel (d)) and canonical sort + dedup of the test
// paths (kernel (e) for TPs).
//
// TP(p) = path(entry -> first p), then p, then path(last p -> exit), joined
// at the shared endpoints (Problem 1 output; the touring of Sec. 7.3), with
// path(a -> b) read from the lowest-id BFS predecessor table.  Because the
// PPs arrive in canonical order, TPs of PPs that share a first vertex share
// their prefix and are already in order among themselves; so the TP list is
// a sequence of sorted runs (one per (graph, first vertex)).  Runs are merged
// pairwise with a merge-path kernel comparing whole sequences, and exact
// duplicates (two PPs of different first vertices can yield the same TP)
// are dropped after the final round.
#include "common.cuh"
#include "kernels.h"
#include "paths_dev.cuh"

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

constexpr int TPM_ITEMS = 4;

// One round of pairwise run merging: pair p = runs (2p, 2p+1).  Thread t
// writes outputs [t*ITEMS, t*ITEMS + ITEMS), locating its pair and merge-path
// split by binary search (A first on ties, so equal TPs stay adjacent).
__global__ void tp_merge_kernel(const long long *perm_in, long long *perm_out, const long long *bounds,
                                long long R, long long P, const long long *off, const int *vert,
                                const int *graph) {
    const long long d0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * TPM_ITEMS;
    if (d0 >= P) return;
    const long long npairs = (R + 1) / 2;
    long long pair = -1, a_lo = 0, a_hi = 0, b_hi = 0, i = 0, j = 0;
    for (int t = 0; t < TPM_ITEMS; ++t) {
        const long long d = d0 + t;
        if (d >= P) break;
        if (pair < 0 || d >= b_hi) {
            // locate the pair containing output position d
            long long lo = 0, hi = npairs - 1;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (bounds[2 * mid] <= d) lo = mid;
                else hi = mid - 1;
            }
            pair = lo;
            a_lo = bounds[2 * pair];
            a_hi = (2 * pair + 1 <= R) ? bounds[2 * pair + 1] : P;
            b_hi = (2 * pair + 2 <= R) ? bounds[2 * pair + 2] : a_hi;
            const long long na = a_hi - a_lo, nb = b_hi - a_hi, diag = d - a_lo;
            long long lo2 = diag > nb ? diag - nb : 0, hi2 = diag < na ? diag : na;
            while (lo2 < hi2) {
                const long long mid = (lo2 + hi2) >> 1;
                if (tp_cmp(perm_in[a_lo + mid], perm_in[a_hi + diag - mid - 1], off, vert, graph) <= 0)
                    lo2 = mid + 1;
                else
                    hi2 = mid;
            }
            i = a_lo + lo2;
            j = a_hi + (diag - lo2);
        }
        bool take_a;
        if (i >= a_hi) take_a = false;
        else if (j >= b_hi) take_a = true;
        else take_a = tp_cmp(perm_in[i], perm_in[j], off, vert, graph) <= 0;
        perm_out[d] = take_a ? perm_in[i++] : perm_in[j++];
    }
}

cudaError_t tp_merge_round(const long long *perm_in, long long *perm_out, const long long *bounds, long long R,
                           long long P, const long long *tp_off, const int *tp_vert, const int *tp_graph,
                           cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const long long threads = (P + TPM_ITEMS - 1) / TPM_ITEMS;
    tp_merge_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(perm_in, perm_out, bounds, R, P, tp_off,
                                                                     tp_vert, tp_graph);
    note_launch();
    return cudaGetLastError();
}

__global__ void halve_bounds_kernel(const long long *bounds, long long R, long long *out) {
    const long long R2 = (R + 1) / 2;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= R2;
         r += (long long)gridDim.x * blockDim.x)
        out[r] = (r < R2) ? bounds[2 * r] : bounds[R];
}

cudaError_t tp_halve_bounds(const long long *bounds, long long R, long long *out, cudaStream_t s) {
    halve_bounds_kernel<<<grid_for((R + 1) / 2 + 1), 256, 0, s>>>(bounds, R, out);
    note_launch();
    return cudaGetLastError();
}

__global__ void dedup_kernel(const long long *perm, long long P, const long long *off, const int *vert,
                             const int *graph, long long *keep_len, int *keep) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = perm[i];
        const int k = (i == 0) || tp_cmp(perm[i - 1], a, off, vert, graph) != 0;
        keep[i] = k;
        keep_len[i] = k ? off[a + 1] - off[a] : 0;
    }
}

cudaError_t tp_dedup_flags(const long long *perm, long long P, const long long *tp_off, const int *tp_vert,
                           const int *tp_graph, long long *keep_len, int *keep, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    dedup_kernel<<<grid_for(P), 256, 0, s>>>(perm, P, tp_off, tp_vert, tp_graph, keep_len, keep);
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
