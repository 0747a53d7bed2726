// Longest-first touring: a smaller TP set.
//
// Sec. 7.3 describes Ammann and Offutt's construction of TPs that tour every
// PP: take the longest PP, extend it to the initial and final vertices, and
// repeat with the longest PP that no TP chosen so far covers.  Here "extend"
// is TP(p) of the one-per-PP construction (lowest-id BFS prefix and suffix),
// a PP is covered when it is a contiguous subpath of a chosen TP, equal
// lengths go in canonical order, and the chosen TPs are returned in canonical
// order -- a subset of the one-per-PP TP list.
//
// The rule reads sequentially (a PP's turn depends on the TPs chosen before
// it), but its outcome has a description that parallelises: in the order
// (longer first, then canonical), p is chosen iff no chosen PP before p
// covers p with its TP.  So, over all graphs at once:
//  1. every PP p (a warp each) builds TP(p) in shared memory, finds the PPs
//     that are windows of it, and emits an edge p -> q for each such q that
//     comes after p in the order;
//  2. the edges are grouped by target;
//  3. sweeps decide the PPs: q is covered once a chosen source reaches it,
//     and chosen once all its sources are covered (or it has none).  The
//     first undecided PP in the order has only decided sources, so each
//     sweep decides at least one PP; sweeps repeat until none is left;
//  4. the chosen PPs' TPs are taken from the one-per-PP TP list.
//
// Which windows of a TP t can be PPs: a PP q at position i of t is the
// longest window t[i..j] that is a simple path (a simple t[i..j+1] would
// extend an acyclic q; a cycle q ends where t[i] comes back).  With nxt[k]
// the next position of t[k]'s vertex after k and S(i) the minimum of nxt over
// [i, L): if S(i) < S(i+1) (then S(i) = nxt[i]) the window is the cycle
// t[i..S(i)], else t[i..S(i)-1] (t[i..L-1] when nothing repeats).  t is a
// prefix path, p and a suffix path, each simple, so nxt comes from two
// per-vertex position tables (of p's part and of the suffix part).  Each
// window's hash comes from prefix hashes of t in O(1); it is looked up in an
// open-addressing table of the PP list and checked vertex by vertex.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "touring.h"

namespace tpg {

namespace {

constexpr int TOUR_WARPS = 8;  // warps per block of the edge launch (fewer if shared memory is short)
constexpr unsigned TOUR_INF = 0xFFFFu;
// polynomial hash of a sequence: raw = sum (s_k + 1) B^(len-1-k) mod 2^64,
// key = MurmurHash3's 64-bit finaliser of raw mixed with graph and length
constexpr unsigned long long HB = 0x9E3779B97F4A7C15ull;
constexpr unsigned long long HG = 0xD6E8FEB86659FD93ull;
constexpr unsigned long long HL = 0xA0761D6478BD642Full;

unsigned grid_for(long long n, int block = 256) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

__device__ __forceinline__ unsigned long long hash_key(unsigned long long raw, int gid, int len) {
    unsigned long long h = raw ^ ((unsigned long long)(unsigned)(gid + 1) * HG) ^ ((unsigned long long)len * HL);
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h ? h : 1ull;
}

// v[0..len) == s[0..len), eight independent loads at a time
__device__ __forceinline__ bool same_seq(const int *v, const unsigned short *s, int len) {
    int e = 0;
    for (; e + 8 <= len; e += 8) {
        int x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = v[e + u];
        bool ok = true;
#pragma unroll
        for (int u = 0; u < 8; ++u) ok &= x[u] == (int)s[e + u];
        if (!ok) return false;
    }
    for (; e < len; ++e)
        if (v[e] != (int)s[e]) return false;
    return true;
}

__global__ void powers_kernel(unsigned long long *pw, int n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long x = 1ull;
        for (int k = 0; k <= n; ++k) {
            pw[k] = x;
            x *= HB;
        }
    }
}

__global__ void table_build_kernel(PathTable t, const long long *off, const int *vert, const int *graph_of,
                                   long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long o = off[i];
        const int len = (int)(off[i + 1] - o);
        unsigned long long raw = 0ull;
        for (int k = 0; k < len; ++k) raw = raw * HB + (unsigned long long)(unsigned)(vert[o + k] + 1);
        const int gid = graph_of ? graph_of[i] : 0;
        const unsigned long long h = hash_key(raw, gid, len);
        const long long t0 = t.tbase[gid], mask = t.tbase[gid + 1] - t0 - 1;
        long long j = (long long)(h & (unsigned long long)mask);
        for (long long probes = 0; probes <= mask; ++probes, j = (j + 1) & mask) {
            if (atomicCAS(t.key + t0 + j, 0ull, h) == 0ull) {
                t.idx[t0 + j] = (int)i;
                break;
            }
        }
    }
}

// shared memory of one warp: t (u16), S (u16), hit list (int), position
// tables of p's part and of the suffix part (short), prefix hashes (u64)
struct TourLayout {
    size_t warp_bytes, o_s, o_hit, o_posp, o_posb, o_pf;
    int lm;
};
__host__ __device__ inline TourLayout tour_layout(int maxn) {
    TourLayout l;
    l.lm = 3 * maxn + 2;
    const size_t LM = (size_t)l.lm;
    l.o_s = (LM * sizeof(unsigned short) + 15) & ~(size_t)15;
    l.o_hit = l.o_s + ((LM * sizeof(unsigned short) + 15) & ~(size_t)15);
    l.o_posp = l.o_hit + ((LM * sizeof(int) + 15) & ~(size_t)15);
    l.o_posb = l.o_posp + (size_t)maxn * sizeof(short);
    l.o_pf = (l.o_posb + (size_t)maxn * sizeof(short) + 15) & ~(size_t)15;
    l.warp_bytes = (l.o_pf + (LM + 1) * sizeof(unsigned long long) + 15) & ~(size_t)15;
    return l;
}

__global__ void __launch_bounds__(32 * TOUR_WARPS) tour_edges_kernel(TourEdgeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_nhit[TOUR_WARPS];
    const GraphDev &g = a.g;
    const int maxn = a.maxn;
    const TourLayout lay = tour_layout(maxn);
    const int LM = lay.lm;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char *wb = smem + (size_t)wid * lay.warp_bytes;
    unsigned short *t = (unsigned short *)wb;
    unsigned short *S = (unsigned short *)(wb + lay.o_s);
    int *hit = (int *)(wb + lay.o_hit);
    short *posP = (short *)(wb + lay.o_posp);
    short *posB = (short *)(wb + lay.o_posb);
    unsigned long long *Pf = (unsigned long long *)(wb + lay.o_pf);
    for (int i = lane; i < maxn; i += 32) posP[i] = posB[i] = -1;
    __syncwarp();
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long p = blockIdx.x * (long long)(blockDim.x >> 5) + wid; p < a.P; p += nw) {
        const int gi = a.pp_graph ? a.pp_graph[p] : 0;
        const long long lo = a.pp_gptr[gi], hi = a.pp_gptr[gi + 1];
        const int vb = g.vbase[gi];
        const long long t0 = a.tab.tbase[gi], tmask = a.tab.tbase[gi + 1] - t0 - 1;
        const unsigned long long *tkey = a.tab.key + t0;
        const int *tidx = a.tab.idx + t0;
        const long long po = a.pp_off[p];
        const int plen = (int)(a.pp_off[p + 1] - po);
        const int *pv = a.pp_vert + po;
        const int f = plen > 0 ? pv[0] : 0, l = plen > 0 ? pv[plen - 1] : 0;
        const int pl = g.pre_len[vb + f], sl = g.suf_len[vb + l];
        if (plen < 1 || pl == 0 || sl == 0 || pl - 1 + plen + sl - 1 > LM) {
            if (lane == 0) atomicOr(a.err, (plen >= 1 && (pl == 0 || sl == 0)) ? ERR_UNREACH : ERR_INVAL);
            continue;
        }
        const int A = pl - 1, L = A + plen + sl - 1;
        // TP(p): the prefix path without its last vertex (p's first), p, the
        // suffix path without its first vertex (p's last)
        const int *pre = g.pre_seq + g.pre_off[vb + f];
        const int *suf = g.suf_seq + g.suf_off[vb + l];
        for (int k = lane; k < L; k += 32)
            t[k] = (unsigned short)(k < A ? pre[k] : (k < A + plen ? pv[k - A] : suf[k - A - plen + 1]));
        __syncwarp();
        const bool cyc = plen > 1 && t[A] == t[A + plen - 1];
        for (int k = A + lane; k < L; k += 32) {
            if (k >= A + plen) posB[t[k]] = (short)k;
            else if (!(cyc && k == A + plen - 1)) posP[t[k]] = (short)k;
        }
        __syncwarp();
        // nxt into S, then S = suffix minimum, chunk by chunk from the end
        unsigned carry = TOUR_INF;
        for (int c = (L - 1) >> 5; c >= 0; --c) {
            const int k = c * 32 + lane;
            unsigned x = TOUR_INF;
            if (k < L) {
                const int v = t[k];
                if (k < A) x = posP[v] >= 0 ? (unsigned)posP[v] : (posB[v] >= 0 ? (unsigned)posB[v] : TOUR_INF);
                else if (k < A + plen)
                    x = (cyc && k == A) ? (unsigned)(A + plen - 1) : (posB[v] >= 0 ? (unsigned)posB[v] : TOUR_INF);
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_down_sync(0xffffffffu, x, o);
                if (lane + o < 32) x = min(x, y);
            }
            x = min(x, carry);
            if (k < L) S[k] = (unsigned short)x;
            carry = __shfl_sync(0xffffffffu, x, 0);
        }
        // prefix hashes Pf[k] = raw(t[0..k)), chunk by chunk: the affine
        // maps x -> x B + (t[k] + 1) composed with a warp scan
        unsigned long long run = 0ull;
        for (int c = 0; c * 32 < L; ++c) {
            const int k = c * 32 + lane;
            unsigned long long m = k < L ? HB : 1ull, b = k < L ? (unsigned long long)(t[k] + 1u) : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long m0 = __shfl_up_sync(0xffffffffu, m, o);
                const unsigned long long b0 = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) {
                    b = b0 * m + b;
                    m = m0 * m;
                }
            }
            const unsigned long long v = run * m + b;
            if (k < L) Pf[k + 1] = v;
            run = __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) {
            Pf[0] = 0ull;
            s_nhit[wid] = 0;
        }
        __syncwarp();
        // the one possible PP per start position, looked up
        for (int i = lane; i < L; i += 32) {
            const unsigned si = S[i], sn = i + 1 < L ? S[i + 1] : TOUR_INF;
            const int e = si < sn ? (int)si : (si >= (unsigned)L ? L - 1 : (int)si - 1);
            const int len = e - i + 1;
            const unsigned long long raw = Pf[e + 1] - Pf[i] * a.pw[len];
            const unsigned long long h = hash_key(raw, gi, len);
            long long j = (long long)(h & (unsigned long long)tmask);
            for (long long probes = 0; probes <= tmask; ++probes, j = (j + 1) & tmask) {
                const unsigned long long kj = tkey[j];
                if (kj == 0ull) break;
                if (kj != h) continue;
                const long long q = tidx[j];
                if (q < lo || q >= hi) continue;
                const long long qo = a.pp_off[q];
                if (a.pp_off[q + 1] - qo != len || !same_seq(a.pp_vert + qo, t + i, len)) continue;
                // q comes after p: shorter, or as long and later in canonical order
                if (len < plen || (len == plen && q > p)) hit[atomicAdd(&s_nhit[wid], 1)] = (int)q;
                break;
            }
        }
        __syncwarp();
        const int n = s_nhit[wid];
        if (n > 0) {
            unsigned long long e0 = 0;
            if (lane == 0) e0 = atomicAdd(a.edge_count, (unsigned long long)n);
            e0 = __shfl_sync(0xffffffffu, e0, 0);
            for (int j = lane; j < n; j += 32)
                if ((long long)(e0 + j) < a.edge_cap) a.edges[e0 + j] = make_int2((int)p, hit[j]);
        }
        for (int k = A + lane; k < L; k += 32) posP[t[k]] = posB[t[k]] = -1;
        __syncwarp();
    }
}

__global__ void indeg_kernel(const int2 *edges, long long E, int *indeg) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < E;
         k += (long long)gridDim.x * blockDim.x)
        atomicAdd(indeg + edges[k].y, 1);
}

__global__ void group_kernel(const int2 *edges, long long E, const long long *in_off, int *indeg, int *in_src) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < E;
         k += (long long)gridDim.x * blockDim.x) {
        const int2 e = edges[k];
        in_src[in_off[e.y] + atomicSub(indeg + e.y, 1) - 1] = e.x;
    }
}

__global__ void sweep_kernel(const long long *in_off, const int *in_src, long long P, unsigned char *state,
                             unsigned long long *undecided) {
    __shared__ unsigned s_left;
    if (threadIdx.x == 0) s_left = 0;
    __syncthreads();
    unsigned left = 0;
    volatile unsigned char *st = state;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < P;
         q += (long long)gridDim.x * blockDim.x) {
        if (st[q]) continue;
        bool chosen_src = false, all_done = true;
        for (long long k = in_off[q], k1 = in_off[q + 1]; k < k1; ++k) {
            const unsigned char s = st[in_src[k]];
            if (s == 1) {
                chosen_src = true;
                break;
            }
            if (s == 0) all_done = false;
        }
        if (chosen_src) st[q] = 2;
        else if (all_done) st[q] = 1;
        else ++left;
    }
    if (left) atomicAdd(&s_left, left);
    __syncthreads();
    if (threadIdx.x == 0 && s_left) atomicAdd(undecided, (unsigned long long)s_left);
}

__global__ void select_kernel(const unsigned char *state, const int *map, long long P, int *sel) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < P;
         q += (long long)gridDim.x * blockDim.x)
        if (state[q] == 1) sel[map[q]] = 1;
}

__global__ void graph_ids_kernel(const long long *gptr, int G, long long n, int *ids) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;  // the last graph g with gptr[g] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (gptr[mid] <= i) lo = mid;
            else hi = mid;
        }
        ids[i] = lo;
    }
}

__global__ void keep_lengths_kernel(const int *sel, const long long *off, long long n, long long *keep_len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        keep_len[i] = sel[i] ? off[i + 1] - off[i] : 0;
}

}  // namespace

long long tour_table_layout(const long long *gptr, int G, long long *tbase) {
    tbase[0] = 0;
    for (int g = 0; g < G; ++g) {
        long long sz = 16;
        while (sz < 2 * (gptr[g + 1] - gptr[g])) sz *= 2;
        tbase[g + 1] = tbase[g] + sz;
    }
    return tbase[G];
}

int tour_max_tp(int maxn) { return 3 * maxn + 2; }

cudaError_t tour_powers(unsigned long long *pw, int n, cudaStream_t s) {
    powers_kernel<<<1, 32, 0, s>>>(pw, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_table_build(PathTable t, const long long *off, const int *vert, const int *graph_of, long long P,
                             cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    table_build_kernel<<<grid_for(P), 256, 0, s>>>(t, off, vert, graph_of, P);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_edges(const TourEdgeArgs &a, int num_sms, int *warps_out, cudaStream_t s) {
    if (a.P <= 0) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const TourLayout lay = tour_layout(a.maxn);
    int warps = TOUR_WARPS;
    while (warps > 1 && (size_t)warps * lay.warp_bytes + 1024 > (size_t)optin) --warps;
    if ((size_t)warps * lay.warp_bytes + 1024 > (size_t)optin) return cudaErrorInvalidValue;
    const size_t smem = (size_t)warps * lay.warp_bytes;
    e = cudaFuncSetAttribute(tour_edges_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tour_edges_kernel, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    const long long need = (a.P + warps - 1) / warps;
    const long long grid =
        std::max(1LL, std::min<long long>(need, (long long)std::max(per_sm, 1) * std::max(num_sms, 1)));
    tour_edges_kernel<<<(unsigned)grid, 32 * warps, smem, s>>>(a);
    note_launch();
    if (warps_out) *warps_out = warps;
    return cudaGetLastError();
}

cudaError_t tour_indegrees(const int2 *edges, long long E, int *indeg, cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    indeg_kernel<<<grid_for(E), 256, 0, s>>>(edges, E, indeg);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_group_edges(const int2 *edges, long long E, const long long *in_off, int *indeg, int *in_src,
                             cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    group_kernel<<<grid_for(E), 256, 0, s>>>(edges, E, in_off, indeg, in_src);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_sweep(const long long *in_off, const int *in_src, long long P, unsigned char *state,
                       unsigned long long *undecided, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    sweep_kernel<<<grid_for(P), 256, 0, s>>>(in_off, in_src, P, state, undecided);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_select(const unsigned char *state, const int *map, long long P, int *sel, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    select_kernel<<<grid_for(P), 256, 0, s>>>(state, map, P, sel);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_graph_ids(const long long *gptr, int G, long long n, int *ids, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    graph_ids_kernel<<<grid_for(n), 256, 0, s>>>(gptr, G, n, ids);
    note_launch();
    return cudaGetLastError();
}

cudaError_t tour_keep_lengths(const int *sel, const long long *off, long long n, long long *keep_len,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    keep_lengths_kernel<<<grid_for(n), 256, 0, s>>>(sel, off, n, keep_len);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
