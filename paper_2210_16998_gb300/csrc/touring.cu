// Longest-first touring: a smaller TP set.
//
// Sec. 7.3 describes Ammann and Offutt's construction of TPs that tour every
// PP: take the longest PP, extend it to the initial and final vertices, and
// repeat with the longest PP that no TP chosen so far covers.  Here "extend"
// is TP(p) of the one-per-PP construction (lowest-id BFS prefix and suffix),
// a PP is covered when it is a contiguous subpath of a chosen TP, equal
// lengths go in canonical order, and the chosen TPs are returned in canonical
// order -- so the result is a subset of the one-per-PP TP list.
//
// GPU design.  The rule is sequential inside a graph, so graphs run in
// parallel: persistent blocks claim whole graphs, those with the most PPs
// first.  A block orders its graph's PPs longest first (counting sort on the
// length, stable) and then runs rounds.  In a round warp 0 collects the next
// NW uncovered PPs in that order; every warp builds its candidate's TP in
// shared memory and finds the PPs that are windows of it; thread 0 takes the
// candidates in order and keeps each one that no kept candidate of the round
// covers -- the sequential rule exactly, since the candidates follow each
// other in the greedy order among the uncovered PPs -- and the warps of the
// kept candidates mark what their TPs cover.
//
// Which windows of a TP t can be PPs: a PP q at position i of t is the
// longest window t[i..j] that is a simple path (a simple t[i..j+1] would
// extend an acyclic q; a cycle q ends where t[i] comes back).  With nxt[k]
// the next position of t[k]'s vertex after k, and S(i) the minimum of nxt
// over [i, L): if nxt[i] < S(i+1) the window is the cycle t[i..nxt[i]],
// else t[i..S(i)-1] (t[i..L-1] when nothing repeats).  t is a prefix path, p
// and a suffix path, each simple, so nxt comes from two per-vertex position
// tables (of p's part and of the suffix part).  Each window is looked up in
// an open-addressing hash table of the PP list and checked vertex by vertex.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "touring.h"

namespace tpg {

namespace {

constexpr int TOUR_MAXW = 16;
constexpr unsigned TOUR_INF = 0xFFFFu;

unsigned grid_for(long long n, int block = 256) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

// (graph, local vertex sequence) -> 64-bit key, never 0: FNV-style mixing of
// each vertex, then the MurmurHash3 64-bit finaliser
__device__ __forceinline__ unsigned long long hash_begin(int gid) {
    return 0xcbf29ce484222325ull ^ ((unsigned long long)(unsigned)gid * 0x9E3779B97F4A7C15ull);
}
__device__ __forceinline__ unsigned long long hash_step(unsigned long long h, int v) {
    return (h ^ (unsigned long long)(unsigned)(v + 1)) * 0x100000001b3ull;
}
__device__ __forceinline__ unsigned long long hash_end(unsigned long long h) {
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    h *= 0xc4ceb9fe1a85ec53ull;
    h ^= h >> 33;
    return h ? h : 1ull;
}

// index in [lo, hi) of the path equal to s[0..len) (graph gid), or -1
template <typename T>
__device__ long long table_find(const PathTable &tab, const long long *off, const int *vert, long long lo,
                                long long hi, int gid, const T *s, int len) {
    unsigned long long h = hash_begin(gid);
    for (int k = 0; k < len; ++k) h = hash_step(h, (int)s[k]);
    h = hash_end(h);
    long long j = (long long)(h & (unsigned long long)tab.mask);
    for (long long probes = 0; probes <= tab.mask; ++probes, j = (j + 1) & tab.mask) {
        const unsigned long long k = tab.key[j];
        if (k == 0ull) return -1;
        if (k != h) continue;
        const long long i = tab.idx[j];
        if (i < lo || i >= hi) continue;
        const long long o = off[i];
        if (off[i + 1] - o != len) continue;
        int e = 0;
        while (e < len && vert[o + e] == (int)s[e]) ++e;
        if (e == len) return i;
    }
    return -1;
}

__device__ __forceinline__ int graph_of_index(const long long *gptr, int G, long long i) {
    int lo = 0, hi = G;  // the last g with gptr[g] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (gptr[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void table_build_kernel(PathTable t, const long long *off, const int *vert, const int *graph_of,
                                   const long long *gptr, int G, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int gid = graph_of ? graph_of[i] : (gptr ? graph_of_index(gptr, G, i) : 0);
        const long long o = off[i], len = off[i + 1] - o;
        unsigned long long h = hash_begin(gid);
        for (long long k = 0; k < len; ++k) h = hash_step(h, vert[o + k]);
        h = hash_end(h);
        long long j = (long long)(h & (unsigned long long)t.mask);
        for (long long probes = 0; probes <= t.mask; ++probes, j = (j + 1) & t.mask) {
            if (atomicCAS(t.key + j, 0ull, h) == 0ull) {
                t.idx[j] = (int)i;
                break;
            }
        }
    }
}

__global__ void graph_ids_kernel(const long long *gptr, int G, long long n, int *ids) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        ids[i] = graph_of_index(gptr, G, i);
}

// shared memory: [block] hist, cursor (maxn + 3 ints each); [per warp] t,
// nxt, S (LM u16 each), posP, posB (maxn shorts each), cover list (LM ints)
struct TourLayout {
    size_t block_bytes, warp_bytes, o_nxt, o_s, o_posp, o_posb, o_cover;
    int lm;
};
__host__ __device__ inline TourLayout tour_layout(int maxn) {
    TourLayout l;
    l.lm = 3 * maxn + 2;
    const size_t LM = (size_t)l.lm;
    l.block_bytes = (2 * sizeof(int) * (size_t)(maxn + 3) + 15) & ~(size_t)15;
    l.o_nxt = LM * sizeof(unsigned short);
    l.o_s = 2 * LM * sizeof(unsigned short);
    l.o_posp = 3 * LM * sizeof(unsigned short);
    l.o_posb = l.o_posp + (size_t)maxn * sizeof(short);
    l.o_cover = (l.o_posb + (size_t)maxn * sizeof(short) + 15) & ~(size_t)15;
    l.warp_bytes = (l.o_cover + LM * sizeof(int) + 15) & ~(size_t)15;
    return l;
}

__global__ void __launch_bounds__(32 * TOUR_MAXW) tour_greedy_kernel(TourArgs a, int G, int NW) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cand[TOUR_MAXW];
    __shared__ unsigned s_M[TOUR_MAXW];
    __shared__ int s_ncov[TOUR_MAXW];
    __shared__ int s_ncand, s_cur, s_graph;
    __shared__ unsigned s_picked;
    const GraphDev &g = a.g;
    const int maxn = a.maxn;
    const TourLayout lay = tour_layout(maxn);
    const int LM = lay.lm;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    int *hist = (int *)smem;
    int *cursor = hist + (maxn + 3);
    unsigned char *wb = smem + lay.block_bytes + (size_t)wid * lay.warp_bytes;
    unsigned short *t = (unsigned short *)wb;
    unsigned short *nxt = (unsigned short *)(wb + lay.o_nxt);
    unsigned short *Sm = (unsigned short *)(wb + lay.o_s);
    short *posP = (short *)(wb + lay.o_posp);
    short *posB = (short *)(wb + lay.o_posb);
    int *cover = (int *)(wb + lay.o_cover);
    for (int i = lane; i < maxn; i += 32) posP[i] = posB[i] = -1;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int c = atomicAdd(a.claim, 1);
            s_graph = c < G ? a.gorder[c] : -1;
        }
        __syncthreads();
        const int gi = s_graph;
        if (gi < 0) break;
        const long long base = a.pp_gptr[gi];
        const int Pg = (int)(a.pp_gptr[gi + 1] - base);
        if (Pg <= 0) continue;
        const int vb = g.vbase[gi];
        const long long tlo = a.tp_gptr[gi], thi = a.tp_gptr[gi + 1];

        // ---- the graph's PPs, longest first (stable counting sort) ----
        for (int i = threadIdx.x; i < maxn + 3; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < Pg; i += blockDim.x) {
            const long long len = a.pp_off[base + i + 1] - a.pp_off[base + i];
            atomicAdd(&hist[len < 0 ? 0 : (len > maxn + 1 ? maxn + 1 : (int)len)], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int l = maxn + 1; l >= 0; --l) {
                cursor[l] = run;
                run += hist[l];
            }
            s_cur = 0;
        }
        __syncthreads();
        if (wid == 0) {
            for (int i0 = 0; i0 < Pg; i0 += 32) {
                const int i = i0 + lane;
                int len = -1;
                if (i < Pg) {
                    const long long l = a.pp_off[base + i + 1] - a.pp_off[base + i];
                    len = l < 0 ? 0 : (l > maxn + 1 ? maxn + 1 : (int)l);
                }
                const unsigned peers = __match_any_sync(0xffffffffu, len);
                const int rank = __popc(peers & lt_mask);
                const int pos = i < Pg ? cursor[len] + rank : 0;
                __syncwarp();
                if (i < Pg && rank == 0) cursor[len] += __popc(peers);
                __syncwarp();
                if (i < Pg) a.ord[base + pos] = i;
            }
        }
        __syncthreads();

        // ---- rounds of up to NW candidates ----
        for (;;) {
            if (wid == 0) {
                int got = 0, i0 = s_cur, last = -1;
                while (got < NW && i0 < Pg) {
                    const int i = i0 + lane;
                    const int q = i < Pg ? a.ord[base + i] : -1;
                    const bool unc = q >= 0 && !a.cov[base + q];
                    const unsigned m = __ballot_sync(0xffffffffu, unc);
                    unsigned take = m;
                    for (int extra = __popc(m) - (NW - got); extra > 0; --extra)
                        take &= ~(1u << (31 - __clz(take)));  // keep the lowest NW - got
                    if (take & (1u << lane)) s_cand[got + __popc(take & lt_mask)] = q;
                    if (take) last = i0 + 31 - __clz(take);
                    got += __popc(take);
                    i0 += 32;
                }
                if (lane == 0) {
                    s_ncand = got;
                    s_cur = got == NW ? last + 1 : Pg;
                }
            }
            __syncthreads();
            const int nc = s_ncand;
            if (nc == 0) break;

            int A = 0, plen = 0, L = 0;
            if (wid < nc) {
                const int q = s_cand[wid];
                const long long po = a.pp_off[base + q];
                plen = (int)(a.pp_off[base + q + 1] - po);
                const int *pv = a.pp_vert + po;
                const int f = plen > 0 ? pv[0] : 0, l = plen > 0 ? pv[plen - 1] : 0;
                const int pl = g.pre_len[vb + f], sl = g.suf_len[vb + l];
                if (plen < 1 || pl == 0 || sl == 0 || pl - 1 + plen + sl - 1 > LM) {
                    if (lane == 0) atomicOr(a.err, (pl == 0 || sl == 0) ? ERR_UNREACH : ERR_INVAL);
                    plen = 0;
                } else {
                    A = pl - 1;
                    L = A + plen + sl - 1;
                }
                // TP(p): prefix path (without its last vertex, p's first), p,
                // suffix path (without its first vertex, p's last)
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
                for (int k = lane; k < L; k += 32) {
                    const int v = t[k];
                    unsigned x = TOUR_INF;
                    if (k < A) x = posP[v] >= 0 ? (unsigned)posP[v] : (posB[v] >= 0 ? (unsigned)posB[v] : TOUR_INF);
                    else if (k < A + plen) x = (cyc && k == A) ? (unsigned)(A + plen - 1)
                                                               : (posB[v] >= 0 ? (unsigned)posB[v] : TOUR_INF);
                    nxt[k] = (unsigned short)x;
                }
                __syncwarp();
                // S = suffix minimum of nxt
                unsigned carry = TOUR_INF;
                for (int c = (L - 1) >> 5; c >= 0; --c) {
                    const int k = c * 32 + lane;
                    unsigned x = k < L ? nxt[k] : TOUR_INF;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned y = __shfl_down_sync(0xffffffffu, x, o);
                        if (lane + o < 32) x = min(x, y);
                    }
                    x = min(x, carry);
                    if (k < L) Sm[k] = (unsigned short)x;
                    carry = __shfl_sync(0xffffffffu, x, 0);
                }
                if (lane == 0) s_ncov[wid] = 0;
                __syncwarp();
                // the one candidate window per start position, looked up
                unsigned mine = 0;
                for (int i = lane; i < L; i += 32) {
                    const unsigned sn = i + 1 < L ? Sm[i + 1] : TOUR_INF;
                    int e;
                    if (nxt[i] < sn) e = nxt[i];
                    else e = Sm[i] >= (unsigned)L ? L - 1 : (int)Sm[i] - 1;
                    const long long r = table_find(a.pp_tab, a.pp_off, a.pp_vert, base, base + Pg, gi, t + i, e - i + 1);
                    if (r >= 0) {
                        const int qq = (int)(r - base);
                        cover[atomicAdd(&s_ncov[wid], 1)] = qq;
                        for (int c = 0; c < nc; ++c)
                            if (s_cand[c] == qq) mine |= 1u << c;
                    }
                }
                mine = __reduce_or_sync(0xffffffffu, mine);
                if (lane == 0) {
                    // TP(p) holds p: its own bit is set (and forced, so that
                    // every round covers its first candidate)
                    if (plen && !(mine & (1u << wid))) atomicOr(a.err, ERR_INVAL);
                    s_M[wid] = mine | (1u << wid);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned covm = 0, picked = 0;
                for (int c = 0; c < nc; ++c)
                    if (!((covm >> c) & 1u)) {
                        picked |= 1u << c;
                        covm |= s_M[c];
                    }
                s_picked = picked;
            }
            __syncthreads();
            if (wid < nc) {
                if ((s_picked >> wid) & 1u) {
                    const int n = s_ncov[wid];
                    for (int j = lane; j < n; j += 32) a.cov[base + cover[j]] = 1;
                    if (lane == 0) {
                        a.cov[base + s_cand[wid]] = 1;
                        if (L > 0) {
                            const long long r = table_find(a.tp_tab, a.tp_off, a.tp_vert, tlo, thi, gi, t, L);
                            if (r >= 0) a.sel[r] = 1;
                            else atomicOr(a.err, ERR_INVAL);
                        }
                    }
                }
                for (int k = A + lane; k < L; k += 32) posP[t[k]] = posB[t[k]] = -1;
            }
            __syncthreads();
        }
    }
}

__global__ void keep_lengths_kernel(const int *sel, const long long *off, long long n, long long *keep_len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        keep_len[i] = sel[i] ? off[i + 1] - off[i] : 0;
}

}  // namespace

long long tour_table_slots(long long n) {
    long long s = 1024;
    while (s < 2 * n) s *= 2;
    return s;
}

cudaError_t tour_table_build(PathTable t, const long long *off, const int *vert, const int *graph_of,
                             const long long *gptr, int G, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    table_build_kernel<<<grid_for(n), 256, 0, s>>>(t, off, vert, graph_of, gptr, G, n);
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

size_t tour_smem_bytes(int maxn, int warps) {
    const TourLayout l = tour_layout(maxn);
    return l.block_bytes + (size_t)warps * l.warp_bytes;
}

int tour_warps(int maxn, size_t smem_max) {
    int w = TOUR_MAXW;
    while (w > 1 && tour_smem_bytes(maxn, w) > smem_max) --w;
    return w;
}

cudaError_t tour_greedy(const TourArgs &a, int G, int warps, int num_sms, cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    if (warps < 1 || warps > TOUR_MAXW) return cudaErrorInvalidValue;
    const size_t smem = tour_smem_bytes(a.maxn, warps);
    cudaError_t e = cudaFuncSetAttribute(tour_greedy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tour_greedy_kernel, 32 * warps, smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(G, (long long)std::max(per_sm, 1) * std::max(num_sms, 1));
    tour_greedy_kernel<<<(unsigned)grid, 32 * warps, smem, s>>>(a, G, warps);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
