// Load-time preprocessing (row a1): union CSR of a batch, device-side CSR
// validation, predecessor CSR, all-pairs BFS tables with the lowest-id
// predecessor tie-break, and the per-vertex tour tables path(entry -> v) and
// path(v -> exit) used to assemble test paths.
#include "common.cuh"
#include "kernels.h"

namespace tpg {

// One block per graph: global ids for the batch (graph g owns vertices
// vbase[g] .. vbase[g+1]-1 and arcs arc_base[g] .. arc_base[g+1]-1).
__global__ void union_csr_kernel(const long long *rp_base, const long long *arc_base, const int *vbase,
                                 const int *rp_cat, const int *col_cat, int G, int N, long long M, int *rp,
                                 int *col, int *vgraph) {
    const int g = blockIdx.x;
    const int vb = vbase[g], ng = vbase[g + 1] - vb;
    const long long rb = rp_base[g], ab = arc_base[g], mg = arc_base[g + 1] - ab;
    for (int i = threadIdx.x; i < ng; i += blockDim.x) {
        rp[vb + i] = (int)(ab + rp_cat[rb + i]);
        vgraph[vb + i] = g;
    }
    for (long long e = threadIdx.x; e < mg; e += blockDim.x) col[ab + e] = col_cat[ab + e] + vb;
    if (g == G - 1 && threadIdx.x == 0) rp[N] = (int)M;
}

cudaError_t build_union_csr(const int *, const long long *rp_base_dev, const long long *arc_base_dev,
                            const int *rp_cat, const int *col_cat, int G, int N, long long M, int *rp, int *col,
                            int *vgraph, int *vbase_dev, cudaStream_t s) {
    union_csr_kernel<<<G, 256, 0, s>>>(rp_base_dev, arc_base_dev, vbase_dev, rp_cat, col_cat, G, N, M, rp, col,
                                       vgraph);
    note_launch();
    return cudaGetLastError();
}

// Device-side validation of one CSR (same rules as the host check): thread
// tid of `stride` checks vertices tid, tid + stride, ...; true if it found a
// violation.
__device__ __forceinline__ bool csr_invalid(const int *rp, const int *col, int n, long long m, int entry, int exit,
                                            int tid, int stride) {
    if (tid == 0) {
        if (rp[0] != 0 || (long long)rp[n] != m) return true;
        if (entry < 0 || entry >= n || exit < 0 || exit >= n || entry == exit) return true;
        if (rp[exit + 1] != rp[exit]) return true;
    }
    for (int u = tid; u < n; u += stride) {
        const int a = rp[u], b = rp[u + 1];
        if (b < a || a < 0 || (long long)b > m) return true;
        for (int e = a; e < b; ++e) {
            const int w = col[e];
            if (w < 0 || w >= n || (e > a && w <= col[e - 1]) || w == entry) return true;
        }
    }
    return false;
}

__global__ void validate_kernel(const int *rp, const int *col, int n, long long m, int entry, int exit,
                                int *err) {
    if (csr_invalid(rp, col, n, m, entry, exit, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x))
        atomicOr(err, ERR_INVAL);
}

cudaError_t validate_csr_device(const int *rp, const int *col, int n, long long m, int entry, int exit, int *err,
                                cudaStream_t s) {
    int blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    validate_kernel<<<blocks, 256, 0, s>>>(rp, col, n, m, entry, exit, err);
    note_launch();
    return cudaGetLastError();
}

__global__ void indeg_kernel(const int *col, long long M, int *indeg) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x)
        atomicAdd(indeg + col[e], 1);
}

__global__ void to_i32_kernel(const long long *in, int *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (int)in[i];
}

__global__ void pred_scatter_kernel(const int *rp, const int *col, int N, int *cursor, int *pcol) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x)
        for (int e = rp[u]; e < rp[u + 1]; ++e) pcol[atomicAdd(cursor + col[e], 1)] = u;
}

// ascending order inside every predecessor list (lists are short)
__global__ void pred_sort_kernel(const int *prp, int *pcol, int N) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const int a = prp[v], b = prp[v + 1];
        for (int i = a + 1; i < b; ++i) {
            const int x = pcol[i];
            int j = i - 1;
            while (j >= a && pcol[j] > x) {
                pcol[j + 1] = pcol[j];
                --j;
            }
            pcol[j + 1] = x;
        }
    }
}

static unsigned grid_for(long long n, int block = 256) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

cudaError_t build_pred_csr(const GraphDev &g, int *prp, int *pcol, int *indeg_tmp, long long *scan_tmp,
                           long long *scan_buf, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(indeg_tmp, 0, sizeof(int) * (size_t)g.N, s);
    if (e != cudaSuccess) return e;
    if (g.M > 0) {
        indeg_kernel<<<grid_for(g.M), 256, 0, s>>>(g.col, g.M, indeg_tmp);
        note_launch();
    }
    if ((e = scan_i32_to_i64(indeg_tmp, scan_buf, g.N, scan_tmp, s)) != cudaSuccess) return e;
    to_i32_kernel<<<grid_for(g.N + 1), 256, 0, s>>>(scan_buf, prp, g.N + 1);
    note_launch();
    to_i32_kernel<<<grid_for(g.N), 256, 0, s>>>(scan_buf, indeg_tmp, g.N);  // cursor = start
    pred_scatter_kernel<<<grid_for(g.N), 256, 0, s>>>(g.rp, g.col, g.N, indeg_tmp, pcol);
    note_launch();
    pred_sort_kernel<<<grid_for(g.N), 256, 0, s>>>(prp, pcol, g.N);
    note_launch();
    return cudaGetLastError();
}

// One block per source vertex a: pull-style BFS inside a's graph.  A vertex
// x first reached at distance d+1 takes as predecessor the lowest-id u with
// an arc u -> x and dist(u) = d.  The graph's predecessor lists are copied to
// shared memory (local ids) when they fit in arc_cap arcs: every level then
// reads shared memory only.
constexpr int BFS_BLOCK = 128;
constexpr int BFS_SMEM_BUDGET = 64 * 1024;

template <bool STAGED>
__device__ __forceinline__ void bfs_levels(const GraphDev &g, int vb, int ng, const int *prp_s, const int *pcol_s,
                                           int *dist_s, int *prow) {
    for (int d = 0;; ++d) {
        int changed = 0;
        for (int x = threadIdx.x; x < ng; x += BFS_BLOCK) {
            if (dist_s[x] != -1) continue;
            int best = 0x7fffffff;
            const int e0 = STAGED ? prp_s[x] : g.prp[vb + x], e1 = STAGED ? prp_s[x + 1] : g.prp[vb + x + 1];
            for (int e = e0; e < e1; ++e) {
                const int u = STAGED ? pcol_s[e] : g.pcol[e] - vb;
                if (dist_s[u] == d && u < best) best = u;
            }
            if (best != 0x7fffffff) {
                dist_s[x] = d + 1;  // other threads only test == d this round
                prow[x] = best;
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
}

__global__ void __launch_bounds__(BFS_BLOCK) bfs_kernel(GraphDev g, const int *gate, int arc_cap) {
    extern __shared__ int smem[];
    if (gate && *gate) return;  // the CSR failed validation
    int *dist_s = smem;                 // [maxn]
    int *prp_s = smem + g.maxn;         // [maxn + 1]
    int *pcol_s = prp_s + g.maxn + 1;   // [arc_cap]
    const int a = blockIdx.x;
    const int gid = g.vgraph ? g.vgraph[a] : 0;
    const int vb = g.vgraph ? g.vbase[gid] : 0;
    const int ng = g.vgraph ? g.vbase[gid + 1] - vb : g.N;
    const int al = a - vb;
    int *drow = g.dist + g.tbl_base[gid] + (long long)al * ng;
    int *prow = g.pred + g.tbl_base[gid] + (long long)al * ng;
    const int a0 = g.prp[vb], mg = g.prp[vb + ng] - a0;
    const bool staged = mg <= arc_cap;
    for (int x = threadIdx.x; x < ng; x += BFS_BLOCK) {
        dist_s[x] = (x == al) ? 0 : -1;
        prow[x] = -1;
    }
    if (staged) {
        for (int x = threadIdx.x; x <= ng; x += BFS_BLOCK) prp_s[x] = g.prp[vb + x] - a0;
        for (int e = threadIdx.x; e < mg; e += BFS_BLOCK) pcol_s[e] = g.pcol[a0 + e] - vb;
    }
    __syncthreads();
    if (staged) bfs_levels<true>(g, vb, ng, prp_s, pcol_s, dist_s, prow);
    else bfs_levels<false>(g, vb, ng, prp_s, pcol_s, dist_s, prow);
    for (int x = threadIdx.x; x < ng; x += BFS_BLOCK) drow[x] = dist_s[x];
}

cudaError_t bfs_all_pairs(const GraphDev &g, cudaStream_t s, const int *gate, long long max_arcs) {
    const size_t base = sizeof(int) * (2 * (size_t)g.maxn + 1);
    const size_t want = base + sizeof(int) * (size_t)max_arcs;
    const int arc_cap = want <= (size_t)BFS_SMEM_BUDGET ? (int)max_arcs : 0;
    const size_t smem = base + sizeof(int) * (size_t)arc_cap;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(bfs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    bfs_kernel<<<g.N, BFS_BLOCK, smem, s>>>(g, gate, arc_cap);
    note_launch();
    return cudaGetLastError();
}

// pre_len[v] = vertices of path(entry -> v) (0 if none); suf_len[v] = vertices
// of path(v -> exit).
__device__ __forceinline__ void tour_len_one(const GraphDev &g, int v) {
    const int gid = g.vgraph ? g.vgraph[v] : 0;
    const int vb = g.vgraph ? g.vbase[gid] : 0;
    const int ng = g.vgraph ? g.vbase[gid + 1] - vb : g.N;
    const int en = g.entry[gid] - vb, ex = g.exit[gid] - vb, vl = v - vb;
    const int *D = g.dist + g.tbl_base[gid];
    const int d1 = D[(long long)en * ng + vl];
    const int d2 = D[(long long)vl * ng + ex];
    g.pre_len[v] = d1 >= 0 ? d1 + 1 : 0;
    g.suf_len[v] = d2 >= 0 ? d2 + 1 : 0;
}

__global__ void tour_len_kernel(GraphDev g) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += gridDim.x * blockDim.x) tour_len_one(g, v);
}

// P: v's graph's predecessor table (global, or a shared-memory copy)
__device__ __forceinline__ void tour_fill_one(const GraphDev &g, int v, const int *P) {
    const int gid = g.vgraph ? g.vgraph[v] : 0;
    const int vb = g.vgraph ? g.vbase[gid] : 0;
    const int ng = g.vgraph ? g.vbase[gid + 1] - vb : g.N;
    const int en = g.entry[gid] - vb, ex = g.exit[gid] - vb, vl = v - vb;
    // path(entry -> v), backwards from v through P[entry][.]
    int len = g.pre_len[v];
    int *dst = g.pre_seq + g.pre_off[v];
    int x = vl;
    for (int i = len - 1; i >= 0; --i) {
        dst[i] = x;
        if (i > 0) x = P[(long long)en * ng + x];
    }
    // path(v -> exit), backwards from exit through P[v][.]
    len = g.suf_len[v];
    dst = g.suf_seq + g.suf_off[v];
    x = ex;
    for (int i = len - 1; i >= 0; --i) {
        dst[i] = x;
        if (i > 0) x = P[(long long)vl * ng + x];
    }
}

__global__ void tour_fill_kernel(GraphDev g) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += gridDim.x * blockDim.x)
        tour_fill_one(g, v, g.pred + g.tbl_base[g.vgraph ? g.vgraph[v] : 0]);
}

cudaError_t tour_lengths(const GraphDev &g, long long *scan_tmp, cudaStream_t s) {
    tour_len_kernel<<<grid_for(g.N), 256, 0, s>>>(g);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = scan_i32_to_i64(g.pre_len, g.pre_off, g.N, scan_tmp, s)) != cudaSuccess) return e;
    return scan_i32_to_i64(g.suf_len, g.suf_off, g.N, scan_tmp, s);
}

cudaError_t tour_fill(const GraphDev &g, cudaStream_t s) {
    tour_fill_kernel<<<grid_for(g.N), 256, 0, s>>>(g);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// one graph of at most PREP_SMALL_N vertices: the steps above in three
// launches (this kernel, the BFS, tour_small_kernel) and no host round trip
// but the final error check
// ---------------------------------------------------------------------------
constexpr int PREP_BLOCK = 1024;
constexpr size_t TOUR_STAGE_BYTES = 96 * 1024;  // predecessor tables up to 156 x 156 go to shared memory

// Optional CSR validation (an invalid CSR sets ERR_INVAL in *err and nothing
// else runs), then the predecessor CSR with ascending lists and the table
// base {0, N*N}.  Dynamic shared memory: N + 1 ints.
__global__ void __launch_bounds__(PREP_BLOCK) prep_small_kernel(GraphDev g, int *prp, int *pcol,
                                                                long long *tbl_base, int validate, int entry,
                                                                int exit, int *err) {
    extern __shared__ int s_cur[];
    __shared__ int s_bad;
    const int N = g.N, tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (validate) {
        if (csr_invalid(g.rp, g.col, N, g.M, entry, exit, tid, PREP_BLOCK)) s_bad = 1;
        __syncthreads();
        if (s_bad) {
            if (tid == 0) atomicOr(err, ERR_INVAL);
            return;
        }
    }
    for (int v = tid; v <= N; v += PREP_BLOCK) s_cur[v] = 0;
    __syncthreads();
    for (long long e = tid; e < g.M; e += PREP_BLOCK) atomicAdd(&s_cur[g.col[e]], 1);
    __syncthreads();
    // exclusive scan of the in-degrees: prp, and the scatter cursors
    long long carry = 0;
    for (int base = 0; base <= N; base += PREP_BLOCK) {
        const int v = base + tid;
        const long long c = v < N ? s_cur[v] : 0;
        long long tot = 0;
        const long long ex = block_excl_scan_i64<PREP_BLOCK>(c, tot);
        if (v <= N) {
            prp[v] = (int)(carry + ex);
            s_cur[v] = (int)(carry + ex);
        }
        carry += tot;
    }
    if (tid == 0) {
        tbl_base[0] = 0;
        tbl_base[1] = (long long)N * N;
    }
    __syncthreads();
    for (int u = tid; u < N; u += PREP_BLOCK)
        for (int e = g.rp[u]; e < g.rp[u + 1]; ++e) pcol[atomicAdd(&s_cur[g.col[e]], 1)] = u;
    __syncthreads();
    for (int v = tid; v < N; v += PREP_BLOCK) {
        const int a = prp[v], b = prp[v + 1];
        for (int i = a + 1; i < b; ++i) {
            const int x = pcol[i];
            int j = i - 1;
            while (j >= a && pcol[j] > x) {
                pcol[j + 1] = pcol[j];
                --j;
            }
            pcol[j + 1] = x;
        }
    }
}

// Successor and predecessor bitsets of vertex v (graph-local bit ids, W
// words each).  Ids outside the graph's W words are skipped, so a CSR that
// failed validation cannot make it write elsewhere (it is never run on one).
__device__ __forceinline__ void vertex_masks(const GraphDev &g, int v, unsigned *smask, unsigned *pmask) {
    const int W = g.W;
    const int vb = g.vgraph ? g.vbase[g.vgraph[v]] : 0;
    for (int j = 0; j < W; ++j) {
        unsigned sm = 0u, pm = 0u;
        for (int e = g.rp[v]; e < g.rp[v + 1]; ++e) {
            const int b = g.col[e] - vb;
            if ((b >> 5) == j && b >= 0) sm |= 1u << (b & 31);
        }
        for (int e = g.prp[v]; e < g.prp[v + 1]; ++e) {
            const int b = g.pcol[e] - vb;
            if ((b >> 5) == j && b >= 0) pm |= 1u << (b & 31);
        }
        smask[(long long)v * W + j] = sm;
        pmask[(long long)v * W + j] = pm;
    }
}

__global__ void masks_kernel(GraphDev g, unsigned *smask, unsigned *pmask, const int *gate) {
    if (gate && *gate) return;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.N; v += (long long)gridDim.x * blockDim.x)
        vertex_masks(g, (int)v, smask, pmask);
}

cudaError_t build_vertex_masks(const GraphDev &g, unsigned *smask, unsigned *pmask, const int *gate, cudaStream_t s) {
    if (g.W > MASK_MAX_W) return cudaErrorInvalidValue;
    masks_kernel<<<grid_for(g.N), 256, 0, s>>>(g, smask, pmask, gate);
    note_launch();
    return cudaGetLastError();
}

// Tour lengths, their offsets and the tour sequences of one graph in one
// block; pre_seq and suf_seq hold N(N+1)/2 entries each, an upper bound (the
// i-th vertex in order of distance from the entry is at most i arcs away, so
// its path has at most i + 1 vertices; the same toward the exit).  With
// stage_pred the N x N predecessor table is first copied to dynamic shared
// memory, so the path walks read shared memory.
__global__ void __launch_bounds__(PREP_BLOCK) tour_small_kernel(GraphDev g, const int *gate, int stage_pred,
                                                                unsigned *smask, unsigned *pmask) {
    extern __shared__ int pred_s[];
    if (*gate) return;
    const int N = g.N, tid = threadIdx.x;
    if (smask)
        for (int v = tid; v < N; v += PREP_BLOCK) vertex_masks(g, v, smask, pmask);
    if (stage_pred) {
        const long long nn = (long long)N * N;
        for (long long i = tid; i < nn; i += PREP_BLOCK) pred_s[i] = g.pred[i];
    }
    for (int v = tid; v < N; v += PREP_BLOCK) tour_len_one(g, v);
    __syncthreads();
    long long cp = 0, cs = 0;
    for (int base = 0; base <= N; base += PREP_BLOCK) {
        const int v = base + tid;
        const long long a = v < N ? g.pre_len[v] : 0, b = v < N ? g.suf_len[v] : 0;
        long long ta = 0, tb = 0;
        const long long ea = block_excl_scan_i64<PREP_BLOCK>(a, ta);
        const long long eb = block_excl_scan_i64<PREP_BLOCK>(b, tb);
        if (v <= N) {
            g.pre_off[v] = cp + ea;
            g.suf_off[v] = cs + eb;
        }
        cp += ta;
        cs += tb;
    }
    __syncthreads();
    for (int v = tid; v < N; v += PREP_BLOCK) tour_fill_one(g, v, stage_pred ? pred_s : g.pred);
}

cudaError_t preprocess_small(const GraphDev &g, int *prp, int *pcol, long long *tbl_base, bool validate, int entry,
                             int exit, int *err, cudaStream_t s, unsigned *smask, unsigned *pmask) {
    if (g.G != 1 || g.N > PREP_SMALL_N) return cudaErrorInvalidValue;
    prep_small_kernel<<<1, PREP_BLOCK, sizeof(int) * (g.N + 1), s>>>(g, prp, pcol, tbl_base, validate ? 1 : 0,
                                                                     entry, exit, err);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = bfs_all_pairs(g, s, err, g.M)) != cudaSuccess) return e;
    const size_t pred_bytes = sizeof(int) * (size_t)g.N * g.N;
    const int stage = pred_bytes <= TOUR_STAGE_BYTES;
    if (stage && pred_bytes > 48 * 1024) {
        if ((e = cudaFuncSetAttribute(tour_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TOUR_STAGE_BYTES)) != cudaSuccess)
            return e;
    }
    tour_small_kernel<<<1, PREP_BLOCK, stage ? pred_bytes : 0, s>>>(g, err, stage, smask, pmask);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
