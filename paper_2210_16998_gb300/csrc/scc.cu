// The per-SCC step of the compositional route (Sec. 2.1; Defs. 3, 5 and 9).
//
// The strongly connected components come from the all-pairs BFS table the
// load already builds: v and u share an SCC iff each reaches the other, and
// an SCC is named by its smallest vertex.  The SCC subgraphs are the graph
// restricted to arcs inside one SCC; their union is a graph whose simple
// paths never leave an SCC, so the regular frontier run on it yields the
// PPs of every SCC's own subgraph at once.  The SccInternalPPs (Def. 9) are
// those that are cycles, or that neither start at an SccEntryVertex (one
// with a predecessor in another SCC) nor end at an SccExitVertex (one with a
// successor in another SCC).
#include "common.cuh"
#include "kernels.h"
#include "scc.h"

namespace tpg {

namespace {

unsigned grid_for(long long n, int block = 256) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

__global__ void scc_ids_kernel(GraphDev g, int *comp) {
    const int n = g.N;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int *dv = g.dist + (long long)v * n;  // d(v, .)
        int c = v;
        for (int u = 0; u < v; ++u)
            if (dv[u] >= 0 && g.dist[(long long)u * n + v] >= 0) {
                c = u;
                break;
            }
        comp[v] = c;
    }
}

__global__ void intra_count_kernel(GraphDev g, const int *comp, int *cnt) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < g.N; u += gridDim.x * blockDim.x) {
        int c = 0;
        for (int e = g.rp[u]; e < g.rp[u + 1]; ++e) c += comp[g.col[e]] == comp[u];
        cnt[u] = c;
    }
}

__global__ void intra_write_kernel(GraphDev g, const int *comp, const long long *off, int *row_ptr, int *col) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u <= g.N; u += gridDim.x * blockDim.x) {
        row_ptr[u] = (int)off[u];
        if (u == g.N) continue;
        long long o = off[u];
        for (int e = g.rp[u]; e < g.rp[u + 1]; ++e)
            if (comp[g.col[e]] == comp[u]) col[o++] = g.col[e];
    }
}

__global__ void boundary_kernel(GraphDev g, const int *comp, unsigned char *is_entry, unsigned char *is_exit) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += gridDim.x * blockDim.x) {
        bool en = false, ex = false;
        for (int e = g.prp[v]; e < g.prp[v + 1]; ++e) en |= comp[g.pcol[e]] != comp[v];
        for (int e = g.rp[v]; e < g.rp[v + 1]; ++e) ex |= comp[g.col[e]] != comp[v];
        is_entry[v] = en;
        is_exit[v] = ex;
    }
}

__global__ void internal_flags_kernel(const long long *off, const int *vert, long long P,
                                      const unsigned char *is_entry, const unsigned char *is_exit, int *keep,
                                      long long *keep_len) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const long long o = off[i], len = off[i + 1] - o;
        const int f = vert[o], l = vert[o + len - 1];
        const bool k = (len >= 2 && f == l) || (!is_entry[f] && !is_exit[l]);
        keep[i] = k;
        keep_len[i] = k ? len : 0;
    }
}

}  // namespace

cudaError_t scc_ids(const GraphDev &g, int *comp, cudaStream_t s) {
    scc_ids_kernel<<<grid_for(g.N, 128), 128, 0, s>>>(g, comp);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scc_intra_counts(const GraphDev &g, const int *comp, int *cnt, cudaStream_t s) {
    intra_count_kernel<<<grid_for(g.N), 256, 0, s>>>(g, comp, cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scc_intra_write(const GraphDev &g, const int *comp, const long long *off, int *row_ptr, int *col,
                            cudaStream_t s) {
    intra_write_kernel<<<grid_for(g.N + 1), 256, 0, s>>>(g, comp, off, row_ptr, col);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scc_boundary(const GraphDev &g, const int *comp, unsigned char *is_entry, unsigned char *is_exit,
                         cudaStream_t s) {
    boundary_kernel<<<grid_for(g.N), 256, 0, s>>>(g, comp, is_entry, is_exit);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scc_internal_flags(const long long *off, const int *vert, long long P, const unsigned char *is_entry,
                               const unsigned char *is_exit, int *keep, long long *keep_len, cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    internal_flags_kernel<<<grid_for(P), 256, 0, s>>>(off, vert, P, is_entry, is_exit, keep, keep_len);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
