// Strongly connected components and the SCC-internal prime paths (scc.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tpg {

// comp[v] = the smallest vertex u with d(v, u) and d(u, v) finite (v's SCC,
// named by its smallest member), from the all-pairs BFS table of a
// one-graph handle
cudaError_t scc_ids(const GraphDev &g, int *comp, cudaStream_t s);
// cnt[u] = successors w of u in u's SCC
cudaError_t scc_intra_counts(const GraphDev &g, const int *comp, int *cnt, cudaStream_t s);
// the intra-SCC CSR: row_ptr (int32, from the exclusive scan `off` of cnt,
// off[n] = arcs) and col
cudaError_t scc_intra_write(const GraphDev &g, const int *comp, const long long *off, int *row_ptr, int *col,
                            cudaStream_t s);
// SccEntryVertex / SccExitVertex flags: a predecessor / successor in another SCC
cudaError_t scc_boundary(const GraphDev &g, const int *comp, unsigned char *is_entry, unsigned char *is_exit,
                         cudaStream_t s);
// keep[i] = PP i of the intra-SCC graph is SCC-internal (a cycle, or its
// first vertex no SccEntryVertex and its last no SccExitVertex);
// keep_len[i] = its length if kept, else 0
cudaError_t scc_internal_flags(const long long *off, const int *vert, long long P, const unsigned char *is_entry,
                               const unsigned char *is_exit, int *keep, long long *keep_len, cudaStream_t s);

}  // namespace tpg
