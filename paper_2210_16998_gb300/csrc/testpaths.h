// Per-graph TP run merging for the host-driven path (testpaths.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tpg {

// run_base[g] / nruns[g]: the first run of graph g and its number of runs,
// from the runs' exclusive prefix run_rank[P + 1] and the graph ranges
// gptr[G + 1] of the (not yet merged) TP list.
cudaError_t tp_run_bases(const long long *gptr, const long long *run_rank, int G, long long *run_base,
                         long long *nruns, cudaStream_t s);
// rounds that merge up to `max_runs` runs per graph
int tp_merge_rounds(long long max_runs);

// Packed comparison keys of the TPs (vertex v as v + 1 in `bits` = 8 or 16
// bits, 64 / bits per word, most significant first; see key_cmp):
// key_len[i] = words of TP i, then (after a scan into key_off) the words.
cudaError_t tp_key_lengths(const long long *tp_off, long long P, int bits, long long *key_len, cudaStream_t s);
cudaError_t tp_write_keys(const long long *tp_off, const int *tp_vert, long long P, int bits, const long long *key_off,
                          unsigned long long *key, cudaStream_t s);
// Round r of merging inside every graph: the graph's runs (its run q starts
// at bounds[run_base[g] + q]; bounds[R] = P) are merged in groups, runs
// [m 2^(r+1), m 2^(r+1) + 2^r) with the next 2^r, comparing packed keys;
// after ceil(log2(runs)) rounds each graph is one sorted run.  Runs of
// different graphs are never compared (the list is grouped by graph
// already), so no graph ids are read.
cudaError_t tp_merge_graph_round_keys(const long long *perm_in, long long *perm_out, const long long *bounds,
                                      const long long *run_base, const long long *nruns, const long long *gptr,
                                      int G, int r, long long P, const long long *key_off,
                                      const unsigned long long *key, cudaStream_t s);
// duplicate flags and kept lengths of the sorted TPs, on packed keys
cudaError_t tp_dedup_flags_keys(const long long *perm, long long P, const long long *tp_off, const long long *key_off,
                                const unsigned long long *key, const int *tp_graph, long long *keep_len, int *keep,
                                cudaStream_t s);

// packed keys (as tp_write_keys) of TP(p) for every PP p, read from the
// TP's parts (prefix path, PP, suffix path) instead of a written TP list;
// tp_off holds the TPs' offsets (for their lengths)
cudaError_t tp_write_keys_parts(const long long *pp_off, const int *pp_vert, const int *pp_graph, long long P,
                                const GraphDev &g, const long long *tp_off, int bits, const long long *key_off,
                                unsigned long long *key, cudaStream_t s);
// as tp_gather, but every kept TP is assembled from its parts
cudaError_t tp_assemble(const long long *perm, const int *keep, const long long *keep_rank, long long P,
                        const long long *pp_off, const int *pp_vert, const int *pp_graph, const GraphDev &g,
                        const long long *tp_off, const long long *keep_off, long long *final_off, int *out_vert,
                        int *out_graph, cudaStream_t s);
// map[perm[i]] = the final index of sorted TP i (keep_rank[i] if it is kept,
// else that of the kept TP it duplicates, keep_rank[i] - 1); with perm null
// the identity map[i] = i
cudaError_t tp_index_map(const long long *perm, const int *keep, const long long *keep_rank, long long P, int *map,
                         cudaStream_t s);

}  // namespace tpg
