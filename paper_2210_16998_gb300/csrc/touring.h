// Longest-first touring: a smaller TP set (touring.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tpg {

// Open-addressing tables of a PP list, one per graph so that the lookups of
// PPs of one graph (which run together) stay in L2: graph g owns slots
// tbase[g] .. tbase[g+1]-1, a power of two at least twice its PPs (16 at
// least); key[j] = hash of (graph, sequence), 0 = empty; idx[j] = the PP.
struct PathTable {
    unsigned long long *key;
    int *idx;
    const long long *tbase;  // [G + 1]
};
// tbase (host, G + 1 entries) from the PP graph pointer gptr; returns the slots
long long tour_table_layout(const long long *gptr, int G, long long *tbase);
// longest window a TP can have (3 maxn - 1 vertices) and the hash powers it needs
int tour_max_tp(int maxn);
// pw[k] = B^k for k = 0 .. n of the sequence hash's base B
cudaError_t tour_powers(unsigned long long *pw, int n, cudaStream_t s);
// insert PPs 0 .. P-1 (offsets off[P + 1], local vertex ids; graph of PP i
// = graph_of[i], or 0 if null).  The table's keys must be zero.
cudaError_t tour_table_build(PathTable t, const long long *off, const int *vert, const int *graph_of, long long P,
                             cudaStream_t s);

struct TourEdgeArgs {
    GraphDev g;
    const long long *pp_off;   // [P + 1] canonical PP list (local ids)
    const int *pp_vert;
    const int *pp_graph;       // [P] graph of each PP, or null for one graph
    const long long *pp_gptr;  // [G + 1]
    long long P;
    PathTable tab;             // the PP list
    const unsigned long long *pw;  // [tour_max_tp(maxn) + 1]
    int2 *edges;               // out: {p, q}: TP(p) covers q, q after p in the order
    long long edge_cap;
    unsigned long long *edge_count;  // zero at launch; counts every edge, also past edge_cap
    int *err;                  // ERR_* flags
    int maxn;
};
// one launch, every PP of every graph (persistent warps, as many as fit
// num_sms SMs); *warps_out receives the warps per block
cudaError_t tour_edges(const TourEdgeArgs &a, int num_sms, int *warps_out, cudaStream_t s);
// in_off[P + 1] (exclusive scan of in-degrees, from a caller scan of indeg)
// and in_src: the edges grouped by target.  indeg must be zero before
// tour_indegrees; tour_group_edges counts it back down to zero.
cudaError_t tour_indegrees(const int2 *edges, long long E, int *indeg, cudaStream_t s);
cudaError_t tour_group_edges(const int2 *edges, long long E, const long long *in_off, int *indeg, int *in_src,
                             cudaStream_t s);
// one sweep of the decisions (state: 0 undecided, 1 chosen, 2 covered by a
// chosen earlier PP); *undecided (zeroed by the caller) receives what is left
cudaError_t tour_sweep(const long long *in_off, const int *in_src, long long P, unsigned char *state,
                       unsigned long long *undecided, cudaStream_t s);
// sel[map[q]] = 1 for every chosen q
cudaError_t tour_select(const unsigned char *state, const int *map, long long P, int *sel, cudaStream_t s);
// graph id of every path of a list grouped by graph (gptr[G + 1])
cudaError_t tour_graph_ids(const long long *gptr, int G, long long n, int *ids, cudaStream_t s);
// keep_len[i] = sel[i] ? length of path i : 0
cudaError_t tour_keep_lengths(const int *sel, const long long *off, long long n, long long *keep_len,
                              cudaStream_t s);

}  // namespace tpg
