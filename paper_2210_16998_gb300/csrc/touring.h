// Longest-first touring: a smaller TP set (touring.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tpg {

// Open-addressing table of a path list: key[j] = hash of (graph, sequence)
// (0 = empty slot), idx[j] = the path's index.  `mask` + 1 slots, a power of
// two at least twice the number of paths.
struct PathTable {
    unsigned long long *key;
    int *idx;
    long long mask;
};
long long tour_table_slots(long long n);
// insert paths 0 .. n-1 (offsets off[n + 1], local vertex ids); the graph of
// path i is graph_of[i] if given, else found in gptr[G + 1], else 0.  The
// table's keys must be zero.
cudaError_t tour_table_build(PathTable t, const long long *off, const int *vert, const int *graph_of,
                             const long long *gptr, int G, long long n, cudaStream_t s);
// graph id of every path of a list grouped by graph (gptr[G + 1])
cudaError_t tour_graph_ids(const long long *gptr, int G, long long n, int *ids, cudaStream_t s);

struct TourArgs {
    GraphDev g;
    const long long *pp_off;   // [P + 1] canonical PP list (local ids)
    const int *pp_vert;
    const long long *pp_gptr;  // [G + 1]
    PathTable pp_tab;          // the PP list
    const long long *tp_off;   // [T + 1] the one-per-PP TP list, canonical
    const int *tp_vert;
    const long long *tp_gptr;  // [G + 1]
    PathTable tp_tab;          // the TP list
    const int *gorder;         // [G] graphs in claim order (most PPs first)
    int *claim;                // zero: next graph to claim
    int *ord;                  // [P] scratch: each graph's PPs, longest first
    unsigned char *cov;        // [P] zero: covered PPs
    int *sel;                  // [T] zero: chosen TPs (out)
    int *err;                  // ERR_* flags
    int maxn;                  // largest graph
};
// shared memory bytes of a tour_greedy launch with `warps` warps
size_t tour_smem_bytes(int maxn, int warps);
// warps per block that fit `smem_max` bytes (1 .. 16)
int tour_warps(int maxn, size_t smem_max);
// one launch over the G graphs (persistent blocks, as many as fit num_sms SMs)
cudaError_t tour_greedy(const TourArgs &a, int G, int warps, int num_sms, cudaStream_t s);
// keep_len[i] = sel[i] ? length of path i : 0
cudaError_t tour_keep_lengths(const int *sel, const long long *off, long long n, long long *keep_len,
                              cudaStream_t s);

}  // namespace tpg
