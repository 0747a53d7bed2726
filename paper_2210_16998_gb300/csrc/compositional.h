// The compositional route's path extraction and merging (compositional.cu).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace tpg {

// the three kinds of SCC paths the merge joins (Defs. 6-8)
enum { SEG_EE = 0, SEG_EX = 1, SEG_EN = 2, SEG_KINDS = 3 };

// One kind's list: paths grouped by first vertex (those starting at v are
// ptr[v] .. ptr[v+1]-1, in canonical order), offsets and vertices.
struct SegList {
    const long long *ptr;  // [n + 1]
    long long *off;        // [count + 1]
    int *vert;
    const long long *vptr;  // [n + 1] vertex offset of the paths starting at v
};

// Per-task outputs of the extraction: per kind, the scanned path and vertex
// offsets of every task (pos[c][T] and vpos[c][T] are the totals) and the
// kind's offsets / vertices arrays.
struct SegTaskOut {
    const long long *pos[SEG_KINDS];
    const long long *vpos[SEG_KINDS];
    long long *off[SEG_KINDS];
    int *vert[SEG_KINDS];
};
struct SegPtrs {
    long long *ptr[SEG_KINDS];
    long long *vptr[SEG_KINDS];
};

// prefix tasks: every acyclic simple path inside one SCC of at most D
// vertices, per first vertex (count pass: task_cnt[n]; write pass: D ints
// per task at task_pos, and the task's length)
cudaError_t comp_prefix_tasks(const GraphDev &g, const int *comp, int D, long long *task_cnt,
                              const long long *task_pos, int *task_vert, int *task_len, bool write, cudaStream_t s);
// extraction: each task's prefix and, for D-vertex prefixes, every acyclic
// simple path inside the SCC that extends it, sorted into entry-exit, exit
// and entry paths; count pass (counts: [2 * SEG_KINDS][T]) or write pass
cudaError_t comp_segments(const GraphDev &g, const int *comp, const unsigned char *is_entry,
                          const unsigned char *is_exit, int D, long long T, const int *task_vert, const int *task_len,
                          long long *counts, const SegTaskOut &out, bool write, cudaStream_t s);
// each kind's per-first-vertex pointers (n + 1) from the per-task scans
cudaError_t comp_group_ptrs(int n, const long long *task_pos, const SegTaskOut &out, const SegPtrs &ptrs,
                            cudaStream_t s);

// One level of the merge: a record is a partial concatenation ending in
// segment seg (an exit path at level 0, an entry-exit path later) with its
// parent record (global index, -1 at level 0).  Count pass: per record, the
// completed PPs (an entry path joined by a crossing arc) and the next
// level's records (an entry-exit path joined by a crossing arc).  Write pass
// at the scanned offsets.
struct MergeLevel {
    const int *seg;          // [n] segment of each record
    long long n;             // records
    long long base;          // global index of the level's first record
    const long long *seg_off;  // offsets of the list the records' segments come from
    const int *seg_vert;
};
cudaError_t comp_merge_level(const GraphDev &g, const int *comp, const MergeLevel &lv, const SegList &ee,
                             const SegList &en, long long *out_cnt, long long *next_cnt, const long long *out_pos,
                             const long long *next_pos, int2 *out_rec, int *next_seg, long long *next_par,
                             bool write, cudaStream_t s);

// Materialise the completed PPs: out_rec[i] = {entry path, last record}.
// Count pass: lengths (len[i]); write pass: vertices at off[i].  rec_seg /
// rec_par / rec_level hold every record of every level (global index);
// level 0 segments index the exit paths, later ones the entry-exit paths.
cudaError_t comp_materialise(const int2 *out_rec, long long n, const int *rec_seg, const long long *rec_par,
                             const int *rec_level, const SegList &ee, const SegList &ex, const SegList &en,
                             long long *len, const long long *off, int *vert, bool write, cudaStream_t s);

// v[i] = x
cudaError_t comp_fill(int *v, long long n, int x, cudaStream_t s);
// level 0 of the merge: seg[i] = i (the exit paths), par[i] = -1
cudaError_t comp_level0(int *seg, long long *par, long long n, cudaStream_t s);
// run_start[i] = 1 at 0 and from first_singletons on (a sorted run, then
// one run per path)
cudaError_t comp_run_starts(int *run_start, long long n, long long first_singletons, cudaStream_t s);
// copy a path list into a bigger one at path index p0 and vertex index v0
cudaError_t comp_append(const long long *off, const int *vert, long long n, long long p0, long long v0,
                        long long *dst_off, int *dst_vert, cudaStream_t s);

}  // namespace tpg
