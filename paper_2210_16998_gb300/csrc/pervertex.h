// Baseline in the paper's per-vertex-list design (pervertex.cu).
#pragma once
#include <cuda_runtime.h>

namespace tpg {

// The paths of k vertices, grouped by end vertex: those ending at v are
// ptr[v] .. ptr[v+1]-1, path i's vertices at verts[i * k .. i * k + k), with
// the paper's flags per path (one byte each, so two successor threads never
// write the same byte with different values).
struct PvLevel {
    const long long *ptr;  // [n + 1]
    int *verts;
    unsigned char *ext;         // extended by a successor (not a PP)
    unsigned char *read_left;   // read by the vertex's first successor
    unsigned char *read_right;  // read by its second successor
    unsigned char *cyc;         // a cycle (first vertex = last)
};

// step k (k >= 2) of the lists: count pass (write = false: cnt[v] = paths
// of k vertices that v appends; labels prev's paths read and extended) or
// write pass (cur.ptr from a scan of cnt)
cudaError_t pv_extend(int k, int n, const int *rp, const int *col, const int *prp, const int *pcol,
                      const PvLevel &prev, const PvLevel &cur, long long *cnt, bool write, cudaStream_t s);
// pruning of every vertex's list (lv: device array of levels 0 .. levels,
// level k holding paths of k vertices): count pass (pp_cnt, vert_cnt per
// vertex) or write pass (offsets and vertices at pp_base / vert_base)
cudaError_t pv_prune(int n, int levels, const PvLevel *lv, long long *pp_cnt, long long *vert_cnt,
                     const long long *pp_base, const long long *vert_base, long long *off, int *out, bool write,
                     cudaStream_t s);

// v[i] = i
cudaError_t pv_iota(int *v, int n, cudaStream_t s);

}  // namespace tpg
