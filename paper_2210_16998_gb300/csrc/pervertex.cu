// Baseline in the paper's own design (Sec. 4 and 5, Alg. 1-4): one thread
// per vertex, each vertex keeping the list of simple paths that end at it as
// whole vertex sequences, with the paper's per-path flags (extended, read by
// the left / right successor, cyclic).
//
// What differs, only where a GPU requires it: the paper's kernel is
// self-stabilising -- every vertex thread loops, reads its predecessors'
// lists as they grow and waits on the other threads' flags until the
// vertices before it are done.  Threads of different blocks that wait on one
// another have no guarantee of running at the same time, so the same reads
// and copies run here as one pair of launches per path length: at step k
// every vertex thread reads the paths of k-1 vertices in its predecessors'
// lists, labels each one read, and extends each eligible one (not cyclic,
// and the vertex not on it unless as its first vertex) by itself, copying
// the whole path (ExtendPath); a count pass sizes the step's lists first.
// Then every vertex thread prunes its own list (Alg. 3's first loop): a path
// that was extended, or that is a proper suffix of a path one vertex longer
// in the same list (a simple u.p exists: "included in"), is not a PP; every
// cycle is one.  Out-degree at most 2 (the two successor flags).
#include "common.cuh"
#include "kernels.h"
#include "pervertex.h"

namespace tpg {

namespace {

unsigned grid_for(long long n, int block = 128) {
    long long b = (n + block - 1) / block;
    return (unsigned)(b < 1 ? 1 : b);
}

// step k: count (write = false) or write (write = true) the paths of k
// vertices ending at each vertex, from the paths of k-1 vertices of its
// predecessors (prev: k-1 vertices each, grouped by end vertex)
template <bool WRITE>
__global__ void extend_kernel(int k, int n, const int *rp, const int *col, const int *prp, const int *pcol,
                              PvLevel prev, PvLevel cur, long long *cnt) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    long long c = 0;
    const long long base = WRITE ? cur.ptr[v] : 0;
    for (int e = prp[v]; e < prp[v + 1]; ++e) {
        const int u = pcol[e];
        const bool left = col[rp[u]] == v;  // u's first successor
        for (long long q = prev.ptr[u]; q < prev.ptr[u + 1]; ++q) {
            if (prev.cyc[q]) continue;  // a cycle is a PP where it ends and is not read on
            const int *qv = prev.verts + q * (k - 1);
            if (!WRITE) {
                if (left) prev.read_left[q] = 1;
                else prev.read_right[q] = 1;
            }
            bool on = false;
            for (int j = 0; j < k - 1; ++j) on |= qv[j] == v;
            if (on && qv[0] != v) continue;
            if (WRITE) {
                int *dst = cur.verts + (base + c) * k;
                for (int j = 0; j < k - 1; ++j) dst[j] = qv[j];
                dst[k - 1] = v;
                cur.cyc[base + c] = qv[0] == v;
                cur.ext[base + c] = 0;
                cur.read_left[base + c] = cur.read_right[base + c] = 0;
            } else {
                prev.ext[q] = 1;
            }
            ++c;
        }
    }
    if (!WRITE) cnt[v] = c;
}

// per vertex: its PPs (count pass) or their offsets and vertices (write pass)
template <bool WRITE>
__global__ void prune_kernel(int n, int levels, const PvLevel *lv, long long *pp_cnt, long long *vert_cnt,
                             const long long *pp_base, const long long *vert_base, long long *off, int *out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    long long np = 0, nv = 0;
    for (int k = 1; k <= levels; ++k) {
        const PvLevel L = lv[k];
        for (long long p = L.ptr[v]; p < L.ptr[v + 1]; ++p) {
            if (L.ext[p]) continue;
            const int *pv = L.verts + p * k;
            bool pp = true;
            if (!L.cyc[p] && k < levels) {
                // a proper suffix of a path of k + 1 vertices ending at v?
                const PvLevel M = lv[k + 1];
                for (long long r = M.ptr[v]; r < M.ptr[v + 1] && pp; ++r) {
                    const int *rv = M.verts + r * (k + 1) + 1;
                    int j = 0;
                    while (j < k && rv[j] == pv[j]) ++j;
                    if (j == k) pp = false;
                }
            }
            if (!pp) continue;
            if (WRITE) {
                off[pp_base[v] + np] = vert_base[v] + nv;
                for (int j = 0; j < k; ++j) out[vert_base[v] + nv + j] = pv[j];
            }
            ++np;
            nv += k;
        }
    }
    if (!WRITE) {
        pp_cnt[v] = np;
        vert_cnt[v] = nv;
    }
}

__global__ void iota_i32_kernel(int *v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

}  // namespace

cudaError_t pv_iota(int *v, int n, cudaStream_t s) {
    iota_i32_kernel<<<grid_for(n), 128, 0, s>>>(v, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t pv_extend(int k, int n, const int *rp, const int *col, const int *prp, const int *pcol,
                      const PvLevel &prev, const PvLevel &cur, long long *cnt, bool write, cudaStream_t s) {
    if (write) extend_kernel<true><<<grid_for(n), 128, 0, s>>>(k, n, rp, col, prp, pcol, prev, cur, cnt);
    else extend_kernel<false><<<grid_for(n), 128, 0, s>>>(k, n, rp, col, prp, pcol, prev, cur, cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t pv_prune(int n, int levels, const PvLevel *lv, long long *pp_cnt, long long *vert_cnt,
                     const long long *pp_base, const long long *vert_base, long long *off, int *out, bool write,
                     cudaStream_t s) {
    if (write)
        prune_kernel<true><<<grid_for(n), 128, 0, s>>>(n, levels, lv, pp_cnt, vert_cnt, pp_base, vert_base, off, out);
    else
        prune_kernel<false><<<grid_for(n), 128, 0, s>>>(n, levels, lv, pp_cnt, vert_cnt, pp_base, vert_base, off,
                                                        out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
