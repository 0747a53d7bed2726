// The compositional route (Sec. 2.1, Defs. 3-11): path extraction per SCC
// and the merge of the extracted paths along the component graph.
//
// A PP that leaves an SCC never comes back (the component graph is a DAG),
// so a PP crossing SCCs is an exit path of its first SCC (Def. 7: an acyclic
// path to an SccExitVertex whose first vertex has every predecessor on it),
// then entry-exit paths of the SCCs it passes (Def. 6: acyclic, from an
// SccEntryVertex to an SccExitVertex), then an entry path of its last SCC
// (Def. 8: from an SccEntryVertex, with every successor of its last vertex
// on it), consecutive parts joined by arcs between SCCs.  The PPs inside one
// SCC are the SccInternalPPs (Def. 9, scc.cu).
//
// GPU design.  Extraction: the acyclic simple paths inside each SCC of at
// most D vertices are enumerated first, one thread per first vertex; each
// becomes a task, and one thread per task walks the paths that extend a
// D-vertex prefix depth-first, holding the path's vertex set as a bitset of
// at most 8 words, and tests the three kinds with the vertex bitsets of the
// graph (a large SCC is so spread over many threads); tasks stay grouped by
// first vertex, so each kind's list is grouped by first vertex; count
// passes size the lists.  Merge: a level-synchronous frontier over
// partial concatenations (records {segment, parent record}), level 0 the
// exit paths; a record ending at x is joined, over every arc x -> y to
// another SCC, to the entry paths starting at y (a completed PP) and to the
// entry-exit paths starting at y (a record of the next level); count pass,
// scan, write pass per level.  The completed PPs are then materialised by
// walking their records' parents.
#include "common.cuh"
#include "compositional.h"
#include "kernels.h"

namespace tpg {

namespace {

constexpr int CW = 8;         // bitset words (graphs of at most 256 vertices)
constexpr int CMAX_N = 256;   // longest path inside an SCC, and longest chain of records

unsigned grid_for(long long n, int block = 128) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

// Prefix tasks: every acyclic simple path inside an SCC of at most D
// vertices, walked depth-first from each first vertex (count pass:
// task_cnt[r]; write pass: the paths at task_pos[r], D ints each, and their
// lengths).  Each is one extraction task (below).
template <bool WRITE>
__global__ void prefix_kernel(GraphDev g, const int *comp, int D, long long *task_cnt, const long long *task_pos,
                              int *task_vert, int *task_len) {
    const int n = g.N;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int path[CMAX_N], eidx[CMAX_N];
    unsigned vis[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) vis[j] = 0u;
    const int cr = comp[r];
    long long c = 0;
    auto emit = [&](int d) {
        if (WRITE) {
            const long long t = task_pos[r] + c;
            for (int i = 0; i <= d; ++i) task_vert[t * D + i] = path[i];
            task_len[t] = d + 1;
        }
        ++c;
    };
    int d = 0;
    path[0] = r;
    eidx[0] = g.rp[r];
    vis[r >> 5] |= 1u << (r & 31);
    emit(0);
    for (;;) {
        const int x = path[d];
        int w = -1;
        while (d + 1 < D && eidx[d] < g.rp[x + 1]) {
            const int y = g.col[eidx[d]++];
            if (comp[y] == cr && !((vis[y >> 5] >> (y & 31)) & 1u)) {
                w = y;
                break;
            }
        }
        if (w >= 0) {
            ++d;
            path[d] = w;
            eidx[d] = g.rp[w];
            vis[w >> 5] |= 1u << (w & 31);
            emit(d);
            continue;
        }
        if (d == 0) break;
        vis[x >> 5] &= ~(1u << (x & 31));
        --d;
    }
    if (!WRITE) task_cnt[r] = c;
}

// One extraction task: its prefix path, and, when the prefix has D
// vertices, every acyclic simple path inside the SCC that extends it,
// depth-first; each path is sorted into entry-exit, exit and entry paths
// (count pass: counts[kind][t] paths and counts[3 + kind][t] vertices;
// write pass at the scanned per-task offsets pos[kind] / vpos[kind]).
template <bool WRITE>
__global__ void segments_kernel(GraphDev g, const int *comp, const unsigned char *is_entry,
                                const unsigned char *is_exit, int D, long long T, const int *task_vert,
                                const int *task_len, long long *counts, SegTaskOut out) {
    const int n = g.N, W = g.W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < T;
         t += (long long)gridDim.x * blockDim.x) {
        int path[CMAX_N], eidx[CMAX_N];
        unsigned vis[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) vis[j] = 0u;
        const int len = task_len[t];
        for (int i = 0; i < len; ++i) {
            const int v = task_vert[t * D + i];
            path[i] = v;
            vis[v >> 5] |= 1u << (v & 31);
        }
        const int r = path[0], cr = comp[r];
        long long np[SEG_KINDS] = {0, 0, 0}, nv[SEG_KINDS] = {0, 0, 0};
        auto visit = [&](int d) {
            const int last = path[d];
            bool pred_in = true, succ_in = true;
            for (int j = 0; j < W; ++j) {
                pred_in &= (g.pmask[(long long)r * W + j] & ~vis[j]) == 0u;
                succ_in &= (g.smask[(long long)last * W + j] & ~vis[j]) == 0u;
            }
            const bool kind[SEG_KINDS] = {is_entry[r] && is_exit[last], is_exit[last] && pred_in,
                                          is_entry[r] && succ_in};
            for (int c = 0; c < SEG_KINDS; ++c) {
                if (!kind[c]) continue;
                if (WRITE) {
                    const long long p = out.pos[c][t] + np[c], v0 = out.vpos[c][t] + nv[c];
                    out.off[c][p] = v0;
                    for (int i = 0; i <= d; ++i) out.vert[c][v0 + i] = path[i];
                }
                ++np[c];
                nv[c] += d + 1;
            }
        };
        const int floor_d = len - 1;
        int d = floor_d;
        visit(d);
        if (len == D) {
            eidx[d] = g.rp[path[d]];
            for (;;) {
                const int x = path[d];
                int w = -1;
                while (eidx[d] < g.rp[x + 1]) {
                    const int y = g.col[eidx[d]++];
                    if (comp[y] == cr && !((vis[y >> 5] >> (y & 31)) & 1u)) {
                        w = y;
                        break;
                    }
                }
                if (w >= 0 && d + 1 < CMAX_N) {
                    ++d;
                    path[d] = w;
                    eidx[d] = g.rp[w];
                    vis[w >> 5] |= 1u << (w & 31);
                    visit(d);
                    continue;
                }
                if (d == floor_d) break;
                vis[x >> 5] &= ~(1u << (x & 31));
                --d;
            }
        }
        if (!WRITE) {
            for (int c = 0; c < SEG_KINDS; ++c) {
                counts[(long long)c * T + t] = np[c];
                counts[(long long)(SEG_KINDS + c) * T + t] = nv[c];
            }
        }
        (void)n;
    }
}

// per first vertex v: where its paths start in each kind's list (the scans
// over tasks, read at v's first task)
__global__ void group_ptr_kernel(int n, const long long *task_pos, SegTaskOut out, SegPtrs ptrs) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        const long long t = task_pos[v];
        for (int c = 0; c < SEG_KINDS; ++c) {
            ptrs.ptr[c][v] = out.pos[c][t];
            ptrs.vptr[c][v] = out.vpos[c][t];
        }
    }
}

template <bool WRITE>
__global__ void merge_level_kernel(GraphDev g, const int *comp, MergeLevel lv, SegList ee, SegList en,
                                   long long *out_cnt, long long *next_cnt, const long long *out_pos,
                                   const long long *next_pos, int2 *out_rec, int *next_seg, long long *next_par) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < lv.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = lv.seg[i];
        const int x = lv.seg_vert[lv.seg_off[s + 1] - 1];
        long long no = 0, nn = 0;
        const long long o0 = WRITE ? out_pos[i] : 0, n0 = WRITE ? next_pos[i] : 0;
        for (int e = g.rp[x]; e < g.rp[x + 1]; ++e) {
            const int y = g.col[e];
            if (comp[y] == comp[x]) continue;
            const long long z0 = en.ptr[y], z1 = en.ptr[y + 1], q0 = ee.ptr[y], q1 = ee.ptr[y + 1];
            if (WRITE) {
                for (long long z = z0; z < z1; ++z) out_rec[o0 + no + (z - z0)] = make_int2((int)z, (int)(lv.base + i));
                for (long long q = q0; q < q1; ++q) {
                    next_seg[n0 + nn + (q - q0)] = (int)q;
                    next_par[n0 + nn + (q - q0)] = lv.base + i;
                }
            }
            no += z1 - z0;
            nn += q1 - q0;
        }
        if (!WRITE) {
            out_cnt[i] = no;
            next_cnt[i] = nn;
        }
    }
}

template <bool WRITE>
__global__ void materialise_kernel(const int2 *out_rec, long long n, const int *rec_seg, const long long *rec_par,
                                   const int *rec_level, SegList ee, SegList ex, SegList en, long long *len,
                                   const long long *off, int *vert) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int2 o = out_rec[i];
        int chain[CMAX_N];
        int depth = 0;
        long long total = en.off[o.x + 1] - en.off[o.x];
        for (long long r = o.y; r >= 0 && depth < CMAX_N; r = rec_par[r]) {
            chain[depth++] = (int)r;
            const SegList &S = rec_level[r] == 0 ? ex : ee;
            total += S.off[rec_seg[r] + 1] - S.off[rec_seg[r]];
        }
        if (!WRITE) {
            len[i] = total;
            continue;
        }
        long long p = off[i];
        for (int t = depth - 1; t >= 0; --t) {
            const int r = chain[t];
            const SegList &S = rec_level[r] == 0 ? ex : ee;
            for (long long k = S.off[rec_seg[r]]; k < S.off[rec_seg[r] + 1]; ++k) vert[p++] = S.vert[k];
        }
        for (long long k = en.off[o.x]; k < en.off[o.x + 1]; ++k) vert[p++] = en.vert[k];
    }
}

__global__ void fill_kernel(int *v, long long n, int x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] = x;
}

__global__ void iota_par_kernel(int *seg, long long *par, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        seg[i] = (int)i;
        par[i] = -1;
    }
}

__global__ void run_starts_kernel(int *run_start, long long n, long long first_singletons) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        run_start[i] = i == 0 || i >= first_singletons;
}

__global__ void append_kernel(const long long *off, const int *vert, long long n, long long p0, long long v0,
                              long long *dst_off, int *dst_vert) {
    const long long base = off[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        dst_off[p0 + i] = v0 + off[i] - base;
        for (long long k = off[i]; k < off[i + 1]; ++k) dst_vert[v0 + k - base] = vert[k];
    }
}

}  // namespace

cudaError_t comp_prefix_tasks(const GraphDev &g, const int *comp, int D, long long *task_cnt,
                              const long long *task_pos, int *task_vert, int *task_len, bool write, cudaStream_t s) {
    if (g.N > CMAX_N || g.W > CW || D < 1 || D > CMAX_N) return cudaErrorInvalidValue;
    if (write)
        prefix_kernel<true><<<grid_for(g.N, 32), 32, 0, s>>>(g, comp, D, task_cnt, task_pos, task_vert, task_len);
    else
        prefix_kernel<false><<<grid_for(g.N, 32), 32, 0, s>>>(g, comp, D, task_cnt, task_pos, task_vert, task_len);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_segments(const GraphDev &g, const int *comp, const unsigned char *is_entry,
                          const unsigned char *is_exit, int D, long long T, const int *task_vert, const int *task_len,
                          long long *counts, const SegTaskOut &out, bool write, cudaStream_t s) {
    if (g.N > CMAX_N || g.W > CW || !g.smask || !g.pmask) return cudaErrorInvalidValue;
    if (T <= 0) return cudaSuccess;
    if (write)
        segments_kernel<true><<<grid_for(T, 64), 64, 0, s>>>(g, comp, is_entry, is_exit, D, T, task_vert, task_len,
                                                             counts, out);
    else
        segments_kernel<false><<<grid_for(T, 64), 64, 0, s>>>(g, comp, is_entry, is_exit, D, T, task_vert, task_len,
                                                              counts, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_group_ptrs(int n, const long long *task_pos, const SegTaskOut &out, const SegPtrs &ptrs,
                            cudaStream_t s) {
    group_ptr_kernel<<<grid_for(n + 1, 128), 128, 0, s>>>(n, task_pos, out, ptrs);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_merge_level(const GraphDev &g, const int *comp, const MergeLevel &lv, const SegList &ee,
                             const SegList &en, long long *out_cnt, long long *next_cnt, const long long *out_pos,
                             const long long *next_pos, int2 *out_rec, int *next_seg, long long *next_par,
                             bool write, cudaStream_t s) {
    if (lv.n <= 0) return cudaSuccess;
    if (write)
        merge_level_kernel<true><<<grid_for(lv.n, 256), 256, 0, s>>>(g, comp, lv, ee, en, out_cnt, next_cnt, out_pos,
                                                                      next_pos, out_rec, next_seg, next_par);
    else
        merge_level_kernel<false><<<grid_for(lv.n, 256), 256, 0, s>>>(g, comp, lv, ee, en, out_cnt, next_cnt,
                                                                       out_pos, next_pos, out_rec, next_seg, next_par);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_materialise(const int2 *out_rec, long long n, const int *rec_seg, const long long *rec_par,
                             const int *rec_level, const SegList &ee, const SegList &ex, const SegList &en,
                             long long *len, const long long *off, int *vert, bool write, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (write)
        materialise_kernel<true><<<grid_for(n, 128), 128, 0, s>>>(out_rec, n, rec_seg, rec_par, rec_level, ee, ex,
                                                                   en, len, off, vert);
    else
        materialise_kernel<false><<<grid_for(n, 128), 128, 0, s>>>(out_rec, n, rec_seg, rec_par, rec_level, ee, ex,
                                                                    en, len, off, vert);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_fill(int *v, long long n, int x, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n, x);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_level0(int *seg, long long *par, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    iota_par_kernel<<<grid_for(n, 256), 256, 0, s>>>(seg, par, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_run_starts(int *run_start, long long n, long long first_singletons, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    run_starts_kernel<<<grid_for(n, 256), 256, 0, s>>>(run_start, n, first_singletons);
    note_launch();
    return cudaGetLastError();
}

cudaError_t comp_append(const long long *off, const int *vert, long long n, long long p0, long long v0,
                        long long *dst_off, int *dst_vert, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    append_kernel<<<grid_for(n, 128), 128, 0, s>>>(off, vert, n, p0, v0, dst_off, dst_vert);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tpg
