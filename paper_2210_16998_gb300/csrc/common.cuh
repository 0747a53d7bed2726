// Shared device helpers and internal structures of libtpg.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tpg.h"

namespace tpg {

// ---------------------------------------------------------------------------
// error flags raised by kernels (bitwise OR into one int in device memory)
// ---------------------------------------------------------------------------
enum : int {
    ERR_OVF_NODES = 1,    // persistent path arena full
    ERR_OVF_LEVEL = 2,    // ping-pong frontier full
    ERR_OVF_PP = 4,       // PP reference list full
    ERR_RESERVED_8 = 8,   // (unused)
    ERR_TIMEOUT = 16,     // a bounded wait ran out
    ERR_UNREACH = 32,     // TP: vertex not reachable / cannot reach exit
    ERR_INVAL = 64,       // device-side validation failed
    ERR_OVF_LEVELS = 128, // more levels than the level table holds
    ERR_OVF_COUNT = 256,  // a level count passed 2^31 - 1
};
constexpr int ERR_OVERFLOW_MASK = ERR_OVF_NODES | ERR_OVF_LEVEL | ERR_OVF_PP;

// wall-clock limit of every device-side spin (nanoseconds)
constexpr unsigned long long SPIN_LIMIT_NS = 4ull * 1000 * 1000 * 1000;

// One frontier level of the path arena.  The arena is a chain of segments;
// a level lives inside one segment, so a level is addressed by a pointer.
// Written while the previous level is processed (nodes, count, pp) and when
// this level's totals are known (pp_count, children).  64 bytes.
struct LevelRec {
    int2 *nodes;            // the level's first node {last vertex, parent index}
    long long count;        // nodes in the level
    int *pp;                // the level's first PP reference
    long long pp_count;     // PPs found in the level
    long long children;     // nodes of the next level (exact, also on overflow)
    long long pad[3];
};

// Device view of one handle's graph(s): the union of all graphs with global
// vertex ids (graph g owns ids vbase[g] .. vbase[g+1]-1).
struct GraphDev {
    int N;            // total vertices
    int G;            // graphs
    int maxn;         // largest graph
    int W;            // 32-bit words of the per-path visited bitset
    long long M;      // total arcs
    const int *rp, *col;     // successor CSR (global ids)
    const int *prp, *pcol;   // predecessor CSR (global ids)
    const int *vgraph;       // [N] graph of each vertex
    const int *vbase;        // [G+1]
    const int *entry, *exit; // [G] global ids
    const long long *tbl_base;  // [G+1] offsets of the per-graph n_g x n_g BFS tables
    int *dist, *pred;           // BFS tables, local ids: [tbl_base[g] + a*n_g + x]
    int *pre_len, *suf_len;     // [N] vertex counts of path(entry->v), path(v->exit), 0 = none
    long long *pre_off, *suf_off;  // [N+1]
    int *pre_seq, *suf_seq;     // local ids
    // successor and predecessor sets of every vertex as W-word bitsets of
    // graph-local ids ([N][W]; built when W <= MASK_MAX_W, else null)
    const unsigned *smask, *pmask;
};
constexpr int MASK_MAX_W = 8;

// ---------------------------------------------------------------------------
// memory-model helpers (PTX ISA: ld/st .relaxed.gpu, %globaltimer)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with tree arrival: a block arrives at one of
// BAR_GROUPS group counters; the last block of a group arrives at the top
// counter; the last group flips the generation that everyone else waits on.
// bar[0] = top count, bar[1] = generation, bar[2 .. 2 + BAR_GROUPS) = group
// counts (all zero at launch; each counter is reset by its last arrival).
// Arrivals on one address are serialised by the L2, so splitting them over
// groups shortens the barrier from ~G to ~G/BAR_GROUPS + BAR_GROUPS steps.
// Every wait is bounded by `limit_ns` (default SPIN_LIMIT_NS; ERR_TIMEOUT,
// false on expiry).  Also false, on every block alike, if an error flag in
// `stop` was raised before the barrier.
constexpr int BAR_GROUPS = 32;
constexpr int BAR_WORDS = 2 + BAR_GROUPS;
__device__ __forceinline__ bool grid_barrier_tree(unsigned *bar, int *err, int stop,
                                                  unsigned long long limit_ns = SPIN_LIMIT_NS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned G = gridDim.x;
        const unsigned grp = blockIdx.x % BAR_GROUPS;
        const unsigned gsize = (G - grp + BAR_GROUPS - 1) / BAR_GROUPS;
        const unsigned ngroups = G < (unsigned)BAR_GROUPS ? G : (unsigned)BAR_GROUPS;
        const unsigned gen = ld_acquire_u32(bar + 1);
        __threadfence();
        bool released = false;
        if (atomicAdd(bar + 2 + grp, 1u) == gsize - 1) {
            atomicExch(bar + 2 + grp, 0u);
            __threadfence();
            if (atomicAdd(bar, 1u) == ngroups - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
                released = true;
            }
        }
        if (!released) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(bar + 1) == gen) {
                __nanosleep(64);
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (__ldcg(err) & stop) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide barrier on one arrival counter that only grows: each block adds
// 1 (a release reduction, no reply to wait for) and waits, polling with
// acquire loads, until the counter reaches `target` (grid size times the
// number of barriers so far in the launch; the counter is zero at launch).
// The wait is bounded by `limit_ns` (ERR_TIMEOUT, false on expiry); false on
// every block alike if an error flag in `stop` was raised before the barrier.
__device__ __forceinline__ bool grid_barrier_count(unsigned *ctr, unsigned target, int *err, int stop,
                                                   unsigned long long limit_ns = SPIN_LIMIT_NS) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // No full fences: the block's writes are ordered before the arrival
        // by __syncthreads and the release, and the acquire load that sees
        // the last arrival (then __syncthreads) orders every later read of
        // the block after the other blocks' writes.
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
        if (ld_acquire_u32(ctr) < target) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(ctr) < target) {
                __nanosleep(32);
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (__ldcg(err) & stop) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// counts of one level saturate here (int32 path indices)
constexpr unsigned long long MAX31 = (1ull << 31) - 1;

// Block-wide exclusive scan of two 32-bit counters packed as (a << 32 | b);
// the per-block sums must stay below 2^32.  Returns the exclusive prefix and
// writes the block total to `total`.  BLOCK threads, BLOCK % 32 == 0.
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v,
                                                                   unsigned long long &total) {
    constexpr int NW = BLOCK / 32;
    __shared__ unsigned long long s_warp[NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = (lane < NW) ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    unsigned long long warp_prefix = wid ? s_warp[wid - 1] : 0ull;
    total = s_warp[NW - 1];
    unsigned long long r = warp_prefix + x - v;
    __syncthreads();
    return r;
}

// Block-wide exclusive scan of int64 values.
template <int BLOCK>
__device__ __forceinline__ long long block_excl_scan_i64(long long v, long long &total) {
    constexpr int NW = BLOCK / 32;
    __shared__ long long s_w[NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < NW) ? s_w[lane] : 0ll;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_w[lane] = w;
    }
    __syncthreads();
    long long wp = wid ? s_w[wid - 1] : 0ll;
    total = s_w[NW - 1];
    long long r = wp + x - v;
    __syncthreads();
    return r;
}

}  // namespace tpg
