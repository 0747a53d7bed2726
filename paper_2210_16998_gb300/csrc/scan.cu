// Device-wide exclusive prefix sums (reduce -> scan of tile sums -> downsweep).
// Three plain launches, no inter-block waiting.
#include "common.cuh"
#include "kernels.h"

namespace tpg {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_ITEMS = 8;
constexpr long long SCAN_TILE = (long long)SCAN_BLOCK * SCAN_ITEMS;

size_t scan_tmp_elems(long long n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 2; }

template <typename T>
__global__ void __launch_bounds__(SCAN_BLOCK) scan_reduce_kernel(const T *in, long long n, long long *tile_sums) {
    const long long base = blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const long long i = base + (long long)j * SCAN_BLOCK + threadIdx.x;
        if (i < n) s += (long long)in[i];
    }
    long long total;
    block_excl_scan_i64<SCAN_BLOCK>(s, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_BLOCK) scan_tile_sums_kernel(long long *tile_sums, long long ntiles) {
    long long carry = 0;
    for (long long base = 0; base < ntiles; base += SCAN_BLOCK) {
        const long long i = base + threadIdx.x;
        const long long v = (i < ntiles) ? tile_sums[i] : 0;
        long long total;
        const long long ex = block_excl_scan_i64<SCAN_BLOCK>(v, total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_BLOCK) scan_down_kernel(const T *in, long long *out, long long n,
                                                               const long long *tile_sums, long long ntiles) {
    const long long base = blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS];
    long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const long long i = base + j;
        v[j] = (i < n) ? (long long)in[i] : 0;
        s += v[j];
    }
    long long total;
    long long run = block_excl_scan_i64<SCAN_BLOCK>(s, total) + tile_sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const long long i = base + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = tile_sums[ntiles];
}

__global__ void scan_empty_kernel(long long *out) { out[0] = 0; }

template <typename T>
static cudaError_t scan_impl(const T *in, long long *out, long long n, long long *tmp, cudaStream_t s) {
    if (n <= 0) {
        scan_empty_kernel<<<1, 1, 0, s>>>(out);
        note_launch();
        return cudaGetLastError();
    }
    const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    scan_reduce_kernel<T><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, n, tmp);
    note_launch();
    scan_tile_sums_kernel<<<1, SCAN_BLOCK, 0, s>>>(tmp, ntiles);
    note_launch();
    scan_down_kernel<T><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, out, n, tmp, ntiles);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scan_i64(const long long *in, long long *out, long long n, long long *tmp, cudaStream_t s) {
    return scan_impl<long long>(in, out, n, tmp, s);
}

// The two halves of scan_i64: the first leaves the tile prefixes in tmp and
// the total at tmp[scan_total_index(n)]; the second writes out[0..n].
cudaError_t scan_i64_sums(const long long *in, long long n, long long *tmp, cudaStream_t s) {
    if (n <= 0) {
        scan_empty_kernel<<<1, 1, 0, s>>>(tmp);
        note_launch();
        return cudaGetLastError();
    }
    const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    scan_reduce_kernel<long long><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, n, tmp);
    scan_tile_sums_kernel<<<1, SCAN_BLOCK, 0, s>>>(tmp, ntiles);
    note_launch(2);
    return cudaGetLastError();
}
long long scan_total_index(long long n) { return n <= 0 ? 0 : (n + SCAN_TILE - 1) / SCAN_TILE; }
cudaError_t scan_i64_finish(const long long *in, long long *out, long long n, const long long *tmp, cudaStream_t s) {
    if (n <= 0) {
        scan_empty_kernel<<<1, 1, 0, s>>>(out);
        note_launch();
        return cudaGetLastError();
    }
    const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    scan_down_kernel<long long><<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(in, out, n, tmp, ntiles);
    note_launch();
    return cudaGetLastError();
}

cudaError_t scan_i32_to_i64(const int *in, long long *out, long long n, long long *tmp, cudaStream_t s) {
    return scan_impl<int>(in, out, n, tmp, s);
}

}  // namespace tpg
