// tpg_prime_paths_noalloc: prime paths of one small graph without any
// memory allocation.
//
// Some callers cannot allocate device memory at the moment they need the
// answer: code that runs under a fixed memory budget handed out up front
// (an allocation in mid-run could fail or break it), and code embedded in a
// host framework that owns every allocation itself.  For them this entry
// point runs the same kernels as tpg_load_cfg + tpg_prime_paths, but every
// temporary buffer (the predecessor lists, the path arena, the frontier, the
// per-chunk level counts, the ordering buffers) lives in one file-scope
// __device__ array of fixed size, and the results go to buffers the caller
// already owns.
//
// The array (NA_SCRATCH_BYTES, about 33 MB) is part of the library image:
// every GPU that loads the library keeps it until the process exits.  All
// calls share it and it keeps the last call's contents, so each call clears
// what has to start at zero; two calls whose work overlaps on the GPU (for
// example on two streams) race on it and must not be issued.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace tpg {
namespace {

constexpr int NA_MAXN = 128;                  // vertices (bitset of 4 words)
constexpr long long NA_MAXM = 16384;          // arcs (NA_MAXN^2)
constexpr long long NA_NODE_CAP = 1LL << 20;  // simple paths in the arena
constexpr long long NA_LVL_CAP = 1LL << 18;   // simple paths in one level
constexpr long long NA_PP_CAP = 1LL << 18;    // prime paths
constexpr int NA_W = 4;
constexpr EnumShape NA_SHAPE = {256, 1};  // tile of 256 paths
constexpr int NA_TILE = 256;
constexpr int NA_MAX_LEVELS = NA_MAXN + 4;
// per-chunk level counts for the frontier launch of up to 8 blocks of 256
// threads on each of up to 160 SMs (a GB300 has 152); a larger grid is
// refused by the launch (TPG_ECUDA)
constexpr long long NA_AGG_WORDS = enum_agg_words(8 * 160, ENUM_UPW * 8);

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NaLayout {
    size_t prp, pcol, indeg, scanbuf, scantmp, vbase, smask, pmask, levels, ctl, nodes, tfl0, tfl1, tvis0, tvis1, tcnt0, tcnt1, pprefs,
        agg, keys0, keys1, refs0, refs1, len, ltmp, total;
};

constexpr NaLayout na_layout() {
    NaLayout L{};
    size_t o = 0;
    L.prp = o;     o = align256(o + sizeof(int) * (NA_MAXN + 1));
    L.pcol = o;    o = align256(o + sizeof(int) * NA_MAXM);
    L.indeg = o;   o = align256(o + sizeof(int) * (NA_MAXN + 1));
    L.scanbuf = o; o = align256(o + sizeof(long long) * (NA_MAXN + 2));
    L.scantmp = o; o = align256(o + sizeof(long long) * 64);
    L.vbase = o;   o = align256(o + sizeof(int) * 2);
    L.smask = o;   o = align256(o + sizeof(unsigned) * NA_MAXN * NA_W);
    L.pmask = o;   o = align256(o + sizeof(unsigned) * NA_MAXN * NA_W);
    L.levels = o;  o = align256(o + sizeof(LevelRec) * NA_MAX_LEVELS);
    L.ctl = o;     o = align256(o + CTL_BYTES);
    L.nodes = o;   o = align256(o + sizeof(int2) * NA_NODE_CAP);
    L.tfl0 = o;    o = align256(o + sizeof(int2) * NA_LVL_CAP);
    L.tfl1 = o;    o = align256(o + sizeof(int2) * NA_LVL_CAP);
    L.tvis0 = o;   o = align256(o + sizeof(unsigned) * NA_W * NA_LVL_CAP);
    L.tvis1 = o;   o = align256(o + sizeof(unsigned) * NA_W * NA_LVL_CAP);
    L.tcnt0 = o;   o = align256(o + sizeof(unsigned short) * NA_LVL_CAP);
    L.tcnt1 = o;   o = align256(o + sizeof(unsigned short) * NA_LVL_CAP);
    L.pprefs = o;  o = align256(o + sizeof(int) * NA_PP_CAP);
    L.agg = o;     o = align256(o + sizeof(long long) * NA_AGG_WORDS);
    L.keys0 = o;   o = align256(o + sizeof(int) * NA_PP_CAP);
    L.keys1 = o;   o = align256(o + sizeof(int) * NA_PP_CAP);
    L.refs0 = o;   o = align256(o + sizeof(long long) * NA_PP_CAP);
    L.refs1 = o;   o = align256(o + sizeof(long long) * NA_PP_CAP);
    L.len = o;     o = align256(o + sizeof(long long) * (NA_PP_CAP + 1));
    L.ltmp = o;    o = align256(o + sizeof(long long) * ((NA_PP_CAP + 1) / 2048 + 4));
    L.total = o;
    return L;
}

constexpr NaLayout NA = na_layout();
constexpr size_t NA_SCRATCH_BYTES = NA.total;
static_assert(NA_SCRATCH_BYTES < (36u << 20), "no-allocation scratch stays under 36 MB");

// the scratch array shared by every call on a device
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
void *g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the array on the current device (looked up once per
// device; in host code the symbol itself is only a host-side stand-in).
int na_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return TPG_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TPG_ECUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return TPG_OK;
}

// CSR checks needed by the enumeration: row_ptr[0] = 0, row_ptr[n] = m,
// non-decreasing, successor ids in range and strictly ascending.
__global__ void na_validate_kernel(const int *rp, const int *col, int n, int m, int *err) {
    int bad = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != m)) bad = 1;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n && !bad; u += gridDim.x * blockDim.x) {
        const int a = rp[u], b = rp[u + 1];
        if (a < 0 || b < a || b > m) {
            bad = 1;
            break;
        }
        for (int e = a; e < b; ++e) {
            const int w = col[e];
            if (w < 0 || w >= n || (e > a && w <= col[e - 1])) {
                bad = 1;
                break;
            }
        }
    }
    if (bad) atomicOr(err, ERR_INVAL);
}

#define NA_CK(x)                           \
    do {                                   \
        if ((x) != cudaSuccess) {          \
            cudaGetLastError();            \
            return TPG_ECUDA;              \
        }                                  \
    } while (0)

}  // namespace
}  // namespace tpg

using namespace tpg;

extern "C" int tpg_prime_paths_noalloc(int32_t n, int32_t m, const int32_t *row_ptr_dev, const int32_t *col_dev,
                                       int64_t *offsets_dev, int64_t cap_paths, int32_t *vertices_dev,
                                       int64_t cap_vertices, void *stream, int64_t *num_paths,
                                       int64_t *num_vertices) {
    if (num_paths) *num_paths = 0;
    if (num_vertices) *num_vertices = 0;
    if (n < 1 || m < 0 || !row_ptr_dev || (m > 0 && !col_dev) || !offsets_dev || !vertices_dev || !num_paths ||
        !num_vertices || cap_paths < 0 || cap_vertices < 0)
        return TPG_EINVAL;
    if (n > NA_MAXN || m > NA_MAXM) return TPG_ETOOBIG;
    void *base = nullptr;
    const int rc0 = na_scratch(&base);
    if (rc0 != TPG_OK) return rc0;
    char *S = (char *)base;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = (int *)(S + NA.ctl);

    // 1. validate the CSR on the device
    int h_err = 0;
    NA_CK(cudaMemsetAsync(err, 0, CTL_BYTES, s));
    na_validate_kernel<<<1, 128, 0, s>>>(row_ptr_dev, col_dev, n, m, err);
    note_launch();
    NA_CK(cudaGetLastError());
    NA_CK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (h_err & ERR_INVAL) return TPG_EINVAL;

    // 2. graph view with predecessor lists in the scratch array
    const int h_vbase[2] = {0, n};
    NA_CK(cudaMemcpyAsync(S + NA.vbase, h_vbase, sizeof(h_vbase), cudaMemcpyHostToDevice, s));
    GraphDev d{};
    d.N = n;
    d.G = 1;
    d.maxn = n;
    d.W = bitset_words_supported(n);
    d.M = m;
    d.rp = row_ptr_dev;
    d.col = col_dev;
    d.prp = (const int *)(S + NA.prp);
    d.pcol = (const int *)(S + NA.pcol);
    d.vgraph = nullptr;
    d.vbase = (const int *)(S + NA.vbase);
    NA_CK(build_pred_csr(d, (int *)(S + NA.prp), (int *)(S + NA.pcol), (int *)(S + NA.indeg),
                         (long long *)(S + NA.scantmp), (long long *)(S + NA.scanbuf), s));
    static_assert(NA_W <= MASK_MAX_W, "the vertex bitsets cover every supported bitset width");
    d.smask = (const unsigned *)(S + NA.smask);
    d.pmask = (const unsigned *)(S + NA.pmask);
    NA_CK(build_vertex_masks(d, (unsigned *)(S + NA.smask), (unsigned *)(S + NA.pmask), nullptr, s));

    // 3. the frontier kernel over the scratch arena
    EnumArgs a{};
    a.g = d;
    a.seg = (int2 *)(S + NA.nodes);
    a.seg_cap = NA_NODE_CAP;
    a.next_nodes = nullptr;
    a.tfl[0] = (int2 *)(S + NA.tfl0);
    a.tfl[1] = (int2 *)(S + NA.tfl1);
    a.tvis[0] = (unsigned *)(S + NA.tvis0);
    a.tvis[1] = (unsigned *)(S + NA.tvis1);
    a.tcnt[0] = (unsigned short *)(S + NA.tcnt0);
    a.tcnt[1] = (unsigned short *)(S + NA.tcnt1);
    a.lvl_cap = NA_LVL_CAP;
    a.pp_seg = (int *)(S + NA.pprefs);
    a.pp_seg_cap = NA_PP_CAP;
    a.levels = (LevelRec *)(S + NA.levels);
    a.max_levels = n + 4;
    a.start_level = 1;
    a.seed_level1 = 1;
    a.split = 1;
    a.agg = (long long *)(S + NA.agg);
    a.agg_cap = NA_AGG_WORDS;
    a.err = err;
    a.stop_level = err + 1;
    a.bar = (unsigned *)(S + NA.ctl + CTL_BAR_OFFSET);
    a.spin_ns = SPIN_LIMIT_NS;
    NA_CK(cudaMemsetAsync(a.levels, 0, sizeof(LevelRec) * NA_MAX_LEVELS, s));
    NA_CK(cudaMemsetAsync(err, 0, CTL_BYTES, s));
    int num_sms = 1, dev = 0, grid = 0;
    NA_CK(cudaGetDevice(&dev));
    NA_CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    NA_CK(launch_enumerate(a, NA_SHAPE, num_sms, s, &grid));
    LevelRec lv[NA_MAX_LEVELS];
    NA_CK(cudaMemcpyAsync(lv, a.levels, sizeof(LevelRec) * NA_MAX_LEVELS, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (h_err & ERR_TIMEOUT) return TPG_ETIMEOUT;
    if (h_err & ERR_INVAL) return TPG_ECUDA;
    if (h_err & (ERR_OVERFLOW_MASK | ERR_OVF_COUNT | ERR_OVF_LEVELS)) return TPG_ETOOBIG;

    // 4. sizes; the caller's buffers must hold them
    int pp_levels[NA_MAX_LEVELS];
    int npl = 0;
    long long P = 0, V = 0;
    for (int k = 1; k < a.max_levels; ++k) {
        if (lv[k].count <= 0) break;
        if (lv[k].pp_count > 0) {
            pp_levels[npl++] = k;
            P += lv[k].pp_count;
            V += (long long)k * lv[k].pp_count;
        }
    }
    *num_paths = P;
    *num_vertices = V;
    if (P > cap_paths || V > cap_vertices) return TPG_ETOOBIG;

    // 5. canonical order and materialisation into the caller's buffers
    const LevelRec *dlev = a.levels;
    if (P == 0) {
        NA_CK(cudaMemsetAsync(offsets_dev, 0, sizeof(long long), s));
    } else if (npl == 1) {
        const int k = pp_levels[0];
        NA_CK(pp_offsets_single_level((long long *)offsets_dev, P, k, s));
        NA_CK(pp_materialize(nullptr, lv[k].pp, k, P, (const long long *)offsets_dev, dlev, a.max_levels, d, vertices_dev,
                             nullptr, s));
    } else {
        int *keys[2] = {(int *)(S + NA.keys0), (int *)(S + NA.keys1)};
        long long *refs[2] = {(long long *)(S + NA.refs0), (long long *)(S + NA.refs1)};
        int cur = 0, cur_level = 0;
        long long na = 0;
        for (int idx = npl - 1; idx >= 0; --idx) {
            const int k = pp_levels[idx];
            const int *lref = lv[k].pp;
            if (na == 0) {
                NA_CK(order_init_run(lref, k, lv[k].pp_count, keys[cur], refs[cur], s));
                na = lv[k].pp_count;
            } else {
                NA_CK(order_merge(keys[cur], refs[cur], na, lref, k, lv[k].pp_count, keys[cur ^ 1], refs[cur ^ 1],
                                  dlev, cur_level, s));
                cur ^= 1;
                na += lv[k].pp_count;
            }
            cur_level = k;
        }
        NA_CK(pp_lengths(refs[cur], P, (long long *)(S + NA.len), s));
        NA_CK(scan_i64((long long *)(S + NA.len), (long long *)offsets_dev, P, (long long *)(S + NA.ltmp), s));
        NA_CK(pp_materialize(refs[cur], nullptr, 0, P, (const long long *)offsets_dev, dlev, a.max_levels, d, vertices_dev,
                             nullptr, s));
    }
    NA_CK(cudaStreamSynchronize(s));
    return TPG_OK;
}
