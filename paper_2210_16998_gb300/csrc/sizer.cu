// Learned sizer: a small message-passing network that predicts, for every
// vertex r, log1p of the enumeration volume rooted at r (simple paths, prime
// paths, prime-path vertices).  Its predictions pre-size the path arena and
// the output buffers of a graph-mode capture, so a new batch can be captured
// and replayed without an exact sizing run; a capture that proves too small
// falls back to the exact path, so results never depend on the network.
//
// Network (hidden H = 64, three message-passing layers):
//   h0 = ReLU(W0 x + b0)                                  x: 8 features
//   h_l = ReLU(W_l [h_{l-1}; sum_{u->v} h_{l-1}[u]; sum_{v->w} h_{l-1}[w]] + b_l)
//   y = Wo h3 + bo                                        3 targets
// Loss: mean squared error against log1p of the exact per-root counts.
// Storage: FP32 master weights (Adam), BF16 working copies and BF16
// activations; every product accumulates in FP32.  The dense layers run as
// BF16 tensor-core MMAs (mma.sync m16n8k16, FP32 accumulators); the
// aggregation, head, weight gradients and optimiser are plain CUDA-core
// kernels.
#include <atomic>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace tpg {
namespace {

constexpr int SZ_H = 64;       // hidden width
constexpr int SZ_F = 8;        // input features
constexpr int SZ_T = 3;        // targets
constexpr int SZ_L = 3;        // message-passing layers
constexpr int SZ_K = 3 * SZ_H; // 192: [self; in-sum; out-sum]

// parameter layout (FP32 master copy)
constexpr int OFF_W0 = 0;
constexpr int OFF_B0 = OFF_W0 + SZ_H * SZ_F;
constexpr int OFF_WL = OFF_B0 + SZ_H;                      // layer l: W at OFF_WL + l*(H*K + H)
constexpr int LAYER_SZ = SZ_H * SZ_K + SZ_H;
constexpr int OFF_WO = OFF_WL + SZ_L * LAYER_SZ;
constexpr int OFF_BO = OFF_WO + SZ_T * SZ_H;
constexpr int NPARAM = OFF_BO + SZ_T;
__host__ __device__ constexpr int off_w(int l) { return OFF_WL + l * LAYER_SZ; }
__host__ __device__ constexpr int off_b(int l) { return OFF_WL + l * LAYER_SZ + SZ_H * SZ_K; }

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// features (from the loaded handle: degrees, entry/exit, SCC size from the
// BFS tables, BFS depth from entry and to exit, graph size)
// ---------------------------------------------------------------------------
__global__ void sz_features_kernel(GraphDev g, float *X) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += gridDim.x * blockDim.x) {
        const int gid = g.vgraph ? g.vgraph[v] : 0;
        const int vb = g.vgraph ? g.vbase[gid] : 0;
        const int ng = g.vgraph ? g.vbase[gid + 1] - vb : g.N;
        const int vl = v - vb, en = g.entry[gid] - vb, ex = g.exit[gid] - vb;
        const int *D = g.dist + g.tbl_base[gid];
        int scc = 0;
        for (int u = 0; u < ng; ++u) scc += (D[(long long)vl * ng + u] >= 0 && D[(long long)u * ng + vl] >= 0);
        const int d1 = D[(long long)en * ng + vl], d2 = D[(long long)vl * ng + ex];
        float *x = X + (long long)v * SZ_F;
        x[0] = log1pf((float)(g.prp[v + 1] - g.prp[v]));
        x[1] = log1pf((float)(g.rp[v + 1] - g.rp[v]));
        x[2] = vl == en ? 1.f : 0.f;
        x[3] = vl == ex ? 1.f : 0.f;
        x[4] = log1pf((float)scc);
        x[5] = d1 >= 0 ? (float)d1 / (float)ng : 2.f;
        x[6] = d2 >= 0 ? (float)d2 / (float)ng : 2.f;
        x[7] = logf((float)ng) / 5.f;
    }
}

// labels: log1p of the exact per-root counts
__global__ void sz_labels_kernel(const unsigned long long *counts, long long N, float *T) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N * SZ_T;
         i += (long long)gridDim.x * blockDim.x)
        T[i] = log1pf((float)counts[i]);
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
__global__ void sz_input_fwd(const float *X, long long N, const float *P, bf16 *H0) {
    __shared__ float w[SZ_H * SZ_F + SZ_H];
    for (int i = threadIdx.x; i < SZ_H * SZ_F + SZ_H; i += blockDim.x) w[i] = P[OFF_W0 + i];
    __syncthreads();
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
        float x[SZ_F];
#pragma unroll
        for (int k = 0; k < SZ_F; ++k) x[k] = X[v * SZ_F + k];
        for (int o = 0; o < SZ_H; ++o) {
            float z = w[SZ_H * SZ_F + o];
#pragma unroll
            for (int k = 0; k < SZ_F; ++k) z = fmaf(w[o * SZ_F + k], x[k], z);
            H0[v * SZ_H + o] = __float2bfloat16(z > 0.f ? z : 0.f);
        }
    }
}

// Xcat[v] = [h[v]; sum over predecessors; sum over successors], one warp per
// vertex, two channels per lane, FP32 sums rounded once to BF16.
__global__ void sz_aggregate(const bf16 *H, long long N, const int *rp, const int *col, const int *prp,
                             const int *pcol, bf16 *Xcat) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long v = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); v < N; v += nw) {
        const __nv_bfloat162 *H2 = (const __nv_bfloat162 *)H;
        const __nv_bfloat162 self = H2[v * (SZ_H / 2) + lane];
        float in0 = 0.f, in1 = 0.f, out0 = 0.f, out1 = 0.f;
        for (int e = prp[v]; e < prp[v + 1]; ++e) {
            const float2 f = __bfloat1622float2(H2[(long long)pcol[e] * (SZ_H / 2) + lane]);
            in0 += f.x;
            in1 += f.y;
        }
        for (int e = rp[v]; e < rp[v + 1]; ++e) {
            const float2 f = __bfloat1622float2(H2[(long long)col[e] * (SZ_H / 2) + lane]);
            out0 += f.x;
            out1 += f.y;
        }
        __nv_bfloat162 *X2 = (__nv_bfloat162 *)(Xcat + v * SZ_K);
        X2[lane] = self;
        X2[SZ_H / 2 + lane] = __floats2bfloat162_rn(in0, in1);
        X2[SZ_H + lane] = __floats2bfloat162_rn(out0, out1);
    }
}

__device__ __forceinline__ unsigned pack_bf16(bf16 lo, bf16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// C[M x NC] = A[M x K] * B, with B given transposed as Bt[NC x K] (both BF16
// row-major), FP32 accumulation on the tensor cores (mma.sync m16n8k16
// row.col).  Block: 4 warps, a 64 x 64 output tile; warp w owns rows
// 16w..16w+15 and eight 8-column MMA tiles.  EPI 0: out_bf16 = ReLU(C + bias)
// (forward layer); EPI 1: out_f32 = C (input gradient).
template <int K, int EPI>
__global__ void __launch_bounds__(128) sz_mma_gemm(const bf16 *A, long long M, const bf16 *Bt, int NC,
                                                   const float *bias, bf16 *out_bf16, float *out_f32) {
    constexpr int LD = K + 8;  // padded row (bank spread)
    extern __shared__ __align__(16) unsigned char sz_smem[];
    bf16 *As = (bf16 *)sz_smem;
    bf16 *Bs = As + 64 * LD;
    const long long row0 = blockIdx.x * 64ll;
    const int col0 = blockIdx.y * 64;
    const int tid = threadIdx.x;
    for (int i = tid; i < 64 * K / 8; i += 128) {
        const int r = i / (K / 8), c = (i % (K / 8)) * 8;
        uint4 va = make_uint4(0, 0, 0, 0);
        if (row0 + r < M) va = *(const uint4 *)(A + (row0 + r) * K + c);
        *(uint4 *)(As + r * LD + c) = va;
        uint4 vb = make_uint4(0, 0, 0, 0);
        if (col0 + r < NC) vb = *(const uint4 *)(Bt + (long long)(col0 + r) * K + c);
        *(uint4 *)(Bs + r * LD + c) = vb;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    float acc[8][4];
#pragma unroll
    for (int t = 0; t < 8; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
    const int r0 = warp * 16 + gid;
#pragma unroll
    for (int kk = 0; kk < K; kk += 16) {
        const int c0 = kk + tig * 2;
        const unsigned a0 = pack_bf16(As[r0 * LD + c0], As[r0 * LD + c0 + 1]);
        const unsigned a1 = pack_bf16(As[(r0 + 8) * LD + c0], As[(r0 + 8) * LD + c0 + 1]);
        const unsigned a2 = pack_bf16(As[r0 * LD + c0 + 8], As[r0 * LD + c0 + 9]);
        const unsigned a3 = pack_bf16(As[(r0 + 8) * LD + c0 + 8], As[(r0 + 8) * LD + c0 + 9]);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int n = t * 8 + gid;
            const unsigned b0 = pack_bf16(Bs[n * LD + c0], Bs[n * LD + c0 + 1]);
            const unsigned b1 = pack_bf16(Bs[n * LD + c0 + 8], Bs[n * LD + c0 + 9]);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long r = row0 + r0 + half * 8;
            const int c = col0 + t * 8 + tig * 2;
            if (r >= M || c >= NC) continue;
            const float v0 = acc[t][half * 2], v1 = acc[t][half * 2 + 1];
            if (EPI == 0) {
                const float z0 = v0 + bias[c], z1 = v1 + bias[c + 1];
                *(__nv_bfloat162 *)(out_bf16 + r * NC + c) =
                    __floats2bfloat162_rn(z0 > 0.f ? z0 : 0.f, z1 > 0.f ? z1 : 0.f);
            } else {
                *(float2 *)(out_f32 + r * NC + c) = make_float2(v0, v1);
            }
        }
    }
}

__global__ void sz_head_fwd(const bf16 *H3, long long N, const float *P, float *Y) {
    __shared__ float w[SZ_T * SZ_H + SZ_T];
    for (int i = threadIdx.x; i < SZ_T * SZ_H + SZ_T; i += blockDim.x) w[i] = P[OFF_WO + i];
    __syncthreads();
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
        float y[SZ_T] = {w[SZ_T * SZ_H], w[SZ_T * SZ_H + 1], w[SZ_T * SZ_H + 2]};
        for (int o = 0; o < SZ_H; ++o) {
            const float h = __bfloat162float(H3[v * SZ_H + o]);
#pragma unroll
            for (int t = 0; t < SZ_T; ++t) y[t] = fmaf(w[t * SZ_H + o], h, y[t]);
        }
#pragma unroll
        for (int t = 0; t < SZ_T; ++t) Y[v * SZ_T + t] = y[t];
    }
}

// ---------------------------------------------------------------------------
// loss and backward
// ---------------------------------------------------------------------------
// dY = 2 (Y - T) / (3N); dZ3 = (dY Wo) * [H3 > 0]; loss = mean (Y - T)^2
__global__ void __launch_bounds__(256) sz_head_bwd(const float *Y, const float *T, const bf16 *H3, long long N,
                                                   const float *P, float *dY, double *loss, float *dZ,
                                                   bf16 *dZb) {
    __shared__ float w[SZ_T * SZ_H];
    __shared__ double sloss;
    for (int i = threadIdx.x; i < SZ_T * SZ_H; i += blockDim.x) w[i] = P[OFF_WO + i];
    if (threadIdx.x == 0) sloss = 0.0;
    __syncthreads();
    const float scale = 2.f / (float)(SZ_T * N);
    double my_loss = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
        float dy[SZ_T];
#pragma unroll
        for (int t = 0; t < SZ_T; ++t) {
            const float d = Y[v * SZ_T + t] - T[v * SZ_T + t];
            my_loss += (double)d * d;
            dy[t] = scale * d;
            dY[v * SZ_T + t] = dy[t];
        }
        for (int o = 0; o < SZ_H; ++o) {
            const float h = __bfloat162float(H3[v * SZ_H + o]);
            float dh = 0.f;
#pragma unroll
            for (int t = 0; t < SZ_T; ++t) dh = fmaf(dy[t], w[t * SZ_H + o], dh);
            const float dz = h > 0.f ? dh : 0.f;
            dZ[v * SZ_H + o] = dz;
            dZb[v * SZ_H + o] = __float2bfloat16(dz);
        }
    }
    atomicAdd(&sloss, my_loss);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(loss, sloss / (double)(SZ_T * N));
}

// dWo[t][o] = sum_v dY[v][t] H3[v][o], dbo[t] = sum_v dY[v][t]: thread
// (t, o) of a 256-thread block (192 + 3 used) walks a strided set of vertices.
__global__ void __launch_bounds__(256) sz_head_dw(const float *dY, const bf16 *H3, long long N, float *G) {
    const int i = threadIdx.x;
    if (i >= SZ_T * SZ_H + SZ_T) return;
    const int t = i < SZ_T * SZ_H ? i / SZ_H : i - SZ_T * SZ_H, o = i % SZ_H;
    float acc = 0.f;
    for (long long v = blockIdx.x; v < N; v += gridDim.x) {
        const float d = dY[v * SZ_T + t];
        acc = i < SZ_T * SZ_H ? fmaf(d, __bfloat162float(H3[v * SZ_H + o]), acc) : acc + d;
    }
    atomicAdd(&G[OFF_WO + i], acc);
}

// dW_l[m][k] += sum_v dZ[v][m] Xcat[v][k]; db_l[m] += sum_v dZ[v][m].
// Thread t owns output row m = t / 4 and 48 columns; each block walks a
// strided set of 32-vertex chunks staged in shared memory.
__global__ void __launch_bounds__(256) sz_dW(const float *dZ, const bf16 *Xcat, long long N, float *gW,
                                             float *gb) {
    __shared__ float sdz[32][SZ_H];
    __shared__ float sx[32][SZ_K];
    const int m = threadIdx.x >> 2, k0 = (threadIdx.x & 3) * 48;
    float acc[48];
#pragma unroll
    for (int q = 0; q < 48; ++q) acc[q] = 0.f;
    float accb = 0.f;
    for (long long base = blockIdx.x * 32ll; base < N; base += gridDim.x * 32ll) {
        for (int i = threadIdx.x; i < 32 * SZ_H; i += 256) {
            const long long v = base + i / SZ_H;
            sdz[i / SZ_H][i % SZ_H] = v < N ? dZ[v * SZ_H + i % SZ_H] : 0.f;
        }
        for (int i = threadIdx.x; i < 32 * SZ_K; i += 256) {
            const long long v = base + i / SZ_K;
            sx[i / SZ_K][i % SZ_K] = v < N ? __bfloat162float(Xcat[v * SZ_K + i % SZ_K]) : 0.f;
        }
        __syncthreads();
        for (int r = 0; r < 32; ++r) {
            const float d = sdz[r][m];
            if (d == 0.f) continue;
            if ((threadIdx.x & 3) == 0) accb += d;
#pragma unroll
            for (int q = 0; q < 48; ++q) acc[q] = fmaf(d, sx[r][k0 + q], acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 48; ++q)
        if (acc[q] != 0.f) atomicAdd(&gW[m * SZ_K + k0 + q], acc[q]);
    if ((threadIdx.x & 3) == 0 && accb != 0.f) atomicAdd(&gb[m], accb);
}

// dH_prev[v] = dX[v][self] + sum_{v->w} dX[w][in] + sum_{u->v} dX[u][out];
// dZ_prev = dH_prev * [H_prev > 0].  One warp per vertex.
__global__ void sz_backprop_agg(const float *dX, const bf16 *Hprev, long long N, const int *rp, const int *col,
                                const int *prp, const int *pcol, float *dZ, bf16 *dZb) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long v = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); v < N; v += nw) {
        for (int c = lane; c < SZ_H; c += 32) {
            float d = dX[v * SZ_K + c];
            for (int e = rp[v]; e < rp[v + 1]; ++e) d += dX[(long long)col[e] * SZ_K + SZ_H + c];
            for (int e = prp[v]; e < prp[v + 1]; ++e) d += dX[(long long)pcol[e] * SZ_K + 2 * SZ_H + c];
            const float dz = __bfloat162float(Hprev[v * SZ_H + c]) > 0.f ? d : 0.f;
            dZ[v * SZ_H + c] = dz;
            if (dZb) dZb[v * SZ_H + c] = __float2bfloat16(dz);
        }
    }
}

__global__ void __launch_bounds__(256) sz_input_bwd(const float *dZ0, const float *X, long long N, float *G) {
    __shared__ float gw[SZ_H * SZ_F + SZ_H];
    for (int i = threadIdx.x; i < SZ_H * SZ_F + SZ_H; i += blockDim.x) gw[i] = 0.f;
    __syncthreads();
    const int o = threadIdx.x & (SZ_H - 1);
    const int lanes = blockDim.x / SZ_H;
    float acc[SZ_F + 1] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long v = blockIdx.x * (long long)lanes + threadIdx.x / SZ_H; v < N; v += (long long)gridDim.x * lanes) {
        const float d = dZ0[v * SZ_H + o];
        if (d == 0.f) continue;
#pragma unroll
        for (int k = 0; k < SZ_F; ++k) acc[k] = fmaf(d, X[v * SZ_F + k], acc[k]);
        acc[SZ_F] += d;
    }
#pragma unroll
    for (int k = 0; k < SZ_F; ++k) atomicAdd(&gw[o * SZ_F + k], acc[k]);
    atomicAdd(&gw[SZ_H * SZ_F + o], acc[SZ_F]);
    __syncthreads();
    for (int i = threadIdx.x; i < SZ_H * SZ_F + SZ_H; i += blockDim.x) atomicAdd(&G[OFF_W0 + i], gw[i]);
}

// Adam (Kingma & Ba) on the FP32 master weights, then BF16 working copies
// of the layer weights in both orientations.
__global__ void sz_adam(float *P, const float *G, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                        float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void sz_refresh_bf16(const float *P, bf16 *Wb, bf16 *Wtb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < SZ_L * SZ_H * SZ_K; i += gridDim.x * blockDim.x) {
        const int l = i / (SZ_H * SZ_K), r = i % (SZ_H * SZ_K);
        const int o = r / SZ_K, k = r % SZ_K;
        const bf16 w = __float2bfloat16(P[off_w(l) + r]);
        Wb[i] = w;                                        // [l][o][k]
        Wtb[l * SZ_H * SZ_K + k * SZ_H + o] = w;          // [l][k][o]
    }
}

// per-graph and total predicted volumes (expm1 of the predictions)
__global__ void sz_sum_pred(const float *Y, long long N, double *tot) {
    __shared__ double s[SZ_T];
    if (threadIdx.x < SZ_T) s[threadIdx.x] = 0.0;
    __syncthreads();
    double acc[SZ_T] = {0.0, 0.0, 0.0};
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int t = 0; t < SZ_T; ++t) acc[t] += expm1((double)fmaxf(Y[v * SZ_T + t], 0.f));
#pragma unroll
    for (int t = 0; t < SZ_T; ++t) atomicAdd(&s[t], acc[t]);
    __syncthreads();
    if (threadIdx.x < SZ_T) atomicAdd(&tot[threadIdx.x], s[threadIdx.x]);
}

unsigned grid_of(long long n, int block, int num_sms) {
    long long b = (n + block - 1) / block;
    const long long cap = (long long)num_sms * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

struct SizerNet {
    cudaStream_t s = nullptr;
    int num_sms = 1;
    float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr;
    bf16 *Wb = nullptr, *Wtb = nullptr;
    double *loss = nullptr, *tot = nullptr;
    int step = 0;
    long long capN = 0;
    bf16 *H[SZ_L + 1] = {};
    bf16 *Xcat[SZ_L] = {};
    float *Y = nullptr, *dY = nullptr, *dX = nullptr, *dZ = nullptr;
    bf16 *dZb = nullptr;
    std::vector<void *> owned;
};

namespace {

void *sz_alloc(SizerNet *n, size_t bytes) {
    void *p = lib_dev_alloc(bytes, n->s);
    if (p) n->owned.push_back(p);
    return p;
}

void sz_free_scratch(SizerNet *n) {
    // the scratch buffers are the owned allocations made after the parameters (index >= 8)
    for (size_t i = 8; i < n->owned.size(); ++i) lib_dev_free(n->owned[i], n->s);
    if (n->owned.size() > 8) n->owned.resize(8);
    for (auto &h : n->H) h = nullptr;
    for (auto &x : n->Xcat) x = nullptr;
    n->Y = n->dY = n->dX = n->dZ = nullptr;
    n->dZb = nullptr;
    n->capN = 0;
}

cudaError_t sz_ensure(SizerNet *n, long long N) {
    if (N <= n->capN) return cudaSuccess;
    sz_free_scratch(n);
    const long long C = N + N / 4 + 64;
    for (auto &h : n->H) h = (bf16 *)sz_alloc(n, sizeof(bf16) * SZ_H * C);
    for (auto &x : n->Xcat) x = (bf16 *)sz_alloc(n, sizeof(bf16) * SZ_K * C);
    n->Y = (float *)sz_alloc(n, sizeof(float) * SZ_T * C);
    n->dY = (float *)sz_alloc(n, sizeof(float) * SZ_T * C);
    n->dX = (float *)sz_alloc(n, sizeof(float) * SZ_K * C);
    n->dZ = (float *)sz_alloc(n, sizeof(float) * SZ_H * C);
    n->dZb = (bf16 *)sz_alloc(n, sizeof(bf16) * SZ_H * C);
    for (auto h : n->H)
        if (!h) return cudaErrorMemoryAllocation;
    for (auto x : n->Xcat)
        if (!x) return cudaErrorMemoryAllocation;
    if (!n->Y || !n->dY || !n->dX || !n->dZ || !n->dZb) return cudaErrorMemoryAllocation;
    n->capN = C;
    return cudaSuccess;
}

template <int K, int EPI>
cudaError_t sz_gemm(SizerNet *n, const bf16 *A, long long M, const bf16 *Bt, int NC, const float *bias, bf16 *ob,
                    float *of) {
    const size_t smem = 2 * 64 * (K + 8) * sizeof(bf16);
    // the shared-memory attribute is set once per device id
    static std::atomic<bool> attr[64];
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev].load()) {
        cudaError_t e = cudaFuncSetAttribute(sz_mma_gemm<K, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr[dev].store(true);
    }
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((NC + 63) / 64));
    sz_mma_gemm<K, EPI><<<grid, 128, smem, n->s>>>(A, M, Bt, NC, bias, ob, of);
    note_launch();
    return cudaGetLastError();
}

// splitmix64 (Steele, Lea, Flood 2014) for the weight initialisation
unsigned long long sm64(unsigned long long &x) {
    unsigned long long z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

int sz_param_count() { return NPARAM; }
int sz_features_per_vertex() { return SZ_F; }
int sz_targets() { return SZ_T; }

SizerNet *sz_create(unsigned long long seed, cudaStream_t s, int num_sms) {
    SizerNet *n = new SizerNet();
    n->s = s;
    n->num_sms = num_sms;
    n->P = (float *)sz_alloc(n, sizeof(float) * NPARAM);
    n->G = (float *)sz_alloc(n, sizeof(float) * NPARAM);
    n->m = (float *)sz_alloc(n, sizeof(float) * NPARAM);
    n->v = (float *)sz_alloc(n, sizeof(float) * NPARAM);
    n->Wb = (bf16 *)sz_alloc(n, sizeof(bf16) * SZ_L * SZ_H * SZ_K);
    n->Wtb = (bf16 *)sz_alloc(n, sizeof(bf16) * SZ_L * SZ_H * SZ_K);
    n->loss = (double *)sz_alloc(n, sizeof(double) * 4);
    n->tot = (double *)sz_alloc(n, sizeof(double) * 4);
    if (n->owned.size() != 8) {
        sz_destroy(n);
        return nullptr;
    }
    // He-uniform weights, zero biases (deterministic in the seed)
    std::vector<float> h(NPARAM, 0.f);
    unsigned long long x = seed;
    auto uni = [&](float bound) { return (float)(((sm64(x) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * bound; };
    for (int i = 0; i < SZ_H * SZ_F; ++i) h[OFF_W0 + i] = uni(sqrtf(6.f / SZ_F));
    for (int l = 0; l < SZ_L; ++l)
        for (int i = 0; i < SZ_H * SZ_K; ++i) h[off_w(l) + i] = uni(sqrtf(6.f / SZ_K));
    for (int i = 0; i < SZ_T * SZ_H; ++i) h[OFF_WO + i] = uni(sqrtf(3.f / SZ_H));
    if (sz_set_params(n, h.data()) != cudaSuccess ||
        cudaMemsetAsync(n->m, 0, sizeof(float) * NPARAM, s) != cudaSuccess ||
        cudaMemsetAsync(n->v, 0, sizeof(float) * NPARAM, s) != cudaSuccess) {
        cudaGetLastError();
        sz_destroy(n);
        return nullptr;
    }
    return n;
}

void sz_destroy(SizerNet *n) {
    if (!n) return;
    cudaStreamSynchronize(n->s);
    for (void *p : n->owned) lib_dev_free(p, n->s);
    cudaStreamSynchronize(n->s);
    delete n;
}

cudaError_t sz_set_params(SizerNet *n, const float *host) {
    cudaError_t e = cudaMemcpyAsync(n->P, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, n->s);
    if (e != cudaSuccess) return e;
    sz_refresh_bf16<<<64, 256, 0, n->s>>>(n->P, n->Wb, n->Wtb);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(n->s);
}

cudaError_t sz_get_params(SizerNet *n, float *host) {
    cudaError_t e = cudaMemcpyAsync(host, n->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, n->s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(n->s);
}

cudaError_t sz_get_grads(SizerNet *n, float *host) {
    cudaError_t e = cudaMemcpyAsync(host, n->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, n->s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(n->s);
}

cudaError_t sz_features(const GraphDev &g, float *X, cudaStream_t s, int num_sms) {
    sz_features_kernel<<<grid_of(g.N, 128, num_sms), 128, 0, s>>>(g, X);
    note_launch();
    return cudaGetLastError();
}

cudaError_t sz_labels(const unsigned long long *counts, long long N, float *T, cudaStream_t s, int num_sms) {
    sz_labels_kernel<<<grid_of(3 * N, 256, num_sms), 256, 0, s>>>(counts, N, T);
    note_launch();
    return cudaGetLastError();
}

cudaError_t sz_forward(SizerNet *n, const SzGraph &b) {
    cudaError_t e = sz_ensure(n, b.N);
    if (e != cudaSuccess) return e;
    const unsigned g256 = grid_of(b.N, 256, n->num_sms);
    sz_input_fwd<<<g256, 256, 0, n->s>>>(b.X, b.N, n->P, n->H[0]);
    note_launch();
    for (int l = 0; l < SZ_L; ++l) {
        sz_aggregate<<<grid_of(b.N * 32, 256, n->num_sms), 256, 0, n->s>>>(n->H[l], b.N, b.rp, b.col, b.prp, b.pcol,
                                                                          n->Xcat[l]);
        note_launch();
        e = sz_gemm<SZ_K, 0>(n, n->Xcat[l], b.N, n->Wb + (size_t)l * SZ_H * SZ_K, SZ_H, n->P + off_b(l),
                             n->H[l + 1], nullptr);
        if (e != cudaSuccess) return e;
    }
    sz_head_fwd<<<g256, 256, 0, n->s>>>(n->H[SZ_L], b.N, n->P, n->Y);
    note_launch();
    return cudaGetLastError();
}

cudaError_t sz_loss_backward(SizerNet *n, const SzGraph &b, double *loss_host) {
    cudaError_t e = sz_forward(n, b);
    if (e != cudaSuccess) return e;
    const unsigned g256 = grid_of(b.N, 256, n->num_sms);
    if ((e = cudaMemsetAsync(n->G, 0, sizeof(float) * NPARAM, n->s))) return e;
    if ((e = cudaMemsetAsync(n->loss, 0, sizeof(double), n->s))) return e;
    sz_head_bwd<<<g256, 256, 0, n->s>>>(n->Y, b.T, n->H[SZ_L], b.N, n->P, n->dY, n->loss, n->dZ, n->dZb);
    sz_head_dw<<<(unsigned)(n->num_sms * 4), 256, 0, n->s>>>(n->dY, n->H[SZ_L], b.N, n->G);
    note_launch(2);
    for (int l = SZ_L - 1; l >= 0; --l) {
        // dX = dZ W_l (input gradient of the layer); dW_l, db_l
        e = sz_gemm<SZ_H, 1>(n, n->dZb, b.N, n->Wtb + (size_t)l * SZ_H * SZ_K, SZ_K, nullptr, nullptr, n->dX);
        if (e != cudaSuccess) return e;
        sz_dW<<<(unsigned)(n->num_sms * 2), 256, 0, n->s>>>(n->dZ, n->Xcat[l], b.N, n->G + off_w(l),
                                                           n->G + off_b(l));
        sz_backprop_agg<<<grid_of(b.N * 32, 256, n->num_sms), 256, 0, n->s>>>(n->dX, n->H[l], b.N, b.rp, b.col,
                                                                             b.prp, b.pcol, n->dZ, n->dZb);
        note_launch(2);
    }
    sz_input_bwd<<<(unsigned)(n->num_sms * 4), 256, 0, n->s>>>(n->dZ, b.X, b.N, n->G);
    note_launch();
    if ((e = cudaGetLastError())) return e;
    if (loss_host) {
        if ((e = cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->s))) return e;
        if ((e = cudaStreamSynchronize(n->s))) return e;
    }
    return cudaSuccess;
}

cudaError_t sz_adam_step(SizerNet *n, float lr) {
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    sz_adam<<<grid_of(NPARAM, 256, n->num_sms), 256, 0, n->s>>>(n->P, n->G, n->m, n->v, NPARAM, lr, b1, b2, 1e-8f, c1,
                                                               c2);
    sz_refresh_bf16<<<64, 256, 0, n->s>>>(n->P, n->Wb, n->Wtb);
    note_launch(2);
    return cudaGetLastError();
}

// expm1 sums of a [N][3] log1p array (labels or predictions) into totals_host[3]
cudaError_t sz_log_totals(SizerNet *n, const float *Y, long long N, double *totals_host) {
    cudaError_t e = cudaMemsetAsync(n->tot, 0, sizeof(double) * SZ_T, n->s);
    if (e != cudaSuccess) return e;
    sz_sum_pred<<<grid_of(N, 256, n->num_sms), 256, 0, n->s>>>(Y, N, n->tot);
    note_launch();
    if ((e = cudaMemcpyAsync(totals_host, n->tot, sizeof(double) * SZ_T, cudaMemcpyDeviceToHost, n->s))) return e;
    return cudaStreamSynchronize(n->s);
}

cudaError_t sz_predict(SizerNet *n, const SzGraph &b, float *Y_host, double *totals_host) {
    cudaError_t e = sz_forward(n, b);
    if (e != cudaSuccess) return e;
    if (totals_host) {
        if ((e = cudaMemsetAsync(n->tot, 0, sizeof(double) * SZ_T, n->s))) return e;
        sz_sum_pred<<<grid_of(b.N, 256, n->num_sms), 256, 0, n->s>>>(n->Y, b.N, n->tot);
        note_launch();
        if ((e = cudaMemcpyAsync(totals_host, n->tot, sizeof(double) * SZ_T, cudaMemcpyDeviceToHost, n->s))) return e;
    }
    if (Y_host && (e = cudaMemcpyAsync(Y_host, n->Y, sizeof(float) * SZ_T * b.N, cudaMemcpyDeviceToHost, n->s)))
        return e;
    return cudaStreamSynchronize(n->s);
}

}  // namespace tpg
