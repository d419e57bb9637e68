// FP32 tensor-entry kernels of the S3CMTF epoch (sm_103a, CUDA cores).
//
//   k_tensor_contrib  minibatch and full-gradient pass: per-entry Eq. (8) row gradients
//                     written to their segment slots, CTA partials of the core gradient.
//   k_tensor_hog      HOGWILD pass (Section 3.3 on the GPU): per-tile row gradients
//                     combined in shared memory, applied with vector atomics.
//   k_tensor_fwd      predictions and squared errors (loss, RMSE, predict).
//
// Layout: one thread per tensor entry, 256 entries per CTA tile, the core in shared memory
// (every warp reads the same core row at the same time, so each load is a broadcast), the
// entry's N factor rows and the N partial products in registers.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"
#include "tensor_fp32.cuh"

namespace s3 {

struct IdxPtrs {
    const int32_t* p[kMaxN];
};

// per-factor offsets (floats) of the HOGWILD row accumulators in shared memory
struct HogSmem {
    int off[kMaxF];
    int nF;
};

template <int N, int JP>
__device__ __forceinline__ float entry_partials(const float* sG, float (&a)[N][JP],
                                                float (&p)[N][JP]) {
    if constexpr (N == 3) return partials3<JP>(sG, a[0], a[1], a[2], p[0], p[1], p[2]);
    else return partials4<JP>(sG, a[0], a[1], a[2], a[3], p[0], p[1], p[2], p[3]);
}

template <int N, int JP>
__device__ __forceinline__ float entry_predict(const float* sG, float (&a)[N][JP]) {
    if constexpr (N == 3) return predict3<JP>(sG, a[0], a[1], a[2]);
    else return predict4<JP>(sG, a[0], a[1], a[2], a[3]);
}

template <int N, int JP>
__device__ __forceinline__ void load_core_smem(float* sG, const float* __restrict__ G) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    for (int l = threadIdx.x * 4; l < Q * JPR; l += kTile * 4) st4(sG + l, ld4_nc(G + l));
}

// ------------------------------------------------------------------ minibatch / gradient
template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_tensor_contrib(DParams P, DGroup Gr, TensorLaunch L) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    extern __shared__ __align__(16) float smem[];
    float* sG = smem;
    float* stage = smem + Q * JPR;
    load_core_smem<N, JP>(sG, P.G);
    const int64_t e0 = L.e_begin + (int64_t)blockIdx.x * kTile;
    const int nb = (int)((L.e_end - e0) < kTile ? (L.e_end - e0) : kTile);
    const int tid = threadIdx.x;
    __syncthreads();
    if (tid < nb) {
        const int64_t e = e0 + tid;
        float a[N][JP];
        int32_t row[N];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            row[n] = __ldg(Gr.tidx[n] + e);
            load_row<JP, false>(P.U[n] + (int64_t)row[n] * JPR, a[n]);
        }
        float p[N][JP];
        const float err = __ldg(Gr.tval + e) - entry_partials<N, JP>(sG, a, p);
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float r = P.lambda_reg * __ldg(P.inv_cnt[n] + row[n]);
            float c[JPR];
#pragma unroll
            for (int j = 0; j < JPR; ++j) c[j] = j < JP ? fmaf(-err, p[n][j], r * a[n][j]) : 0.f;
            float* dst = L.contrib[n] + (int64_t)__ldg(Gr.tpos[n] + e) * JPR;
#pragma unroll
            for (int q = 0; q < JPR / 4; ++q)
                st4(dst + 4 * q, make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
            float* sp = stage + (n * kTile + tid) * JPR;
#pragma unroll
            for (int j = 0; j < JP; ++j) sp[j] = n == 0 ? err * a[n][j] : a[n][j];
        }
    }
    __syncthreads();
    CoreAcc<N, JP> acc;
    acc.init();
    acc.add_tile(stage, nb);
    __syncthreads();
    acc.store(L.core_part + (int64_t)blockIdx.x * (Q * JP), stage);
}

// ------------------------------------------------------------------ HOGWILD
template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_tensor_hog(DParams P, DGroup Gr, int64_t t_begin,
                                                      int64_t t_end, const float* eta_p,
                                                      int row_mean, float* core_part,
                                                      HogSmem H) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    extern __shared__ __align__(16) float smem[];
    float* sG = smem;
    float* stage = smem + Q * JPR;
    const float eta = *eta_p;
    const int tid = threadIdx.x;
    load_core_smem<N, JP>(sG, P.G);
    CoreAcc<N, JP> acc;
    acc.init();
    for (int64_t t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
        // clear this tile's row accumulators
        for (int F = 0; F < H.nF; ++F) {
            const int nseg = (int)(Gr.seg_off[F][t + 1] - Gr.seg_off[F][t]);
            float* sa = smem + H.off[F];
            for (int l = tid * 4; l < nseg * JPR; l += kTile * 4) st4(sa + l, make_float4(0, 0, 0, 0));
        }
        __syncthreads();
        const int64_t e0 = Gr.t_off[t];
        const int nb = (int)(Gr.t_off[t + 1] - e0);
        if (tid < nb) {
            const int64_t e = e0 + tid;
            float a[N][JP];
            int32_t row[N];
#pragma unroll
            for (int n = 0; n < N; ++n) {
                row[n] = __ldg(Gr.tidx[n] + e);
                load_row<JP, true>(P.U[n] + (int64_t)row[n] * JPR, a[n]);
            }
            float p[N][JP];
            const float err = __ldg(Gr.tval + e) - entry_partials<N, JP>(sG, a, p);
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const float r = P.lambda_reg * __ldg(P.inv_cnt[n] + row[n]);
                float* sa = smem + H.off[n] + __ldg(Gr.tpos[n] + e) * JPR;
#pragma unroll
                for (int j = 0; j < JP; ++j) atomicAdd(sa + j, fmaf(-err, p[n][j], r * a[n][j]));
                float* sp = stage + (n * kTile + tid) * JPR;
#pragma unroll
                for (int j = 0; j < JP; ++j) sp[j] = n == 0 ? err * a[n][j] : a[n][j];
            }
        }
        // coupled entries of the tile
        for (int m = 0; m < P.M; ++m) {
            const int c = P.cmode[m];
            const int64_t c0 = Gr.c_off[m][t], c1 = Gr.c_off[m][t + 1];
            const float lm = P.lambda_m;
            for (int64_t e = c0 + tid; e < c1; e += kTile) {
                const int32_t r = __ldg(Gr.cr[m] + e), k = __ldg(Gr.cc[m] + e);
                float u[JP], v[JP];
                load_row<JP, true>(P.U[c] + (int64_t)r * JPR, u);
                load_row<JP, true>(P.V[m] + (int64_t)k * JPR, v);
                float yh = 0.f;
#pragma unroll
                for (int j = 0; j < JP; ++j) yh = fmaf(u[j], v[j], yh);
                const float err = __ldg(Gr.cval[m] + e) - yh;
                const float rv = lm * P.lambda_reg * __ldg(P.inv_cnt[P.N + m] + k);
                float* su = smem + H.off[c] + __ldg(Gr.cpos_u[m] + e) * JPR;
                float* sv = smem + H.off[P.N + m] + __ldg(Gr.cpos_v[m] + e) * JPR;
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    atomicAdd(su + j, -lm * err * v[j]);
                    atomicAdd(sv + j, fmaf(-lm * err, u[j], rv * v[j]));
                }
            }
        }
        __syncthreads();
        acc.add_tile(stage, nb);
        // apply this tile's steps: one vector atomic per 4 values of every touched row
        for (int F = 0; F < H.nF; ++F) {
            const int64_t sg0 = Gr.seg_off[F][t];
            const int nseg = (int)(Gr.seg_off[F][t + 1] - sg0);
            const float* sa = smem + H.off[F];
            float* base = F < P.N ? P.U[F] : P.V[F - P.N];
            for (int l = tid; l < nseg * (JPR / 4); l += kTile) {
                const int s = l / (JPR / 4), q = l % (JPR / 4);
                const int32_t rr = __ldg(Gr.seg_row[F] + sg0 + s);
                const float den = row_mean ? (float)__ldg(Gr.seg_cnt[F] + sg0 + s) : 1.f;
                const float sc = -eta * __ldg(P.damp[F] + rr) / den;
                const float4 v = *reinterpret_cast<const float4*>(sa + s * JPR + 4 * q);
                red_add_v4(base + (int64_t)rr * JPR + 4 * q, sc * v.x, sc * v.y, sc * v.z, sc * v.w);
            }
        }
        __syncthreads();
    }
    acc.store(core_part + (int64_t)blockIdx.x * (Q * JP), stage);
}

// ------------------------------------------------------------------ forward
__device__ __forceinline__ void block_reduce_pair(Kahan k, float* out2) {
    __shared__ float ws[2][kTile / 32];
    // warp level: merge (s, c) pairs in a fixed tree
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_down_sync(0xffffffffu, k.s, o);
        const float oc = __shfl_down_sync(0xffffffffu, k.c, o);
        k.c += oc;
        k.add(os);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { ws[0][w] = k.s; ws[1][w] = k.c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        Kahan t;
        t.init();
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { t.c += ws[1][i]; t.add(ws[0][i]); }
        out2[0] = t.s;
        out2[1] = t.c;
    }
}

template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_tensor_fwd(DParams P, IdxPtrs idx, const float* x,
                                                      int64_t n, float* pred, float* sq_part) {
    constexpr int JPR = round4(JP);
    extern __shared__ __align__(16) float smem[];
    float* sG = smem;
    load_core_smem<N, JP>(sG, P.G);
    __syncthreads();
    Kahan k;
    k.init();
    for (int64_t e = (int64_t)blockIdx.x * kTile + threadIdx.x; e < n; e += (int64_t)gridDim.x * kTile) {
        float a[N][JP];
#pragma unroll
        for (int m = 0; m < N; ++m)
            load_row<JP, false>(P.U[m] + (int64_t)__ldg(idx.p[m] + e) * JPR, a[m]);
        const float xt = entry_predict<N, JP>(sG, a);
        if (pred) pred[e] = xt;
        if (x) {
            const float d = __ldg(x + e) - xt;
            k.add(d * d);
        }
    }
    if (sq_part) block_reduce_pair(k, sq_part + 2 * blockIdx.x);
}

// ------------------------------------------------------------------ dispatch
#define S3_FOR_EACH_TENSOR_SHAPE(X) \
    X(3, 2) X(3, 4) X(3, 5) X(3, 8) X(3, 10) X(3, 16) X(3, 20) X(3, 32) X(4, 2) X(4, 4) X(4, 8)

int tensor_supported_jp(int N, int J) {
    static const int jp3[] = {2, 4, 5, 8, 10, 16, 20, 32};
    static const int jp4[] = {2, 4, 8};
    if (N == 3) {
        for (int v : jp3) if (v >= J) return v;
    } else if (N == 4) {
        for (int v : jp4) if (v >= J) return v;
    }
    return 0;
}

static size_t core_floats(int N, int JP) {
    size_t q = 1;
    for (int n = 0; n < N - 1; ++n) q *= JP;
    return q * round4(JP);
}

size_t tensor_contrib_smem(int N, int JP) {
    return sizeof(float) * (core_floats(N, JP) + (size_t)N * kTile * round4(JP));
}

size_t tensor_hog_smem(int N, int JP, const int64_t* max_segs, int nF) {
    size_t b = tensor_contrib_smem(N, JP) / sizeof(float);
    for (int F = 0; F < nF; ++F) b += (size_t)max_segs[F] * round4(JP);
    return b * sizeof(float);
}

template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

cudaError_t launch_tensor_contrib(int N, int JP, const DParams& P, const DGroup& G,
                                  const TensorLaunch& L, cudaStream_t s) {
    const int64_t n = L.e_end - L.e_begin;
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + kTile - 1) / kTile);
    const size_t smem = tensor_contrib_smem(N, JP);
#define X(NN, JJ)                                                              \
    if (N == NN && JP == JJ) {                                                 \
        cudaError_t e = prep(k_tensor_contrib<NN, JJ>, smem);                  \
        if (e != cudaSuccess) return e;                                        \
        k_tensor_contrib<NN, JJ><<<grid, kTile, smem, s>>>(P, G, L);           \
        return cudaGetLastError();                                             \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tensor_hog(int N, int JP, const DParams& P, const DGroup& G,
                               int64_t t_begin, int64_t t_end, int grid, const float* eta,
                               int row_mean, float* core_part, const int64_t* max_segs,
                               cudaStream_t s) {
    if (t_end <= t_begin) return cudaSuccess;
    HogSmem H;
    H.nF = P.N + P.M;
    size_t off = tensor_contrib_smem(N, JP) / sizeof(float);
    for (int F = 0; F < H.nF; ++F) {
        H.off[F] = (int)off;
        off += (size_t)max_segs[F] * round4(JP);
    }
    const size_t smem = off * sizeof(float);
#define X(NN, JJ)                                                                        \
    if (N == NN && JP == JJ) {                                                           \
        cudaError_t e = prep(k_tensor_hog<NN, JJ>, smem);                                \
        if (e != cudaSuccess) return e;                                                  \
        k_tensor_hog<NN, JJ><<<grid, kTile, smem, s>>>(P, G, t_begin, t_end, eta,        \
                                                       row_mean, core_part, H);          \
        return cudaGetLastError();                                                       \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tensor_fwd(int N, int JP, const DParams& P, const int32_t* const* idx,
                              const float* x, int64_t n, float* pred, float* sq_part,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    IdxPtrs ip;
    for (int m = 0; m < kMaxN; ++m) ip.p[m] = m < N ? idx[m] : nullptr;
    const unsigned grid = (unsigned)std::min<int64_t>((n + kTile - 1) / kTile, 4096);
    const size_t smem = sizeof(float) * core_floats(N, JP);
#define X(NN, JJ)                                                                 \
    if (N == NN && JP == JJ) {                                                    \
        cudaError_t e = prep(k_tensor_fwd<NN, JJ>, smem);                         \
        if (e != cudaSuccess) return e;                                           \
        k_tensor_fwd<NN, JJ><<<grid, kTile, smem, s>>>(P, ip, x, n, pred, sq_part); \
        return cudaGetLastError();                                                \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t tensor_prepare(int N, int JP, size_t hog_smem) {
#define X(NN, JJ)                                                                  \
    if (N == NN && JP == JJ) {                                                     \
        cudaError_t e = prep(k_tensor_contrib<NN, JJ>, tensor_contrib_smem(NN, JJ)); \
        if (e == cudaSuccess) e = prep(k_tensor_fwd<NN, JJ>, sizeof(float) * core_floats(NN, JJ)); \
        if (e == cudaSuccess && hog_smem > 0) e = prep(k_tensor_hog<NN, JJ>, hog_smem); \
        return e;                                                                  \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

int tensor_hog_blocks_per_sm(int N, int JP, size_t smem) {
    int nb = 0;
#define X(NN, JJ)                                                                          \
    if (N == NN && JP == JJ) {                                                             \
        if (prep(k_tensor_hog<NN, JJ>, smem) != cudaSuccess) return 0;                     \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tensor_hog<NN, JJ>, kTile, \
                                                          smem) != cudaSuccess)            \
            return 0;                                                                      \
        return nb;                                                                         \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return 0;
}

int tensor_fwd_blocks(int64_t n) {
    return (int)std::min<int64_t>((n + kTile - 1) / kTile, 4096);
}

}  // namespace s3
