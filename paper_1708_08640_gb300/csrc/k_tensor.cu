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
#include "hog_common.cuh"
#include "tensor_fp32.cuh"

namespace s3 {

struct IdxPtrs {
    const int32_t* p[kMaxN];
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
// One persistent launch per epoch.  CTAs claim tiles in visiting order from a global
// counter; a tile reads the current rows and core (coherent loads: other CTAs update them
// concurrently), combines its row gradients in shared memory, adds the row steps with vector
// atomics and adds its share of the core step to G (lock-free, like the rows).
template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_tensor_hog(DParams P, DGroup Gr, int64_t n_tiles,
                                                      int* tile_counter, const float* eta_p,
                                                      int row_mean, float core_step_scale,
                                                      HogSmem H) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_tile;
    float* sG = smem;
    float* stage = smem + Q * JPR;
    const float eta = *eta_p;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1);
        // current core (coherent: other CTAs add to it)
        for (int l = tid * 4; l < Q * JPR; l += kTile * 4) st4(sG + l, ld4_cg(P.G + l));
        __syncthreads();
        const int64_t t = s_tile;
        if (t >= n_tiles) break;
        hog_clear<JPR>(smem, Gr, t, H);
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
        hog_coupled<JP>(P, Gr, t, smem, H);
        __syncthreads();
        // core: this tile's share of the core step,
        //   G += eta * cs / W * (sum_b e_b a1 o..o aN / n_t - lambda_reg / |Omega| * G)
        if (nb > 0) {
            const float sc = eta * core_step_scale / (float)nb;
            const float rg = eta * core_step_scale * P.lambda_reg * P.inv_nnz;
            CoreTile<N, JP>::apply(stage, nb, sG, P.G, sc, rg);
        }
        hog_flush<JPR>(P, Gr, t, smem, H, eta, row_mean);
        __syncthreads();
    }
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

// the opt-in above 48 KB counts static shared memory too, so set the limit whenever the
// dynamic part is large
template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
    if (smem > 32 * 1024)
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

cudaError_t launch_tensor_hog(int N, int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                              int* tile_counter, int grid, const float* eta, int row_mean,
                              float core_step_scale, const int64_t* max_segs, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
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
        k_tensor_hog<NN, JJ><<<grid, kTile, smem, s>>>(P, G, n_tiles, tile_counter, eta, \
                                                       row_mean, core_step_scale, H);    \
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

// the forward pass with one CTA per 256 entries (no grid-stride loop): ceil(n / 256) pairs
cudaError_t launch_tensor_fwd_one_pass(int N, int JP, const DParams& P, const int32_t* const* idx,
                                       const float* x, int64_t n, float* sq_part, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    IdxPtrs ip;
    for (int m = 0; m < kMaxN; ++m) ip.p[m] = m < N ? idx[m] : nullptr;
    const unsigned grid = (unsigned)((n + kTile - 1) / kTile);
    const size_t smem = sizeof(float) * core_floats(N, JP);
#define X(NN, JJ)                                                                      \
    if (N == NN && JP == JJ) {                                                         \
        cudaError_t e = prep(k_tensor_fwd<NN, JJ>, smem);                              \
        if (e != cudaSuccess) return e;                                                \
        k_tensor_fwd<NN, JJ><<<grid, kTile, smem, s>>>(P, ip, x, n, nullptr, sq_part); \
        return cudaGetLastError();                                                     \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

int tensor_fwd_blocks(int64_t n) {
    return (int)std::min<int64_t>((n + kTile - 1) / kTile, 4096);
}

}  // namespace s3
