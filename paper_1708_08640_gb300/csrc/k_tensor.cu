// FP32 tensor-entry kernels of the S3CMTF epoch (sm_103a, CUDA cores).
//
//   k_tensor_contrib  minibatch and full-gradient pass: per-entry Eq. (8) row gradients
//                     written to their segment slots, CTA partials of the core gradient.
//   k_tensor_hog      HOGWILD pass (Section 3.3 on the GPU), in tensor_hog.cuh; its
//                     variants are compiled in k_tensor_hog2.cu and k_tensor_hog4.cu.
//   k_tensor_fwd      predictions and squared errors (loss, RMSE, predict).
//
// Layout: one thread per tensor entry, 256 entries per CTA tile, the core in shared memory
// (every warp reads the same core row at the same time, so each load is a broadcast), the
// entry's N factor rows and the N partial products in registers.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"
#include "tensor_hog.cuh"

namespace s3 {

// Coordinates of the forward kernel: SoA index arrays, each mode's extent I_n, and an
// optional flag raised when some index lies outside [0, I_n) (the entry is then skipped:
// no row is read for it, its prediction is NaN and it adds nothing to the sums).
struct IdxPtrs {
    const int32_t* p[kMaxN];
    int32_t lim[kMaxN];
    int* bad;
};

template <int N, int JP>
__device__ __forceinline__ void load_core_smem(float* sG, const float* __restrict__ G) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    for (int l = threadIdx.x * 4; l < Q * JPR; l += kTile * 4) st4(sG + l, ld4_nc(G + l));
}

// ------------------------------------------------------------------ gradient
// Grid-stride over tiles of kTile entries: every entry's Eq. (8) row gradients go to their
// segment slots; each CTA accumulates its tiles' sum e a1 o..o aN (compensated across tiles)
// and writes one partial at the end.
template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_tensor_contrib(DParams P, DGroup Gr, TensorLaunch L) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    extern __shared__ __align__(16) float smem[];
    float* sG = smem;
    float* stage = smem + Q * JPR;
    load_core_smem<N, JP>(sG, P.G);
    const int tid = threadIdx.x;
    CoreAcc<N, JP> acc;
    acc.init();
    __syncthreads();
    for (int64_t e0 = L.e_begin + (int64_t)blockIdx.x * kTile; e0 < L.e_end;
         e0 += (int64_t)gridDim.x * kTile) {
        const int nb = (int)((L.e_end - e0) < kTile ? (L.e_end - e0) : kTile);
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
            const float xt = entry_partials<N, JP>(sG, a, p);
            // the data terms' weight -err: the error (loss) or the caller's weight
            const float err = L.w ? -__ldg(L.w + e) : __ldg(Gr.tval + e) - xt;
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
        acc.add_tile(stage, nb);
        __syncthreads();
    }
    acc.store(L.core_part + (int64_t)blockIdx.x * (Q * JP), stage);
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
        int32_t r[N];
        bool inside = true;
#pragma unroll
        for (int m = 0; m < N; ++m) {
            r[m] = __ldg(idx.p[m] + e);
            inside = inside && (uint32_t)r[m] < (uint32_t)idx.lim[m];
        }
        if (!inside) {
            if (idx.bad) atomicExch(idx.bad, 1);
            if (pred) pred[e] = __int_as_float(0x7fc00000);
            continue;
        }
        float a[N][JP];
#pragma unroll
        for (int m = 0; m < N; ++m) load_row<JP, false>(P.U[m] + (int64_t)r[m] * JPR, a[m]);
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

int tensor_hog_lanes(int N, int JP, int64_t tile) {
    if (N != 3) return 1;
    return tile <= hog_compute_threads(N, JP) / 4 ? 4 : 2;
}

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

size_t tensor_hog_smem(int N, int JP, int L, const int64_t* max_events, const int64_t* max_segs,
                       int64_t ccap, int nF) {
    return hog_layout(N, JP, L, max_events, max_segs, ccap, nF, nullptr) * sizeof(float);
}

cudaError_t launch_tensor_contrib(int N, int JP, const DParams& P, const DGroup& G,
                                  const TensorLaunch& L, int max_grid, int* grid_out,
                                  cudaStream_t s) {
    const int64_t n = L.e_end - L.e_begin;
    *grid_out = 0;
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kTile - 1) / kTile, max_grid));
    *grid_out = (int)grid;
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

cudaError_t launch_tensor_hog(int N, int JP, int L, const DParams& P, const DGroup& G,
                              int64_t n_tiles, int* tile_counter, int grid, const float* eta,
                              int row_mean, float core_step_scale, const int64_t* max_events,
                              const int64_t* max_segs, int64_t ccap, cudaStream_t s) {
    if (L == 2)
        return launch_tensor_hog_l2(N, JP, P, G, n_tiles, tile_counter, grid, eta, row_mean,
                                    core_step_scale, max_events, max_segs, ccap, s);
    return launch_tensor_hog_l41(N, JP, L, P, G, n_tiles, tile_counter, grid, eta, row_mean,
                                 core_step_scale, max_events, max_segs, ccap, s);
}

static IdxPtrs idx_ptrs(int N, const int32_t* const* idx, const int64_t* dims, int* bad) {
    IdxPtrs ip;
    for (int m = 0; m < kMaxN; ++m) {
        ip.p[m] = m < N ? idx[m] : nullptr;
        ip.lim[m] = m < N ? (int32_t)dims[m] : 0;
    }
    ip.bad = bad;
    return ip;
}

cudaError_t launch_tensor_fwd(int N, int JP, const DParams& P, const int32_t* const* idx,
                              const int64_t* dims, int* bad, const float* x, int64_t n,
                              float* pred, float* sq_part, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const IdxPtrs ip = idx_ptrs(N, idx, dims, bad);
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

cudaError_t tensor_prepare(int N, int JP) {
#define X(NN, JJ)                                                                  \
    if (N == NN && JP == JJ) {                                                     \
        cudaError_t e = prep(k_tensor_contrib<NN, JJ>, tensor_contrib_smem(NN, JJ)); \
        if (e == cudaSuccess) e = prep(k_tensor_fwd<NN, JJ>, sizeof(float) * core_floats(NN, JJ)); \
        return e;                                                                  \
    }
    S3_FOR_EACH_TENSOR_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

int tensor_hog_blocks_per_sm(int N, int JP, int L, size_t smem) {
    return L == 2 ? tensor_hog_blocks_l2(N, JP, smem) : tensor_hog_blocks_l41(N, JP, L, smem);
}

// the forward pass with one CTA per 256 entries (no grid-stride loop): ceil(n / 256) pairs
cudaError_t launch_tensor_fwd_one_pass(int N, int JP, const DParams& P, const int32_t* const* idx,
                                       const int64_t* dims, int* bad, const float* x, int64_t n,
                                       float* sq_part, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const IdxPtrs ip = idx_ptrs(N, idx, dims, bad);
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
