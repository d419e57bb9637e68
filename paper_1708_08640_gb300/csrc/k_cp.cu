// S3CMTF-CP (Section 4.2: the method with a hyper-diagonal core) on the GPU, FP32.
//
// With G = diag(l), Eq. (4) becomes x~ = sum_j l_j prod_n a_n[j] and Eq. (3) p_n[j] =
// l_j prod_{m != n} a_m[j]: O(N J) work per entry instead of O(J^N), so the epoch is bound
// by the row gathers, not by arithmetic.  k_cp_hog is the HOGWILD epoch of this model: one
// thread per tensor entry, tiles claimed from a counter by persistent CTAs, row gradients
// to slots in shared memory and summed per row (the same tile bookkeeping as the Tucker
// kernels), and the diagonal's share of the core step reduced over the tile and added
// lock-free.  The core keeps the padded dense layout with zeros off the diagonal.
#include <cuda_runtime.h>

#include "hog_common.cuh"
#include "kernels.h"

namespace s3 {

constexpr int kCpThreads = 256;

// flattened position of the diagonal element (j, .., j) in the padded core
__device__ __forceinline__ int64_t cp_diag(int N, int JP, int ldg, int j) {
    int64_t l = j;
    for (int n = 1; n < N - 1; ++n) l = l * JP + j;
    return l * ldg + j;
}

template <int N, int JP>
__global__ void __launch_bounds__(kCpThreads) k_cp_hog(DParams P, DGroup Gr, int64_t n_tiles,
                                                       int* tile_counter, const float* eta_p,
                                                       int row_mean, float core_step_scale,
                                                       HogSmem H) {
    constexpr int JPR = round4(JP);
    extern __shared__ __align__(16) float smem[];
    __shared__ float s_lam[JPR];
    __shared__ float s_red[kCpThreads / 32][JPR];
    __shared__ int64_t s_cur, s_nxt;        // this tile and the one claimed after it
    __shared__ int64_t s_lo[32], s_hi[32];  // array ranges of this tile (hog_ranges lanes)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float eta = *eta_p;
    // tiles claimed two ahead, their ranges read one ahead (as in the BF16 Tucker kernel):
    // the segment table goes out as asynchronous copies at the tile's start
    if (tid == 0) {
        s_cur = atomicAdd(tile_counter, 1);
        s_nxt = atomicAdd(tile_counter, 1);
    }
    __syncthreads();
    if (tid < 32) hog_ranges(P, Gr, s_cur, n_tiles, H, tid, s_lo[tid], s_hi[tid]);
    __syncthreads();
    for (;;) {
        const int64_t t = s_cur;
        if (t >= n_tiles) break;
        int claim = 0;
        if (tid == 0) claim = atomicAdd(tile_counter, 1);   // needed only at the tile's end
        const int64_t e0 = s_lo[0];
        const int nb = (int)(s_hi[0] - e0);
        hog_tables_async(P, Gr, s_lo, s_hi, smem, H, tid, kCpThreads);
        // the diagonal is read by the warp after the one whose threads add to it, so that no
        // load waits for the same thread's reduction of the previous tile
        if (tid >= 32 && tid < 32 + JP) s_lam[tid - 32] = __ldcg(P.G + cp_diag(N, JP, P.ldg, tid - 32));
        __syncthreads();
        float gd[JP];   // this entry's e * prod_n a_n, the diagonal's gradient (negated)
#pragma unroll
        for (int j = 0; j < JP; ++j) gd[j] = 0.f;
        if (tid < nb) {
            const int64_t e = e0 + tid;
            float a[N][JP], inv[N];
            int32_t tp[N];
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const int32_t row = __ldg(Gr.tidx[n] + e);
                tp[n] = __ldg(Gr.tpos[n] + e);
                load_row<JP, true>(P.U[n] + (int64_t)row * JPR, a[n]);
                inv[n] = __ldg(P.inv_cnt[n] + row);
            }
            float prod[JP];
            float xt = 0.f;
#pragma unroll
            for (int j = 0; j < JP; ++j) {
                float pr = a[0][j];
#pragma unroll
                for (int n = 1; n < N; ++n) pr *= a[n][j];
                prod[j] = pr;
                xt = fmaf(s_lam[j], pr, xt);
            }
            const float err = __ldg(Gr.tval + e) - xt;
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const float r = P.lambda_reg * inv[n];
                float c[JPR];
#pragma unroll
                for (int j = 0; j < JPR; ++j) {
                    float pn = 0.f;
                    if (j < JP) {
                        pn = s_lam[j];
#pragma unroll
                        for (int m = 0; m < N; ++m)
                            if (m != n) pn *= a[m][j];
                    }
                    c[j] = j < JP ? fmaf(-err, pn, r * a[n][j]) : 0.f;
                }
                put_slot<JPR>(smem, H, n, tp[n], c);
            }
#pragma unroll
            for (int j = 0; j < JP; ++j) gd[j] = err * prod[j];
        }
        hog_coupled<JP>(P, Gr, s_lo, s_hi, smem, H, tid, kCpThreads);
        // the tile's diagonal gradient: warp butterflies, then the warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < JP; ++j) gd[j] += __shfl_xor_sync(0xffffffffu, gd[j], o);
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < JP; ++j) s_red[warp][j] = gd[j];
        cp_async_wait_all();   // this thread's table copies
        __syncthreads();
        hog_tables_damp(P, Gr, s_lo, s_hi, smem, H, tid, kCpThreads);
        // G_jj += eta cs / W (sum_b e_b prod_n a_n[j] / n_t - lambda_reg / |Omega| G_jj)
        if (tid < JP && nb > 0) {
            float s = 0.f;
            for (int w = 0; w < kCpThreads / 32; ++w) s += s_red[w][tid];
            const float sc = eta * core_step_scale / (float)nb;
            const float rg = eta * core_step_scale * P.lambda_reg * P.inv_nnz;
            float* gd = P.G + cp_diag(N, JP, P.ldg, tid);
            atomicAdd(gd, fmaf(sc, s, -rg * s_lam[tid]));
            if (P.nonneg) red_proj(gd);
        }
        cp_async_wait_all();   // this thread's step-scale copies
        __syncthreads();
        // the next tile's ranges are read while this one's row steps go out (nothing reads
        // s_lo / s_hi / s_nxt past the barrier above until the one below)
        int64_t lo = 0, hi = 0;
        if (tid < 32) hog_ranges(P, Gr, s_nxt, n_tiles, H, tid, lo, hi);
        hog_flush<JPR>(P, smem, H, eta, row_mean, threadIdx.x, blockDim.x);
        __syncwarp();   // warp 0's lanes have read s_nxt before thread 0 moves it
        if (tid < 32) {
            s_lo[tid] = lo;
            s_hi[tid] = hi;
        }
        if (tid == 0) {
            s_cur = s_nxt;
            s_nxt = claim;
        }
        __syncthreads();
    }
}

// zero every off-diagonal element of the padded core (the CP model's core is hyper-diagonal)
__global__ void k_cp_mask(float* G, int N, int JP, int ldg) {
    int64_t total = ldg;
    for (int n = 0; n < N - 1; ++n) total *= JP;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < total;
         l += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = l;
        const int j0 = (int)(r % ldg);
        r /= ldg;
        bool diag = true;
        for (int n = 0; n < N - 1; ++n) {
            diag &= (int)(r % JP) == j0;
            r /= JP;
        }
        if (!diag) G[l] = 0.f;
    }
}

#define S3_FOR_EACH_CP_SHAPE(X) \
    X(3, 2) X(3, 4) X(3, 5) X(3, 8) X(3, 10) X(3, 16) X(3, 20) X(3, 32) X(4, 2) X(4, 4) X(4, 8)

static size_t cp_smem(int JP, const int64_t* max_events, const int64_t* max_segs, int nF, HogSmem* H) {
    if (H) *H = HogSmem{};
    return hog_smem_floats(round4(JP), max_events, max_segs, nF, H, 0) * sizeof(float);
}

size_t tensor_cp_smem(int JP, const int64_t* max_events, const int64_t* max_segs, int nF) {
    return cp_smem(JP, max_events, max_segs, nF, nullptr);
}

int tensor_cp_blocks_per_sm(int N, int JP, size_t smem) {
    int nb = 0;
#define X(NN, JJ)                                                                           \
    if (N == NN && JP == JJ) {                                                              \
        if (smem > 32 * 1024 &&                                                             \
            cudaFuncSetAttribute(k_cp_hog<NN, JJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem) != cudaSuccess)                                 \
            return 0;                                                                       \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cp_hog<NN, JJ>, kCpThreads,  \
                                                          smem) != cudaSuccess)             \
            return 0;                                                                       \
        return nb;                                                                          \
    }
    S3_FOR_EACH_CP_SHAPE(X)
#undef X
    return 0;
}

cudaError_t launch_tensor_cp_hog(int N, int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                 int* tile_counter, int grid, const float* eta, int row_mean,
                                 float core_step_scale, const int64_t* max_events,
                                 const int64_t* max_segs, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    HogSmem H;
    const size_t smem = cp_smem(JP, max_events, max_segs, P.N + P.M, &H);
#define X(NN, JJ)                                                                           \
    if (N == NN && JP == JJ) {                                                              \
        if (smem > 32 * 1024) {                                                             \
            cudaError_t e = cudaFuncSetAttribute(k_cp_hog<NN, JJ>,                          \
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            if (e != cudaSuccess) return e;                                                 \
        }                                                                                   \
        k_cp_hog<NN, JJ><<<grid, kCpThreads, smem, s>>>(P, G, n_tiles, tile_counter, eta,    \
                                                        row_mean, core_step_scale, H);      \
        return cudaGetLastError();                                                          \
    }
    S3_FOR_EACH_CP_SHAPE(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_cp_mask(float* G, int N, int JP, int ldg, cudaStream_t s) {
    k_cp_mask<<<64, 256, 0, s>>>(G, N, JP, ldg);
    return cudaGetLastError();
}

}  // namespace s3
