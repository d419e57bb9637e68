// The deterministic minibatch epoch as one cooperative launch (sm_103a, FP32 form).
//
// Every batch of the visiting order takes two phases separated by grid-wide barriers:
//   A  the batch's tensor entries (spread over all CTAs, one per thread) and coupled entries
//      compute their Eq. (8) row gradients at the batch-start parameters and write them to
//      their segment slots; each CTA writes its partial of sum_b e_b a1 o .. o aN;
//   B  one warp per touched row sums the row's slots in slot order (compensated) and applies
//      the row step; one warp per core element sums the CTA partials in CTA order and
//      applies the core step.
// The slot layout, the sums' order and the CTA partitioning are fixed, so the epoch is
// deterministic.  Parameters change inside the launch, so every parameter read is a
// coherent (L2) load.  The barrier waits are bounded: after ~1 s without progress a CTA sets
// the error flag and leaves, and the others leave at their next barrier.
#include <cuda_runtime.h>

#include "kernels.h"
#include "tensor_fp32.cuh"

namespace s3 {

constexpr int kBarrierSpins = 1 << 24;   // x 64 ns sleeps: about one second

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// sense-free grid barrier: a counter of arrivals and a generation number that the last
// arriving CTA advances.  Returns false (for the whole CTA) when the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire_u32(gen);
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            int it = 0;
            while (ld_acquire_u32(gen) == g && it < kBarrierSpins) {
                __nanosleep(64);
                ++it;
            }
            if (ld_acquire_u32(gen) == g) *s_ok = 0;
        }
        __threadfence();
    }
    __syncthreads();
    return *s_ok != 0;
}

struct MbArgs {
    float* contrib[kMaxF];
    float* core_part;       // gridDim.x partials of JP^N floats
    unsigned* bar_count;
    unsigned* bar_gen;
    int* err_flag;
    const float* eta;
    float core_scale;
    int row_mean;
    int64_t n_batches;
};

template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_mb_epoch(DParams P, DGroup Gr, MbArgs A) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    constexpr int Pd = Q * JP;
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_ok;
    float* sG = smem;
    float* stage = smem + Q * JPR;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nF = P.N + P.M;
    const float eta = *A.eta;
    if (tid == 0) s_ok = 1;
    __syncthreads();
    for (int64_t b = 0; b < A.n_batches; ++b) {
        // ------------------------------------------------ phase A: gradients into slots
        for (int l = tid * 4; l < Q * JPR; l += kTile * 4) st4(sG + l, ld4_cg(P.G + l));
        const int64_t t0 = Gr.t_off[b], t1 = Gr.t_off[b + 1];
        const int64_t per = (t1 - t0 + gridDim.x - 1) / gridDim.x;
        const int64_t my0 = t0 + (int64_t)blockIdx.x * per;
        const int nb = (int)max((int64_t)0, min(per, t1 - my0));
        __syncthreads();
        if (tid < nb) {
            const int64_t e = my0 + tid;
            float a[N][JP];
            int32_t row[N];
#pragma unroll
            for (int n = 0; n < N; ++n) {
                row[n] = __ldg(Gr.tidx[n] + e);
                load_row<JP, true>(P.U[n] + (int64_t)row[n] * JPR, a[n]);
            }
            float p[N][JP];
            float xt;
            if constexpr (N == 3) xt = partials3<JP>(sG, a[0], a[1], a[2], p[0], p[1], p[2]);
            else xt = partials4<JP>(sG, a[0], a[1], a[2], a[3], p[0], p[1], p[2], p[3]);
            const float err = __ldg(Gr.tval + e) - xt;
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const float r = P.lambda_reg * __ldg(P.inv_cnt[n] + row[n]);
                float c[JPR];
#pragma unroll
                for (int j = 0; j < JPR; ++j) c[j] = j < JP ? fmaf(-err, p[n][j], r * a[n][j]) : 0.f;
                float* dst = A.contrib[n] + (int64_t)__ldg(Gr.tpos[n] + e) * JPR;
#pragma unroll
                for (int q = 0; q < JPR / 4; ++q)
                    st4(dst + 4 * q, make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
                float* sp = stage + (n * kTile + tid) * JPR;
#pragma unroll
                for (int j = 0; j < JP; ++j) sp[j] = n == 0 ? err * a[n][j] : a[n][j];
            }
        }
        // coupled entries of the batch, spread the same way
        for (int m = 0; m < P.M; ++m) {
            const int c = P.cmode[m];
            const int64_t c0 = Gr.c_off[m][b], c1 = Gr.c_off[m][b + 1];
            const int64_t cper = (c1 - c0 + gridDim.x - 1) / gridDim.x;
            const int64_t cm0 = c0 + (int64_t)blockIdx.x * cper;
            const int64_t cm1 = min(c1, cm0 + cper);
            for (int64_t e = cm0 + tid; e < cm1; e += kTile) {
                const int32_t r = __ldg(Gr.cr[m] + e), k = __ldg(Gr.cc[m] + e);
                float u[JP], v[JP];
                load_row<JP, true>(P.U[c] + (int64_t)r * JPR, u);
                load_row<JP, true>(P.V[m] + (int64_t)k * JPR, v);
                float yh = 0.f;
#pragma unroll
                for (int j = 0; j < JP; ++j) yh = fmaf(u[j], v[j], yh);
                const float am = -P.lambda_m * (__ldg(Gr.cval[m] + e) - yh);
                const float rv = P.lambda_m * P.lambda_reg * __ldg(P.inv_cnt[P.N + m] + k);
                float du[JPR], dv[JPR];
#pragma unroll
                for (int j = 0; j < JPR; ++j) {
                    du[j] = j < JP ? am * v[j] : 0.f;
                    dv[j] = j < JP ? fmaf(am, u[j], rv * v[j]) : 0.f;
                }
                float* pu = A.contrib[c] + (int64_t)__ldg(Gr.cpos_u[m] + e) * JPR;
                float* pv = A.contrib[P.N + m] + (int64_t)__ldg(Gr.cpos_v[m] + e) * JPR;
#pragma unroll
                for (int q = 0; q < JPR / 4; ++q) {
                    st4(pu + 4 * q, make_float4(du[4 * q], du[4 * q + 1], du[4 * q + 2], du[4 * q + 3]));
                    st4(pv + 4 * q, make_float4(dv[4 * q], dv[4 * q + 1], dv[4 * q + 2], dv[4 * q + 3]));
                }
            }
        }
        __syncthreads();
        {
            CoreAcc<N, JP> acc;
            acc.init();
            acc.add_tile(stage, nb);
            __syncthreads();
            acc.store(A.core_part + (int64_t)blockIdx.x * Pd, stage);
        }
        if (!grid_barrier(A.bar_count, A.bar_gen, &s_ok)) break;
        // ------------------------------------------------ phase B: ordered sums and steps
        int64_t seg_begin[kMaxF + 1];
        seg_begin[0] = 0;
        for (int F = 0; F < nF; ++F)
            seg_begin[F + 1] = seg_begin[F] + (Gr.seg_off[F][b + 1] - Gr.seg_off[F][b]);
        const int64_t n_seg = seg_begin[nF];
        const int64_t n_items = n_seg + Pd;
        const int64_t gwarp = ((int64_t)blockIdx.x * kTile + tid) >> 5;
        const int64_t nwarps = ((int64_t)gridDim.x * kTile) >> 5;
        for (int64_t w = gwarp; w < n_items; w += nwarps) {
            if (w < n_seg) {
                int F = 0;
                while (F + 1 < nF && w >= seg_begin[F + 1]) ++F;
                const int64_t sg = Gr.seg_off[F][b] + (w - seg_begin[F]);
                const int32_t row = __ldg(Gr.seg_row[F] + sg);
                const int32_t st = __ldg(Gr.seg_start[F] + sg);
                const int32_t cnt = __ldg(Gr.seg_cnt[F] + sg);
                float sum[JPR];
                {
                    Kahan k[JPR];
#pragma unroll
                    for (int j = 0; j < JPR; ++j) k[j].init();
                    const float* src = A.contrib[F] + (int64_t)st * JPR;
                    for (int e = lane; e < cnt; e += 32) {
#pragma unroll
                        for (int q = 0; q < JPR / 4; ++q) {
                            const float4 v = ld4_cg(src + (int64_t)e * JPR + 4 * q);
                            k[4 * q + 0].add(v.x);
                            k[4 * q + 1].add(v.y);
                            k[4 * q + 2].add(v.z);
                            k[4 * q + 3].add(v.w);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < JPR; ++j) sum[j] = k[j].value();
                }
                if (cnt > 1) {
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1)
#pragma unroll
                        for (int j = 0; j < JPR; ++j) sum[j] += __shfl_xor_sync(0xffffffffu, sum[j], o);
                } else {
#pragma unroll
                    for (int j = 0; j < JPR; ++j) sum[j] = __shfl_sync(0xffffffffu, sum[j], 0);
                }
                if (lane < JPR / 4) {
                    const float sc = -eta / (A.row_mean ? (float)cnt : 1.f);
                    float* base = (F < P.N ? P.U[F] : P.V[F - P.N]) + (int64_t)row * JPR + 4 * lane;
                    float4 u = ld4_cg(base);
                    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < JPR / 4; ++q)
                        if (q == lane) d = make_float4(sum[4 * q], sum[4 * q + 1], sum[4 * q + 2], sum[4 * q + 3]);
                    u.x = fmaf(sc, d.x, u.x);
                    u.y = fmaf(sc, d.y, u.y);
                    u.z = fmaf(sc, d.z, u.z);
                    u.w = fmaf(sc, d.w, u.w);
                    st4(base, u);
                }
            } else {
                const int64_t l = w - n_seg;
                Kahan k;
                k.init();
                for (int64_t pi = lane; pi < gridDim.x; pi += 32) k.add(__ldcg(A.core_part + pi * Pd + l));
                float sum = k.value();
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                const int64_t ntb = t1 - t0;
                if (lane == 0 && ntb > 0) {
                    float* g = P.G + (l / JP) * JPR + (l % JP);
                    const float gv = *g;
                    *g = gv + eta * A.core_scale * (sum / (float)ntb) -
                         eta * A.core_scale * P.lambda_reg * P.inv_nnz * gv;
                }
            }
        }
        if (!grid_barrier(A.bar_count, A.bar_gen, &s_ok)) break;
    }
    if (tid == 0 && !s_ok) atomicExch(A.err_flag, 1);
}

#define S3_FOR_EACH_TENSOR_SHAPE_MB(X) \
    X(3, 2) X(3, 4) X(3, 5) X(3, 8) X(3, 10) X(3, 16) X(3, 20) X(3, 32) X(4, 2) X(4, 4) X(4, 8)

static size_t mb_smem(int N, int JP) {
    size_t q = 1;
    for (int n = 0; n < N - 1; ++n) q *= JP;
    return sizeof(float) * (q * round4(JP) + (size_t)N * kTile * round4(JP));
}

int minibatch_epoch_grid(int N, int JP, int num_sms) {
    int per = 0;
    const size_t smem = mb_smem(N, JP);
#define X(NN, JJ)                                                                            \
    if (N == NN && JP == JJ) {                                                               \
        if (smem > 32 * 1024 &&                                                              \
            cudaFuncSetAttribute(k_mb_epoch<NN, JJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem) != cudaSuccess)                                  \
            return 0;                                                                        \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mb_epoch<NN, JJ>, kTile,   \
                                                          smem) != cudaSuccess)              \
            return 0;                                                                        \
        return per * num_sms;                                                                \
    }
    S3_FOR_EACH_TENSOR_SHAPE_MB(X)
#undef X
    return 0;
}

cudaError_t launch_minibatch_epoch(int N, int JP, const DParams& P, const DGroup& G,
                                   const MbLaunch& L, cudaStream_t s) {
    MbArgs A;
    for (int F = 0; F < kMaxF; ++F) A.contrib[F] = L.contrib[F];
    A.core_part = L.core_part;
    A.bar_count = L.bar_count;
    A.bar_gen = L.bar_gen;
    A.err_flag = L.err_flag;
    A.eta = L.eta;
    A.core_scale = L.core_scale;
    A.row_mean = L.row_mean;
    A.n_batches = L.n_batches;
    DParams Pc = P;
    DGroup Gc = G;
    void* args[] = {&Pc, &Gc, &A};
    const size_t smem = mb_smem(N, JP);
#define X(NN, JJ)                                                                          \
    if (N == NN && JP == JJ && smem > 32 * 1024 &&                                         \
        cudaFuncSetAttribute(k_mb_epoch<NN, JJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem) != cudaSuccess)                                    \
        return cudaErrorInvalidValue;                                                      \
    if (N == NN && JP == JJ)                                                               \
        return cudaLaunchCooperativeKernel((const void*)k_mb_epoch<NN, JJ>, dim3(L.grid),  \
                                           dim3(kTile), args, smem, s);
    S3_FOR_EACH_TENSOR_SHAPE_MB(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace s3
