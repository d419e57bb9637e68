// Per-tile bookkeeping shared by the HOGWILD kernels (FP32 and BF16 forms): the tile's row
// accumulators in shared memory, its coupled-matrix entries, and the final row steps.
#pragma once
#include "common.cuh"
#include "tensor_fp32.cuh"

namespace s3 {

// per-factor offsets (floats) of the HOGWILD row accumulators in shared memory
struct HogSmem {
    int off[kMaxF];
    int nF;
};

// zero the accumulators of tile t's segments
template <int JPR>
__device__ __forceinline__ void hog_clear(float* smem, const DGroup& Gr, int64_t t, const HogSmem& H) {
    for (int F = 0; F < H.nF; ++F) {
        const int nseg = (int)(Gr.seg_off[F][t + 1] - Gr.seg_off[F][t]);
        float* sa = smem + H.off[F];
        for (int l = threadIdx.x * 4; l < nseg * JPR; l += blockDim.x * 4)
            st4(sa + l, make_float4(0, 0, 0, 0));
    }
}

// Eq. (8), coupled rows, for the coupled entries of tile t: read the current rows, add the
// gradients into the tile's accumulators (shared-memory atomics)
template <int JP>
__device__ __forceinline__ void hog_coupled(const DParams& P, const DGroup& Gr, int64_t t,
                                            float* smem, const HogSmem& H) {
    constexpr int JPR = round4(JP);
    for (int m = 0; m < P.M; ++m) {
        const int c = P.cmode[m];
        const int64_t c0 = Gr.c_off[m][t], c1 = Gr.c_off[m][t + 1];
        const float lm = P.lambda_m;
        for (int64_t e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
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
}

// apply tile t's row steps: one vector atomic per 4 values of every touched row,
// step = -eta * damp[row] * (sum or mean of the row's gradients in the tile)
template <int JPR>
__device__ __forceinline__ void hog_flush(const DParams& P, const DGroup& Gr, int64_t t,
                                          const float* smem, const HogSmem& H, float eta,
                                          int row_mean) {
    for (int F = 0; F < H.nF; ++F) {
        const int64_t sg0 = Gr.seg_off[F][t];
        const int nseg = (int)(Gr.seg_off[F][t + 1] - sg0);
        const float* sa = smem + H.off[F];
        float* base = F < P.N ? P.U[F] : P.V[F - P.N];
        for (int l = threadIdx.x; l < nseg * (JPR / 4); l += blockDim.x) {
            const int s = l / (JPR / 4), q = l % (JPR / 4);
            const int32_t rr = __ldg(Gr.seg_row[F] + sg0 + s);
            const float den = row_mean ? (float)__ldg(Gr.seg_cnt[F] + sg0 + s) : 1.f;
            const float sc = -eta * __ldg(P.damp[F] + rr) / den;
            const float4 v = *reinterpret_cast<const float4*>(sa + s * JPR + 4 * q);
            red_add_v4(base + (int64_t)rr * JPR + 4 * q, sc * v.x, sc * v.y, sc * v.z, sc * v.w);
        }
    }
}

}  // namespace s3
