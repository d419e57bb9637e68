// BF16 tensor-core form of the S3CMTF tensor pass (3-way, padded rank JP = 16), sm_103a.
//
// For a tile of 256 tensor entries (two halves of 128 = the MMA's M) the three dense
// contractions of the per-entry work run on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands in shared memory, FP32 accumulators in tensor memory):
//   stage 1   T  = A3 . G_(3)^T      [128 entries x JP^2 pairs]  (Def. 4, Alg. 3: the core
//                                      contracted with the last mode's rows)
//   partial   P3 = KR . G_(3)        [128 entries x JP]          (p_3 = G x_{-3} {a})
//   core      dG = KR^T . (e o A3)   [JP^2 pairs x JP]           (sum_b e_b a1 o a2 o a3)
// with KR[b] = a1_b (x) a2_b (the Khatri-Rao row of the entry).  The rest runs on CUDA cores
// in FP32: p_1 = T a_2, p_2 = T^T a_1 and x~ = a_1 . p_1 from each thread's TMEM lane, the
// error e = x - x~, the row gradients of Eq. (8) and the row / core steps.  FP32 master
// parameters; BF16 only for the tensor-core operands.
//
// Shared-memory operands (no swizzle, 8 x 16-byte core matrices; see tc.cuh):
//   sG   the core once, element (j3, pair) at (pair/8)*(JP/8)*128 + (j3/8)*128
//        + (j3%8)*16 + (pair%8)*2: MN-major B of stage 1 (K = j3, N = pair) and K-major B of
//        the partial (K = pair, N = j3), both read from the same bytes
//   sA3  per half, K-major A (M = entry, K = j3)
//   sKR  per half and 128-pair chunk, K-major A of the partial (M = entry, K = pair) and,
//        read as MN-major, the A operand of the core GEMM (M = pair, K = entry)
//   sEA3 e*a3 of all 256 entries, MN-major B of the core GEMM (K = entry, N = j3)
// TMEM (512 columns): T of both halves [0, 256), P3 of both halves [256, 256 + 2 JP),
// dG per chunk [256 + 2 JP, 256 + 2 JP + NC JP).
#include <cuda_runtime.h>

#include "hog_common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace s3 {

constexpr int kBfTile = 256;    // entries per tile (two MMA halves)
constexpr int kChunk = 128;     // pairs per chunk (the N of stage 1, the M of the core GEMM)
constexpr int kWaitLimit = 1 << 24;

template <int JP>
struct BfLayout {
    static_assert(JP == 16, "the BF16 form is built for padded rank 16");
    static constexpr int NPAIR = JP * JP;
    static constexpr int NC = NPAIR / kChunk;
    static constexpr uint32_t G_BYTES = JP * NPAIR * 2;
    static constexpr uint32_t A3_BYTES = 128 * JP * 2;           // per half
    static constexpr uint32_t KR_BYTES = 128 * kChunk * 2;       // per half
    static constexpr uint32_t EA3_BYTES = kBfTile * JP * 2;
    static constexpr uint32_t OFF_G = 0;
    static constexpr uint32_t OFF_A3 = OFF_G + G_BYTES;
    static constexpr uint32_t OFF_KR = OFF_A3 + 2 * A3_BYTES;
    static constexpr uint32_t OFF_EA3 = OFF_KR + 2 * KR_BYTES;
    static constexpr uint32_t OFF_ACC = OFF_EA3 + EA3_BYTES;     // row accumulators (floats)
    static constexpr uint32_t COL_T = 0;
    static constexpr uint32_t COL_P3 = 256;
    static constexpr uint32_t COL_DG = 256 + 2 * JP;
    static_assert(COL_DG + NC * JP <= 512, "TMEM budget");
};

// one 16-byte chunk of 8 BF16 values
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d) : "memory");
}

template <int JP>
__global__ void __launch_bounds__(kBfTile, 1)
k_tensor_hog_bf16(DParams P, DGroup Gr, int64_t n_tiles, int* tile_counter, const float* eta_p,
                  int row_mean, float core_step_scale, HogSmem H, int* err_flag) {
    using Lt = BfLayout<JP>;
    constexpr int JPR = JP;          // JP is a multiple of 4
    constexpr int NC = Lt::NC;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_tile;
    __shared__ int s_fail;   // set when a bounded wait ran out; read after barriers only
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int half = tid >> 7, r = tid & 127;
    const uint32_t sbase = smem_u32(smem_raw);
    const uint32_t sG = sbase + Lt::OFF_G;
    const uint32_t sA3 = sbase + Lt::OFF_A3 + half * Lt::A3_BYTES;
    const uint32_t sKR0 = sbase + Lt::OFF_KR;
    const uint32_t sKR = sKR0 + half * Lt::KR_BYTES;
    const uint32_t sEA3 = sbase + Lt::OFF_EA3;
    const float eta = *eta_p;
    if (warp == 0) tmem_alloc(&s_tmem, 512);
    if (tid == 0) {
        mbar_init(&s_mbar, 1);
        s_fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1);
        __syncthreads();
        const int64_t t = s_tile;
        if (t >= n_tiles || s_fail) break;
        // ---- the current core as BF16 operand (two 16-byte chunks of 8 pairs per thread)
        for (int ch = tid; ch < JP * Lt::NPAIR / 8; ch += kBfTile) {
            const int pg = ch / JP, j3 = ch % JP;      // 8 pairs starting at 8 pg, one j3
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __ldcg(P.G + (int64_t)(8 * pg + i) * JPR + j3);
            const uint32_t off = pg * (JP / 8) * 128 + (j3 / 8) * 128 + (j3 % 8) * 16;
            st_shared_v4(sG + off, pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                         pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
        }
        hog_clear<JPR>(smem, Gr, t, H);
        // ---- this thread's entry
        const int64_t e0 = Gr.t_off[t];
        const int nb = (int)(Gr.t_off[t + 1] - e0);
        const bool valid = tid < nb;
        const int64_t e = e0 + tid;
        float a1[JP], a2[JP], a3[JP];
        int32_t row[3] = {0, 0, 0};
        float x = 0.f;
        if (valid) {
            row[0] = __ldg(Gr.tidx[0] + e);
            row[1] = __ldg(Gr.tidx[1] + e);
            row[2] = __ldg(Gr.tidx[2] + e);
            load_row<JP, true>(P.U[0] + (int64_t)row[0] * JPR, a1);
            load_row<JP, true>(P.U[1] + (int64_t)row[1] * JPR, a2);
            load_row<JP, true>(P.U[2] + (int64_t)row[2] * JPR, a3);
            x = __ldg(Gr.tval + e);
        } else {
#pragma unroll
            for (int j = 0; j < JP; ++j) { a1[j] = 0.f; a2[j] = 0.f; a3[j] = 0.f; }
        }
        // A3 row (K-major, M = entry)
#pragma unroll
        for (int kg = 0; kg < JP / 8; ++kg) {
            const uint32_t off = (r / 8) * (JP / 8) * 128 + kg * 128 + (r % 8) * 16;
            st_shared_v4(sA3 + off, pack_bf16x2(a3[8 * kg], a3[8 * kg + 1]),
                         pack_bf16x2(a3[8 * kg + 2], a3[8 * kg + 3]),
                         pack_bf16x2(a3[8 * kg + 4], a3[8 * kg + 5]),
                         pack_bf16x2(a3[8 * kg + 6], a3[8 * kg + 7]));
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        // ---- stage 1, chunk by chunk; p1 and p2 from this thread's lane of T
        float p1[JP], p2[JP];
#pragma unroll
        for (int j = 0; j < JP; ++j) { p1[j] = 0.f; p2[j] = 0.f; }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (tid == 0) {
                tc_fence_after();
                constexpr uint32_t idesc = tc_idesc_bf16(128, kChunk, 0, 1);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < JP / 16; ++ks) {
                        const uint64_t ad = tc_sdesc(sbase + Lt::OFF_A3 + h * Lt::A3_BYTES + ks * 256,
                                                     128, (JP / 8) * 128);
                        const uint64_t bd = tc_sdesc(sG + (kChunk / 8) * c * (JP / 8) * 128 + ks * 256,
                                                     128, (JP / 8) * 128);
                        tc_mma(tmem + Lt::COL_T + h * kChunk, ad, bd, idesc, ks > 0);
                    }
                tc_commit(&s_mbar);
            }
            if (!mbar_wait(&s_mbar, phase, kWaitLimit)) s_fail = 1;
            phase ^= 1;
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < kChunk / 32; ++q) {
                float v[32];
                tmem_ld32(lane_base + Lt::COL_T + half * kChunk + 32 * q, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int pair = kChunk * c + 32 * q + i;
                    const int j1 = pair / JP, j2 = pair % JP;
                    p1[j1] = fmaf(v[i], a2[j2], p1[j1]);
                    p2[j2] = fmaf(v[i], a1[j1], p2[j2]);
                }
            }
            tc_fence_before();
            __syncthreads();
        }
        float xt = 0.f;
#pragma unroll
        for (int j = 0; j < JP; ++j) xt = fmaf(a1[j], p1[j], xt);
        const float err = valid ? x - xt : 0.f;
        // e * a3 (MN-major B of the core GEMM: K = entry, N = j3)
#pragma unroll
        for (int jg = 0; jg < JP / 8; ++jg) {
            const uint32_t off = jg * (kBfTile / 8) * 128 + (tid / 8) * 128 + (tid % 8) * 16;
            st_shared_v4(sEA3 + off, pack_bf16x2(err * a3[8 * jg], err * a3[8 * jg + 1]),
                         pack_bf16x2(err * a3[8 * jg + 2], err * a3[8 * jg + 3]),
                         pack_bf16x2(err * a3[8 * jg + 4], err * a3[8 * jg + 5]),
                         pack_bf16x2(err * a3[8 * jg + 6], err * a3[8 * jg + 7]));
        }
        // ---- partial p3 and core gradient, chunk by chunk of Khatri-Rao rows
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int kg = 0; kg < kChunk / 8; ++kg) {
                float w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int pair = kChunk * c + 8 * kg + i;
                    w[i] = a1[pair / JP] * a2[pair % JP];
                }
                const uint32_t off = (r / 8) * (kChunk / 8) * 128 + kg * 128 + (r % 8) * 16;
                st_shared_v4(sKR + off, pack_bf16x2(w[0], w[1]), pack_bf16x2(w[2], w[3]),
                             pack_bf16x2(w[4], w[5]), pack_bf16x2(w[6], w[7]));
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                // P3[h] += KR[h] . G_(3)[chunk]   (M = 128 entries, N = JP, K = 128 pairs)
                constexpr uint32_t id_p3 = tc_idesc_bf16(128, JP, 0, 0);
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < kChunk / 16; ++ks) {
                        const uint64_t ad = tc_sdesc(sKR0 + h * Lt::KR_BYTES + ks * 256, 128,
                                                     (kChunk / 8) * 128);
                        const uint64_t bd = tc_sdesc(sG + ((kChunk / 8) * c + 2 * ks) * (JP / 8) * 128,
                                                     (JP / 8) * 128, 128);
                        tc_mma(tmem + Lt::COL_P3 + h * JP, ad, bd, id_p3, (c > 0 || ks > 0));
                    }
                // dG[c] = KR^T . (e o A3)   (M = 128 pairs, N = JP, K = 256 entries)
                constexpr uint32_t id_dg = tc_idesc_bf16(128, JP, 1, 1);
#pragma unroll
                for (int ks = 0; ks < kBfTile / 16; ++ks) {
                    const int h = ks / 8, kk = ks % 8;
                    const uint64_t ad = tc_sdesc(sKR0 + h * Lt::KR_BYTES + kk * 2 * (kChunk / 8) * 128,
                                                 (kChunk / 8) * 128, 128);
                    const uint64_t bd = tc_sdesc(sEA3 + ks * 256, 128, (kBfTile / 8) * 128);
                    tc_mma(tmem + Lt::COL_DG + c * JP, ad, bd, id_dg, ks > 0);
                }
                tc_commit(&s_mbar);
            }
            if (!mbar_wait(&s_mbar, phase, kWaitLimit)) s_fail = 1;
            phase ^= 1;
            tc_fence_after();
        }
        // ---- row gradients (Eq. (8)) into the tile's accumulators
        {
            float p3[JP];
            tmem_ld16(lane_base + Lt::COL_P3 + half * JP, p3);
            if (valid) {
                const float r0 = P.lambda_reg * __ldg(P.inv_cnt[0] + row[0]);
                const float r1 = P.lambda_reg * __ldg(P.inv_cnt[1] + row[1]);
                const float r2 = P.lambda_reg * __ldg(P.inv_cnt[2] + row[2]);
                float* s0 = smem + H.off[0] + __ldg(Gr.tpos[0] + e) * JPR;
                float* s1 = smem + H.off[1] + __ldg(Gr.tpos[1] + e) * JPR;
                float* s2 = smem + H.off[2] + __ldg(Gr.tpos[2] + e) * JPR;
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    atomicAdd(s0 + j, fmaf(-err, p1[j], r0 * a1[j]));
                    atomicAdd(s1 + j, fmaf(-err, p2[j], r1 * a2[j]));
                    atomicAdd(s2 + j, fmaf(-err, p3[j], r2 * a3[j]));
                }
            }
        }
        // ---- this tile's share of the core step, lock-free:
        //      G += eta cs / W (dG / n_t - lambda_reg / |Omega| G)
        if (nb > 0) {
            const float sc = eta * core_step_scale / (float)nb;
            const float rg = eta * core_step_scale * P.lambda_reg * P.inv_nnz;
            for (int c = half; c < NC; c += 2) {
                float d[JP];
                tmem_ld16(lane_base + Lt::COL_DG + c * JP, d);
                const int pair = kChunk * c + r;
                float* g = P.G + (int64_t)pair * JPR;
#pragma unroll
                for (int q = 0; q < JP / 4; ++q) {
                    const float4 gv = ld4_cg(g + 4 * q);
                    red_add_v4(g + 4 * q, fmaf(sc, d[4 * q], -rg * gv.x),
                               fmaf(sc, d[4 * q + 1], -rg * gv.y),
                               fmaf(sc, d[4 * q + 2], -rg * gv.z),
                               fmaf(sc, d[4 * q + 3], -rg * gv.w));
                }
            }
        }
        hog_coupled<JP>(P, Gr, t, smem, H);
        tc_fence_before();
        __syncthreads();
        hog_flush<JPR>(P, Gr, t, smem, H, eta, row_mean);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail && tid == 0) atomicExch(err_flag, 1);
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

size_t tensor_hog_bf16_smem(int JP, const int64_t* max_segs, int nF) {
    if (JP != 16) return 0;
    size_t b = BfLayout<16>::OFF_ACC;
    for (int F = 0; F < nF; ++F) b += (size_t)max_segs[F] * JP * sizeof(float);
    return b;
}

cudaError_t launch_tensor_hog_bf16(int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                   int* tile_counter, int grid, const float* eta, int row_mean,
                                   float core_step_scale, const int64_t* max_segs, int* err_flag,
                                   cudaStream_t s) {
    if (JP != 16 || P.N != 3) return cudaErrorInvalidValue;
    if (n_tiles <= 0) return cudaSuccess;
    HogSmem H;
    H.nF = P.N + P.M;
    // accumulator offsets in floats from the start of dynamic shared memory
    size_t off = BfLayout<16>::OFF_ACC / sizeof(float);
    for (int F = 0; F < H.nF; ++F) {
        H.off[F] = (int)off;
        off += (size_t)max_segs[F] * JP;
    }
    const size_t smem = off * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_tensor_hog_bf16<16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_tensor_hog_bf16<16><<<grid, kBfTile, smem, s>>>(P, G, n_tiles, tile_counter, eta, row_mean,
                                                      core_step_scale, H, err_flag);
    return cudaGetLastError();
}

}  // namespace s3
