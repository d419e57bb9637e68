// BF16 tensor-core form of the S3CMTF tensor pass (3-way, ranks up to 32), sm_103a.  A
// kernel variant computes on a JQ x JQ grid of (j1, j2) pairs and a last-mode rank JK:
// (16, 16), (20, 32) or (32, 32) (see BfLayout).  The parameters keep the context's FP32
// layout (rows of P.ld floats, the core P.jp x P.jp x P.ldg); the kernel zero-extends them.
//
// A CTA of 128 threads takes tiles of 128 tensor entries (the MMA's M), one entry per
// thread and TMEM lane.  The three dense contractions of the per-entry work run on the
// 5th-generation tensor cores (tcgen05.mma, BF16 operands in shared memory, FP32
// accumulators in tensor memory), chunk by chunk of 128 (j1, j2) pairs:
//   stage 1   T  = A3 . G_(3)^T      [128 entries x 128 pairs]   (Def. 4, Alg. 3: the core
//                                      contracted with the last mode's rows)
//   partial   P3 = KR . G_(3)        [128 entries x JK]           (p_3 = G x_{-3} {a})
//   core      dG = KR^T . (e o A3)   [128 pairs x JK]             (sum_b e_b a1 o a2 o a3)
// with KR[b] = a1_b (x) a2_b (the Khatri-Rao row of the entry).  The rest runs on CUDA cores
// in FP32: p_1 = T a_2, p_2 = T^T a_1 and x~ = a_1 . p_1 from each thread's TMEM lane, the
// error e = x - x~, the row gradients of Eq. (8) and the row / core steps.  FP32 master
// parameters; BF16 only for the tensor-core operands.
//
// Shared-memory operands (no swizzle, 8 x 16-byte core matrices; see tc.cuh):
//   sG   the core, element (j3, pair) at (pair/8)*(JK/8)*128 + (j3/8)*128 + (j3%8)*16
//        + (pair%8)*2: MN-major B of stage 1 (K = j3, N = pair) and K-major B of the
//        partial (K = pair, N = j3), both read from the same bytes
//   sA3  K-major A of stage 1 (M = entry, K = j3)
//   sKR  one 128-pair chunk, K-major A of the partial (M = entry, K = pair) and, read as
//        MN-major, the A operand of the core GEMM (M = pair, K = entry)
//   sEA3 e*a3, MN-major B of the core GEMM (K = entry, N = j3)
// TMEM (256 columns, so that two CTAs share an SM): T of one chunk [0, 128), P3
// [128, 128 + JK), dG of one chunk [128 + JK, 128 + 2 JK).
#include <cuda_runtime.h>

#include "hog_common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace s3 {

constexpr int kBfTile = 128;    // entries per tile (the MMA's M)
constexpr int kChunk = 128;     // pairs per chunk (the N of stage 1, the M of the core GEMM)
constexpr int kWaitLimit = 1 << 24;
constexpr uint32_t kTmemCols = 256;
// more than a third of an SM's shared memory, so that no more than two CTAs (2 x 256 TMEM
// columns) are ever resident on one SM
constexpr size_t kBfMinSmem = 80 * 1024;

// JQ: the side of the (j1, j2) pair grid (the rank of modes 1 and 2 the kernel computes
// at); JK: the last mode's rank, padded to the MMAs' K and N granularity.  (16, 16) and
// (32, 32) for padded ranks up to 16 and 32; (20, 20 x 20 pairs, j3 padded to 32) for
// rank 20, whose pairs (padded to whole chunks of 128) cost half those of (32, 32).
template <int JQ, int JK>
struct BfLayout {
    static_assert((JQ == 16 && JK == 16) || (JQ == 20 && JK == 32) || (JQ == 32 && JK == 32),
                  "the BF16 form is built for padded ranks 16, 20 and 32");
    static constexpr int NQ = JQ * JQ;                                  // pairs of the grid
    static constexpr int NPAIR = (NQ + kChunk - 1) / kChunk * kChunk;   // in whole chunks
    static constexpr int NC = NPAIR / kChunk;
    static constexpr uint32_t G_BYTES = JK * NPAIR * 2;
    static constexpr uint32_t A3_BYTES = kBfTile * JK * 2;
    static constexpr uint32_t KR_BYTES = kBfTile * kChunk * 2;
    static constexpr uint32_t EA3_BYTES = kBfTile * JK * 2;
    static constexpr uint32_t OFF_G = 0;
    static constexpr uint32_t OFF_A3 = OFF_G + G_BYTES;
    static constexpr uint32_t OFF_KR = OFF_A3 + A3_BYTES;
    static constexpr uint32_t OFF_EA3 = OFF_KR + KR_BYTES;
    static constexpr uint32_t OFF_SLOTS = OFF_EA3 + EA3_BYTES;   // row gradient slots (floats)
    static constexpr uint32_t COL_T = 0;
    static constexpr uint32_t COL_P3 = kChunk;
    static constexpr uint32_t COL_DG = kChunk + JK;
    static_assert(COL_DG + JK <= kTmemCols, "TMEM budget");
    static_assert(OFF_SLOTS % 16 == 0, "slot rows are written with 16-byte stores");
};

// one 16-byte chunk of 8 BF16 values
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d) : "memory");
}

// byte offset of core element (j3, pair) in sG
template <int JK>
__device__ __forceinline__ uint32_t g_off(int pair, int j3) {
    return (uint32_t)((pair / 8) * (JK / 8) * 128 + (j3 / 8) * 128 + (j3 % 8) * 16 + (pair % 8) * 2);
}

template <int JQ, int JK>
__global__ void __launch_bounds__(kBfTile, 2)
k_tensor_hog_bf16(DParams P, DGroup Gr, int64_t n_tiles, int* tile_counter, const float* eta_p,
                  int row_mean, float core_step_scale, HogSmem H, int* err_flag) {
    using Lt = BfLayout<JQ, JK>;
    constexpr int JPR = JQ;          // slot rows (JQ is a multiple of 4)
    constexpr int NQ = Lt::NQ;
    constexpr int NC = Lt::NC;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int64_t s_cur, s_nxt;        // this tile and the one claimed after it
    __shared__ int64_t s_lo[32], s_hi[32];  // array ranges of this tile (hog_ranges lanes)
    __shared__ int s_fail;   // set when a bounded wait ran out; read after barriers only
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = smem_u32(smem_raw);
    const uint32_t sG = sbase + Lt::OFF_G;
    const uint32_t sA3 = sbase + Lt::OFF_A3;
    const uint32_t sKR = sbase + Lt::OFF_KR;
    const uint32_t sEA3 = sbase + Lt::OFF_EA3;
    const __nv_bfloat16* gbf = reinterpret_cast<const __nv_bfloat16*>(smem_raw + Lt::OFF_G);
    const float eta = *eta_p;
    if (warp == 0) tmem_alloc(&s_tmem, kTmemCols);
    if (tid == 0) {
        mbar_init(&s_mbar, 1);
        s_fail = 0;
    }
    // the BF16 core's padding (past the layout's jp, ldg) is zero for the whole launch
    for (int l = tid * 16; l < (int)Lt::G_BYTES; l += kBfTile * 16)
        st_shared_v4(sbase + Lt::OFF_G + l, 0u, 0u, 0u, 0u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    uint32_t phase = 0;

    // Tiles are claimed two ahead and their array ranges read one ahead, so that a tile
    // starts with its ranges (entries, coupled entries, segments) in shared memory: its
    // segment table goes out as asynchronous copies at once, and its critical path is the
    // entries' index loads, then their rows.
    if (tid == 0) {
        s_cur = atomicAdd(tile_counter, 1);
        s_nxt = atomicAdd(tile_counter, 1);
    }
    __syncthreads();
    if (tid < 32) hog_ranges(P, Gr, s_cur, n_tiles, H, tid, s_lo[tid], s_hi[tid]);
    __syncthreads();
    for (;;) {
        const int64_t t = s_cur;
        if (t >= n_tiles || s_fail) break;
        // the tile after the next one is claimed now; it is needed only at this one's end
        int claim = 0;
        if (tid == 0) claim = atomicAdd(tile_counter, 1);
        hog_tables_async(P, Gr, s_lo, s_hi, smem, H, tid, kBfTile);
        // ---- this thread's entry: indices first, so that their round trip overlaps the
        //      core's reload
        const int64_t e0 = s_lo[0];
        const int nb = (int)(s_hi[0] - e0);
        const bool valid = tid < nb;
        const int64_t e = e0 + tid;
        int32_t row[3] = {0, 0, 0};
        int32_t tp[3] = {0, 0, 0};
        float x = 0.f;
        if (valid) {
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                row[n] = __ldg(Gr.tidx[n] + e);
                tp[n] = __ldg(Gr.tpos[n] + e);
            }
            x = __ldg(Gr.tval + e);
        }
        // ---- the current core as BF16 operand: coalesced float4 reads of G (the layout's
        //      jp x jp x ldg), each element stored at its place in the (j3, pair) core-matrix
        //      layout (pair = j1 JQ + j2); the padding past jp stays zero
        if (P.jp == JQ && P.ldg == JQ) {
            // the layout's rank is the kernel's: pair = l / JQ with compile-time divisions
            for (int l = tid * 4; l < NQ * JQ; l += kBfTile * 4) {
                const float4 v = ld4_cg(P.G + l);
                const int pair = l / JQ, j0 = l % JQ;
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<__nv_bfloat16*>(smem_raw + Lt::OFF_G + g_off<JK>(pair, j0 + i)) =
                        __float2bfloat16_rn(vv[i]);
            }
        } else {
            const int jp = P.jp, ldg = P.ldg;
            for (int l = tid * 4; l < jp * jp * ldg; l += kBfTile * 4) {
                const float4 v = ld4_cg(P.G + l);
                const int j3 = l % ldg, j12 = l / ldg;
                const int pair = (j12 / jp) * JQ + j12 % jp;
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<__nv_bfloat16*>(smem_raw + Lt::OFF_G + g_off<JK>(pair, j3 + i)) =
                        __float2bfloat16_rn(vv[i]);
            }
        }
        // ---- the entry's rows, and the rows' 1 / |Omega^{n,i}| (used after the MMAs)
        float a1[JQ], a2[JQ], a3[JK];
        float inv[3] = {0.f, 0.f, 0.f};
        if (valid) {
            load_row_ld<JQ>(P.U[0] + (int64_t)row[0] * P.ld, P.ld, a1);
            load_row_ld<JQ>(P.U[1] + (int64_t)row[1] * P.ld, P.ld, a2);
            load_row_ld<JK>(P.U[2] + (int64_t)row[2] * P.ld, P.ld, a3);
#pragma unroll
            for (int n = 0; n < 3; ++n) inv[n] = __ldg(P.inv_cnt[n] + row[n]);
        } else {
#pragma unroll
            for (int j = 0; j < JQ; ++j) { a1[j] = 0.f; a2[j] = 0.f; }
#pragma unroll
            for (int j = 0; j < JK; ++j) a3[j] = 0.f;
        }
        // A3 row (K-major, M = entry)
#pragma unroll
        for (int kg = 0; kg < JK / 8; ++kg) {
            const uint32_t off = (tid / 8) * (JK / 8) * 128 + kg * 128 + (tid % 8) * 16;
            st_shared_v4(sA3 + off, pack_bf16x2(a3[8 * kg], a3[8 * kg + 1]),
                         pack_bf16x2(a3[8 * kg + 2], a3[8 * kg + 3]),
                         pack_bf16x2(a3[8 * kg + 4], a3[8 * kg + 5]),
                         pack_bf16x2(a3[8 * kg + 6], a3[8 * kg + 7]));
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        // ---- stage 1, chunk by chunk; p1 and p2 from this thread's lane of T
        float p1[JQ], p2[JQ];
#pragma unroll
        for (int j = 0; j < JQ; ++j) { p1[j] = 0.f; p2[j] = 0.f; }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (tid == 0) {
                tc_fence_after();
                constexpr uint32_t idesc = tc_idesc_bf16(128, kChunk, 0, 1);
#pragma unroll
                for (int ks = 0; ks < JK / 16; ++ks) {
                    const uint64_t ad = tc_sdesc(sA3 + ks * 256, 128, (JK / 8) * 128);
                    const uint64_t bd = tc_sdesc(sG + (kChunk / 8) * c * (JK / 8) * 128 + ks * 256,
                                                 128, (JK / 8) * 128);
                    tc_mma(tmem + Lt::COL_T, ad, bd, idesc, ks > 0);
                }
                tc_commit(&s_mbar);
            }
            if (!mbar_wait(&s_mbar, phase, kWaitLimit)) s_fail = 1;
            phase ^= 1;
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < kChunk / 32; ++q) {
                float v[32];
                tmem_ld32(lane_base + Lt::COL_T + 32 * q, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int pair = kChunk * c + 32 * q + i;
                    if (pair >= NQ) continue;   // past the grid (its T is zero)
                    const int j1 = pair / JQ, j2 = pair % JQ;
                    p1[j1] = fmaf(v[i], a2[j2], p1[j1]);
                    p2[j2] = fmaf(v[i], a1[j1], p2[j2]);
                }
            }
            // every lane has read T before the next chunk's MMA overwrites it; after the
            // last chunk, every thread's table copies have landed too
            if (c == NC - 1) cp_async_wait_all();
            tc_fence_before();
            __syncthreads();
        }
        // the segments' step scales, gathered by the rows the table copies brought
        hog_tables_damp(Gr, smem, H, tid, kBfTile);
        float xt = 0.f;
#pragma unroll
        for (int j = 0; j < JQ; ++j) xt = fmaf(a1[j], p1[j], xt);
        const float err = valid ? x - xt : 0.f;
        // e * a3 (MN-major B of the core GEMM: K = entry, N = j3)
#pragma unroll
        for (int jg = 0; jg < JK / 8; ++jg) {
            const uint32_t off = jg * (kBfTile / 8) * 128 + (tid / 8) * 128 + (tid % 8) * 16;
            st_shared_v4(sEA3 + off, pack_bf16x2(err * a3[8 * jg], err * a3[8 * jg + 1]),
                         pack_bf16x2(err * a3[8 * jg + 2], err * a3[8 * jg + 3]),
                         pack_bf16x2(err * a3[8 * jg + 4], err * a3[8 * jg + 5]),
                         pack_bf16x2(err * a3[8 * jg + 6], err * a3[8 * jg + 7]));
        }
        // ---- partial p3 and core gradient, chunk by chunk of Khatri-Rao rows; each chunk's
        //      share of the core step leaves as soon as its dG is in TMEM:
        //      G += eta cs / W (dG / n_t - lambda_reg / |Omega| G)   (lock-free)
        const float sc = nb > 0 ? eta * core_step_scale / (float)nb : 0.f;
        const float rg = eta * core_step_scale * P.lambda_reg * P.inv_nnz;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int kg = 0; kg < kChunk / 8; ++kg) {
                float w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int pair = kChunk * c + 8 * kg + i;
                    const int pq = pair < NQ ? pair : 0;   // (a compile-time index)
                    w[i] = pair < NQ ? a1[pq / JQ] * a2[pq % JQ] : 0.f;
                }
                const uint32_t off = (tid / 8) * (kChunk / 8) * 128 + kg * 128 + (tid % 8) * 16;
                st_shared_v4(sKR + off, pack_bf16x2(w[0], w[1]), pack_bf16x2(w[2], w[3]),
                             pack_bf16x2(w[4], w[5]), pack_bf16x2(w[6], w[7]));
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                // P3 += KR . G_(3)[chunk]   (M = 128 entries, N = JK, K = 128 pairs)
                constexpr uint32_t id_p3 = tc_idesc_bf16(128, JK, 0, 0);
#pragma unroll
                for (int ks = 0; ks < kChunk / 16; ++ks) {
                    const uint64_t ad = tc_sdesc(sKR + ks * 256, 128, (kChunk / 8) * 128);
                    const uint64_t bd = tc_sdesc(sG + ((kChunk / 8) * c + 2 * ks) * (JK / 8) * 128,
                                                 (JK / 8) * 128, 128);
                    tc_mma(tmem + Lt::COL_P3, ad, bd, id_p3, (c > 0 || ks > 0));
                }
                // dG[chunk] = KR^T . (e o A3)   (M = 128 pairs, N = JK, K = 128 entries)
                constexpr uint32_t id_dg = tc_idesc_bf16(128, JK, 1, 1);
#pragma unroll
                for (int ks = 0; ks < kBfTile / 16; ++ks) {
                    const uint64_t ad = tc_sdesc(sKR + ks * 2 * (kChunk / 8) * 128, (kChunk / 8) * 128, 128);
                    const uint64_t bd = tc_sdesc(sEA3 + ks * 256, 128, (kBfTile / 8) * 128);
                    tc_mma(tmem + Lt::COL_DG, ad, bd, id_dg, ks > 0);
                }
                tc_commit(&s_mbar);
            }
            if (!mbar_wait(&s_mbar, phase, kWaitLimit)) s_fail = 1;
            phase ^= 1;
            tc_fence_after();
            if (nb > 0) {
                // lane tid holds pair kChunk*c + tid = j1 JQ + j2 (inside the layout when
                // j1, j2 < jp, and then its j3 < ldg go out); the regulariser reads the BF16
                // copy of G (its term, eta cs lambda / (W |Omega|) G, sits far below G's
                // FP32 ulp)
                const int pair = kChunk * c + tid;
                const int j1 = pair / JQ, j2 = pair % JQ;
                const bool inside = pair < NQ && j1 < P.jp && j2 < P.jp;
                float* g = P.G + ((int64_t)j1 * P.jp + j2) * P.ldg;
#pragma unroll
                for (int h = 0; h < JK / 16; ++h) {
                    float d[16];
                    tmem_ld16(lane_base + Lt::COL_DG + 16 * h, d);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!inside || 16 * h + 4 * q >= P.ldg) continue;
                        float gv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            gv[i] = __bfloat162float(gbf[g_off<JK>(pair, 16 * h + 4 * q + i) / 2]);
                        red_add_v4(g + 16 * h + 4 * q, fmaf(sc, d[4 * q], -rg * gv[0]),
                                   fmaf(sc, d[4 * q + 1], -rg * gv[1]),
                                   fmaf(sc, d[4 * q + 2], -rg * gv[2]),
                                   fmaf(sc, d[4 * q + 3], -rg * gv[3]));
                        if (P.nonneg) red_proj_v4(g + 16 * h + 4 * q);
                    }
                }
            }
            // every lane has read dG, and the MMAs have read KR, before the next chunk
            tc_fence_before();
            __syncthreads();
        }
        // ---- row gradients (Eq. (8)) into the tile's slots
        {
            float p3[JK];
#pragma unroll
            for (int h = 0; h < JK / 16; ++h) {
                float v[16];
                tmem_ld16(lane_base + Lt::COL_P3 + 16 * h, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) p3[16 * h + i] = v[i];
            }
            if (valid) {
                const float r0 = P.lambda_reg * inv[0];
                const float r1 = P.lambda_reg * inv[1];
                const float r2 = P.lambda_reg * inv[2];
                float c[JPR];
#pragma unroll
                for (int j = 0; j < JQ; ++j) c[j] = fmaf(-err, p1[j], r0 * a1[j]);
                put_slot<JPR>(smem, H, 0, tp[0], c);
#pragma unroll
                for (int j = 0; j < JQ; ++j) c[j] = fmaf(-err, p2[j], r1 * a2[j]);
                put_slot<JPR>(smem, H, 1, tp[1], c);
#pragma unroll
                for (int j = 0; j < JQ; ++j) c[j] = fmaf(-err, p3[j], r2 * a3[j]);
                put_slot<JPR>(smem, H, 2, tp[2], c);
            }
        }
        hog_coupled<JQ>(P, Gr, s_lo, s_hi, smem, H, tid, kBfTile);
        cp_async_wait_all();
        tc_fence_before();
        __syncthreads();
        // the next tile's ranges are read while this one's row steps go out (nothing reads
        // s_lo / s_hi / s_nxt past the barrier above until the one below)
        int64_t lo = 0, hi = 0;
        if (tid < 32) hog_ranges(P, Gr, s_nxt, n_tiles, H, tid, lo, hi);
        hog_flush<JPR>(P, smem, H, eta, row_mean);
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
    tc_fence_before();
    __syncthreads();
    if (s_fail && tid == 0) atomicExch(err_flag, 1);
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// JP: the rank the form computes at, 16, 20 or 32 (the slot rows hold JP floats)
static size_t bf16_fixed_bytes(int JP) {
    return JP == 16 ? BfLayout<16, 16>::OFF_SLOTS
         : JP == 20 ? BfLayout<20, 32>::OFF_SLOTS
         : JP == 32 ? BfLayout<32, 32>::OFF_SLOTS : 0;
}

size_t tensor_hog_bf16_smem(int JP, const int64_t* max_events, const int64_t* max_segs, int nF) {
    const size_t fixed = bf16_fixed_bytes(JP);
    if (!fixed) return 0;
    const size_t b = hog_smem_floats(JP, max_events, max_segs, nF, nullptr, fixed / sizeof(float)) *
                     sizeof(float);
    return b < kBfMinSmem ? kBfMinSmem : b;
}

int tensor_hog_bf16_tile() { return kBfTile; }

// the dynamic shared-memory limit, and the largest shared-memory carveout: two CTAs of this
// kernel need most of an SM's shared memory
template <typename K>
static cudaError_t prep_bf16(K kernel, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int JQ, int JK>
static cudaError_t launch_bf16(const DParams& P, const DGroup& G, int64_t n_tiles, int* tile_counter,
                               int grid, const float* eta, int row_mean, float core_step_scale,
                               const HogSmem& H, size_t smem, int* err_flag, cudaStream_t s) {
    cudaError_t e = prep_bf16(k_tensor_hog_bf16<JQ, JK>, smem);
    if (e != cudaSuccess) return e;
    k_tensor_hog_bf16<JQ, JK><<<grid, kBfTile, smem, s>>>(P, G, n_tiles, tile_counter, eta, row_mean,
                                                          core_step_scale, H, err_flag);
    return cudaGetLastError();
}

cudaError_t launch_tensor_hog_bf16(int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                   int* tile_counter, int grid, const float* eta, int row_mean,
                                   float core_step_scale, const int64_t* max_events,
                                   const int64_t* max_segs, int* err_flag, cudaStream_t s) {
    const size_t fixed = bf16_fixed_bytes(JP);
    if (!fixed || P.N != 3) return cudaErrorInvalidValue;
    if (n_tiles <= 0) return cudaSuccess;
    HogSmem H{};
    size_t smem = hog_smem_floats(JP, max_events, max_segs, P.N + P.M, &H, fixed / sizeof(float)) *
                  sizeof(float);
    if (smem < kBfMinSmem) smem = kBfMinSmem;
    if (JP == 16)
        return launch_bf16<16, 16>(P, G, n_tiles, tile_counter, grid, eta, row_mean, core_step_scale,
                                   H, smem, err_flag, s);
    if (JP == 20)
        return launch_bf16<20, 32>(P, G, n_tiles, tile_counter, grid, eta, row_mean, core_step_scale,
                                   H, smem, err_flag, s);
    return launch_bf16<32, 32>(P, G, n_tiles, tile_counter, grid, eta, row_mean, core_step_scale, H,
                               smem, err_flag, s);
}

// CTAs of the BF16 kernel that fit on one SM with this much dynamic shared memory (at most
// two: two CTAs take all 512 TMEM columns), from the device's shared-memory and register
// limits and the kernel's static resources.  (A CTA launched beyond what fits only runs once
// another has finished: the kernel has no inter-CTA waits, so it would find no tile left.)
int tensor_hog_bf16_blocks_per_sm(int JP, size_t smem) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaErrorInvalidValue;
    if (JP == 16) {
        e = prep_bf16(k_tensor_hog_bf16<16, 16>, smem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tensor_hog_bf16<16, 16>);
    } else if (JP == 20) {
        e = prep_bf16(k_tensor_hog_bf16<20, 32>, smem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tensor_hog_bf16<20, 32>);
    } else if (JP == 32) {
        e = prep_bf16(k_tensor_hog_bf16<32, 32>, smem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tensor_hog_bf16<32, 32>);
    }
    if (e != cudaSuccess) return 0;
    int dev = 0, sm_smem = 0, reserved = 0, sm_regs = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
    const int by_smem = (int)((size_t)sm_smem / per_cta);
    // registers are allocated per warp in units of 256
    const int warp_regs = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = sm_regs / (warp_regs * (kBfTile / 32));
    int nb = by_smem < by_regs ? by_smem : by_regs;
    return nb < 2 ? nb : 2;
}

}  // namespace s3
