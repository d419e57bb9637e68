// BF16 tensor-core form of the S3CMTF tensor pass (3-way, ranks up to 32), sm_103a.  A
// kernel variant computes on a JQ x JQ grid of (j1, j2) pairs and a last-mode rank JK:
// (16, 16), (20, 32) or (32, 32) (see BfLayout).  The parameters keep the context's FP32
// layout (rows of P.ld floats, the core P.jp x P.jp x P.ldg); the kernel zero-extends them.
//
// A CTA takes tiles of up to 128 tensor entries (the MMA's M), one entry per thread of its
// four entry warps and per TMEM lane.  The three dense contractions of the per-entry work
// run on the 5th-generation tensor cores (tcgen05.mma, BF16 operands in shared memory, FP32
// accumulators in tensor memory):
//   stage 1   T  = A3 . G_(3)^T      [128 entries x 64 pairs] per MMA group, double-buffered
//                                      (Def. 4, Alg. 3: the core contracted with the last
//                                      mode's rows)
//   partial   P3 = KR . G_(3)        [128 entries x JK]        (p_3 = G x_{-3} {a})
//   core      dG += KR^T . (e o A3)  [128 pairs x JK] per chunk (sum_b e_b a1 o a2 o a3)
// with KR[b] = a1_b (x) a2_b (the Khatri-Rao row of the entry), in chunks of 128 pairs.  The
// rest runs on CUDA cores in FP32: p_1 = T a_2, p_2 = T^T a_1 and x~ = a_1 . p_1 from each
// thread's TMEM lane (packed two-lane FMAs), the error e = x - x~, the row gradients of
// Eq. (8) and the row steps.  FP32 master parameters; BF16 only for the tensor-core operands.
//
// A fifth warp issues every MMA (one elected thread) and hands buffers back and forth with
// the entry warps through mbarriers, so that the MMAs of the next 128 pairs run while the
// entry warps read the current 64, and the next Khatri-Rao chunk is built (and, with two
// buffers, stored) while the current one is multiplied.
//
// The core step: a tile's core gradient (its entries' mean, e / n_b folded into e o A3)
// accumulates in TMEM across the tiles a CTA takes, and is added to G (lock-free,
// red.global.add) every `core_sync` tiles, when the CTA also re-reads the current core into
// its BF16 copy; between two such points the CTA computes with its copy.  With core_sync = 1
// this is the per-tile core step of the FP32 form.
//
// Shared-memory operands (no swizzle, 8 x 16-byte core matrices; see tc.cuh):
//   sG   the core, element (j3, pair) at (pair/8)*(JK/8)*128 + (j3/8)*128 + (j3%8)*16
//        + (pair%8)*2: MN-major B of stage 1 (K = j3, N = pair) and K-major B of the
//        partial (K = pair, N = j3), both read from the same bytes
//   sA3  K-major A of stage 1 (M = entry, K = j3)
//   sKR  one or two 128-pair chunks, K-major A of the partial (M = entry, K = pair) and,
//        read as MN-major, the A operand of the core GEMM (M = pair, K = entry)
//   sEA3 (e / n_b) a3, MN-major B of the core GEMM (K = entry, N = j3)
// TMEM: dG of every chunk [0, NC JK), P3 [COL_P3, + JK), three stage-1 buffers of 64 columns.
#include <cuda_runtime.h>

#include "hog_common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace s3 {

constexpr int kBfTile = 128;    // entries per tile at most (the MMA's M)
constexpr int kChunk = 128;     // pairs per Khatri-Rao chunk (the M of the core GEMM)
constexpr int kTN = 64;         // pairs per stage-1 MMA group (its N)
constexpr int kNB = 3;          // stage-1 TMEM buffers
constexpr int kMaxKr = 2;       // Khatri-Rao chunk buffers in shared memory, at most
constexpr int kBfThreads = kBfTile + 32;   // four entry warps and the MMA warp
// the wait for the MMA warp's last commit before the TMEM is released: never shorter than
// this, whatever the launch's wait limit
constexpr uint64_t kEndWaitNs = 2000000000ull;

// JQ: the side of the (j1, j2) pair grid (the rank of modes 1 and 2 the kernel computes
// at); JK: the last mode's rank, padded to the MMAs' K and N granularity.  (16, 16) and
// (32, 32) for padded ranks up to 16 and 32; (20, 20 x 20 pairs, j3 padded to 32) for
// rank 20, whose pairs (padded to whole chunks of 128) cost half those of (32, 32).
template <int JQ, int JK>
struct BfLayout {
    static_assert((JQ == 16 && JK == 16) || (JQ == 20 && JK == 32) || (JQ == 32 && JK == 32),
                  "the BF16 form is built for padded ranks 16, 20 and 32");
    static_assert(JQ % 2 == 0, "pairs (2k, 2k + 1) share j1");
    static constexpr int NQ = JQ * JQ;                                  // pairs of the grid
    static constexpr int NPAIR = (NQ + kChunk - 1) / kChunk * kChunk;   // in whole chunks
    static constexpr int NC = NPAIR / kChunk;
    static constexpr int NH = NPAIR / kTN;                              // stage-1 MMA groups
    static constexpr uint32_t G_BYTES = JK * NPAIR * 2;
    static constexpr uint32_t A3_BYTES = kBfTile * JK * 2;
    // TMEM columns, each area 32-column aligned, the stage-1 buffers 64-column aligned
    static constexpr uint32_t COL_DG = 0;
    static constexpr uint32_t COL_P3 = (NC * JK + 31) / 32 * 32;
    static constexpr uint32_t COL_T = (COL_P3 + JK + 63) / 64 * 64;
    static constexpr uint32_t TMEM_USED = COL_T + kNB * kTN;
    static constexpr uint32_t TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
    static constexpr int CTAS_PER_SM = TMEM_COLS == 256 ? 2 : 1;
    // two Khatri-Rao buffers when one CTA has the SM (the next chunk is stored while the
    // MMAs read the current one), one when two CTAs share it
    static constexpr int NKR = CTAS_PER_SM == 1 ? 2 : 1;
    static constexpr uint32_t KR1_BYTES = kBfTile * kChunk * 2;
    static constexpr uint32_t KR_BYTES = NKR * KR1_BYTES;
    static constexpr uint32_t EA3_BYTES = kBfTile * JK * 2;
    static constexpr uint32_t OFF_G = 0;
    static constexpr uint32_t OFF_A3 = OFF_G + G_BYTES;
    static constexpr uint32_t OFF_KR = OFF_A3 + A3_BYTES;
    static constexpr uint32_t OFF_EA3 = OFF_KR + KR_BYTES;
    static constexpr uint32_t OFF_SLOTS = OFF_EA3 + EA3_BYTES;   // row gradient slots (floats)
    static_assert(TMEM_USED <= 512, "TMEM budget");
    static_assert(OFF_SLOTS % 16 == 0, "slot rows are written with 16-byte stores");
};

// Dynamic shared memory of at least a third of an SM for layouts that allocate 256 TMEM
// columns (no more than two CTAs share an SM: their allocations fit together), and of more
// than half of one for layouts that allocate 512 (one CTA per SM).
template <int JQ, int JK>
constexpr size_t bf_min_smem() {
    return BfLayout<JQ, JK>::TMEM_COLS == 256 ? 80 * 1024 : 116 * 1024;
}

// mbarriers of the kernel
enum {
    kBarA3 = 0,                 // entry warps: the tile's A3 is in shared memory (or: no more
                                // tiles)
    kBarKr = 1,                 // [kMaxKr] entry warps: a Khatri-Rao chunk (and, first, e o A3)
                                // is in its buffer
    kBarKrFree = 1 + kMaxKr,    // [kMaxKr] MMA warp: the MMAs reading a buffer have completed
    kBarP3 = 1 + 2 * kMaxKr,    // MMA warp: the tile's P3 and dG MMAs have completed
    kBarTFull = 2 + 2 * kMaxKr, // [kNB] MMA warp: a stage-1 buffer holds its 64 pairs of T
    kBarTFree = kBarTFull + kNB,   // [kNB] entry warps: a stage-1 buffer has been read
    kBarEnd = kBarTFree + kNB,     // MMA warp: everything it issued has completed
    kNBars = kBarEnd + 1
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

// Where a bounded wait ran out, for the host's message: the first failure of the launch is
// kept as (site << 24) | (tiles this CTA had finished, at most 2^24 - 1).
enum { kSiteA3 = 1, kSiteTFree = 2, kSiteKr = 3, kSiteEnd = 4, kSiteTFull = 5, kSiteKrFree = 6,
       kSiteP3 = 7 };
__device__ __forceinline__ void record_fail(int* err_flag, int* s_fail, int site, uint32_t tiles) {
    atomicCAS(err_flag, 0, (site << 24) | (int)(tiles < 0xFFFFFFu ? tiles : 0xFFFFFFu));
    *s_fail = 1;
}

// the entry warps' own barrier (the MMA warp runs a separate loop)
__device__ __forceinline__ void entry_sync() {
    asm volatile("bar.sync 1, %0;" :: "r"(kBfTile) : "memory");
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 h) {
    return *reinterpret_cast<uint32_t*>(&h);
}

// The current core as BF16 operand: coalesced float4 reads of G (the layout's
// jp x jp x ldg), each element stored at its place in the (j3, pair) core-matrix layout
// (pair = j1 JQ + j2); the padding past jp stays zero.  Sixteen loads in flight per thread.
template <int JQ, int JK>
__device__ __forceinline__ void load_core_bf16(const DParams& P, uint8_t* smem_raw, int tid) {
    using Lt = BfLayout<JQ, JK>;
    constexpr int U = 16;
    uint8_t* gb = smem_raw + Lt::OFF_G;
    if (P.jp == JQ && P.ldg == JQ) {
        // the layout's rank is the kernel's: compile-time divisions
        constexpr int n4 = Lt::NQ * JQ / 4;                 // float4s
        for (int b = 0; b < n4; b += kBfTile * U) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = b + u * kBfTile + tid;
                v[u] = k < n4 ? ld4_cg(P.G + 4 * k) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = b + u * kBfTile + tid;
                if (k >= n4) continue;
                const int l = 4 * k, pair = l / JQ, j0 = l % JQ;
                const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<__nv_bfloat16*>(gb + g_off<JK>(pair, j0 + i)) = __float2bfloat16_rn(vv[i]);
            }
        }
    } else {
        const int jp = P.jp, ldg = P.ldg;
        const int n4 = jp * jp * ldg / 4;
        for (int b = 0; b < n4; b += kBfTile * U) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = b + u * kBfTile + tid;
                v[u] = k < n4 ? ld4_cg(P.G + 4 * k) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = b + u * kBfTile + tid;
                if (k >= n4) continue;
                const int l = 4 * k, j3 = l % ldg, j12 = l / ldg;
                const int pair = (j12 / jp) * JQ + j12 % jp;
                const float vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<__nv_bfloat16*>(gb + g_off<JK>(pair, j3 + i)) = __float2bfloat16_rn(vv[i]);
            }
        }
    }
}

// The tile's row steps (hog_flush) with the rows' quad count fixed at compile time when the
// context's rows are as wide as the slots (ranks 16, 20, 32): an item's (segment, quad) split
// is then a shift or a multiply instead of a division by a runtime value, and the step's
// division by the event count is taken only under the MEAN rule.  The same sums, steps and
// order as hog_flush; at rank 32 each SM sub-partition runs one entry warp, so every
// instruction of this loop is on the tile's critical path.
template <int JPR>
__device__ __forceinline__ void flush_rows_bf16(const DParams& P, const float* smem, const HogSmem& H,
                                                float eta, int row_mean, int first, int stride) {
    if (P.ld != JPR) {
        hog_flush<JPR>(P, smem, H, eta, row_mean, first, stride);
        return;
    }
    constexpr int SS = slot_stride(JPR), NQ = JPR / 4;
    const int* cnts = reinterpret_cast<const int*>(smem + H.noff);
    for (int F = 0; F < H.nF; ++F) {
        const int nseg = cnts[F];
        const float* sa = smem + H.off[F];
        const int4* tab = reinterpret_cast<const int4*>(smem + H.toff[F]);
        float* base = F < P.N ? P.U[F] : P.V[F - P.N];
        for (int l = first; l < nseg * NQ; l += stride) {
            const int s = l / NQ, q = l % NQ;
            const int4 sg = tab[s];   // row, first slot, events, step scale
            const int32_t rr = sg.x, st = sg.y, cnt = sg.z;
            float4 acc = *reinterpret_cast<const float4*>(sa + st * SS + 4 * q);
            for (int k = 1; k < cnt; ++k) {
                const float4 v = *reinterpret_cast<const float4*>(sa + (st + k) * SS + 4 * q);
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
            float sc = -eta * __int_as_float(sg.w);
            if (row_mean) sc /= (float)cnt;
            float* dst = base + (int64_t)rr * JPR + 4 * q;
            red_add_v4(dst, sc * acc.x, sc * acc.y, sc * acc.z, sc * acc.w);
            if (P.nonneg) red_proj_v4(dst);
        }
    }
}

template <int JQ, int JK>
__global__ void __launch_bounds__(kBfThreads, BfLayout<JQ, JK>::CTAS_PER_SM)
k_tensor_hog_bf16(DParams P, DGroup Gr, int64_t n_tiles, int* tile_counter, const float* eta_p,
                  int row_mean, float core_step_scale, int core_sync, HogSmem H, int* err_flag,
                  uint64_t wait_ns) {
    using Lt = BfLayout<JQ, JK>;
    constexpr int JPR = JQ;          // slot rows (JQ is a multiple of 4)
    constexpr int NQ = Lt::NQ;
    constexpr int NC = Lt::NC;
    constexpr int NH = Lt::NH;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    float* smem = reinterpret_cast<float*>(smem_raw);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[kNBars];
    __shared__ int64_t s_cur, s_nxt;        // this tile and the one claimed after it
    __shared__ int64_t s_lo[32], s_hi[32];  // array ranges of this tile (hog_ranges lanes)
    __shared__ int s_fail;   // set when a bounded wait ran out
    __shared__ int s_go;     // the entry warps take another tile (read by the MMA warp)
    __shared__ int s_fresh;  // the tile's core GEMM starts a new accumulation in TMEM
    __shared__ int s_stop;   // thread 0's view of s_fail, the same for every entry thread
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem_raw);
    const uint32_t sG = sbase + Lt::OFF_G;
    const uint32_t sA3 = sbase + Lt::OFF_A3;
    const uint32_t sKR = sbase + Lt::OFF_KR;
    const uint32_t sEA3 = sbase + Lt::OFF_EA3;
    if (warp == 0) tmem_alloc(&s_tmem, Lt::TMEM_COLS);
    if (tid == 0) {
        mbar_init(&s_bar[kBarA3], kBfTile / 32);
        for (int b = 0; b < kMaxKr; ++b) {
            mbar_init(&s_bar[kBarKr + b], kBfTile / 32);
            mbar_init(&s_bar[kBarKrFree + b], 1);
        }
        mbar_init(&s_bar[kBarP3], 1);
        for (int b = 0; b < kNB; ++b) {
            mbar_init(&s_bar[kBarTFull + b], 1);
            mbar_init(&s_bar[kBarTFree + b], kBfTile / 32);
        }
        mbar_init(&s_bar[kBarEnd], 1);
        s_fail = 0;
        s_fresh = 1;
    }
    // the BF16 core's padding (past the layout's jp, ldg) is zero for the whole launch
    for (int l = tid * 16; l < (int)Lt::G_BYTES; l += kBfThreads * 16)
        st_shared_v4(sG + l, 0u, 0u, 0u, 0u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == kBfTile / 32) {
        // ------------------------------------------------------------ the MMA warp
        if (lane == 0) {
            uint32_t ph_a3 = 0, nh = 0, nk = 0, tiles = 0;
            bool ok = true;
            for (;; ++tiles) {
                if (!mbar_wait_ns(&s_bar[kBarA3], ph_a3, wait_ns)) {
                    record_fail(err_flag, &s_fail, kSiteA3, tiles);
                    ok = false;
                    break;
                }
                ph_a3 ^= 1;
                if (!s_go) break;
                const bool fresh = s_fresh != 0;
                tc_fence_after();
                // stage 1: T[buffer] = A3 . G_(3)^T over 64 pairs (M = 128, N = 64, K = JK)
                constexpr uint32_t id_t = tc_idesc_bf16(128, kTN, 0, 1);
                for (int h = 0; h < NH && ok; ++h, ++nh) {
                    const uint32_t b = nh % kNB;
                    if (nh >= (uint32_t)kNB &&
                        !mbar_wait_ns(&s_bar[kBarTFree + b], ((nh / kNB) - 1) & 1, wait_ns)) {
                        record_fail(err_flag, &s_fail, kSiteTFree, tiles);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < JK / 16; ++ks) {
                        const uint64_t ad = tc_sdesc(sA3 + ks * 256, 128, (JK / 8) * 128);
                        const uint64_t bd = tc_sdesc(sG + (kTN / 8) * h * (JK / 8) * 128 + ks * 256, 128,
                                                     (JK / 8) * 128);
                        tc_mma(tmem + Lt::COL_T + b * kTN, ad, bd, id_t, ks > 0);
                    }
                    tc_commit(&s_bar[kBarTFull + b]);
                }
                if (!ok) break;
                // the Khatri-Rao chunks: P3 += KR . G_(3)[chunk], dG[chunk] += KR^T . (e o A3)
                constexpr uint32_t id_p3 = tc_idesc_bf16(128, JK, 0, 0);
                constexpr uint32_t id_dg = tc_idesc_bf16(128, JK, 1, 1);
                for (int c = 0; c < NC; ++c, ++nk) {
                    const uint32_t kb = nk % Lt::NKR;
                    const uint32_t kr = sKR + kb * Lt::KR1_BYTES;
                    if (!mbar_wait_ns(&s_bar[kBarKr + kb], (nk / Lt::NKR) & 1, wait_ns)) {
                        record_fail(err_flag, &s_fail, kSiteKr, tiles);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int ks = 0; ks < kChunk / 16; ++ks) {
                        const uint64_t ad = tc_sdesc(kr + ks * 256, 128, (kChunk / 8) * 128);
                        const uint64_t bd = tc_sdesc(sG + ((kChunk / 8) * c + 2 * ks) * (JK / 8) * 128,
                                                     (JK / 8) * 128, 128);
                        tc_mma(tmem + Lt::COL_P3, ad, bd, id_p3, (c > 0 || ks > 0));
                    }
#pragma unroll
                    for (int ks = 0; ks < kBfTile / 16; ++ks) {
                        const uint64_t ad = tc_sdesc(kr + ks * 2 * (kChunk / 8) * 128, (kChunk / 8) * 128, 128);
                        const uint64_t bd = tc_sdesc(sEA3 + ks * 256, 128, (kBfTile / 8) * 128);
                        tc_mma(tmem + Lt::COL_DG + c * JK, ad, bd, id_dg, (!fresh || ks > 0));
                    }
                    tc_commit(&s_bar[kBarKrFree + kb]);
                    if (c == NC - 1) tc_commit(&s_bar[kBarP3]);
                }
                if (!ok) break;
            }
            // nothing this thread issued may still run when the TMEM is released
            tc_commit(&s_bar[kBarEnd]);
            if (!mbar_wait_ns(&s_bar[kBarEnd], 0, wait_ns > kEndWaitNs ? wait_ns : kEndWaitNs))
                record_fail(err_flag, &s_fail, kSiteEnd, tiles);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ the entry warps
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        const float eta = *eta_p;
        uint32_t ph_p3 = 0, nh = 0, nk = 0, tiles = 0;
        int since_sync = 0, acc_tiles = 0;
        // Tiles are claimed two ahead and their array ranges read one ahead, so that a tile
        // starts with its ranges (entries, coupled entries, segments) in shared memory.
        if (tid == 0) {
            s_cur = atomicAdd(tile_counter, 1);
            s_nxt = atomicAdd(tile_counter, 1);
        }
        entry_sync();
        if (tid < 32) hog_ranges(P, Gr, s_cur, n_tiles, H, tid, s_lo[tid], s_hi[tid]);
        load_core_bf16<JQ, JK>(P, smem_raw, tid);
        fence_proxy_async();
        if (tid == 0) s_go = s_cur < n_tiles;
        entry_sync();
        for (;;) {
            if (!s_go) {
                // the MMA warp learns that no tile follows
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_bar[kBarA3]);
                break;
            }
            // whether this is the CTA's last tile, read while s_nxt is the same for every
            // thread (thread 0 moves it at the tile's end, and warp 0 may get there first)
            const bool last = s_nxt >= n_tiles;
            // the tile after the next one is claimed now; it is needed only at this one's end
            int claim = 0;
            if (tid == 0) claim = atomicAdd(tile_counter, 1);
            hog_tables_async(P, Gr, s_lo, s_hi, smem, H, tid, kBfTile);
            // ---- this thread's entry and its rows
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
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_bar[kBarA3]);
            // ---- stage 1: p1 = T a2 and p2 = T^T a1 from this lane of T, 64 pairs at a time
            float p1[JQ];
            float2 p2v[JQ / 2];
#pragma unroll
            for (int j = 0; j < JQ; ++j) p1[j] = 0.f;
#pragma unroll
            for (int j = 0; j < JQ / 2; ++j) p2v[j] = make_float2(0.f, 0.f);
#pragma unroll
            for (int h = 0; h < NH; ++h, ++nh) {
                const uint32_t b = nh % kNB;
                bool got = mbar_wait_ns(&s_bar[kBarTFull + b], (nh / kNB) & 1, wait_ns);
                if (!got) record_fail(err_flag, &s_fail, kSiteTFull, tiles);
                // after a wait that ran out the warp reads nothing (an MMA may still write)
                got = __all_sync(0xffffffffu, got);
                tc_fence_after();
                uint32_t r[2][32];
                if (got) {
                    tmem_ld32_nw(lane_base + Lt::COL_T + b * kTN, r[0]);
                    tmem_ld32_nw(lane_base + Lt::COL_T + b * kTN + 32, r[1]);
                    tmem_wait_ld();
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) { r[0][i] = 0u; r[1][i] = 0u; }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_bar[kBarTFree + b]);
                // pairs h*64 + i, i even: (i, i + 1) share j1 (JQ is even); two running
                // accumulators of p1[j1] keep the FMA chains short
                float2 run[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                int run_j1 = -1;
#pragma unroll
                for (int i = 0; i < kTN; i += 2) {
                    const int pair = h * kTN + i;
                    if (pair >= NQ) break;   // past the grid (its T is zero)
                    const int j1 = pair / JQ, j2 = pair % JQ;
                    if (j1 != run_j1) {
                        if (run_j1 >= 0)
                            p1[run_j1] += (run[0].x + run[0].y) + (run[1].x + run[1].y);
                        run[0] = make_float2(0.f, 0.f);
                        run[1] = make_float2(0.f, 0.f);
                        run_j1 = j1;
                    }
                    const float2 tv = make_float2(__uint_as_float(r[i / 32][i % 32]),
                                                  __uint_as_float(r[i / 32][i % 32 + 1]));
                    run[(i / 2) & 1] = __ffma2_rn(tv, make_float2(a2[j2], a2[j2 + 1]), run[(i / 2) & 1]);
                    p2v[j2 / 2] = __ffma2_rn(tv, make_float2(a1[j1], a1[j1]), p2v[j2 / 2]);
                }
                if (run_j1 >= 0) p1[run_j1] += (run[0].x + run[0].y) + (run[1].x + run[1].y);
            }
            // the segment table copies have landed; each segment's step scale is gathered
            // by its row
            cp_async_wait_all();
            hog_tables_damp(P, Gr, s_lo, s_hi, smem, H, tid, kBfTile);
            float xt = 0.f;
#pragma unroll
            for (int j = 0; j < JQ; ++j) xt = fmaf(a1[j], p1[j], xt);
            const float err = valid ? x - xt : 0.f;
            // ---- row gradients of modes 1 and 2 (Eq. (8)) into the tile's slots
            if (valid) {
                const float r0 = P.lambda_reg * inv[0];
                const float r1 = P.lambda_reg * inv[1];
                float c[JPR];
#pragma unroll
                for (int j = 0; j < JQ; ++j) c[j] = fmaf(-err, p1[j], r0 * a1[j]);
                put_slot<JPR>(smem, H, 0, tp[0], c);
#pragma unroll
                for (int j = 0; j < JQ / 2; ++j) {
                    c[2 * j] = fmaf(-err, p2v[j].x, r1 * a2[2 * j]);
                    c[2 * j + 1] = fmaf(-err, p2v[j].y, r1 * a2[2 * j + 1]);
                }
                put_slot<JPR>(smem, H, 1, tp[1], c);
            }
            // ---- (e / n_b) a3: MN-major B of the core GEMM (K = entry, N = j3); the tile's
            //      mean is folded in, so that dG accumulates means across tiles
            {
                const float w = nb > 0 ? err / (float)nb : 0.f;
#pragma unroll
                for (int jg = 0; jg < JK / 8; ++jg) {
                    const uint32_t off = jg * (kBfTile / 8) * 128 + (tid / 8) * 128 + (tid % 8) * 16;
                    st_shared_v4(sEA3 + off, pack_bf16x2(w * a3[8 * jg], w * a3[8 * jg + 1]),
                                 pack_bf16x2(w * a3[8 * jg + 2], w * a3[8 * jg + 3]),
                                 pack_bf16x2(w * a3[8 * jg + 4], w * a3[8 * jg + 5]),
                                 pack_bf16x2(w * a3[8 * jg + 6], w * a3[8 * jg + 7]));
                }
            }
            // ---- Khatri-Rao chunks: products of the BF16 rows, two per instruction
            __nv_bfloat162 b1[JQ], b2[JQ / 2];
#pragma unroll
            for (int j = 0; j < JQ; ++j) b1[j] = __float2bfloat162_rn(a1[j]);
#pragma unroll
            for (int j = 0; j < JQ / 2; ++j) b2[j] = __floats2bfloat162_rn(a2[2 * j], a2[2 * j + 1]);
#pragma unroll
            for (int c = 0; c < NC; ++c, ++nk) {
                uint32_t kr[kChunk / 2];
#pragma unroll
                for (int i = 0; i < kChunk; i += 2) {
                    const int pair = kChunk * c + i;
                    const int pq = pair < NQ ? pair : 0;   // (a compile-time index)
                    kr[i / 2] = pair < NQ ? bf2_bits(__hmul2(b1[pq / JQ], b2[(pq % JQ) / 2])) : 0u;
                }
                // the MMAs of the chunk this buffer held before have read it
                const uint32_t kb = nk % Lt::NKR;
                if (nk >= (uint32_t)Lt::NKR &&
                    !mbar_wait_ns(&s_bar[kBarKrFree + kb], ((nk / Lt::NKR) - 1) & 1, wait_ns))
                    record_fail(err_flag, &s_fail, kSiteKrFree, tiles);
#pragma unroll
                for (int kg = 0; kg < kChunk / 8; ++kg) {
                    const uint32_t off = (tid / 8) * (kChunk / 8) * 128 + kg * 128 + (tid % 8) * 16;
                    st_shared_v4(sKR + kb * Lt::KR1_BYTES + off, kr[4 * kg], kr[4 * kg + 1], kr[4 * kg + 2],
                                 kr[4 * kg + 3]);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_bar[kBarKr + kb]);
            }
            // ---- P3, the mode-3 row gradient, the coupled entries
            bool p3_ok = mbar_wait_ns(&s_bar[kBarP3], ph_p3, wait_ns);
            if (!p3_ok) record_fail(err_flag, &s_fail, kSiteP3, tiles);
            p3_ok = __all_sync(0xffffffffu, p3_ok);
            ph_p3 ^= 1;
            tc_fence_after();
            {
                float p3[JK];
#pragma unroll
                for (int hh = 0; hh < JK / 16; ++hh) {
                    float v[16];
                    if (p3_ok) {
                        tmem_ld16(lane_base + Lt::COL_P3 + 16 * hh, v);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) p3[16 * hh + i] = v[i];
                }
                if (valid) {
                    const float r2 = P.lambda_reg * inv[2];
                    float c[JPR];
#pragma unroll
                    for (int j = 0; j < JQ; ++j) c[j] = fmaf(-err, p3[j], r2 * a3[j]);
                    put_slot<JPR>(smem, H, 2, tp[2], c);
                }
            }
            hog_coupled<JQ>(P, Gr, s_lo, s_hi, smem, H, tid, kBfTile);
            cp_async_wait_all();
            tc_fence_before();
            if (tid == 0) s_stop = s_fail;
            entry_sync();
            // ---- the row steps; the next tile's ranges are read meanwhile (nothing reads
            //      s_lo / s_hi / s_nxt past the barrier above until the one below).  A wait
            //      that ran out leaves this tile's TMEM values undefined: nothing is written.
            const bool failed = s_stop != 0;
            int64_t lo = 0, hi = 0;
            if (tid < 32) hog_ranges(P, Gr, s_nxt, n_tiles, H, tid, lo, hi);
            if (!failed) flush_rows_bf16<JPR>(P, smem, H, eta, row_mean, tid, kBfTile);
            since_sync += 1;
            acc_tiles += nb > 0;
            // ---- the core step of the tiles since the last one, when due (and always at the
            //      CTA's last tile):  G += eta cs / W (sum of tile means - n lambda / |Omega| G)
            if (since_sync >= core_sync || last || failed) {
                const float sc = eta * core_step_scale;
                const float rg = eta * core_step_scale * P.lambda_reg * P.inv_nnz * (float)acc_tiles;
                const __nv_bfloat16* gbf = reinterpret_cast<const __nv_bfloat16*>(smem_raw + Lt::OFF_G);
#pragma unroll 1
                for (int c = 0; c < NC && !failed; ++c) {
                    float d[JK];
#pragma unroll
                    for (int hh = 0; hh < JK / 16; ++hh) {
                        float v[16];
                        tmem_ld16(lane_base + Lt::COL_DG + c * JK + 16 * hh, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) d[16 * hh + i] = v[i];
                    }
                    // lane tid holds pair kChunk*c + tid = j1 JQ + j2 (inside the layout when
                    // j1, j2 < jp, and then its j3 < ldg go out); the regulariser reads the
                    // BF16 copy of G (its term sits far below G's FP32 ulp)
                    const int pair = kChunk * c + tid;
                    const int j1 = pair / JQ, j2 = pair % JQ;
                    const bool inside = !failed && acc_tiles > 0 && pair < NQ && j1 < P.jp && j2 < P.jp;
                    float* g = P.G + ((int64_t)j1 * P.jp + j2) * P.ldg;
#pragma unroll
                    for (int q = 0; q < JK / 4; ++q) {
                        if (!inside || 4 * q >= P.ldg) continue;
                        float gv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) gv[i] = __bfloat162float(gbf[g_off<JK>(pair, 4 * q + i) / 2]);
                        red_add_v4(g + 4 * q, fmaf(sc, d[4 * q], -rg * gv[0]),
                                   fmaf(sc, d[4 * q + 1], -rg * gv[1]),
                                   fmaf(sc, d[4 * q + 2], -rg * gv[2]),
                                   fmaf(sc, d[4 * q + 3], -rg * gv[3]));
                        if (P.nonneg) red_proj_v4(g + 4 * q);
                    }
                }
                tc_fence_before();
                entry_sync();    // every lane has read dG and the old copy before it changes
                load_core_bf16<JQ, JK>(P, smem_raw, tid);
                fence_proxy_async();
                since_sync = 0;
                acc_tiles = 0;
                if (tid == 0) s_fresh = 1;
            } else if (tid == 0) {
                s_fresh = 0;
            }
            __syncwarp();   // warp 0's lanes have read s_nxt before thread 0 moves it
            if (tid < 32) {
                s_lo[tid] = lo;
                s_hi[tid] = hi;
            }
            if (tid == 0) {
                s_cur = s_nxt;
                s_nxt = claim;
                s_go = s_cur < n_tiles && !failed;
            }
            ++tiles;
            entry_sync();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail && tid == 0) atomicCAS(err_flag, 0, 1);
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, Lt::TMEM_COLS);
}

// JP: the rank the form computes at, 16, 20 or 32 (the slot rows hold JP floats)
static size_t bf16_fixed_bytes(int JP) {
    return JP == 16 ? BfLayout<16, 16>::OFF_SLOTS
         : JP == 20 ? BfLayout<20, 32>::OFF_SLOTS
         : JP == 32 ? BfLayout<32, 32>::OFF_SLOTS : 0;
}

static size_t bf16_min_smem(int JP) {
    return JP == 16 ? bf_min_smem<16, 16>() : JP == 20 ? bf_min_smem<20, 32>() : bf_min_smem<32, 32>();
}

size_t tensor_hog_bf16_smem(int JP, const int64_t* max_events, const int64_t* max_segs, int nF) {
    const size_t fixed = bf16_fixed_bytes(JP);
    if (!fixed) return 0;
    const size_t b = hog_smem_floats(JP, max_events, max_segs, nF, nullptr, fixed / sizeof(float)) *
                     sizeof(float);
    return b < bf16_min_smem(JP) ? bf16_min_smem(JP) : b;
}

int tensor_hog_bf16_tile() { return kBfTile; }

int tensor_hog_bf16_core_sync(int JP) {
    // tiles between two core steps of a CTA by default, by the context's padded rank: 1 up to
    // rank 10 (the FP32 form's per-tile step), 2 up to rank 20, 4 above.  On the cfg1 data at
    // rank 16, 1, 2 and 4 tiles gave 7.58, 7.31 and 7.17 ms per epoch and test-RMSE curves
    // within 0.49%, 0.38% and 0.63% of Algorithm 1's over 5 epochs.
    return JP <= 10 ? 1 : JP <= 20 ? 2 : 4;
}

// the dynamic shared-memory limit, and the largest shared-memory carveout
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
                               int core_sync, const HogSmem& H, size_t smem, int* err_flag,
                               uint64_t wait_ns, cudaStream_t s) {
    cudaError_t e = prep_bf16(k_tensor_hog_bf16<JQ, JK>, smem);
    if (e != cudaSuccess) return e;
    k_tensor_hog_bf16<JQ, JK><<<grid, kBfThreads, smem, s>>>(P, G, n_tiles, tile_counter, eta, row_mean,
                                                             core_step_scale, core_sync, H, err_flag,
                                                             wait_ns);
    return cudaGetLastError();
}

cudaError_t launch_tensor_hog_bf16(int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                   int* tile_counter, int grid, const float* eta, int row_mean,
                                   float core_step_scale, int core_sync, const int64_t* max_events,
                                   const int64_t* max_segs, int* err_flag, uint64_t wait_ns,
                                   cudaStream_t s) {
    const size_t fixed = bf16_fixed_bytes(JP);
    if (!fixed || P.N != 3 || core_sync < 1) return cudaErrorInvalidValue;
    if (n_tiles <= 0) return cudaSuccess;
    HogSmem H{};
    size_t smem = hog_smem_floats(JP, max_events, max_segs, P.N + P.M, &H, fixed / sizeof(float)) *
                  sizeof(float);
    if (smem < bf16_min_smem(JP)) smem = bf16_min_smem(JP);
    if (JP == 16)
        return launch_bf16<16, 16>(P, G, n_tiles, tile_counter, grid, eta, row_mean, core_step_scale,
                                   core_sync, H, smem, err_flag, wait_ns, s);
    if (JP == 20)
        return launch_bf16<20, 32>(P, G, n_tiles, tile_counter, grid, eta, row_mean, core_step_scale,
                                   core_sync, H, smem, err_flag, wait_ns, s);
    return launch_bf16<32, 32>(P, G, n_tiles, tile_counter, grid, eta, row_mean, core_step_scale,
                               core_sync, H, smem, err_flag, wait_ns, s);
}

// CTAs of the BF16 kernel that fit on one SM with this much dynamic shared memory (at most
// two at rank 16, one at ranks 20 and 32: their TMEM allocations of 256 or 512 columns must
// fit together), from the device's shared-memory and register limits and the kernel's
// static resources.  (A CTA launched beyond what fits only runs once another has finished:
// the kernel has no inter-CTA waits, so it would find no tile left.)
int tensor_hog_bf16_blocks_per_sm(int JP, size_t smem) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaErrorInvalidValue;
    int cap = 1;
    if (JP == 16) {
        e = prep_bf16(k_tensor_hog_bf16<16, 16>, smem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tensor_hog_bf16<16, 16>);
        cap = BfLayout<16, 16>::CTAS_PER_SM;
    } else if (JP == 20) {
        e = prep_bf16(k_tensor_hog_bf16<20, 32>, smem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tensor_hog_bf16<20, 32>);
        cap = BfLayout<20, 32>::CTAS_PER_SM;
    } else if (JP == 32) {
        e = prep_bf16(k_tensor_hog_bf16<32, 32>, smem);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tensor_hog_bf16<32, 32>);
        cap = BfLayout<32, 32>::CTAS_PER_SM;
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
    const int by_regs = sm_regs / (warp_regs * (kBfThreads / 32));
    int nb = by_smem < by_regs ? by_smem : by_regs;
    return nb < cap ? nb : cap;
}

}  // namespace s3
