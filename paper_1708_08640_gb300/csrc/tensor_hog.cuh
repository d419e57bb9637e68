// The FP32 HOGWILD tensor kernel (sm_103a, CUDA cores), shared by the translation units
// that compile its variants (k_tensor_hog2.cu: two lanes per entry; k_tensor_hog4.cu: four
// lanes, and the 4-way one-lane form).
#pragma once
#include <cuda_runtime.h>

#include "hog_common.cuh"
#include "kernels.h"
#include "tensor_fp32.cuh"

namespace s3 {

// ------------------------------------------------------------------ HOGWILD
// One persistent launch per epoch.  CTAs claim tiles in visiting order from a global
// counter; a tile reads the current rows and core (coherent loads: other CTAs update them
// concurrently), writes its row gradients to slots in shared memory, sums every row's slots
// and adds the row steps with vector atomics, and adds its share of the core step to G
// (lock-free, like the rows).
// L adjacent lanes share an entry (3-way: the j1 range is split, the lanes' parts of p2, p3
// and x~ are added with shuffles), so a tile holds T / L entries: fewer entries in flight
// (less staleness) for the same number of threads.
// A CTA has T = hog_compute_threads(N, JP) compute threads and one prefetch warp.  While the
// compute threads work on
// a tile, the prefetch warp loads everything the next tile will read besides the parameters
// (indices, values, slot positions, coupled entries, segment table) into the other metadata
// buffer, so that a tile's critical path starts at its row gathers; the core is re-read at
// the start of every tile, while those gathers are in flight.  The prefetch warp runs its
// own three-stage pipeline: it claims a tile three tiles ahead, reads the array ranges of
// the tile two ahead and copies the tile one ahead, so that only the copies' round trips
// fall into a tile.
// threads of a CTA: T = hog_compute_threads(N, JP) compute threads and the prefetch warp
__host__ __device__ constexpr int hog_threads(int N, int JP) { return hog_compute_threads(N, JP) + 32; }

template <int N, int JP>
struct HogCore {
    static constexpr int Q = ipow_t<JP, N - 1>::v;
    static constexpr int floats = Q * round4(JP);
};

template <int T>
__device__ __forceinline__ void compute_barrier() {
    asm volatile("bar.sync 1, %0;" :: "r"(T) : "memory");
}
// the end of a tile, for the compute threads and the prefetch warp (which run separate loops)
template <int T>
__device__ __forceinline__ void tile_barrier() {
    asm volatile("bar.sync 2, %0;" :: "r"(T + 32) : "memory");
}

// one CTA per SM (two for 4-way tensors up to padded rank 8: at most 112 registers a thread)
template <int N, int JP, int L>
__global__ void __launch_bounds__(hog_threads(N, JP), (N == 4 ? 2 : 1))
k_tensor_hog(DParams P, DGroup Gr, int64_t n_tiles,
                                                            int* tile_counter, const float* eta_p,
                                                            int row_mean, float core_step_scale,
                                                            HogSmem H) {
    static_assert(L == 1 || N == 3, "lanes per entry > 1 is built for 3-way tensors");
    constexpr int JPR = round4(JP);
    constexpr int JH = (JP + L - 1) / L;
    constexpr int kT = hog_compute_threads(N, JP);   // compute threads
    constexpr int ST = kT / L;             // entries per tile at most: rows per stage block
    constexpr int GF = HogCore<N, JP>::floats;
    // coupled rows of the first round are gathered together with the tensor rows when they
    // fit in the registers
    constexpr bool kEarlyCpl = JP <= 10;
    extern __shared__ __align__(16) float smem[];
    float* sG = smem;                  // the core (see hog_layout)
    float* stage = smem + GF;
    const float eta = *eta_p;
    const int tid = threadIdx.x;
    const bool pf = tid >= kT;             // the prefetch warp
    const int lane = tid & 31;
    const int slot = tid / L, lsub = tid % L;
    (void)slot;
    (void)lsub;
    int* meta_base = reinterpret_cast<int*>(smem);
    if (pf) {
        // the prefetch pipeline: the tile in the buffer being computed, the tile to copy next,
        // the tile after it (its ranges in flight) and the claim after that
        int c0 = 0, c1 = 0, claim = 0;
        if (lane == 0) {
            c0 = atomicAdd(tile_counter, 1);
            c1 = atomicAdd(tile_counter, 1);
            claim = atomicAdd(tile_counter, 1);
        }
        int64_t t_cur = __shfl_sync(0xffffffffu, c0, 0);
        int64_t t_after = __shfl_sync(0xffffffffu, c1, 0);
        int64_t lo, hi, lo_after, hi_after;
        hog_ranges(P, Gr, t_cur, n_tiles, H, lane, lo, hi);
        hog_ranges(P, Gr, t_after, n_tiles, H, lane, lo_after, hi_after);
        hog_prefetch<N>(P, Gr, t_cur, n_tiles, lo, hi, meta_base + H.meta[0], H, ST, lane);
        tile_barrier<kT>();
        for (int it = 0; t_cur < n_tiles; ++it) {
            const int64_t t_next = t_after;
            lo = lo_after;
            hi = hi_after;
            t_after = __shfl_sync(0xffffffffu, claim, 0);
            if (lane == 0) claim = atomicAdd(tile_counter, 1);
            hog_ranges(P, Gr, t_after, n_tiles, H, lane, lo_after, hi_after);
            hog_prefetch<N>(P, Gr, t_next, n_tiles, lo, hi, meta_base + H.meta[(it & 1) ^ 1], H, ST, lane);
            tile_barrier<kT>();
            t_cur = t_next;
        }
        return;
    }
    tile_barrier<kT>();
    for (int it = 0;; ++it) {
        const int b = it & 1;
        const int* mb = meta_base + H.meta[b];
        const int64_t t = *reinterpret_cast<const int64_t*>(mb + kMetaTile);
        if (t >= n_tiles) break;
        {
            // the current core (coherent: other CTAs add to it), once the tile's row gathers
            // are in flight.  Thread t reloads the quads that thread t + 32 reduced in the
            // previous tile's core step, not its own: a load after the same thread's reduction
            // to the same address waits until the reduction is done at L2, which put the
            // whole reduction round trip in front of every tile.
            auto reload_core = [&]() {
                for (int l = ((tid + 32) % kT) * 4; l < GF; l += kT * 4) st4(sG + l, ld4_cg(P.G + l));
                compute_barrier<kT>();
            };
            const int nb = mb[kMetaNb];
            const int nc = mb[kMetaNc];
            const HogMeta& M = H.M;
            // the first round of coupled entries: indices from the buffer, rows gathered now
            const bool hc = kEarlyCpl && tid < nc;
            float cu[kEarlyCpl ? JP : 1], cv[kEarlyCpl ? JP : 1];
            int cm = 0;
            float cinv = 0.f;   // 1 / |Omega_Y^{2,k}| of the entry's column, loaded with its rows
            if constexpr (kEarlyCpl) {
                if (hc) {
                    cm = mb[M.c_m + tid];
                    const int ck = mb[M.c_k + tid];
                    load_row<JP, true>(P.U[P.cmode[cm]] + (int64_t)mb[M.c_r + tid] * JPR, cu);
                    load_row<JP, true>(P.V[cm] + (int64_t)ck * JPR, cv);
                    cinv = __ldg(P.inv_cnt[P.N + cm] + ck);
                }
            }
            if constexpr (L == 1) {
                float a[N][JP];
                float inv[N];   // 1 / |Omega^{n,i}| of the entry's rows, loaded with the rows
                if (tid < nb) {
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        const int32_t row = mb[M.tidx + n * ST + tid];
                        load_row<JP, true>(P.U[n] + (int64_t)row * JPR, a[n]);
                        inv[n] = __ldg(P.inv_cnt[n] + row);
                    }
                }
                reload_core();
                if (tid < nb) {
                    float p[N][JP];
                    const float err = __int_as_float(mb[M.tval + tid]) - entry_partials<N, JP>(sG, a, p);
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        const float r = P.lambda_reg * inv[n];
                        float c[JPR];
#pragma unroll
                        for (int j = 0; j < JPR; ++j) c[j] = j < JP ? fmaf(-err, p[n][j], r * a[n][j]) : 0.f;
                        put_slot<JPR>(smem, H, n, mb[M.tpos + n * ST + tid], c);
                        float* sp = stage + (n * ST + tid) * JPR;
#pragma unroll
                        for (int j = 0; j < JP; ++j) sp[j] = n == 0 ? err * a[n][j] : a[n][j];
                    }
                }
            } else {
                // every lane runs the shuffles, so invalid slots work on zero rows
                const bool valid = slot < nb;
                const int sl = valid ? slot : 0;
                int32_t row[3] = {0, 0, 0};
                float a1s[JH], a2[JP], a3[JP];
                float x = 0.f;
                // 1 / |Omega^{n,i}| of mode 1's row and of the row this lane writes in modes 2
                // or 3, loaded with the rows
                float inv1 = 0.f, inv23 = 0.f;
                const int j1base = lsub * JH;
                if (valid) {
#pragma unroll
                    for (int n = 0; n < 3; ++n) row[n] = mb[M.tidx + n * ST + sl];
                    const float* u1 = P.U[0] + (int64_t)row[0] * JPR;
#pragma unroll
                    for (int jj = 0; jj < JH; ++jj) a1s[jj] = j1base + jj < JP ? __ldcg(u1 + j1base + jj) : 0.f;
                    load_row<JP, true>(P.U[1] + (int64_t)row[1] * JPR, a2);
                    load_row<JP, true>(P.U[2] + (int64_t)row[2] * JPR, a3);
                    inv1 = __ldg(P.inv_cnt[0] + row[0]);
                    if (lsub < 2) inv23 = lsub == 0 ? __ldg(P.inv_cnt[1] + row[1]) : __ldg(P.inv_cnt[2] + row[2]);
                    x = __int_as_float(mb[M.tval + sl]);
                } else {
#pragma unroll
                    for (int jj = 0; jj < JH; ++jj) a1s[jj] = 0.f;
#pragma unroll
                    for (int j = 0; j < JP; ++j) { a2[j] = 0.f; a3[j] = 0.f; }
                }
                reload_core();
                float p1s[JH], p2[JP], p3[JP];
                float xt = partials3_lane<JP, L>(sG, j1base, a1s, a2, a3, p1s, p2, p3);
#pragma unroll
                for (int o = 1; o < L; o <<= 1) {
                    xt += __shfl_xor_sync(0xffffffffu, xt, o);
#pragma unroll
                    for (int j = 0; j < JP; ++j) {
                        p2[j] += __shfl_xor_sync(0xffffffffu, p2[j], o);
                        p3[j] += __shfl_xor_sync(0xffffffffu, p3[j], o);
                    }
                }
                if (valid) {
                    const float err = x - xt;
                    // mode 1: this lane's j1 values (the slot's padding is written by the last lane)
                    {
                        const float r = P.lambda_reg * inv1;
                        float* sa = smem + H.off[0] + mb[M.tpos + sl] * slot_stride(JPR);
                        float* sp = stage + (0 * ST + slot) * JPR;
#pragma unroll
                        for (int jj = 0; jj < JH; ++jj) {
                            const int j1 = j1base + jj;
                            if (j1 < JP) {
                                sa[j1] = fmaf(-err, p1s[jj], r * a1s[jj]);
                                sp[j1] = err * a1s[jj];
                            }
                        }
                        if (lsub == L - 1)
#pragma unroll
                            for (int j = JP; j < JPR; ++j) sa[j] = 0.f;
                    }
                    // modes 2 and 3: lanes 0 and 1 write one each (every lane holds the whole
                    // p2 and p3)
                    if (lsub < 2) {
                        // (element-wise selects: a pointer to either register array would move
                        // both arrays to local memory)
                        const int n = 1 + lsub;
                        const float r = P.lambda_reg * inv23;
                        float c[JPR];
                        float* sp = stage + (n * ST + slot) * JPR;
#pragma unroll
                        for (int j = 0; j < JPR; ++j) {
                            const float pj = lsub == 0 ? p2[j < JP ? j : 0] : p3[j < JP ? j : 0];
                            const float aj = lsub == 0 ? a2[j < JP ? j : 0] : a3[j < JP ? j : 0];
                            c[j] = j < JP ? fmaf(-err, pj, r * aj) : 0.f;
                            if (j < JP) sp[j] = aj;
                        }
                        put_slot<JPR>(smem, H, n, mb[M.tpos + n * ST + sl], c);
                    }
                }
            }
            // coupled entries, Eq. (8): the first round from the rows gathered above, then
            // any further rounds in full
            if constexpr (kEarlyCpl) {
                if (hc) hog_coupled_one<JP>(P, smem, H, cm, cinv, mb[M.c_pu + tid], mb[M.c_pv + tid],
                                            __int_as_float(mb[M.c_y + tid]), cu, cv);
            }
            for (int e = kEarlyCpl ? tid + kT : tid; e < nc; e += kT) {
                float u[JP], v[JP];
                const int m = mb[M.c_m + e], k = mb[M.c_k + e];
                load_row<JP, true>(P.U[P.cmode[m]] + (int64_t)mb[M.c_r + e] * JPR, u);
                load_row<JP, true>(P.V[m] + (int64_t)k * JPR, v);
                const float kinv = __ldg(P.inv_cnt[P.N + m] + k);
                hog_coupled_one<JP>(P, smem, H, m, kinv, mb[M.c_pu + e], mb[M.c_pv + e],
                                    __int_as_float(mb[M.c_y + e]), u, v);
            }
            compute_barrier<kT>();
            // the row steps first: their reductions drain while the core step computes, not in
            // front of the next tile's gathers
            hog_flush_meta<JPR>(P, smem, H, mb, eta, row_mean, tid, kT);
            // core: this tile's share of the core step,
            //   G += eta * cs / W * (sum_b e_b a1 o..o aN / n_t - lambda_reg / |Omega| * G)
            if (nb > 0) {
                const float sc = eta * core_step_scale / (float)nb;
                const float rg = eta * core_step_scale * P.lambda_reg * P.inv_nnz;
                CoreTile<N, JP, ST, kT>::apply(stage, nb, sG, P.G, sc, rg, P.nonneg);
            }
        }
        tile_barrier<kT>();
    }
}

static inline size_t hog_core_floats(int N, int JP) {
    size_t q = 1;
    for (int n = 0; n < N - 1; ++n) q *= JP;
    return q * round4(JP);
}

// the HOGWILD kernel's fixed shared memory (floats): the core and a stage of T / L rows
// per mode
static inline size_t hog_fixed_floats(int N, int JP, int L) {
    return hog_core_floats(N, JP) + (size_t)N * (hog_compute_threads(N, JP) / L) * round4(JP);
}

// the whole layout: core, stage, slots, metadata buffers
static inline size_t hog_layout(int N, int JP, int L, const int64_t* max_events,
                                const int64_t* max_segs, int64_t ccap, int nF, HogSmem* H) {
    return hog_meta_smem_floats(round4(JP), N, hog_compute_threads(N, JP) / L, max_events, max_segs, ccap, nF, H,
                                hog_fixed_floats(N, JP, L));
}

// launcher and occupancy query over a list of (N, JP, L) variants, for one translation unit
#define S3_DEFINE_HOG_VARIANTS(SHAPES, LAUNCH_NAME, BLOCKS_NAME)                                 \
    cudaError_t LAUNCH_NAME(int N, int JP, int L, const DParams& P, const DGroup& G,              \
                            int64_t n_tiles, int* tile_counter, int grid, const float* eta,       \
                            int row_mean, float core_step_scale, const int64_t* max_events,       \
                            const int64_t* max_segs, int64_t ccap, cudaStream_t s) {              \
        if (n_tiles <= 0) return cudaSuccess;                                                     \
        HogSmem H{};                                                                              \
        const size_t smem = hog_layout(N, JP, L, max_events, max_segs, ccap, P.N + P.M, &H) *     \
                            sizeof(float);                                                        \
        SHAPES(S3_HOG_LAUNCH_ONE)                                                                 \
        return cudaErrorInvalidValue;                                                             \
    }                                                                                             \
    int BLOCKS_NAME(int N, int JP, int L, size_t smem) {                                          \
        int nb = 0;                                                                               \
        SHAPES(S3_HOG_BLOCKS_ONE)                                                                 \
        return 0;                                                                                 \
    }

#define S3_HOG_LAUNCH_ONE(NN, JJ, LL)                                                          \
    if (N == NN && JP == JJ && L == LL) {                                                      \
        cudaError_t e = prep(k_tensor_hog<NN, JJ, LL>, smem);                                  \
        if (e != cudaSuccess) return e;                                                        \
        k_tensor_hog<NN, JJ, LL><<<grid, hog_threads(NN, JJ), smem, s>>>(P, G, n_tiles, tile_counter, eta, \
                                                           row_mean, core_step_scale, H);      \
        return cudaGetLastError();                                                             \
    }

#define S3_HOG_BLOCKS_ONE(NN, JJ, LL)                                                          \
    if (N == NN && JP == JJ && L == LL) {                                                      \
        if (prep(k_tensor_hog<NN, JJ, LL>, smem) != cudaSuccess) return 0;                     \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tensor_hog<NN, JJ, LL>, hog_threads(NN, JJ), \
                                                          smem) != cudaSuccess)                \
            return 0;                                                                          \
        return nb;                                                                             \
    }

}  // namespace s3
