// The deterministic minibatch epoch as one cooperative launch (sm_103a, FP32 form).
//
// Every batch of the visiting order takes two phases separated by grid-wide barriers:
//   A  the batch's tensor entries (chunks of 32 to 256 entries, one chunk per CTA) and
//      coupled entries (spread over the other CTAs) compute their Eq. (8) row gradients at
//      the batch-start parameters and write them to their segment slots; each CTA with a
//      tensor chunk writes its partial of sum_b e_b a1 o .. o aN;
//   B  one thread per short segment, or one warp per long one, sums a touched row's slots in
//      slot order (compensated) and applies the row step; one warp per core element sums
//      the CTA partials in CTA order and applies the core step.
// The slot layout, the sums' order and the CTA partitioning are fixed, so the epoch is
// deterministic.  Parameters change inside the launch, so every parameter read is a
// coherent (L2) load.  Inputs that do not change (a thread's first entries of the next phase:
// indices, values, slot positions, segment tables, and the batch offsets) are loaded before
// the grid barrier that precedes their phase, so their latency overlaps the wait.  The
// barrier waits are bounded (by the context's wait limit, 2 s by
// default): a CTA whose wait runs out sets the error flag and leaves, and the others leave at
// their next barrier.
#include <cuda_runtime.h>

#include "kernels.h"
#include "tensor_fp32.cuh"

namespace s3 {

__device__ __forceinline__ uint64_t mb_globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier on a cumulative arrival counter that is zero before the launch: the k-th
// barrier of the launch is passed once the counter has reached k * gridDim.x (compared with
// wrap-around arithmetic).  Thread 0 of each CTA publishes the CTA's writes (ordered before
// it by the CTA barrier) with one release add and waits with acquire loads; no CTA resets
// anything, so an arrival is one reduction and a release is seen by the next poll.
// `target` is thread 0's count of arrivals expected so far.  Returns false (for the whole
// CTA) when the wait ran out (after about wait_ns nanoseconds).
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned& target, int* s_ok,
                                             uint64_t wait_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(count) : "memory");
        if ((int)(ld_acquire_u32(count) - target) < 0) {
            const uint64_t t0 = mb_globaltimer();
            while ((int)(ld_acquire_u32(count) - target) < 0) {
                if (mb_globaltimer() - t0 > wait_ns) {
                    *s_ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    __syncthreads();
    return *s_ok != 0;
}

// entries of a phase-A chunk at most: two lanes per entry for 3-way tensors, one for 4-way
__host__ __device__ constexpr int mb_stage_rows(int N) { return N == 3 ? kTile / 2 : kTile; }

struct MbArgs {
    float* contrib[kMaxF];
    float* core_part;       // gridDim.x partials of JP^N floats
    unsigned* bar_count;
    int* err_flag;
    const float* eta;
    float core_scale;
    int row_mean;
    int64_t n_batches;
    uint64_t wait_ns;
};

// How a batch's tensor entries [t0, t1) are cut into phase-A chunks: chunks of 32 to
// mb_stage_rows entries (spread over the CTAs, at least 32 per chunk), chunk c on CTA
// c mod grid; only the first n_part CTAs hold a core partial, which keeps phase B's core sums
// short.  The coupled entries go to the CTAs without a chunk (to all when every one has one).
template <int ST>
struct BatchCut {
    int64_t t0, t1, chunk, n_chunks;
    int n_part, c_first, c_ctas;
    __device__ __forceinline__ BatchCut(int64_t a, int64_t b) : t0(a), t1(b) {
        chunk = min((int64_t)ST, max((int64_t)32, (t1 - t0 + gridDim.x - 1) / gridDim.x));
        n_chunks = (t1 - t0 + chunk - 1) / chunk;
        n_part = (int)min(n_chunks, (int64_t)gridDim.x);
        c_first = n_part < (int)gridDim.x ? n_part : 0;
        c_ctas = (int)gridDim.x - c_first;
    }
    // this CTA's share [cm0, cm1) of a coupled range [c0, c1)
    __device__ __forceinline__ void coupled_share(int64_t c0, int64_t c1, int64_t& cm0, int64_t& cm1) const {
        const int c_me = (int)blockIdx.x - c_first;
        const int64_t cper = (c1 - c0 + c_ctas - 1) / c_ctas;
        cm0 = c0 + (int64_t)c_me * cper;
        cm1 = min(c1, cm0 + cper);
    }
};

// The constant inputs (indices, value, slot positions) of one tensor entry and of one
// coupled entry: a thread's first items of a phase are loaded while the grid barrier before
// the phase is waited for.
template <int N>
struct TensorIn {
    int32_t row[N], pos[N];
    float x;
    __device__ __forceinline__ void load(const DGroup& Gr, int64_t e) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            row[n] = __ldg(Gr.tidx[n] + e);
            pos[n] = __ldg(Gr.tpos[n] + e);
        }
        x = __ldg(Gr.tval + e);
    }
};
struct CoupledIn {
    int32_t r, k, pu, pv;
    float y;
    __device__ __forceinline__ void load(const DGroup& Gr, int m, int64_t e) {
        r = __ldg(Gr.cr[m] + e);
        k = __ldg(Gr.cc[m] + e);
        pu = __ldg(Gr.cpos_u[m] + e);
        pv = __ldg(Gr.cpos_v[m] + e);
        y = __ldg(Gr.cval[m] + e);
    }
};
// a segment's table entries (phase B)
struct SegIn {
    int32_t cnt, row, st;
    __device__ __forceinline__ void load(const DGroup& Gr, int F, int64_t sg) {
        cnt = __ldg(Gr.seg_cnt[F] + sg);
        row = __ldg(Gr.seg_row[F] + sg);
        st = __ldg(Gr.seg_start[F] + sg);
    }
};

template <int N, int JP>
__global__ void __launch_bounds__(kTile) k_mb_epoch(DParams P, DGroup Gr, MbArgs A) {
    constexpr int JPR = round4(JP);
    constexpr int Q = ipow_t<JP, N - 1>::v;
    constexpr int Pd = Q * JP;
    constexpr int ST = mb_stage_rows(N);   // entries per chunk at most: rows per stage block
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_ok;
    // batch offsets, fetched one phase ahead: tensor and first coupled matrix ranges of the
    // batch (by batch parity), and the current batch's segment ranges per factor
    __shared__ __align__(8) int64_t s_toff[2][2];
    __shared__ __align__(8) int64_t s_coff[2][2];
    __shared__ __align__(8) int64_t s_seg[kMaxF][2];
    __shared__ int32_t s_nlong[kMaxF];
    __shared__ int64_t s_long_begin[kMaxF + 1], s_short_begin[kMaxF + 1];
    float* sG = smem;
    float* stage = smem + Q * JPR;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nF = P.N + P.M;
    const float eta = *A.eta;
    const int64_t gthread = (int64_t)blockIdx.x * kTile + tid;
    const int64_t nthreads = (int64_t)gridDim.x * kTile;
    const int64_t gwarp = gthread >> 5;
    const int64_t nwarps = nthreads >> 5;
    constexpr int L3 = 2;   // lanes per entry of a 3-way chunk
    const int ent = N == 3 ? tid / L3 : tid;   // this thread's entry of a chunk
    unsigned bar_target = 0;
    if (tid == 0) {
        s_ok = 1;
        if (A.n_batches > 0) {
            s_toff[0][0] = Gr.t_off[0];
            s_toff[0][1] = Gr.t_off[1];
            if (P.M > 0) {
                s_coff[0][0] = Gr.c_off[0][0];
                s_coff[0][1] = Gr.c_off[0][1];
            }
        }
    }
    __syncthreads();
    // a thread's first tensor and coupled entries of the next phase A
    TensorIn<N> pre_t;
    CoupledIn pre_c;
    bool have_t = false, have_c = false;
    auto prefetch_a = [&](int par) {
        const BatchCut<ST> cut(s_toff[par][0], s_toff[par][1]);
        have_t = false;
        have_c = false;
        if ((int64_t)blockIdx.x < cut.n_chunks) {
            const int64_t my0 = cut.t0 + (int64_t)blockIdx.x * cut.chunk;
            const int nb = (int)min(cut.chunk, cut.t1 - my0);
            if (ent < nb) {
                pre_t.load(Gr, my0 + ent);
                have_t = true;
            }
        }
        if (P.M > 0 && (int)blockIdx.x >= cut.c_first) {
            int64_t cm0, cm1;
            cut.coupled_share(s_coff[par][0], s_coff[par][1], cm0, cm1);
            if (cm0 + tid < cm1) {
                pre_c.load(Gr, 0, cm0 + tid);
                have_c = true;
            }
        }
    };
    if (A.n_batches > 0) prefetch_a(0);
    for (int64_t b = 0; b < A.n_batches; ++b) {
        const int par = (int)(b & 1);
        // ------------------------------------------------ phase A: gradients into slots
        // offsets of the next phases, copied to shared memory while this phase runs
        if (tid < nF) {
            cp_async8(&s_seg[tid][0], Gr.seg_off[tid] + b);
            cp_async8(&s_seg[tid][1], Gr.seg_off[tid] + b + 1);
            cp_async4(&s_nlong[tid], Gr.seg_nlong[tid] + b);
        } else if (tid == 32 && b + 1 < A.n_batches) {
            cp_async8(&s_toff[par ^ 1][0], Gr.t_off + b + 1);
            cp_async8(&s_toff[par ^ 1][1], Gr.t_off + b + 2);
        } else if (tid == 64 && b + 1 < A.n_batches && P.M > 0) {
            cp_async8(&s_coff[par ^ 1][0], Gr.c_off[0] + b + 1);
            cp_async8(&s_coff[par ^ 1][1], Gr.c_off[0] + b + 2);
        }
        const BatchCut<ST> cut(s_toff[par][0], s_toff[par][1]);
        const int64_t t0 = cut.t0, t1 = cut.t1;
        CoreAcc<N, JP, ST> acc;
        acc.init();
        // the core is loaded once the first chunk's rows are in flight (inside the loop)
        bool core_loaded = false;
        auto load_core = [&]() {
            if (!core_loaded) {
                for (int l = tid * 4; l < Q * JPR; l += kTile * 4) st4(sG + l, ld4_cg(P.G + l));
                __syncthreads();
                core_loaded = true;
            }
        };
        for (int64_t ch = blockIdx.x; ch < cut.n_chunks; ch += gridDim.x) {
            const int64_t my0 = t0 + ch * cut.chunk;
            const int nb = (int)min(cut.chunk, t1 - my0);
            const bool first = ch == (int64_t)blockIdx.x;
            if constexpr (N == 3) {
                // two lanes per entry (halves each entry's latency); invalid slots run on zeros so
                // that every lane takes part in the shuffles
                constexpr int L = L3;
                constexpr int JH = (JP + L - 1) / L;
                const int slot = ent, lsub = tid % L;
                const bool valid = slot < nb;
                TensorIn<3> in;
                if (valid) {
                    if (first && have_t) in = pre_t;
                    else in.load(Gr, my0 + slot);
                }
                float a1s[JH], a2[JP], a3[JP];
                const int j1base = lsub * JH;
                if (valid) {
                    const float* u1 = P.U[0] + (int64_t)in.row[0] * JPR;
#pragma unroll
                    for (int jj = 0; jj < JH; ++jj) a1s[jj] = j1base + jj < JP ? __ldcg(u1 + j1base + jj) : 0.f;
                    load_row<JP, true>(P.U[1] + (int64_t)in.row[1] * JPR, a2);
                    load_row<JP, true>(P.U[2] + (int64_t)in.row[2] * JPR, a3);
                } else {
#pragma unroll
                    for (int jj = 0; jj < JH; ++jj) a1s[jj] = 0.f;
#pragma unroll
                    for (int j = 0; j < JP; ++j) { a2[j] = 0.f; a3[j] = 0.f; }
                }
                load_core();
                float p1s[JH], p2[JP], p3[JP];
                float xt = partials3_lane<JP, L>(sG, j1base, a1s, a2, a3, p1s, p2, p3);
                xt += __shfl_xor_sync(0xffffffffu, xt, 1);
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    p2[j] += __shfl_xor_sync(0xffffffffu, p2[j], 1);
                    p3[j] += __shfl_xor_sync(0xffffffffu, p3[j], 1);
                }
                if (valid) {
                    const float err = in.x - xt;
                    // mode 1: this lane's j1 values (its slot holds all JPR components: the two
                    // lanes write disjoint ones, the padding is written by lane 1)
                    const float r1 = P.lambda_reg * __ldg(P.inv_cnt[0] + in.row[0]);
                    float* d1 = A.contrib[0] + (int64_t)in.pos[0] * JPR;
                    float* sp1 = stage + (0 * ST + slot) * JPR;
#pragma unroll
                    for (int jj = 0; jj < JH; ++jj) {
                        const int j1 = j1base + jj;
                        if (j1 < JP) {
                            d1[j1] = fmaf(-err, p1s[jj], r1 * a1s[jj]);
                            sp1[j1] = err * a1s[jj];
                        }
                    }
                    if (lsub == L - 1)
                        for (int j = JP; j < JPR; ++j) d1[j] = 0.f;
                    // modes 2 and 3: each lane writes the whole slot of one mode
                    // (element-wise selects keep p2, p3, a2, a3 in registers)
                    const int n = 1 + lsub;
                    const int rown = lsub == 0 ? in.row[1] : in.row[2];
                    const int posn = lsub == 0 ? in.pos[1] : in.pos[2];
                    const float r = P.lambda_reg * __ldg(P.inv_cnt[n] + rown);
                    float c[JPR];
                    float* sp = stage + (n * ST + slot) * JPR;
#pragma unroll
                    for (int j = 0; j < JPR; ++j) {
                        const float pj = lsub == 0 ? p2[j < JP ? j : 0] : p3[j < JP ? j : 0];
                        const float aj = lsub == 0 ? a2[j < JP ? j : 0] : a3[j < JP ? j : 0];
                        c[j] = j < JP ? fmaf(-err, pj, r * aj) : 0.f;
                        if (j < JP) sp[j] = aj;
                    }
                    float* dst = A.contrib[n] + (int64_t)posn * JPR;
#pragma unroll
                    for (int q = 0; q < JPR / 4; ++q)
                        st4(dst + 4 * q, make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
                }
            } else {
                const bool valid = tid < nb;
                TensorIn<N> in;
                float a[N][JP];
                if (valid) {
                    if (first && have_t) in = pre_t;
                    else in.load(Gr, my0 + tid);
#pragma unroll
                    for (int n = 0; n < N; ++n) load_row<JP, true>(P.U[n] + (int64_t)in.row[n] * JPR, a[n]);
                }
                load_core();
                if (valid) {
                    float p[N][JP];
                    const float xt = partials4<JP>(sG, a[0], a[1], a[2], a[3], p[0], p[1], p[2], p[3]);
                    const float err = in.x - xt;
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        const float r = P.lambda_reg * __ldg(P.inv_cnt[n] + in.row[n]);
                        float c[JPR];
#pragma unroll
                        for (int j = 0; j < JPR; ++j) c[j] = j < JP ? fmaf(-err, p[n][j], r * a[n][j]) : 0.f;
                        float* dst = A.contrib[n] + (int64_t)in.pos[n] * JPR;
#pragma unroll
                        for (int q = 0; q < JPR / 4; ++q)
                            st4(dst + 4 * q, make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
                        float* sp = stage + (n * ST + tid) * JPR;
#pragma unroll
                        for (int j = 0; j < JP; ++j) sp[j] = n == 0 ? err * a[n][j] : a[n][j];
                    }
                }
            }
            __syncthreads();
            acc.add_tile(stage, nb);
            __syncthreads();
        }
        // coupled entries of the batch, spread evenly over the CTAs without a tensor chunk
        // (over all CTAs when every one has one)
        for (int m = 0; m < P.M && (int)blockIdx.x >= cut.c_first; ++m) {
            const int c = P.cmode[m];
            const int64_t c0 = m == 0 ? s_coff[par][0] : Gr.c_off[m][b];
            const int64_t c1 = m == 0 ? s_coff[par][1] : Gr.c_off[m][b + 1];
            int64_t cm0, cm1;
            cut.coupled_share(c0, c1, cm0, cm1);
            for (int64_t e = cm0 + tid; e < cm1; e += kTile) {
                CoupledIn in;
                if (m == 0 && e == cm0 + tid && have_c) in = pre_c;
                else in.load(Gr, m, e);
                float u[JP], v[JP];
                load_row<JP, true>(P.U[c] + (int64_t)in.r * JPR, u);
                load_row<JP, true>(P.V[m] + (int64_t)in.k * JPR, v);
                float yh = 0.f;
#pragma unroll
                for (int j = 0; j < JP; ++j) yh = fmaf(u[j], v[j], yh);
                const float am = -P.lambda_m * (in.y - yh);
                const float rv = P.lambda_m * P.lambda_reg * __ldg(P.inv_cnt[P.N + m] + in.k);
                float du[JPR], dv[JPR];
#pragma unroll
                for (int j = 0; j < JPR; ++j) {
                    du[j] = j < JP ? am * v[j] : 0.f;
                    dv[j] = j < JP ? fmaf(am, u[j], rv * v[j]) : 0.f;
                }
                float* pu = A.contrib[c] + (int64_t)in.pu * JPR;
                float* pv = A.contrib[P.N + m] + (int64_t)in.pv * JPR;
#pragma unroll
                for (int q = 0; q < JPR / 4; ++q) {
                    st4(pu + 4 * q, make_float4(du[4 * q], du[4 * q + 1], du[4 * q + 2], du[4 * q + 3]));
                    st4(pv + 4 * q, make_float4(dv[4 * q], dv[4 * q + 1], dv[4 * q + 2], dv[4 * q + 3]));
                }
            }
        }
        if ((int)blockIdx.x < cut.n_part) acc.store(A.core_part + (int64_t)blockIdx.x * Pd, stage);
        // phase B's segment ranges (each group lists its long segments, of more than
        // kShortSeg events, first) and this thread's first segments, loaded before the barrier
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            s_long_begin[0] = s_short_begin[0] = 0;
            for (int F = 0; F < nF; ++F) {
                s_long_begin[F + 1] = s_long_begin[F] + s_nlong[F];
                s_short_begin[F + 1] = s_short_begin[F] + (s_seg[F][1] - s_seg[F][0]) - s_nlong[F];
            }
        }
        __syncthreads();
        const int64_t n_short = s_short_begin[nF], n_long = s_long_begin[nF];
        const int64_t n_items = Pd + n_long;
        SegIn pre_s, pre_l;
        int pre_sF = 0, pre_lF = 0;
        if (gthread < n_short) {
            int F = 0;
            while (F + 1 < nF && gthread >= s_short_begin[F + 1]) ++F;
            pre_sF = F;
            pre_s.load(Gr, F, s_seg[F][0] + s_nlong[F] + (gthread - s_short_begin[F]));
        }
        if (gwarp >= Pd && gwarp < n_items) {
            const int64_t wl = gwarp - Pd;
            int F = 0;
            while (F + 1 < nF && wl >= s_long_begin[F + 1]) ++F;
            pre_lF = F;
            pre_l.load(Gr, F, s_seg[F][0] + (wl - s_long_begin[F]));
        }
        if (!grid_barrier(A.bar_count, bar_target, &s_ok, A.wait_ns)) break;
        // ------------------------------------------------ phase B: ordered sums and steps
        // pass 1: a thread per short segment (the common case: rows touched a few times)
        for (int64_t w = gthread; w < n_short; w += nthreads) {
            int F;
            SegIn sgi;
            if (w == gthread) {
                F = pre_sF;
                sgi = pre_s;
            } else {
                F = 0;
                while (F + 1 < nF && w >= s_short_begin[F + 1]) ++F;
                sgi.load(Gr, F, s_seg[F][0] + s_nlong[F] + (w - s_short_begin[F]));
            }
            const float* src = A.contrib[F] + (int64_t)sgi.st * JPR;
            const float sc = -eta / (A.row_mean ? (float)sgi.cnt : 1.f);
            float* base = (F < P.N ? P.U[F] : P.V[F - P.N]) + (int64_t)sgi.row * JPR;
            float4 row[JPR / 4];   // loaded with the slots
#pragma unroll
            for (int q = 0; q < JPR / 4; ++q) row[q] = ld4_cg(base + 4 * q);
            Kahan k[JPR];
#pragma unroll
            for (int j = 0; j < JPR; ++j) k[j].init();
            rows_sum<JPR / 4>(src, JPR, 0, 1, sgi.cnt, k);
#pragma unroll
            for (int q = 0; q < JPR / 4; ++q) {
                float4 u = row[q];
                u.x = fmaf(sc, k[4 * q].value(), u.x);
                u.y = fmaf(sc, k[4 * q + 1].value(), u.y);
                u.z = fmaf(sc, k[4 * q + 2].value(), u.z);
                u.w = fmaf(sc, k[4 * q + 3].value(), u.w);
                if (P.nonneg) project4(u);
                st4(base + 4 * q, u);
            }
        }
        // pass 2: a warp per long segment and per core element
        // (the core elements first: every batch has them, and their warps start at once)
        for (int64_t w = gwarp; w < n_items; w += nwarps) {
            if (w >= Pd) {
                int F;
                SegIn sgi;
                if (w == gwarp) {
                    F = pre_lF;
                    sgi = pre_l;
                } else {
                    const int64_t wl = w - Pd;
                    F = 0;
                    while (F + 1 < nF && wl >= s_long_begin[F + 1]) ++F;
                    sgi.load(Gr, F, s_seg[F][0] + (wl - s_long_begin[F]));
                }
                float* base = (F < P.N ? P.U[F] : P.V[F - P.N]) + (int64_t)sgi.row * JPR + 4 * (lane % (JPR / 4));
                const float4 u0 = ld4_cg(base);   // loaded with the slots (used by the first lanes)
                float sum[JPR];
                {
                    Kahan k[JPR];
#pragma unroll
                    for (int j = 0; j < JPR; ++j) k[j].init();
                    rows_sum<JPR / 4>(A.contrib[F] + (int64_t)sgi.st * JPR, JPR, lane, 32, sgi.cnt, k);
#pragma unroll
                    for (int j = 0; j < JPR; ++j) sum[j] = k[j].value();
                }
#pragma unroll
                for (int o = 1; o < 32; o <<= 1)
#pragma unroll
                    for (int j = 0; j < JPR; ++j) sum[j] += __shfl_xor_sync(0xffffffffu, sum[j], o);
                if (lane < JPR / 4) {
                    const float sc = -eta / (A.row_mean ? (float)sgi.cnt : 1.f);
                    float4 u = u0;
                    float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < JPR / 4; ++q)
                        if (q == lane) d = make_float4(sum[4 * q], sum[4 * q + 1], sum[4 * q + 2], sum[4 * q + 3]);
                    u.x = fmaf(sc, d.x, u.x);
                    u.y = fmaf(sc, d.y, u.y);
                    u.z = fmaf(sc, d.z, u.z);
                    u.w = fmaf(sc, d.w, u.w);
                    if (P.nonneg) project4(u);
                    st4(base, u);
                }
            } else {
                const int64_t l = w;
                float* g = P.G + (l / JP) * JPR + (l % JP);
                const float gv = lane == 0 ? __ldcg(g) : 0.f;   // loaded with the partials
                Kahan k;
                k.init();
                // four partials' loads in flight per lane (predicated), added in partial order
                for (int64_t pi = lane; pi < cut.n_part; pi += 128) {
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = pi + 32 * u < cut.n_part ? __ldcg(A.core_part + (pi + 32 * u) * Pd + l) : 0.f;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (pi + 32 * u < cut.n_part) k.add(v[u]);
                }
                float sum = k.value();
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                const int64_t ntb = t1 - t0;
                bool core_elem = true;   // S3CMTF-CP: only the diagonal is a parameter
                if (P.cp) {
                    int64_t r = l;
                    const int j0 = (int)(r % JP);
                    for (int n = 1; n < N; ++n) {
                        r /= JP;
                        core_elem &= (int)(r % JP) == j0;
                    }
                }
                if (lane == 0 && ntb > 0 && core_elem) {
                    const float nv = gv + eta * A.core_scale * (sum / (float)ntb) -
                                     eta * A.core_scale * P.lambda_reg * P.inv_nnz * gv;
                    *g = P.nonneg ? project(nv) : nv;
                }
            }
        }
        // the next batch's first entries, loaded before the barrier
        if (b + 1 < A.n_batches) prefetch_a(par ^ 1);
        if (!grid_barrier(A.bar_count, bar_target, &s_ok, A.wait_ns)) break;
    }
    if (tid == 0 && !s_ok) atomicExch(A.err_flag, 1);
}

#define S3_FOR_EACH_TENSOR_SHAPE_MB(X) \
    X(3, 2) X(3, 4) X(3, 5) X(3, 8) X(3, 10) X(3, 16) X(3, 20) X(3, 32) X(4, 2) X(4, 4) X(4, 8)

static size_t mb_smem(int N, int JP) {
    size_t q = 1;
    for (int n = 0; n < N - 1; ++n) q *= JP;
    return sizeof(float) * (q * round4(JP) + (size_t)N * mb_stage_rows(N) * round4(JP));
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
    A.err_flag = L.err_flag;
    A.eta = L.eta;
    A.core_scale = L.core_scale;
    A.row_mean = L.row_mean;
    A.n_batches = L.n_batches;
    A.wait_ns = L.wait_ns;
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
