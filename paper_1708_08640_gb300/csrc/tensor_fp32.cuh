// FP32 (CUDA-core) per-tensor-entry arithmetic of S3CMTF, templated on the order N and
// the padded rank JP.  Shared by the minibatch/gradient, HOGWILD and forward kernels.
//
// For an entry alpha = (i_1..i_N) with rows a_n = u^(n)_{i_n} the kernels need
//   x~    = G x {a}                    (Eq. (4))
//   p_n   = G x_{-n} {a}, n = 1..N      (the partial products of Eq. (8), Eq. (3))
//   e a_1 o a_2 o ... o a_N            (the data part of the core gradient, Eq. (8))
// S3CMTF-opt (Section 3.5, Alg. 3) gets the partials from the intermediate data S by
// Collapse and element-wise division.  Here they come from one sweep over the core that
// reuses the contraction with the last mode's row: T = G x_N a_N gives p_n (n < N) by
// contracting T with the other rows, and the same core values weighted by the products of
// the first N-1 rows give p_N.  No division, so zero rows are harmless.
#pragma once
#include "common.cuh"

namespace s3 {

template <int B, int E>
struct ipow_t { static constexpr int v = B * ipow_t<B, E - 1>::v; };
template <int B>
struct ipow_t<B, 0> { static constexpr int v = 1; };

// loads JP values of a row (stride JPR, 16-byte aligned) into registers
template <int JP, bool kCoherent>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&a)[JP]) {
    constexpr int JPR = round4(JP);
    float t[JPR];
#pragma unroll
    for (int q = 0; q < JPR / 4; ++q) {
        float4 v = kCoherent ? ld4_cg(p + 4 * q) : ld4_nc(p + 4 * q);
        t[4 * q + 0] = v.x;
        t[4 * q + 1] = v.y;
        t[4 * q + 2] = v.z;
        t[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < JP; ++j) a[j] = t[j];
}

// one core row (the last mode) from shared memory
template <int JP>
__device__ __forceinline__ void load_grow(const float* __restrict__ g, float (&r)[JP]) {
    constexpr int JPR = round4(JP);
    float t[JPR];
#pragma unroll
    for (int q = 0; q < JPR / 4; ++q) {
        float4 v = *reinterpret_cast<const float4*>(g + 4 * q);
        t[4 * q + 0] = v.x;
        t[4 * q + 1] = v.y;
        t[4 * q + 2] = v.z;
        t[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < JP; ++j) r[j] = t[j];
}

// ---------------------------------------------------------------- N = 3
// Returns x~; fills p1, p2, p3.  sG: core in shared memory, [JP][JP][JPR].
template <int JP>
__device__ __forceinline__ float partials3(const float* __restrict__ sG, const float (&a1)[JP],
                                           const float (&a2)[JP], const float (&a3)[JP],
                                           float (&p1)[JP], float (&p2)[JP], float (&p3)[JP]) {
    constexpr int JPR = round4(JP);
    constexpr int U1 = JP <= 12 ? JP : 1;
#pragma unroll
    for (int j = 0; j < JP; ++j) { p1[j] = 0.f; p2[j] = 0.f; p3[j] = 0.f; }
#pragma unroll U1
    for (int j1 = 0; j1 < JP; ++j1) {
        const float a1j = a1[j1];
        float p1j = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < JP; ++j2) {
            float g[JP];
            load_grow<JP>(sG + (j1 * JP + j2) * JPR, g);
            const float w = a1j * a2[j2];
            float t = 0.f;
#pragma unroll
            for (int j3 = 0; j3 < JP; ++j3) {
                t = fmaf(g[j3], a3[j3], t);
                p3[j3] = fmaf(g[j3], w, p3[j3]);
            }
            p1j = fmaf(t, a2[j2], p1j);
            p2[j2] = fmaf(t, a1j, p2[j2]);
        }
        p1[j1] = p1j;
    }
    float xt = 0.f;
#pragma unroll
    for (int j = 0; j < JP; ++j) xt = fmaf(a1[j], p1[j], xt);
    return xt;
}

// The same sweep for one of L lanes that share an entry: this lane takes the JH = JP/L
// (rounded up) values of j1 starting at j1base and gets p1 for those, and its parts of p2, p3
// and x~ (the lanes add their parts).  a1s holds a1[j1base .. j1base + JH), zero past JP.
template <int JP, int L>
__device__ __forceinline__ float partials3_lane(const float* __restrict__ sG, int j1base,
                                                const float (&a1s)[(JP + L - 1) / L],
                                                const float (&a2)[JP], const float (&a3)[JP],
                                                float (&p1s)[(JP + L - 1) / L], float (&p2)[JP],
                                                float (&p3)[JP]) {
    constexpr int JPR = round4(JP);
    constexpr int JH = (JP + L - 1) / L;
    constexpr int U1 = JH <= 12 ? JH : 1;
#pragma unroll
    for (int j = 0; j < JP; ++j) { p2[j] = 0.f; p3[j] = 0.f; }
#pragma unroll U1
    for (int jj = 0; jj < JH; ++jj) {
        const int j1 = min(j1base + jj, JP - 1);   // past JP, a1s is zero
        const float a1j = a1s[jj];
        float p1j = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < JP; ++j2) {
            float g[JP];
            load_grow<JP>(sG + (j1 * JP + j2) * JPR, g);
            const float w = a1j * a2[j2];
            float t = 0.f;
#pragma unroll
            for (int j3 = 0; j3 < JP; ++j3) {
                t = fmaf(g[j3], a3[j3], t);
                p3[j3] = fmaf(g[j3], w, p3[j3]);
            }
            p1j = fmaf(t, a2[j2], p1j);
            p2[j2] = fmaf(t, a1j, p2[j2]);
        }
        p1s[jj] = p1j;
    }
    float xt = 0.f;
#pragma unroll
    for (int jj = 0; jj < JH; ++jj) xt = fmaf(a1s[jj], p1s[jj], xt);
    return xt;
}

// prediction only: x~ = sum_j1 a1 sum_j2 a2 sum_j3 g a3
template <int JP>
__device__ __forceinline__ float predict3(const float* __restrict__ sG, const float (&a1)[JP],
                                          const float (&a2)[JP], const float (&a3)[JP]) {
    constexpr int JPR = round4(JP);
    constexpr int U1 = JP <= 12 ? JP : 1;
    float xt = 0.f;
#pragma unroll U1
    for (int j1 = 0; j1 < JP; ++j1) {
        float s = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < JP; ++j2) {
            float g[JP];
            load_grow<JP>(sG + (j1 * JP + j2) * JPR, g);
            float t = 0.f;
#pragma unroll
            for (int j3 = 0; j3 < JP; ++j3) t = fmaf(g[j3], a3[j3], t);
            s = fmaf(t, a2[j2], s);
        }
        xt = fmaf(s, a1[j1], xt);
    }
    return xt;
}

// ---------------------------------------------------------------- N = 4
template <int JP>
__device__ __forceinline__ float partials4(const float* __restrict__ sG, const float (&a1)[JP],
                                           const float (&a2)[JP], const float (&a3)[JP],
                                           const float (&a4)[JP], float (&p1)[JP],
                                           float (&p2)[JP], float (&p3)[JP], float (&p4)[JP]) {
    constexpr int JPR = round4(JP);
    constexpr int U1 = JP <= 4 ? JP : 1;
    // the inner products over j4 and the p4 updates in pairs of j4 (packed FMAs); the j3
    // terms of p1 and p2 share one sum s3 = sum_j3 t a3[j3] per (j1, j2)
    constexpr int J2 = JP / 2;
    static_assert(JP % 2 == 0, "packed form for even ranks");
    float2 p4v[J2];
#pragma unroll
    for (int j = 0; j < J2; ++j) p4v[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < JP; ++j) { p1[j] = 0.f; p2[j] = 0.f; p3[j] = 0.f; }
#pragma unroll U1
    for (int j1 = 0; j1 < JP; ++j1) {
        const float a1j = a1[j1];
        float p1j = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < JP; ++j2) {
            const float w12 = a1j * a2[j2];
            float s3 = 0.f;   // sum_j3 t(j3) a3[j3]
#pragma unroll
            for (int j3 = 0; j3 < JP; ++j3) {
                float g[JP];
                load_grow<JP>(sG + ((j1 * JP + j2) * JP + j3) * JPR, g);
                const float w = w12 * a3[j3];
                const float2 ww = make_float2(w, w);
                float2 tt = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < J2; ++j) {
                    const float2 gg = make_float2(g[2 * j], g[2 * j + 1]);
                    tt = __ffma2_rn(gg, make_float2(a4[2 * j], a4[2 * j + 1]), tt);
                    p4v[j] = __ffma2_rn(gg, ww, p4v[j]);
                }
                const float t = tt.x + tt.y;
                p3[j3] = fmaf(t, w12, p3[j3]);
                s3 = fmaf(t, a3[j3], s3);
            }
            p1j = fmaf(s3, a2[j2], p1j);
            p2[j2] = fmaf(s3, a1j, p2[j2]);
        }
        p1[j1] = p1j;
    }
#pragma unroll
    for (int j = 0; j < J2; ++j) {
        p4[2 * j] = p4v[j].x;
        p4[2 * j + 1] = p4v[j].y;
    }
    float xt = 0.f;
#pragma unroll
    for (int j = 0; j < JP; ++j) xt = fmaf(a1[j], p1[j], xt);
    return xt;
}

template <int JP>
__device__ __forceinline__ float predict4(const float* __restrict__ sG, const float (&a1)[JP],
                                          const float (&a2)[JP], const float (&a3)[JP],
                                          const float (&a4)[JP]) {
    constexpr int JPR = round4(JP);
    constexpr int U1 = JP <= 4 ? JP : 1;
    float xt = 0.f;
#pragma unroll U1
    for (int j1 = 0; j1 < JP; ++j1) {
        float s1 = 0.f;
#pragma unroll
        for (int j2 = 0; j2 < JP; ++j2) {
            float s2 = 0.f;
#pragma unroll
            for (int j3 = 0; j3 < JP; ++j3) {
                float g[JP];
                load_grow<JP>(sG + ((j1 * JP + j2) * JP + j3) * JPR, g);
                float t = 0.f;
#pragma unroll
                for (int j4 = 0; j4 < JP; ++j4) t = fmaf(g[j4], a4[j4], t);
                s2 = fmaf(t, a3[j3], s2);
            }
            s1 = fmaf(s2, a2[j2], s1);
        }
        xt = fmaf(s1, a1[j1], xt);
    }
    return xt;
}

// ---------------------------------------------------------------- core-gradient accumulator
// Accumulates sum_b e_b a1_b o ... o aN_b over the entries of a CTA.  The N staged rows of
// each entry sit in shared memory: stage[n][b][JPR] (stage[0] already multiplied by e_b).
// Thread t owns multi-indices q over the first N-1 modes and all JP values of the last
// mode; when there are fewer multi-indices than threads the entries are split into KS
// slices.  Running sums are Neumaier-compensated across tiles.
// ST: rows between the stage's per-mode blocks (at least the entries of a tile)
template <int N, int JP, int ST = kTile>
struct CoreAcc {
    static constexpr int JPR = round4(JP);
    static constexpr int Q = ipow_t<JP, N - 1>::v;
    static constexpr int KS = (kTile / Q) > 0 ? (kTile / Q) : 1;
    static constexpr int QPT = (Q + kTile - 1) / kTile;
    float s[QPT][JP];
    float c[QPT][JP];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < QPT; ++k)
#pragma unroll
            for (int j = 0; j < JP; ++j) { s[k][j] = 0.f; c[k][j] = 0.f; }
    }

    // stage: shared memory [N][ST][JPR]; nb valid entries
    __device__ __forceinline__ void add_tile(const float* __restrict__ stage, int nb) {
        const int t = threadIdx.x;
        const int slice = KS > 1 ? t / Q : 0;
#pragma unroll
        for (int k = 0; k < QPT; ++k) {
            const int q = KS > 1 ? (t % Q) : (t + k * kTile);
            if (slice >= KS || q >= Q) continue;
            int jj[N - 1];
            {
                int r = q;
#pragma unroll
                for (int n = N - 2; n >= 0; --n) { jj[n] = r % JP; r /= JP; }
            }
            float tile[JP];
#pragma unroll
            for (int j = 0; j < JP; ++j) tile[j] = 0.f;
            for (int b = slice; b < nb; b += KS) {
                float w = stage[(0 * ST + b) * JPR + jj[0]];
#pragma unroll
                for (int n = 1; n < N - 1; ++n) w *= stage[(n * ST + b) * JPR + jj[n]];
                float r[JP];
                load_grow<JP>(stage + ((N - 1) * ST + b) * JPR, r);
#pragma unroll
                for (int j = 0; j < JP; ++j) tile[j] = fmaf(w, r[j], tile[j]);
            }
#pragma unroll
            for (int j = 0; j < JP; ++j) {
                const float x = tile[j];
                const float tt = s[k][j] + x;
                if (fabsf(s[k][j]) >= fabsf(x)) c[k][j] += (s[k][j] - tt) + x;
                else c[k][j] += (x - tt) + s[k][j];
                s[k][j] = tt;
            }
        }
    }

    // Writes this CTA's partial (dense [Q][JP]) to out.  scratch: shared memory of at
    // least KS * Q * JP floats (only used when KS > 1).  Ends with __syncthreads.
    __device__ __forceinline__ void store(float* __restrict__ out, float* scratch) {
        const int t = threadIdx.x;
        if (KS == 1) {
#pragma unroll
            for (int k = 0; k < QPT; ++k) {
                const int q = t + k * kTile;
                if (q >= Q) continue;
#pragma unroll
                for (int j = 0; j < JP; ++j) out[q * JP + j] = s[k][j] + c[k][j];
            }
            __syncthreads();
            return;
        }
        const int slice = t / Q, q = t % Q;
        if (slice < KS) {
#pragma unroll
            for (int j = 0; j < JP; ++j) scratch[(slice * Q + q) * JP + j] = s[0][j] + c[0][j];
        }
        __syncthreads();
        for (int l = t; l < Q * JP; l += kTile) {
            float a = 0.f;
            for (int sl = 0; sl < KS; ++sl) a += scratch[sl * Q * JP + l];
            out[l] = a;
        }
        __syncthreads();
    }
};

// One tile's core step added lock-free to the core in global memory.  The multi-indices q
// of the first N - 1 modes come in pairs (q, q + 1) that differ in mode N - 1's index; thread
// (pair, slice) sums its slice of the tile's entries for both multi-indices and all JP values
// of the last mode (the last mode's row is loaded once for the pair).  With several slices,
// every slice leaves its sums in the stage (read by then), and then every thread takes
// (multi-index, 4 values of the last mode) items: the slices' sums in slice order, and
// sc * sum - rg * G added with one atomic.
template <int N, int JP, int ST = kTile, int T = kTile>
struct CoreTile {
    static constexpr int JPR = round4(JP);
    static constexpr int Q = ipow_t<JP, N - 1>::v;
    static constexpr int JH2 = (JP + 1) / 2;     // pairs per row of mode N - 1 (padding is zero)
    static constexpr int QP = Q / JP * JH2;      // pairs of multi-indices
    // slices: enough threads, at most 16 (each item of the final sum reads one per slice),
    // and as many as leave their sums in the stage
    static constexpr int KS0 = (T / QP) > 16 ? 16 : ((T / QP) > 0 ? (T / QP) : 1);
    static constexpr int KSM = (N * ST) / (2 * QP);
    static constexpr int KS = KS0 < KSM ? KS0 : (KSM > 1 ? KSM : 1);
    static constexpr int QPT = (QP + T - 1) / T;
    // entries per step of the accumulation loop: their shared-memory loads are independent of
    // the accumulation chain, which keeps the entries' order
    static constexpr int U = JP <= 10 ? 4 : (JP <= 20 ? 2 : 1);

    // pair p's sums over slice `slice` of the tile's entries (b = slice, slice + KS, ...)
    __device__ __forceinline__ static void accumulate(const float* __restrict__ stage, int nb, int p,
                                                      int slice, float (&tile)[2][JP]) {
        int jj[N - 1];
        jj[N - 2] = 2 * (p % JH2);
        {
            int r = p / JH2;
#pragma unroll
            for (int n = N - 3; n >= 0; --n) { jj[n] = r % JP; r /= JP; }
        }
#pragma unroll
        for (int j = 0; j < JP; ++j) { tile[0][j] = 0.f; tile[1][j] = 0.f; }
        auto weights = [&](int b, float& wa, float& wb) {
            float w = 1.f;
#pragma unroll
            for (int n = 0; n < N - 2; ++n) w *= stage[(n * ST + b) * JPR + jj[n]];
            const float2 s = *reinterpret_cast<const float2*>(stage + ((N - 2) * ST + b) * JPR + jj[N - 2]);
            wa = w * s.x;
            wb = w * s.y;
        };
        int b = slice;
        for (; b + (U - 1) * KS < nb; b += U * KS) {
            float wa[U], wb[U], r[U][JP];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                weights(b + u * KS, wa[u], wb[u]);
                load_grow<JP>(stage + ((N - 1) * ST + b + u * KS) * JPR, r[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int j = 0; j < JP; ++j) {
                    tile[0][j] = fmaf(wa[u], r[u][j], tile[0][j]);
                    tile[1][j] = fmaf(wb[u], r[u][j], tile[1][j]);
                }
        }
        for (; b < nb; b += KS) {
            float wa, wb, r[JP];
            weights(b, wa, wb);
            load_grow<JP>(stage + ((N - 1) * ST + b) * JPR, r);
#pragma unroll
            for (int j = 0; j < JP; ++j) {
                tile[0][j] = fmaf(wa, r[j], tile[0][j]);
                tile[1][j] = fmaf(wb, r[j], tile[1][j]);
            }
        }
    }

    // G[q] += sc * tile - rg * G[q] for both multi-indices of pair p (the second only when it
    // exists: JP odd pads the pair); nonneg: each add is followed by the projection
    __device__ __forceinline__ static void add(float* G, const float* __restrict__ sG, int p,
                                               const float (&tile)[2][JP], float sc, float rg,
                                               int nonneg) {
        const int q0 = (p / JH2) * JP + 2 * (p % JH2);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && 2 * (p % JH2) + 1 >= JP) break;
            const int q = q0 + h;
            float g[JP];
            load_grow<JP>(sG + q * JPR, g);
            float d[JPR];
#pragma unroll
            for (int j = 0; j < JPR; ++j) d[j] = j < JP ? fmaf(sc, tile[h][j], -rg * g[j]) : 0.f;
#pragma unroll
            for (int c = 0; c < JPR / 4; ++c) {
                red_add_v4(G + q * JPR + 4 * c, d[4 * c], d[4 * c + 1], d[4 * c + 2], d[4 * c + 3]);
                if (nonneg) red_proj_v4(G + q * JPR + 4 * c);
            }
        }
    }

    // Every one of the T threads calls apply (with several slices it has CTA barriers over
    // T threads, and the stage is overwritten).
    __device__ __forceinline__ static void apply(float* stage, int nb, const float* __restrict__ sG,
                                                 float* G, float sc, float rg, int nonneg) {
        const int t = threadIdx.x;
        if constexpr (KS > 1) {
            // (every thread reaches each barrier at the same instruction: warps can straddle
            // the last slice)
            const int p = t % QP, slice = t / QP;
            const bool act = slice < KS;
            float tile[2][JP];
            if (act) accumulate(stage, nb, p, slice, tile);
            asm volatile("bar.sync 1, %0;" :: "r"(T) : "memory");
            if (act) {
                float* o = stage + (slice * QP + p) * 2 * JPR;
#pragma unroll
                for (int j = 0; j < JPR; ++j) {
                    o[j] = j < JP ? tile[0][j] : 0.f;
                    o[JPR + j] = j < JP ? tile[1][j] : 0.f;
                }
            }
            asm volatile("bar.sync 1, %0;" :: "r"(T) : "memory");
            for (int i = t; i < Q * (JPR / 4); i += T) {
                const int q = i / (JPR / 4), c = i % (JPR / 4);
                const int jl = q % JP;
                const int pp = (q / JP) * JH2 + jl / 2;
                const float* o = stage + (pp * 2 + (jl & 1)) * JPR + 4 * c;
                float4 acc = *reinterpret_cast<const float4*>(o);
                for (int sl = 1; sl < KS; ++sl) {
                    const float4 v = *reinterpret_cast<const float4*>(o + sl * QP * 2 * JPR);
                    acc.x += v.x;
                    acc.y += v.y;
                    acc.z += v.z;
                    acc.w += v.w;
                }
                const float4 g = *reinterpret_cast<const float4*>(sG + q * JPR + 4 * c);
                red_add_v4(G + q * JPR + 4 * c, fmaf(sc, acc.x, -rg * g.x), fmaf(sc, acc.y, -rg * g.y),
                           fmaf(sc, acc.z, -rg * g.z), fmaf(sc, acc.w, -rg * g.w));
                if (nonneg) red_proj_v4(G + q * JPR + 4 * c);
            }
        } else {
#pragma unroll
            for (int k = 0; k < QPT; ++k) {
                const int p = t + k * T;
                if (p >= QP) continue;
                float tile[2][JP];
                accumulate(stage, nb, p, 0, tile);
                add(G, sG, p, tile, sc, rg, nonneg);
            }
        }
    }
};

// the N partial products and the prediction of one entry (3- or 4-way)
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

// the opt-in above 48 KB counts static shared memory too, so set the limit whenever the
// dynamic part is large
template <typename K>
static inline cudaError_t prep(K kernel, size_t smem) {
    if (smem > 32 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

}  // namespace s3
