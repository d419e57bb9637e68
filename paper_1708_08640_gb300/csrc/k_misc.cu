// Coupled-matrix, segmented-reduction, core-step and utility kernels of the S3CMTF path.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "kernels.h"

namespace s3 {

// ------------------------------------------------------------------ coupled entries
// Eq. (8), coupled rows: e = y - u^(c)_{j1} . v_{j2};
//   d/du = -lambda_m e v;   d/dv = -lambda_m e u + lambda_m lambda_reg / |Omega_Y^{2,j2}| v
template <int C4>
__global__ void __launch_bounds__(256) k_coupled_contrib(DParams P, DGroup Gr, int m,
                                                         int64_t c0, int64_t c1, float* cu,
                                                         float* cv) {
    const int64_t e = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= c1) return;
    const int ld = 4 * C4;
    const int c = P.cmode[m];
    const int32_t r = __ldg(Gr.cr[m] + e), k = __ldg(Gr.cc[m] + e);
    float4 u[C4], v[C4];
    float yh = 0.f;
#pragma unroll
    for (int q = 0; q < C4; ++q) {
        u[q] = ld4_nc(P.U[c] + (int64_t)r * ld + 4 * q);
        v[q] = ld4_nc(P.V[m] + (int64_t)k * ld + 4 * q);
        yh = fmaf(u[q].x, v[q].x, yh);
        yh = fmaf(u[q].y, v[q].y, yh);
        yh = fmaf(u[q].z, v[q].z, yh);
        yh = fmaf(u[q].w, v[q].w, yh);
    }
    const float err = __ldg(Gr.cval[m] + e) - yh;
    const float a = -P.lambda_m * err;
    const float rv = P.lambda_m * P.lambda_reg * __ldg(P.inv_cnt[P.N + m] + k);
    float* du = cu + (int64_t)__ldg(Gr.cpos_u[m] + e) * ld;
    float* dv = cv + (int64_t)__ldg(Gr.cpos_v[m] + e) * ld;
#pragma unroll
    for (int q = 0; q < C4; ++q) {
        st4(du + 4 * q, make_float4(a * v[q].x, a * v[q].y, a * v[q].z, a * v[q].w));
        st4(dv + 4 * q, make_float4(fmaf(a, u[q].x, rv * v[q].x), fmaf(a, u[q].y, rv * v[q].y),
                                    fmaf(a, u[q].z, rv * v[q].z), fmaf(a, u[q].w, rv * v[q].w)));
    }
}

__device__ __forceinline__ void block_pair_reduce(Kahan k, float* out2) {
    __shared__ float ws[2][32];
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

template <int C4>
__global__ void __launch_bounds__(256) k_coupled_fwd(DParams P, int m, const int32_t* rr,
                                                     const int32_t* cc, const float* y,
                                                     int64_t n, float* sq_part) {
    const int ld = 4 * C4;
    const int c = P.cmode[m];
    Kahan k;
    k.init();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = __ldg(rr + e), kk = __ldg(cc + e);
        float yh = 0.f;
#pragma unroll
        for (int q = 0; q < C4; ++q) {
            const float4 u = ld4_nc(P.U[c] + (int64_t)r * ld + 4 * q);
            const float4 v = ld4_nc(P.V[m] + (int64_t)kk * ld + 4 * q);
            yh = fmaf(u.x, v.x, yh);
            yh = fmaf(u.y, v.y, yh);
            yh = fmaf(u.z, v.z, yh);
            yh = fmaf(u.w, v.w, yh);
        }
        const float d = __ldg(y + e) - yh;
        k.add(d * d);
    }
    block_pair_reduce(k, sq_part + 2 * blockIdx.x);
}

#define S3_DISPATCH_C4(C4V, CALL)                 \
    switch (C4V) {                                \
        case 1: { constexpr int C4 = 1; CALL; } break; \
        case 2: { constexpr int C4 = 2; CALL; } break; \
        case 3: { constexpr int C4 = 3; CALL; } break; \
        case 4: { constexpr int C4 = 4; CALL; } break; \
        case 5: { constexpr int C4 = 5; CALL; } break; \
        case 6: { constexpr int C4 = 6; CALL; } break; \
        case 7: { constexpr int C4 = 7; CALL; } break; \
        case 8: { constexpr int C4 = 8; CALL; } break; \
        default: return cudaErrorInvalidValue;    \
    }

cudaError_t launch_coupled_contrib(const DParams& P, const DGroup& G, int m, int64_t c_begin,
                                   int64_t c_end, float* contrib_u, float* contrib_v,
                                   cudaStream_t s) {
    const int64_t n = c_end - c_begin;
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((n + 255) / 256);
    S3_DISPATCH_C4(P.ld / 4, (k_coupled_contrib<C4><<<grid, 256, 0, s>>>(P, G, m, c_begin, c_end,
                                                                        contrib_u, contrib_v)));
    return cudaGetLastError();
}

int coupled_fwd_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048)); }

cudaError_t launch_coupled_fwd(const DParams& P, int m, const int32_t* r, const int32_t* c,
                               const float* y, int64_t n, float* sq_part, cudaStream_t s) {
    const unsigned grid = (unsigned)coupled_fwd_blocks(n);
    S3_DISPATCH_C4(P.ld / 4, (k_coupled_fwd<C4><<<grid, 256, 0, s>>>(P, m, r, c, y, n, sq_part)));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ segments
// Every segment's events are summed in slot order with Neumaier compensation.  Short
// segments (the common case: rows touched a few times in a group) take one thread each;
// long ones a warp whose lanes stride over the events, huge ones (the hottest rows of a
// large group) a CTA whose threads stride over them.  Strided partial sums are combined
// with a fixed xor butterfly and, across warps, in warp order, so every sum is run-to-run
// identical.
template <int C4>
__device__ __forceinline__ void segment_finish(const DParams& P, const SegmentLaunch& S, int F,
                                               int32_t row, int32_t cnt, const float* sum,
                                               const float* eta_p, int row_mean, int mode,
                                               int j_begin, int j_end) {
    const int ld = 4 * C4;
    if (mode == 0) {
        const float sc = -(*eta_p) / (row_mean ? (float)cnt : 1.f);
        float* base = (F < P.N ? P.U[F] : P.V[F - P.N]) + (int64_t)row * ld;
        for (int j = j_begin; j < j_end; ++j) base[j] = fmaf(sc, sum[j], base[j]);
    } else {
        const int Jf = S.Jf[F];
        float* o = S.out[F] + (int64_t)row * Jf;
        float* cmp = S.comp[F] + (int64_t)row * Jf;
        for (int j = j_begin; j < min(j_end, Jf); ++j) {
            Kahan k;
            k.s = o[j];
            k.c = cmp[j];
            k.add(sum[j]);
            o[j] = k.s;
            cmp[j] = k.c;
        }
    }
}

template <int C4>
__global__ void __launch_bounds__(256) k_segments(DParams P, DGroup Gr, SegmentLaunch S,
                                                  const float* eta_p, int row_mean, int mode) {
    const int ld = 4 * C4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gthread = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    __shared__ float red[8][4 * C4];
    // pass 0: kHugeParts CTAs per huge segment, each on a contiguous piece of its events (a
    // fixed cut, whatever the grid); the CTA that completes a segment adds the pieces' sums in
    // piece order (deterministic), so one segment's events stream on many SMs at once
    __shared__ int s_last;
    for (int64_t w = blockIdx.x; w < S.huge_begin[S.nF] * kHugeParts; w += gridDim.x) {
        const int64_t h = w / kHugeParts;
        const int part = (int)(w % kHugeParts);
        int F = 0;
        while (F + 1 < S.nF && h >= S.huge_begin[F + 1]) ++F;
        const int64_t sg = Gr.seg_off[F][S.g] + (h - S.huge_begin[F]);
        const int32_t cnt = __ldg(Gr.seg_cnt[F] + sg);
        const int32_t row = __ldg(Gr.seg_row[F] + sg);
        const int64_t e0 = (int64_t)cnt * part / kHugeParts, e1 = (int64_t)cnt * (part + 1) / kHugeParts;
        const float* src = S.contrib[F] + ((int64_t)__ldg(Gr.seg_start[F] + sg) + e0) * ld;
        float sum[4 * C4];
        {
            Kahan k[4 * C4];
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) k[j].init();
            rows_sum<C4>(src, ld, threadIdx.x, blockDim.x, (int)(e1 - e0), k);
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) sum[j] = k[j].value();
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) sum[j] += __shfl_xor_sync(0xffffffffu, sum[j], o);
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) red[warp][j] = sum[j];
        __syncthreads();
        float* mine = S.part_sums + (h * kHugeParts + part) * ld;
        if (threadIdx.x < ld) {
            const int j = threadIdx.x;
            Kahan k;
            k.init();
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) k.add(red[i][j]);
            mine[j] = k.value();
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int done = atomicAdd(S.part_done + h, 1);
            s_last = done == kHugeParts - 1;
            if (s_last) {
                S.part_done[h] = 0;   // ready for the next launch
                __threadfence();
            }
        }
        __syncthreads();
        if (s_last && threadIdx.x < ld) {
            const int j = threadIdx.x;
            Kahan k;
            k.init();
            const float* all = S.part_sums + h * kHugeParts * ld;
            for (int q = 0; q < kHugeParts; ++q) k.add(__ldcg(all + q * ld + j));
            float one[4 * C4];
#pragma unroll
            for (int i = 0; i < 4 * C4; ++i) one[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 4 * C4; ++i)
                if (i == j) one[i] = k.value();
            segment_finish<C4>(P, S, F, row, cnt, one, eta_p, row_mean, mode, j, j + 1);
        }
        __syncthreads();
    }
    // pass 1: a thread per short segment
    for (int64_t w = gthread; w < S.short_begin[S.nF]; w += nthreads) {
        int F = 0;
        while (F + 1 < S.nF && w >= S.short_begin[F + 1]) ++F;
        const int64_t sg = Gr.seg_off[F][S.g] + S.nlong[F] + (w - S.short_begin[F]);
        const int32_t cnt = __ldg(Gr.seg_cnt[F] + sg);
        const int32_t row = __ldg(Gr.seg_row[F] + sg);
        const float* src = S.contrib[F] + (int64_t)__ldg(Gr.seg_start[F] + sg) * ld;
        float sum[4 * C4];
        Kahan k[4 * C4];
#pragma unroll
        for (int j = 0; j < 4 * C4; ++j) k[j].init();
        rows_sum<C4>(src, ld, 0, 1, cnt, k);
#pragma unroll
        for (int j = 0; j < 4 * C4; ++j) sum[j] = k[j].value();
        segment_finish<C4>(P, S, F, row, cnt, sum, eta_p, row_mean, mode, 0, ld);
    }
    // pass 2: a warp per long (not huge) segment
    const int64_t gwarp = gthread >> 5, nwarps = nthreads >> 5;
    for (int64_t w = gwarp; w < S.long_begin[S.nF]; w += nwarps) {
        int F = 0;
        while (F + 1 < S.nF && w >= S.long_begin[F + 1]) ++F;
        const int64_t sg = Gr.seg_off[F][S.g] + S.nhuge[F] + (w - S.long_begin[F]);
        const int32_t cnt = __ldg(Gr.seg_cnt[F] + sg);
        const int32_t row = __ldg(Gr.seg_row[F] + sg);
        const float* src = S.contrib[F] + (int64_t)__ldg(Gr.seg_start[F] + sg) * ld;
        float sum[4 * C4];
        {
            Kahan k[4 * C4];
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) k[j].init();
            rows_sum<C4>(src, ld, lane, 32, cnt, k);
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) sum[j] = k[j].value();
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1)
#pragma unroll
            for (int j = 0; j < 4 * C4; ++j) sum[j] += __shfl_xor_sync(0xffffffffu, sum[j], o);
        // each lane finishes one or two components
        const int per = (ld + 31) / 32;
        segment_finish<C4>(P, S, F, row, cnt, sum, eta_p, row_mean, mode, lane * per,
                           min(ld, (lane + 1) * per));
    }
}

cudaError_t launch_segments(const DParams& P, const DGroup& G, const SegmentLaunch& S,
                            const float* eta, int row_mean, int mode, cudaStream_t s) {
    if (S.huge_begin[S.nF] > 0 && (!S.part_sums || !S.part_done)) return cudaErrorInvalidValue;
    const int64_t work = std::max({S.short_begin[S.nF], 32 * S.long_begin[S.nF],
                                   256 * kHugeParts * S.huge_begin[S.nF]});
    if (work <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((work + 255) / 256, 4096);
    S3_DISPATCH_C4(P.ld / 4, (k_segments<C4><<<grid, 256, 0, s>>>(P, G, S, eta, row_mean, mode)));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ core step
// parts: nparts partials, each dense [JP^N] (last mode fastest); G: padded [JP^(N-1)][JPR].
// One warp per core element: the lanes stride over the partials with compensated sums and
// combine them with a fixed xor butterfly (deterministic).
__global__ void __launch_bounds__(256) k_core(DParams P, int N, int JP, int4 Jv,
                                              const float* parts, int64_t nparts, int64_t n_t,
                                              const float* eta_p, float cs, int mode, float* out,
                                              float* comp) {
    int64_t Pd = 1;
    for (int n = 0; n < N; ++n) Pd *= JP;
    const int JPR = round4(JP);
    const int Jn[4] = {Jv.x, Jv.y, Jv.z, Jv.w};
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < Pd; l += nwarps) {
        Kahan k;
        k.init();
        // four partials' loads in flight per lane, added in partial order
        int64_t p = lane;
        for (; p + 96 < nparts; p += 128) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcg(parts + (p + 32 * u) * Pd + l);
#pragma unroll
            for (int u = 0; u < 4; ++u) k.add(v[u]);
        }
        for (; p < nparts; p += 32) k.add(__ldcg(parts + p * Pd + l));
        float sum = k.value();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane != 0) continue;
        const int64_t q = l / JP;
        const int jl = (int)(l % JP);
        if (mode == 0) {
            if (n_t <= 0) continue;
            const float eta = *eta_p;
            float* g = P.G + q * JPR + jl;
            const float gv = *g;
            *g = gv + eta * cs * (sum / (float)n_t) - eta * cs * P.lambda_reg * P.inv_nnz * gv;
        } else {
            // unpadded destination index; skip padded positions
            int64_t r = l, dst = 0, mul = 1;
            bool ok = true;
            for (int n = N - 1; n >= 0; --n) {
                const int j = (int)(r % JP);
                r /= JP;
                if (j >= Jn[n]) ok = false;
                dst += j * mul;
                mul *= Jn[n];
            }
            if (!ok) continue;
            if (P.cp) {   // S3CMTF-CP: only the diagonal is a parameter
                int64_t r2 = l;
                const int j0 = (int)(r2 % JP);
                bool diag = true;
                for (int n = 1; n < N; ++n) {
                    r2 /= JP;
                    diag &= (int)(r2 % JP) == j0;
                }
                if (!diag) continue;
            }
            Kahan a;
            a.s = out[dst];
            a.c = comp[dst];
            a.add(-sum);
            out[dst] = a.s;
            comp[dst] = a.c;
        }
    }
}

cudaError_t launch_core(const DParams& P, int N, int JP, const int* J, const float* parts,
                        int64_t nparts, int64_t n_t, const float* eta, float core_scale, int mode,
                        float* out, float* comp, cudaStream_t s) {
    int64_t Pd = 1;
    for (int n = 0; n < N; ++n) Pd *= JP;
    const unsigned grid = (unsigned)std::min<int64_t>((Pd * 32 + 255) / 256, 4096);
    int4 Jv = make_int4(J[0], N > 1 ? J[1] : 1, N > 2 ? J[2] : 1, N > 3 ? J[3] : 1);
    k_core<<<grid, 256, 0, s>>>(P, N, JP, Jv, parts, nparts, n_t, eta, core_scale, mode, out, comp);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ norms and reductions
struct RowsArg {
    int64_t rows[kMaxF + 1];
};

// blockIdx.y = sum index: 0 -> ||G||^2 over the padded core (padding is zero), F+1 ->
// sum over rows of factor F that have observed entries of ||row||^2.
__global__ void __launch_bounds__(256) k_sqnorms(DParams P, RowsArg R, int JP, float* parts) {
    const int k = blockIdx.y;
    Kahan acc;
    acc.init();
    const int ld = P.ld;
    if (k == 0) {
        const int64_t n = R.rows[0];
        for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
             l += (int64_t)gridDim.x * blockDim.x) {
            const float g = P.G[l];
            acc.add(g * g);
        }
    } else {
        const int F = k - 1;
        const float* base = F < P.N ? P.U[F] : P.V[F - P.N];
        const int64_t rows = R.rows[k];
        const int64_t n = rows * ld;
        for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
             l += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = l / ld;
            if (__ldg(P.inv_cnt[F] + i) > 0.f) {
                const float v = base[l];
                acc.add(v * v);
            }
        }
    }
    block_pair_reduce(acc, parts + 2 * ((int64_t)k * gridDim.x + blockIdx.x));
}

cudaError_t launch_sqnorms(const DParams& P, int nF, const int64_t* rows, int JP, float* parts,
                           int blocks_per_sum, cudaStream_t s) {
    RowsArg R;
    for (int k = 0; k <= nF; ++k) R.rows[k] = rows[k];
    dim3 grid(blocks_per_sum, nF + 1);
    k_sqnorms<<<grid, 256, 0, s>>>(P, R, JP, parts);
    return cudaGetLastError();
}

// FP64 final reduction (the only FP64 arithmetic on the GPU): one CTA, fixed order.
__global__ void __launch_bounds__(256) k_reduce_f64(const float* parts, int64_t count, double* out) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x)
        a += (double)parts[2 * i] + (double)parts[2 * i + 1];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

cudaError_t launch_reduce_f64(const float* parts, int64_t count, double* out, cudaStream_t s) {
    k_reduce_f64<<<1, 256, 0, s>>>(parts, count, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ initial parameters
// Counter-based generator: splitmix64 finalizer (Steele, Lea, Flood 2014) applied to
// seed + golden_gamma * (stream * 2^40 + k + 1).  uniform = (bits >> 11) * 2^-53.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t stream, uint64_t k) {
    const uint64_t z = mix64(seed + 0x9E3779B97F4A7C15ull * ((stream << 40) + k + 1));
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

struct InitArg {
    int64_t rows[kMaxF];
    int cols[kMaxF];
    int nF;
    int N;
    int J[kMaxN];
    int JP;
    double sigma;
};

// blockIdx.y = factor (0..nF-1) or nF for the core
__global__ void __launch_bounds__(256) k_init(DParams P, InitArg A, uint64_t seed) {
    const int f = blockIdx.y;
    if (f < A.nF) {
        float* base = f < P.N ? P.U[f] : P.V[f - P.N];
        const int cols = A.cols[f];
        const int64_t n = A.rows[f] * cols;
        for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
             l += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = l / cols;
            const int j = (int)(l % cols);
            base[i * P.ld + j] = (float)uniform01(seed, 1 + f, (uint64_t)l);
        }
    } else {
        int64_t Pd = 1;
        for (int n = 0; n < A.N; ++n) Pd *= A.J[n];
        const int JPR = round4(A.JP);
        for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Pd;
             l += (int64_t)gridDim.x * blockDim.x) {
            const double u1 = 1.0 - uniform01(seed, 0, 2 * (uint64_t)l);
            const double u2 = uniform01(seed, 0, 2 * (uint64_t)l + 1);
            const double g = A.sigma * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
            // dense index l over J_1..J_N -> padded position
            int64_t r = l, q = 0, mul = 1;
            int jl = 0;
            for (int n = A.N - 1; n >= 0; --n) {
                const int j = (int)(r % A.J[n]);
                r /= A.J[n];
                if (n == A.N - 1) jl = j;
                else { q += j * mul; mul *= A.JP; }
            }
            P.G[q * JPR + jl] = (float)g;
        }
    }
}

cudaError_t launch_init_params(const DParams& P, const int64_t* I, const int* J, const int64_t* K,
                               int JP, uint64_t seed, cudaStream_t s) {
    InitArg A;
    A.N = P.N;
    A.nF = P.N + P.M;
    A.JP = JP;
    double prodJ = 1.0;
    for (int n = 0; n < P.N; ++n) {
        A.rows[n] = I[n];
        A.cols[n] = J[n];
        A.J[n] = J[n];
        prodJ *= J[n];
    }
    for (int m = 0; m < P.M; ++m) {
        A.rows[P.N + m] = K[m];
        A.cols[P.N + m] = J[P.cmode[m]];
    }
    A.sigma = sqrt(pow(3.0, P.N) / prodJ);
    dim3 grid(1024, A.nF + 1);
    k_init<<<grid, 256, 0, s>>>(P, A, seed);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ checks and packing
__global__ void k_check_finite(const float* p, int64_t n, int* flag) {
    bool bad = false;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(p[l])) bad = true;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const float* p, int64_t n, int* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 2048);
    k_check_finite<<<grid, 256, 0, s>>>(p, n, flag);
    return cudaGetLastError();
}

__global__ void k_pack_rows(float* dst, int ld, const float* src, int64_t rows, int J) {
    const int64_t n = rows * ld;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = l / ld;
        const int j = (int)(l % ld);
        dst[l] = j < J ? src[i * J + j] : 0.f;
    }
}
__global__ void k_unpack_rows(float* dst, const float* src, int ld, int64_t rows, int J) {
    const int64_t n = rows * J;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        dst[l] = src[(l / J) * ld + (l % J)];
}

cudaError_t launch_pack_rows(float* dst, int ld, const float* src, int64_t rows, int J,
                             cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((rows * ld + 255) / 256, 4096);
    k_pack_rows<<<grid, 256, 0, s>>>(dst, ld, src, rows, J);
    return cudaGetLastError();
}
cudaError_t launch_unpack_rows(float* dst, const float* src, int ld, int64_t rows, int J,
                               cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((rows * J + 255) / 256, 4096);
    k_unpack_rows<<<grid, 256, 0, s>>>(dst, src, ld, rows, J);
    return cudaGetLastError();
}

// padded core index (q over JP^(N-1), jl < JPR) <-> dense unpadded index
__global__ void k_core_copy(float* dst, const float* src, int N, int4 Jv, int JP, int pack) {
    const int JPR = round4(JP);
    const int Jn[4] = {Jv.x, Jv.y, Jv.z, Jv.w};
    int64_t Q = 1;
    for (int n = 0; n < N - 1; ++n) Q *= JP;
    const int64_t total = Q * JPR;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < total;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int jl = (int)(l % JPR);
        int64_t q = l / JPR;
        bool ok = jl < Jn[N - 1];
        int64_t dense = jl, mul = Jn[N - 1];
        for (int n = N - 2; n >= 0; --n) {
            const int j = (int)(q % JP);
            q /= JP;
            if (j >= Jn[n]) ok = false;
            dense += j * mul;
            mul *= Jn[n];
        }
        if (pack) dst[l] = ok ? src[dense] : 0.f;
        else if (ok) dst[dense] = src[l];
    }
}

cudaError_t launch_pack_core(float* dst, const float* src, int N, const int* J, int JP,
                             cudaStream_t s) {
    int4 Jv = make_int4(J[0], N > 1 ? J[1] : 1, N > 2 ? J[2] : 1, N > 3 ? J[3] : 1);
    k_core_copy<<<64, 256, 0, s>>>(dst, src, N, Jv, JP, 1);
    return cudaGetLastError();
}
cudaError_t launch_unpack_core(float* dst, const float* src, int N, const int* J, int JP,
                               cudaStream_t s) {
    int4 Jv = make_int4(J[0], N > 1 ? J[1] : 1, N > 2 ? J[2] : 1, N > 3 ? J[3] : 1);
    k_core_copy<<<64, 256, 0, s>>>(dst, src, N, Jv, JP, 0);
    return cudaGetLastError();
}

__global__ void k_gather(float* dst, const float* src, const int64_t* idx, int64_t n) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        dst[l] = src[idx[l]];
}

cudaError_t launch_gather_f32(float* dst, const float* src, const int64_t* idx, int64_t n,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (!dst || !src || !idx) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    k_gather<<<grid, 256, 0, s>>>(dst, src, idx, n);
    return cudaGetLastError();
}

}  // namespace s3

namespace s3 {
__global__ void k_add_comp(float* out, const float* comp, int64_t n) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        out[l] += comp[l];
}
cudaError_t launch_add_comp(float* out, const float* comp, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_add_comp<<<grid, 256, 0, s>>>(out, comp, n);
    return cudaGetLastError();
}
// dG (dense unpadded) += lambda_reg * G (the core regulariser summed over all entries)
__global__ void k_core_reg(float* out, const float* G, int N, int4 Jv, int JP, float lam) {
    const int JPR = round4(JP);
    const int Jn[4] = {Jv.x, Jv.y, Jv.z, Jv.w};
    int64_t Pd = 1;
    for (int n = 0; n < N; ++n) Pd *= Jn[n];
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Pd;
         l += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = l, q = 0, mul = 1;
        int jl = 0;
        for (int n = N - 1; n >= 0; --n) {
            const int j = (int)(r % Jn[n]);
            r /= Jn[n];
            if (n == N - 1) jl = j;
            else { q += j * mul; mul *= JP; }
        }
        out[l] += lam * G[q * JPR + jl];
    }
}
cudaError_t launch_core_reg(float* out, const float* G, int N, const int* J, int JP, float lam,
                            cudaStream_t s) {
    int4 Jv = make_int4(J[0], N > 1 ? J[1] : 1, N > 2 ? J[2] : 1, N > 3 ? J[3] : 1);
    k_core_reg<<<64, 256, 0, s>>>(out, G, N, Jv, JP, lam);
    return cudaGetLastError();
}

// A step from a given gradient: rows P[i][j] += alpha * g[i][j] (g dense unpadded, rows of J;
// P padded to ld), then max(0, .) in the non-negative form
__global__ void k_rows_step(float* P, int ld, const float* g, int64_t rows, int J, float alpha,
                            int nonneg) {
    const int64_t n = rows * J;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x) {
        float* p = P + (l / J) * ld + (l % J);
        const float v = fmaf(alpha, g[l], *p);
        *p = nonneg ? project(v) : v;
    }
}
cudaError_t launch_rows_step(float* P, int ld, const float* g, int64_t rows, int J, float alpha,
                             int nonneg, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((rows * J + 255) / 256, 4096);
    k_rows_step<<<grid, 256, 0, s>>>(P, ld, g, rows, J, alpha, nonneg);
    return cudaGetLastError();
}

// the same for the core: G (padded) += alpha * dG (dense unpadded); with cp only the
// hyper-diagonal is a parameter
__global__ void k_core_step(float* G, const float* dG, int N, int4 Jv, int JP, float alpha, int nonneg,
                            int cp) {
    const int JPR = round4(JP);
    const int Jn[4] = {Jv.x, Jv.y, Jv.z, Jv.w};
    int64_t Pd = 1;
    for (int n = 0; n < N; ++n) Pd *= Jn[n];
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < Pd;
         l += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = l, q = 0, mul = 1;
        int jl = 0, j0 = -1;
        bool diag = true;
        for (int n = N - 1; n >= 0; --n) {
            const int j = (int)(r % Jn[n]);
            r /= Jn[n];
            if (j0 < 0) j0 = j;
            diag = diag && j == j0;
            if (n == N - 1) jl = j;
            else { q += j * mul; mul *= JP; }
        }
        if (cp && !diag) continue;
        float* p = G + q * JPR + jl;
        const float v = fmaf(alpha, dG[l], *p);
        *p = nonneg ? project(v) : v;
    }
}
cudaError_t launch_core_step(float* G, const float* dG, int N, const int* J, int JP, float alpha,
                             int nonneg, int cp, cudaStream_t s) {
    int4 Jv = make_int4(J[0], N > 1 ? J[1] : 1, N > 2 ? J[2] : 1, N > 3 ? J[3] : 1);
    k_core_step<<<64, 256, 0, s>>>(G, dG, N, Jv, JP, alpha, nonneg, cp);
    return cudaGetLastError();
}
}  // namespace s3
