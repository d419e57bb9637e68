// Shared device-side definitions of the S3CMTF sm_103a path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace s3 {

constexpr int kMaxN = 4;               // tensor order supported by the kernels: 3 or 4
constexpr int kMaxM = 8;               // coupled matrices
constexpr int kMaxF = kMaxN + kMaxM;   // factor matrices: U^(1..N), then V_1..V_M
constexpr int kTile = 256;             // tensor entries per CTA tile (one per thread)

// Parameters and per-row constants, all device pointers.  Every factor matrix is stored
// row-major with row stride `ld` floats (J padded to a multiple of 4, zero padding); the
// core is stored padded to JP in every mode with the last mode's rows padded to `ldg`.
struct DParams {
    float* G;
    float* U[kMaxN];
    float* V[kMaxM];
    const float* inv_cnt[kMaxF];   // 1/|Omega^{n,i}| for factor n, 1/|Omega_Y^{2,k}| for
                                   // factor N+m; 0 for rows without observed entries
    int ld;                        // row stride (floats) of every factor matrix
    int ldg;                       // row stride (floats) of the padded core's last mode
    int jp;                        // padded rank: the core is jp x .. x jp x ldg
    int cp;                        // 1: S3CMTF-CP, the core is hyper-diagonal
    int nonneg;                    // 1: every step is followed by max(0, .) (projected SGD)
    int N, M;
    int cmode[kMaxM];
    float lambda_reg, lambda_m, inv_nnz;
};

// One grouping of the items (minibatches, HOGWILD tiles or gradient chunks), device arrays.
// Tensor entries and coupled entries are stored in group order.  For every factor F each
// group's occurrences ("events") of rows are sorted by row into segments; `tpos`/`cpos_*`
// give an event's local slot (position among the group's sorted events of that factor) or
// local segment, depending on the grouping's kind.
// Segments of up to kShortSeg events are summed by one thread, longer ones by a warp, and
// (where a grouping marks them) those of more than kHugeSeg events by a whole CTA.
constexpr int kShortSeg = 16;
constexpr int kHugeSeg = 1024;

struct DGroup {
    const int64_t* t_off;
    const int32_t* tidx[kMaxN];
    const float* tval;
    const int32_t* tpos[kMaxN];
    const int64_t* c_off[kMaxM];
    const int32_t* cr[kMaxM];
    const int32_t* cc[kMaxM];
    const float* cval[kMaxM];
    const int32_t* cpos_u[kMaxM];
    const int32_t* cpos_v[kMaxM];
    const int64_t* seg_off[kMaxF];     // [groups + 1] global segment range of each group
    const int32_t* seg_row[kMaxF];     // row of each segment
    const int32_t* seg_start[kMaxF];   // local slot of the segment's first event
    const int32_t* seg_cnt[kMaxF];     // events in the segment
    const int32_t* seg_nlong[kMaxF];   // [groups] segments of more than kShortSeg events, which
                                       // come first in their group (slot-positioned groupings)
    const int64_t* slot_off[kMaxF];    // [groups + 1] global slot range of each group
    const float* row_damp[kMaxF];      // HOGWILD groupings: step scale of every row of each
                                       // factor (the staleness-aware step), else null
};

__host__ __device__ constexpr int round4(int x) { return (x + 3) & ~3; }

__device__ __forceinline__ float4 ld4_nc(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4_cg(const float* p) {
    return __ldcg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ void st4(float* p, float4 v) {
    *reinterpret_cast<float4*>(p) = v;
}

// Asynchronous 4- and 8-byte copies global -> shared (no register round trip; both addresses
// aligned to the size); cp_async_wait_all waits for every copy the thread issued.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                 :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Vector atomic add of 4 consecutive floats (16-byte aligned) in global memory.
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// max(0, v) of the non-negative form, for values one thread owns; a NaN becomes 0
__device__ __forceinline__ float project(float v) { return v > 0.f ? v : 0.f; }
__device__ __forceinline__ void project4(float4& u) {
    u.x = project(u.x);
    u.y = project(u.y);
    u.z = project(u.z);
    u.w = project(u.w);
}

// The projection max(0, v) of 4 consecutive floats in global memory that other threads may
// be adding to: an atomic max of each value's bit pattern, read as a signed integer, with 0.
// A float with its sign bit clear is a non-negative integer and keeps its value; one with it
// set (negative, -0, or a NaN with the sign bit set) is a negative integer and becomes +0.
// Issued by the thread that has just added to the same values, after its add (one thread's
// operations on one address take effect in program order), so the last operation on every
// touched value is a projection.
__device__ __forceinline__ void red_proj_v4(float* p) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
        asm volatile("red.global.max.s32 [%0], %1;" :: "l"(p + i), "r"(0) : "memory");
}
__device__ __forceinline__ void red_proj(float* p) {
    asm volatile("red.global.max.s32 [%0], %1;" :: "l"(p), "r"(0) : "memory");
}

// Neumaier-compensated FP32 accumulation.
struct Kahan {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

// Compensated sums, component by component, of the rows src + e * ld (4 * C4 floats each,
// 16-byte aligned) for e = e0, e0 + step, ... < cnt, added in that order; U rows' loads are
// issued together (the last batch's with predicates), so a short sum costs one round trip.
template <int C4>
__device__ __forceinline__ void rows_sum(const float* src, int64_t ld, int e0, int step, int cnt,
                                         Kahan (&k)[4 * C4]) {
    constexpr int U = C4 <= 4 ? 4 : 2;
    for (int e = e0; e < cnt; e += U * step) {
        float4 v[U][C4];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < C4; ++q)
                v[u][q] = e + u * step < cnt
                              ? __ldcg(reinterpret_cast<const float4*>(src + (int64_t)(e + u * step) * ld + 4 * q))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (e + u * step >= cnt) break;
#pragma unroll
            for (int q = 0; q < C4; ++q) {
                k[4 * q].add(v[u][q].x);
                k[4 * q + 1].add(v[u][q].y);
                k[4 * q + 2].add(v[u][q].z);
                k[4 * q + 3].add(v[u][q].w);
            }
        }
    }
}

}  // namespace s3
