// Per-tile bookkeeping shared by the HOGWILD kernels (FP32 and BF16 forms): the tile's row
// gradient slots in shared memory, its coupled-matrix entries, and the final row steps.
#pragma once
#include "common.cuh"
#include "tensor_fp32.cuh"

namespace s3 {

// A tile's row gradients go to slots in shared memory, one slot per event (the grouping
// numbers a group's events of every factor in row order, so the events of one row occupy
// consecutive slots); the flush sums each row's slots in slot order.  No shared-memory
// atomics, and a fixed summation order inside the tile.
//
// The FP32 kernel's prefetch warp loads, one tile ahead, everything a tile reads besides the
// parameters into one of two metadata buffers (HogMeta): the tile index, its tensor entries'
// indices, values and slot positions, its coupled entries and its segment table.  Offsets
// inside a buffer, in 4-byte words:
struct HogMeta {
    int tidx;           // [N][ST] row indices of the tile's tensor entries
    int tpos;           // [N][ST] their slot positions
    int tval;           // [ST] their values
    int c_r, c_k, c_pu, c_pv, c_y, c_m;   // [ccap] coupled entries: row, column, slots, value,
                                          // matrix (all matrices of the tile in order)
    int tab[kMaxF];     // [max_seg[F]] x 16 bytes: segment table of factor F
    int size;           // words per buffer (a multiple of 4)
};
// header words of a metadata buffer
constexpr int kMetaTile = 0;    // tile index (int64 in words 0-1)
constexpr int kMetaNb = 2;      // tensor entries
constexpr int kMetaNc = 3;      // coupled entries (all matrices)
constexpr int kMetaNseg = 4;    // [kMaxF] segments per factor
constexpr int kMetaHeader = 16; // words (4 + kMaxF)

struct HogSmem {
    int off[kMaxF];    // per-factor offset (floats) of the slot rows in dynamic shared memory
    int toff[kMaxF];   // per-factor offset (floats) of the tile's segment table (BF16 kernel)
    int noff;          // offset (floats) of the tile's segment counts (kMaxF ints; BF16 kernel)
    int nF;
    int meta[2];       // FP32 kernel: offsets (words) of the two metadata buffers
    HogMeta M;
};

// Floats per slot row.  Rows are written with 16-byte stores, which a warp issues in phases
// of 8 lanes; an odd number of 16-byte units per row puts the 8 lanes' rows on distinct banks.
__host__ __device__ constexpr int slot_stride(int JPR) { return (JPR / 4) % 2 ? JPR : JPR + 4; }

// one gradient row (JPR values, zero padding included) into its slot
template <int JPR>
__device__ __forceinline__ void put_slot(float* smem, const HogSmem& H, int F, int32_t slot,
                                         const float (&c)[JPR]) {
    float* d = smem + H.off[F] + slot * slot_stride(JPR);
#pragma unroll
    for (int q = 0; q < JPR / 4; ++q) st4(d + 4 * q, make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]));
}

// A row of P.ld floats (coherent loads) into JP >= P.ld registers, zero beyond: the BF16
// form computes at a rank padded past the layout's.
template <int JP>
__device__ __forceinline__ void load_row_ld(const float* __restrict__ p, int ld, float (&a)[JP]) {
#pragma unroll
    for (int q = 0; q < JP / 4; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * q < ld) v = ld4_cg(p + 4 * q);
        a[4 * q] = v.x;
        a[4 * q + 1] = v.y;
        a[4 * q + 2] = v.z;
        a[4 * q + 3] = v.w;
    }
}

// Eq. (8), coupled rows, for the coupled entries of a tile whose array ranges are in shared
// memory (slo / shi, indexed as the lanes of hog_ranges: lane 1 + m holds matrix m): read the
// current rows (P.ld floats each, zero-extended to JP) and write the gradients to their
// slots (JP floats).  Threads first, first + stride, ... take the entries.
template <int JP>
__device__ __forceinline__ void hog_coupled(const DParams& P, const DGroup& Gr, const int64_t* slo,
                                            const int64_t* shi, float* smem, const HogSmem& H,
                                            int first, int stride) {
    constexpr int JPR = round4(JP);
    for (int m = 0; m < P.M; ++m) {
        const int c = P.cmode[m];
        const int64_t c0 = slo[1 + m], c1 = shi[1 + m];
        const float lm = P.lambda_m;
        for (int64_t e = c0 + first; e < c1; e += stride) {
            const int32_t r = __ldg(Gr.cr[m] + e), k = __ldg(Gr.cc[m] + e);
            float u[JPR], v[JPR];
            load_row_ld<JPR>(P.U[c] + (int64_t)r * P.ld, P.ld, u);
            load_row_ld<JPR>(P.V[m] + (int64_t)k * P.ld, P.ld, v);
            float yh = 0.f;
#pragma unroll
            for (int j = 0; j < JP; ++j) yh = fmaf(u[j], v[j], yh);
            const float err = __ldg(Gr.cval[m] + e) - yh;
            const float rv = lm * P.lambda_reg * __ldg(P.inv_cnt[P.N + m] + k);
            float du[JPR], dv[JPR];
#pragma unroll
            for (int j = 0; j < JPR; ++j) {
                du[j] = j < JP ? -lm * err * v[j] : 0.f;
                dv[j] = j < JP ? fmaf(-lm * err, u[j], rv * v[j]) : 0.f;
            }
            put_slot<JPR>(smem, H, c, __ldg(Gr.cpos_u[m] + e), du);
            put_slot<JPR>(smem, H, P.N + m, __ldg(Gr.cpos_v[m] + e), dv);
        }
    }
}

// A tile's segment table, per factor and segment: (row, first slot, events, step scale),
// 16 bytes, in shared memory, with the segment counts, for a tile whose array ranges are in
// shared memory (slo / shi, the lanes of hog_ranges).  hog_tables_async issues the first
// three words as cp.async copies and stores the counts; once a thread has waited for its own
// copies (cp_async_wait_all), hog_tables_damp gathers the step scale of each segment it
// copied (indexed by the segment's row) the same way; the flush reads the table after a
// second wait and a barrier.  No thread stalls on these loads: the table is
// needed only by the flush, so its round trips overlap the tile's arithmetic.  Threads
// first, first + stride, ... take part.
__device__ __forceinline__ void hog_tables_async(const DParams& P, const DGroup& Gr,
                                                 const int64_t* slo, const int64_t* shi, float* smem,
                                                 const HogSmem& H, int first, int stride) {
    int* cnts = reinterpret_cast<int*>(smem + H.noff);
    for (int F = 0; F < H.nF; ++F) {
        const int64_t s0 = slo[1 + P.M + F];
        const int ns = (int)(shi[1 + P.M + F] - s0);
        if (first == 0) cnts[F] = ns;
        int* tab = reinterpret_cast<int*>(smem + H.toff[F]);
        for (int l = first; l < ns; l += stride) {
            cp_async4(tab + 4 * l, Gr.seg_row[F] + s0 + l);
            cp_async4(tab + 4 * l + 1, Gr.seg_start[F] + s0 + l);
            cp_async4(tab + 4 * l + 2, Gr.seg_cnt[F] + s0 + l);
        }
    }
}

__device__ __forceinline__ void hog_tables_damp(const DParams& P, const DGroup& Gr, const int64_t* slo,
                                                const int64_t* shi, float* smem, const HogSmem& H,
                                                int first, int stride) {
    for (int F = 0; F < H.nF; ++F) {
        const int ns = (int)(shi[1 + P.M + F] - slo[1 + P.M + F]);
        int* tab = reinterpret_cast<int*>(smem + H.toff[F]);
        for (int l = first; l < ns; l += stride) cp_async4(tab + 4 * l + 3, Gr.row_damp[F] + tab[4 * l]);
    }
}

// Eq. (8), coupled rows, for one coupled entry of matrix m (row u of U^(c), column k of
// V_m with kinv = 1 / |Omega_Y^{2,k}|, value y) whose rows were gathered already: the
// gradients to slots pu and pv
template <int JP>
__device__ __forceinline__ void hog_coupled_one(const DParams& P, float* smem, const HogSmem& H,
                                                int m, float kinv, int32_t pu, int32_t pv, float y,
                                                const float (&u)[JP], const float (&v)[JP]) {
    constexpr int JPR = round4(JP);
    float yh = 0.f;
#pragma unroll
    for (int j = 0; j < JP; ++j) yh = fmaf(u[j], v[j], yh);
    const float lm = P.lambda_m;
    const float err = y - yh;
    const float rv = lm * P.lambda_reg * kinv;
    float du[JPR], dv[JPR];
#pragma unroll
    for (int j = 0; j < JPR; ++j) {
        du[j] = j < JP ? -lm * err * v[j] : 0.f;
        dv[j] = j < JP ? fmaf(-lm * err, u[j], rv * v[j]) : 0.f;
    }
    put_slot<JPR>(smem, H, P.cmode[m], pu, du);
    put_slot<JPR>(smem, H, P.N + m, pv, dv);
}

// apply tile t's row steps: per touched row and 4 components, the sum of its slots in slot
// order, then one vector atomic, step = -eta * (step scale of the row) * (sum or mean of the
// row's gradients in the tile).  Slot rows hold JPR floats; global rows P.ld <= JPR, whose
// P.ld / 4 quads are written.  Threads first, first + stride, ... take the (segment, quad)
// items.
template <int JPR>
__device__ __forceinline__ void hog_flush(const DParams& P, const float* smem, const HogSmem& H,
                                          float eta, int row_mean, int first, int stride) {
    constexpr int SS = slot_stride(JPR);
    const int* cnts = reinterpret_cast<const int*>(smem + H.noff);
    const int nq = P.ld / 4;
    for (int F = 0; F < H.nF; ++F) {
        const int nseg = cnts[F];
        const float* sa = smem + H.off[F];
        const int4* tab = reinterpret_cast<const int4*>(smem + H.toff[F]);
        float* base = F < P.N ? P.U[F] : P.V[F - P.N];
        for (int l = first; l < nseg * nq; l += stride) {
            const int s = l / nq, q = l % nq;
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
            const float sc = -eta * __int_as_float(sg.w) / (row_mean ? (float)cnt : 1.f);
            float* dst = base + (int64_t)rr * P.ld + 4 * q;
            red_add_v4(dst, sc * acc.x, sc * acc.y, sc * acc.z, sc * acc.w);
            if (P.nonneg) red_proj_v4(dst);
        }
    }
}

// The prefetch warp's part.  Its lanes hold the ranges of one tile: lane 0 its tensor
// entries, lanes 1..M its coupled entries of matrix lane - 1, the next nF lanes its segments
// of factor lane - 1 - M (lo = hi = 0 elsewhere, and for t >= n_tiles).  hog_ranges issues
// the loads; their values are first used one tile later, so the round trip overlaps the
// copies of the tile in between.
__device__ __forceinline__ void hog_ranges(const DParams& P, const DGroup& Gr, int64_t t,
                                           int64_t n_tiles, const HogSmem& H, int lane,
                                           int64_t& lo, int64_t& hi) {
    lo = 0;
    hi = 0;
    if (t >= n_tiles) return;
    if (lane == 0) {
        lo = Gr.t_off[t];
        hi = Gr.t_off[t + 1];
    } else if (lane <= P.M) {
        lo = Gr.c_off[lane - 1][t];
        hi = Gr.c_off[lane - 1][t + 1];
    } else if (lane <= P.M + H.nF) {
        lo = Gr.seg_off[lane - 1 - P.M][t];
        hi = Gr.seg_off[lane - 1 - P.M][t + 1];
    }
}

// Tile t's metadata into the buffer at meta (see HogMeta), from the ranges of hog_ranges:
// every array as asynchronous copies, then each segment's row damping (indexed by the
// segment's row, a second round trip).  Only the copying lanes touch the buffer; the CTA
// barrier that follows publishes it.  t >= n_tiles writes only the tile index (the CTA
// stops there).
template <int N>
__device__ __forceinline__ void hog_prefetch(const DParams& P, const DGroup& Gr, int64_t t,
                                             int64_t n_tiles, int64_t lo, int64_t hi, int* meta,
                                             const HogSmem& H, int ST, int lane) {
    if (lane == 0) *reinterpret_cast<int64_t*>(meta + kMetaTile) = t;
    if (t >= n_tiles) return;
    const HogMeta& M = H.M;
    const int cnt = (int)(hi - lo);
    const int64_t e0 = __shfl_sync(0xffffffffu, lo, 0);
    const int nb = __shfl_sync(0xffffffffu, cnt, 0);
    for (int l = lane; l < nb; l += 32) {
#pragma unroll
        for (int n = 0; n < N; ++n) {
            cp_async4(meta + M.tidx + n * ST + l, Gr.tidx[n] + e0 + l);
            cp_async4(meta + M.tpos + n * ST + l, Gr.tpos[n] + e0 + l);
        }
        cp_async4(meta + M.tval + l, Gr.tval + e0 + l);
    }
    int nc = 0;
    for (int m = 0; m < P.M; ++m) {
        const int64_t c0 = __shfl_sync(0xffffffffu, lo, 1 + m);
        const int n = __shfl_sync(0xffffffffu, cnt, 1 + m);
        for (int l = lane; l < n; l += 32) {
            const int w = nc + l;
            cp_async4(meta + M.c_r + w, Gr.cr[m] + c0 + l);
            cp_async4(meta + M.c_k + w, Gr.cc[m] + c0 + l);
            cp_async4(meta + M.c_pu + w, Gr.cpos_u[m] + c0 + l);
            cp_async4(meta + M.c_pv + w, Gr.cpos_v[m] + c0 + l);
            cp_async4(meta + M.c_y + w, Gr.cval[m] + c0 + l);
            meta[M.c_m + w] = m;
        }
        nc += n;
    }
    for (int F = 0; F < H.nF; ++F) {
        const int64_t s0 = __shfl_sync(0xffffffffu, lo, 1 + P.M + F);
        const int ns = __shfl_sync(0xffffffffu, cnt, 1 + P.M + F);
        if (lane == 0) meta[kMetaNseg + F] = ns;
        int* tab = meta + M.tab[F];
        for (int l = lane; l < ns; l += 32) {
            cp_async4(tab + 4 * l, Gr.seg_row[F] + s0 + l);
            cp_async4(tab + 4 * l + 1, Gr.seg_start[F] + s0 + l);
            cp_async4(tab + 4 * l + 2, Gr.seg_cnt[F] + s0 + l);
        }
    }
    cp_async_wait_all();
    // each lane reads back only the rows it copied itself
    for (int F = 0; F < H.nF; ++F) {
        const int ns = __shfl_sync(0xffffffffu, cnt, 1 + P.M + F);
        int* tab = meta + M.tab[F];
        for (int l = lane; l < ns; l += 32) cp_async4(tab + 4 * l + 3, Gr.row_damp[F] + tab[4 * l]);
    }
    cp_async_wait_all();
    if (lane == 0) {
        meta[kMetaNb] = nb;
        meta[kMetaNc] = nc;
    }
}

// hog_flush over the segment table of a metadata buffer; threads first, first + stride, ...
// take the (segment, quad) items of all factors in one sequence, so that the long segments
// at the head of every factor's table land on different threads.
template <int JPR>
__device__ __forceinline__ void hog_flush_meta(const DParams& P, const float* smem, const HogSmem& H,
                                               const int* meta, float eta, int row_mean, int first,
                                               int stride) {
    constexpr int SS = slot_stride(JPR), QD = JPR / 4;
    int F = 0, fbase = 0, fend = meta[kMetaNseg] * QD;
    for (int l = first;; l += stride) {
        while (l >= fend && F < H.nF) {
            ++F;
            fbase = fend;
            if (F < H.nF) fend += meta[kMetaNseg + F] * QD;
        }
        if (F >= H.nF) break;
        const float* sa = smem + H.off[F];
        const int4* tab = reinterpret_cast<const int4*>(meta + H.M.tab[F]);
        float* base = F < P.N ? P.U[F] : P.V[F - P.N];
        const int s = (l - fbase) / QD, q = (l - fbase) % QD;
        const int4 sg = tab[s];   // row, first slot, events, step scale
        const int32_t rr = sg.x, st = sg.y, cnt = sg.z;
        const float* src = sa + st * SS + 4 * q;
        float4 acc = *reinterpret_cast<const float4*>(src);
#pragma unroll 4
        for (int k = 1; k < cnt; ++k) {
            const float4 v = *reinterpret_cast<const float4*>(src + k * SS);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        const float sc = -eta * __int_as_float(sg.w) / (row_mean ? (float)cnt : 1.f);
        float* dst = base + (int64_t)rr * JPR + 4 * q;
        red_add_v4(dst, sc * acc.x, sc * acc.y, sc * acc.z, sc * acc.w);
        if (P.nonneg) red_proj_v4(dst);
    }
}

// Layout of the FP32 kernel's shared memory after base_floats (the core copies and the
// stage): slot rows of every factor, then the two metadata buffers (ST tensor entries and
// ccap coupled entries at most per tile).  Returns the total in floats.
__host__ inline size_t hog_meta_smem_floats(int JPR, int N, int ST, const int64_t* max_events,
                                            const int64_t* max_segs, int64_t ccap, int nF,
                                            HogSmem* H, size_t base_floats) {
    size_t off = base_floats;
    for (int F = 0; F < nF; ++F) {
        if (H) H->off[F] = (int)off;
        off += (size_t)max_events[F] * slot_stride(JPR);
    }
    HogMeta M{};
    size_t w = kMetaHeader;
    M.tidx = (int)w; w += (size_t)N * ST;
    M.tpos = (int)w; w += (size_t)N * ST;
    M.tval = (int)w; w += (size_t)ST;
    M.c_r = (int)w; w += (size_t)ccap;
    M.c_k = (int)w; w += (size_t)ccap;
    M.c_pu = (int)w; w += (size_t)ccap;
    M.c_pv = (int)w; w += (size_t)ccap;
    M.c_y = (int)w; w += (size_t)ccap;
    M.c_m = (int)w; w += (size_t)ccap;
    w = (w + 3) & ~(size_t)3;
    for (int F = 0; F < kMaxF; ++F) {
        M.tab[F] = (int)w;
        if (F < nF) w += (size_t)max_segs[F] * 4;
    }
    M.size = (int)((w + 3) & ~(size_t)3);
    if (H) {
        H->M = M;
        H->meta[0] = (int)off;
        H->meta[1] = (int)(off + M.size);
        H->nF = nF;
        H->noff = 0;
        for (int F = 0; F < kMaxF; ++F) H->toff[F] = 0;
    }
    return off + 2 * (size_t)M.size;
}

// Shared-memory layout after base_floats: every factor's slot rows (max_events[F] rows),
// then its segment table (max_segs[F] x 16 bytes), then the kMaxF segment counts; each area
// 16-byte aligned.  Returns the total in floats.
__host__ inline size_t hog_smem_floats(int JPR, const int64_t* max_events, const int64_t* max_segs,
                                       int nF, HogSmem* H, size_t base_floats) {
    size_t off = base_floats;
    for (int F = 0; F < nF; ++F) {
        if (H) H->off[F] = (int)off;
        off += (size_t)max_events[F] * slot_stride(JPR);
    }
    for (int F = 0; F < nF; ++F) {
        if (H) H->toff[F] = (int)off;
        off += (size_t)max_segs[F] * 4;
    }
    if (H) H->noff = (int)off;
    off += kMaxF;
    off = (off + 3) & ~(size_t)3;
    if (H) H->nF = nF;
    return off;
}

}  // namespace s3
