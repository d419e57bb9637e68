// C ABI of the S3CMTF sm_103a path (declared in include/s3cmtf.h).  Host code: argument
// validation, the layout build, device buffers and the launch sequence of each call.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "layout.h"
#include "s3cmtf.h"

using namespace s3;

static constexpr size_t kMaxSmem = 227 * 1024;   // dynamic shared memory per CTA on sm_103a
// default HOGWILD staleness budget for 3-way tensors up to rank 10: tensor entries in flight
// at once (152 CTAs x 192 entries)
static constexpr int64_t kHogInflight = 29184;

// The default budget at the largest rank J: kHogInflight up to rank 10, then shrinking as
// (10 / J)^0.6 (22 029 at rank 16, 19 155 at 20, 14 385 at 32).  Measured on the cfg1 rating
// tensor against Algorithm 1's test-RMSE curve: at rank 10, 29 184 entries in flight keep the
// HOGWILD curve within 0.85%; at rank 16 the same number sits 1.2% above it and 21 888 within
// 0.5% (both forms).
static int64_t hog_inflight_budget(int jmax) {
    if (jmax <= 10) return kHogInflight;
    return (int64_t)std::llround((double)kHogInflight * std::pow(10.0 / (double)jmax, 0.6));
}

namespace {

// device copy of one grouping plus the host metadata needed to size launches
struct DevGrouping {
    DGroup d{};
    int64_t ngroups = 0;
    int nF = 0;
    std::vector<int64_t> t_off, c_off[kMaxM], seg_off[kMaxF], slot_off[kMaxF];
    std::vector<int32_t> seg_nlong[kMaxF], seg_nhuge[kMaxF];
    int64_t max_t = 0, max_c[kMaxM] = {}, max_seg[kMaxF] = {}, max_ev[kMaxF] = {};
    int64_t* t_src = nullptr;
    int64_t* c_src[kMaxM] = {};
    float* tval = nullptr;          // mutable aliases of d.tval / d.cval
    float* cval[kMaxM] = {};
};

}  // namespace

struct s3_ctx {
    int N = 0, M = 0, JP = 0, JPR = 0;
    int64_t I[kMaxN] = {};
    int J[kMaxN] = {};
    int cmode[kMaxM] = {};
    int64_t K[kMaxM] = {};
    int64_t nnz = 0, ynnz[kMaxM] = {}, n_union = 0;
    int64_t nnz_total = 0;          // |Omega| of the whole problem (s3_set_counts), else nnz
    s3_hparams hp{};
    uint64_t seed = 0;
    int64_t epoch = 0;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    bool failed = false;
    std::string err;
    std::vector<void*> allocs;
    int64_t bytes_allocated = 0;    // device memory taken by dalloc (against hp.device_bytes_cap)
    DParams P{};
    float* inv_cnt[kMaxF] = {};
    int64_t hog_grid = 1;
    int64_t hog_bf_grid = 0;        // BF16 HOGWILD CTAs (0: the form is not available)
    int bf_jp = 16;                 // the rank the BF16 form computes at (16, 20 or 32)
    size_t cp_smem = 0;             // S3CMTF-CP kernel's dynamic shared memory
    size_t hog_bf_smem = 0;
    int64_t hog_tile = 0, hog_per_sm = 0, hog_bf_per_sm = 0, hog_bf_tile = 0, hog_ccap = 0;
    int hog_bf_sync = 1;            // BF16 HOGWILD: tiles between two core steps of a CTA
    double* qr_parts = nullptr;     // final QR step scratch (allocated at its first call)
    double* qr_R = nullptr;
    int* qr_bad = nullptr;
    float* qr_core = nullptr;
    int64_t qr_grid = 0;
    DevGrouping mb, hog, grad, hog_bf;   // hog_bf: tiles of the BF16 kernel
    float* contrib[kMaxF] = {};
    float* core_part = nullptr;
    int64_t core_part_n = 0;       // partial slots
    float* seg_parts = nullptr;    // gradient pass: sums of the huge segments' pieces
    int* seg_done = nullptr;       // and their completion counts (zero between launches)
    float* red_parts = nullptr;
    int64_t red_parts_n = 0;       // float pairs
    double* d_red = nullptr;
    double* h_red = nullptr;       // pinned
    float* d_eta = nullptr;
    float* h_eta = nullptr;        // pinned
    int* d_flag = nullptr;
    int* h_flag = nullptr;         // pinned
    int* d_tile_counter = nullptr; // HOGWILD tile claims
    int* d_kerr = nullptr;         // set by a kernel whose bounded wait ran out
    int* d_idx_bad = nullptr;      // set by the forward kernel on an out-of-range index
    int* h_idx_bad = nullptr;      // pinned
    float* grad_w = nullptr;       // s3_gradient's weights in the gradient grouping's order
    float* grad_comp = nullptr;    // compensation buffers of the gradient (all parameters)
    int64_t grad_comp_n = 0;
    float* values_stage = nullptr; // s3_update_values staging (nnz + sum ynnz floats)
    // per grouping (minibatch, HOGWILD, gradient, BF16 HOGWILD): whether its tensor values and
    // each coupled matrix's values still wait to be gathered from values_stage
    uint8_t stale_t[4] = {};
    uint8_t stale_c[4][kMaxM] = {};
    int64_t ntest = 0;
    int32_t* test_idx[kMaxN] = {};
    float* test_val = nullptr;
    size_t hog_smem = 0;
    int hog_lanes = 1;
    int mb_grid = 0;               // CTAs of the persistent minibatch epoch
    unsigned* d_bar = nullptr;     // its grid-barrier arrival counter
    // measurement (s3_profile)
    bool prof = false;
    int64_t launches = 0;
    struct Family {
        std::vector<cudaEvent_t> ev;   // start/stop pairs
        int64_t launches = 0, entries = 0;
    } fam[4];
};

// ------------------------------------------------------------------ helpers
static int fail(s3_ctx* c, int code, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (code == S3_ERR_CUDA) c->failed = true;
    }
    return code;
}

#define CK(expr)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? S3_ERR_OOM : S3_ERR_CUDA,  \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));              \
    } while (0)

// a kernel launch of the library: counted, errors handled like CK
#define KL(expr)             \
    do {                     \
        ctx->launches += 1;  \
        CK(expr);            \
    } while (0)

// CUDA events around one launch of a measured kernel family (only while profiling)
static cudaError_t prof_mark(s3_ctx* ctx, int family) {
    if (!ctx->prof) return cudaSuccess;
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ctx->fam[family].ev.push_back(e);
    return cudaEventRecord(e, ctx->stream);
}
static void prof_count(s3_ctx* ctx, int family, int64_t entries) {
    if (!ctx->prof) return;
    ctx->fam[family].launches += 1;
    ctx->fam[family].entries += entries;
}

// every device allocation of a context; the cap of hp.device_bytes_cap makes an allocation
// beyond it fail as if the device were full
template <typename T>
static cudaError_t dalloc(s3_ctx* ctx, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    const int64_t bytes = (int64_t)(n * sizeof(T));
    if (ctx->hp.device_bytes_cap > 0 && ctx->bytes_allocated + bytes > ctx->hp.device_bytes_cap)
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) {
        ctx->allocs.push_back(*p);
        ctx->bytes_allocated += bytes;
    }
    return e;
}

static uint64_t wait_ns(const s3_ctx* ctx) {
    return ctx->hp.wait_limit_us > 0 ? (uint64_t)ctx->hp.wait_limit_us * 1000ull : 2000000000ull;
}

template <typename T>
static cudaError_t upload(s3_ctx* ctx, T** p, const std::vector<T>& v) {
    cudaError_t e = dalloc(ctx, p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
}

static bool usable(const s3_ctx* c) { return c && !c->failed; }

static float eta_of(const s3_ctx* c, int64_t t) {
    return (float)((double)c->hp.lr0 / (1.0 + (double)c->hp.mu * (double)t));
}

static int upload_grouping(s3_ctx* ctx, const HostGrouping& H, DevGrouping& D) {
    D.ngroups = H.ngroups;
    D.nF = H.nF;
    D.t_off = H.t_off;
    D.max_t = H.max_t;
    int64_t* toff = nullptr;
    CK(upload(ctx, &toff, H.t_off));
    D.d.t_off = toff;
    for (int n = 0; n < ctx->N; ++n) {
        int32_t *a = nullptr, *b = nullptr;
        CK(upload(ctx, &a, H.tidx[n]));
        CK(upload(ctx, &b, H.tpos[n]));
        D.d.tidx[n] = a;
        D.d.tpos[n] = b;
    }
    CK(upload(ctx, &D.tval, H.tval));
    D.d.tval = D.tval;
    CK(upload(ctx, &D.t_src, H.t_src));
    for (int m = 0; m < ctx->M; ++m) {
        D.c_off[m] = H.c_off[m];
        D.max_c[m] = H.max_c[m];
        int64_t* co = nullptr;
        int32_t *r = nullptr, *c = nullptr, *pu = nullptr, *pv = nullptr;
        CK(upload(ctx, &co, H.c_off[m]));
        CK(upload(ctx, &r, H.cr[m]));
        CK(upload(ctx, &c, H.cc[m]));
        CK(upload(ctx, &D.cval[m], H.cval[m]));
        CK(upload(ctx, &pu, H.cpos_u[m]));
        CK(upload(ctx, &pv, H.cpos_v[m]));
        CK(upload(ctx, &D.c_src[m], H.c_src[m]));
        D.d.c_off[m] = co;
        D.d.cr[m] = r;
        D.d.cc[m] = c;
        D.d.cval[m] = D.cval[m];
        D.d.cpos_u[m] = pu;
        D.d.cpos_v[m] = pv;
    }
    for (int F = 0; F < H.nF; ++F) {
        D.seg_off[F] = H.seg_off[F];
        D.seg_nlong[F] = H.seg_nlong[F];
        D.seg_nhuge[F] = H.seg_nhuge[F];
        D.slot_off[F] = H.slot_off[F];
        D.max_seg[F] = H.max_seg[F];
        D.max_ev[F] = H.max_ev[F];
        int64_t *so = nullptr, *sl = nullptr;
        int32_t *sr = nullptr, *ss = nullptr, *sc = nullptr, *sn = nullptr;
        CK(upload(ctx, &so, H.seg_off[F]));
        CK(upload(ctx, &sn, H.seg_nlong[F]));
        CK(upload(ctx, &sl, H.slot_off[F]));
        CK(upload(ctx, &sr, H.seg_row[F]));
        CK(upload(ctx, &ss, H.seg_start[F]));
        CK(upload(ctx, &sc, H.seg_cnt[F]));
        D.d.seg_off[F] = so;
        D.d.slot_off[F] = sl;
        D.d.seg_row[F] = sr;
        D.d.seg_start[F] = ss;
        D.d.seg_cnt[F] = sc;
        D.d.seg_nlong[F] = sn;
    }
    // keep the host vectors alive until the async copies are done
    CK(cudaStreamSynchronize(ctx->stream));
    return S3_OK;
}

// frees a host grouping's per-item arrays once they are on the device (its per-group offsets
// and sizes stay: the launches are sized from them)
static void release_items(HostGrouping& H) {
    auto drop = [](auto& v) { std::decay_t<decltype(v)>().swap(v); };
    for (auto& v : H.tidx) drop(v);
    for (auto& v : H.tpos) drop(v);
    drop(H.tval);
    drop(H.t_src);
    for (int m = 0; m < 8; ++m) {
        drop(H.cr[m]);
        drop(H.cc[m]);
        drop(H.cval[m]);
        drop(H.cpos_u[m]);
        drop(H.cpos_v[m]);
        drop(H.c_src[m]);
    }
    for (int F = 0; F < 12; ++F) {
        drop(H.seg_row[F]);
        drop(H.seg_start[F]);
        drop(H.seg_cnt[F]);
    }
}

static void fill_params(s3_ctx* ctx) {
    DParams& P = ctx->P;
    P.N = ctx->N;
    P.M = ctx->M;
    P.ld = ctx->JPR;
    P.ldg = ctx->JPR;
    P.jp = ctx->JP;
    P.cp = ctx->hp.cp;
    P.nonneg = ctx->hp.nonneg;
    for (int m = 0; m < ctx->M; ++m) P.cmode[m] = ctx->cmode[m];
    for (int F = 0; F < ctx->N + ctx->M; ++F) P.inv_cnt[F] = ctx->inv_cnt[F];
    P.lambda_reg = ctx->hp.lambda_reg;
    P.lambda_m = ctx->hp.lambda_m;
    P.inv_nnz = (float)(1.0 / (double)ctx->nnz);
}

static int64_t factor_rows(const s3_ctx* ctx, int F) {
    return F < ctx->N ? ctx->I[F] : ctx->K[F - ctx->N];
}
static int factor_cols(const s3_ctx* ctx, int F) {
    return F < ctx->N ? ctx->J[F] : ctx->J[ctx->cmode[F - ctx->N]];
}
static float* factor_ptr(const s3_ctx* ctx, int F) {
    return F < ctx->N ? ctx->P.U[F] : ctx->P.V[F - ctx->N];
}

// reads a host-or-device array into a host vector
template <typename T>
static cudaError_t to_host(const T* p, int64_t n, int device_ptrs, std::vector<T>& out) {
    out.resize((size_t)n);
    if (n == 0) return cudaSuccess;
    if (device_ptrs) return cudaMemcpy(out.data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost);
    memcpy(out.data(), p, (size_t)n * sizeof(T));
    return cudaSuccess;
}

static int ensure_red(s3_ctx* ctx, int64_t pairs) {
    if (pairs <= ctx->red_parts_n) return S3_OK;
    if (ctx->red_parts) {
        cudaFree(ctx->red_parts);
        ctx->bytes_allocated -= ctx->red_parts_n * 2 * (int64_t)sizeof(float);
    }
    ctx->allocs.erase(std::remove(ctx->allocs.begin(), ctx->allocs.end(), (void*)ctx->red_parts),
                      ctx->allocs.end());
    CK(dalloc(ctx, &ctx->red_parts, (size_t)pairs * 2));
    ctx->red_parts_n = pairs;
    return S3_OK;
}

// ------------------------------------------------------------------ init
extern "C" int s3_init(s3_ctx** out, const s3_coo_tensor* train, const s3_coo_matrix* Y,
                       int n_coupled, const int* J, const s3_hparams* hp, uint64_t seed,
                       const int64_t* order, int device_ptrs, void* stream) {
    if (!out) return S3_ERR_ARG;
    *out = nullptr;
    s3_ctx* ctx = new s3_ctx();
    auto bail = [&](int code, const std::string& m) {
        // keep the context so the caller can read the message; it is marked failed
        ctx->err = m;
        ctx->failed = true;
        *out = ctx;
        return code;
    };
    if (!train || !J || !hp) return bail(S3_ERR_ARG, "train, J and hp are required");
    const int N = train->n_modes;
    if (N != 3 && N != 4) return bail(S3_ERR_ARG, "n_modes must be 3 or 4");
    if (n_coupled < 0 || n_coupled > kMaxM) return bail(S3_ERR_ARG, "n_coupled must be 0..8");
    if (n_coupled > 0 && !Y) return bail(S3_ERR_ARG, "Y is NULL but n_coupled > 0");
    if (!train->dims || !train->idx || !train->val) return bail(S3_ERR_ARG, "train arrays missing");
    if (train->nnz < 1) return bail(S3_ERR_ARG, "train needs at least one entry");
    if (train->nnz > INT32_MAX) return bail(S3_ERR_ARG, "more than 2^31-1 train entries");
    ctx->N = N;
    ctx->M = n_coupled;
    ctx->hp = *hp;
    ctx->seed = seed;
    ctx->nnz = train->nnz;
    ctx->nnz_total = train->nnz;
    ctx->stream = (cudaStream_t)stream;
    int Jmax = 0;
    for (int n = 0; n < N; ++n) {
        ctx->I[n] = train->dims[n];
        ctx->J[n] = J[n];
        if (ctx->I[n] < 1 || ctx->I[n] > INT32_MAX) return bail(S3_ERR_ARG, "dims out of range");
        if (J[n] < 1 || J[n] > 32) return bail(S3_ERR_ARG, "J_n must be in 1..32");
        Jmax = std::max(Jmax, J[n]);
    }
    ctx->JP = tensor_supported_jp(N, Jmax);
    if (!ctx->JP) return bail(S3_ERR_ARG, "unsupported rank for this order (N=4 supports J<=8)");
    ctx->JPR = round4(ctx->JP);
    if (hp->cp)
        for (int n = 1; n < N; ++n)
            if (J[n] != J[0]) return bail(S3_ERR_ARG, "S3CMTF-CP (hp.cp = 1) needs equal ranks in every mode");
    if (!(hp->lr0 > 0.f) || !(hp->mu >= 0.f) || !(hp->lambda_reg >= 0.f) || !(hp->lambda_m >= 0.f) ||
        !(hp->core_scale >= 0.f) || hp->batch < 1 || (hp->row_rule != 0 && hp->row_rule != 1) ||
        hp->hog_tile < 0 || hp->hog_ctas < 0 || hp->mb_ctas < 0 || (hp->cp != 0 && hp->cp != 1) ||
        (hp->nonneg != 0 && hp->nonneg != 1) || hp->grad_chunk < 0 || hp->hog_core_sync < 0 ||
        hp->wait_limit_us < 0 || hp->device_bytes_cap < 0)
        return bail(S3_ERR_ARG, "invalid hyper-parameters");
    for (int m = 0; m < n_coupled; ++m) {
        const s3_coo_matrix& y = Y[m];
        if (y.coupled_mode < 0 || y.coupled_mode >= N) return bail(S3_ERR_ARG, "coupled_mode out of range");
        if (y.rows != ctx->I[y.coupled_mode]) return bail(S3_ERR_ARG, "coupled rows != dims[coupled_mode]");
        if (y.cols < 1 || y.cols > INT32_MAX) return bail(S3_ERR_ARG, "coupled cols out of range");
        if (y.nnz < 0 || (y.nnz > 0 && (!y.r || !y.c))) return bail(S3_ERR_ARG, "coupled arrays missing");
        ctx->cmode[m] = y.coupled_mode;
        ctx->K[m] = y.cols;
        ctx->ynnz[m] = y.nnz;
    }
    ctx->n_union = ctx->nnz;
    for (int m = 0; m < n_coupled; ++m) ctx->n_union += ctx->ynnz[m];
    // ---- bring the inputs to the host and validate them
    HostInput in;
    in.N = N;
    in.M = n_coupled;
    in.nnz = ctx->nnz;
    std::vector<int32_t> hidx[kMaxN], hyr[kMaxM], hyc[kMaxM];
    std::vector<float> hval, hyv[kMaxM];
    std::vector<int64_t> hord;
    {
        cudaError_t e = cudaSuccess;
        for (int n = 0; n < N && e == cudaSuccess; ++n) e = to_host(train->idx[n], ctx->nnz, device_ptrs, hidx[n]);
        if (e == cudaSuccess) e = to_host(train->val, ctx->nnz, device_ptrs, hval);
        for (int m = 0; m < n_coupled && e == cudaSuccess; ++m) {
            e = to_host(Y[m].r, Y[m].nnz, device_ptrs, hyr[m]);
            if (e == cudaSuccess) e = to_host(Y[m].c, Y[m].nnz, device_ptrs, hyc[m]);
            if (e == cudaSuccess) {
                if (Y[m].val) e = to_host(Y[m].val, Y[m].nnz, device_ptrs, hyv[m]);
                else hyv[m].assign((size_t)Y[m].nnz, 1.0f);
            }
        }
        if (e == cudaSuccess && order) e = to_host(order, ctx->n_union, device_ptrs, hord);
        if (e != cudaSuccess) return bail(S3_ERR_ARG, std::string("reading inputs: ") + cudaGetErrorString(e));
    }
    for (int n = 0; n < N; ++n) {
        for (int64_t e = 0; e < ctx->nnz; ++e) {
            const int32_t v = hidx[n][(size_t)e];
            if (v < 0 || v >= ctx->I[n])
                return bail(S3_ERR_INDEX, "tensor index out of range: mode " + std::to_string(n) +
                                              ", entry " + std::to_string(e));
        }
        in.I[n] = ctx->I[n];
        in.idx[n] = hidx[n].data();
    }
    for (int64_t e = 0; e < ctx->nnz; ++e)
        if (!std::isfinite(hval[(size_t)e])) return bail(S3_ERR_ARG, "non-finite tensor value at " + std::to_string(e));
    in.val = hval.data();
    for (int m = 0; m < n_coupled; ++m) {
        for (int64_t b = 0; b < ctx->ynnz[m]; ++b) {
            if (hyr[m][(size_t)b] < 0 || hyr[m][(size_t)b] >= Y[m].rows || hyc[m][(size_t)b] < 0 ||
                hyc[m][(size_t)b] >= Y[m].cols)
                return bail(S3_ERR_INDEX, "coupled index out of range: matrix " + std::to_string(m) +
                                              ", entry " + std::to_string(b));
            if (!std::isfinite(hyv[m][(size_t)b])) return bail(S3_ERR_ARG, "non-finite coupled value");
        }
        in.cmode[m] = ctx->cmode[m];
        in.K[m] = ctx->K[m];
        in.ynnz[m] = ctx->ynnz[m];
        in.yr[m] = hyr[m].data();
        in.yc[m] = hyc[m].data();
        in.yv[m] = hyv[m].data();
    }
    if (order) {
        std::vector<uint8_t> seen((size_t)ctx->n_union, 0);
        for (int64_t k = 0; k < ctx->n_union; ++k) {
            const int64_t v = hord[(size_t)k];
            if (v < 0 || v >= ctx->n_union || seen[(size_t)v])
                return bail(S3_ERR_INDEX, "order is not a permutation of the items");
            seen[(size_t)v] = 1;
        }
    } else {
        seeded_order(seed, ctx->n_union, hord);
    }
    // ---- layouts
    // the device (its SM count sizes the HOGWILD launches below)
    {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e != cudaSuccess) return bail(S3_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    HostGrouping hmb, hhog, hgrad, hhog_bf;
    const int nF = N + n_coupled;
    // each grouping goes to the device as soon as it is built, and its per-item host arrays
    // are freed then, so that the host holds one grouping at a time (about 70 bytes per item)
    *out = ctx;
    auto place = [&](HostGrouping& H, DevGrouping& D) -> int {
        const int rc = upload_grouping(ctx, H, D);
        if (rc == S3_OK) release_items(H);
        return rc;
    };
    int rc_up = S3_OK;
    // FP32 HOGWILD tiles hold at most T / 2 entries for 3-way tensors (T compute threads,
    // two lanes per entry; tiles of up to T / 4 entries take four), T for 4-way (one lane),
    // T = hog_compute_threads.  Default for 3-way tensors: the largest tile (192 entries up
    // to padded rank 16, 128 at 20, 64 at 32, whose core fills most of shared memory) and
    // about hog_inflight_budget(largest rank) entries in flight (CTAs capped at budget / tile):
    // the HOGWILD test-RMSE curve then stays within 1% of Algorithm 1's on the cfg1 workload
    // at ranks 10 and 16.
    const int64_t hog_t = hog_compute_threads(N, ctx->JP);
    const int64_t tile_max = N == 3 ? hog_t / 2 : hog_t;
    // (S3CMTF-CP runs its own one-thread-per-entry kernel on these tiles: 128 entries on 228
    // CTAs, the same budget in flight)
    const int64_t tile_default = N != 3 ? tile_max
                                 : hp->cp ? std::min<int64_t>(128, tile_max)
                                 : (ctx->JP <= 20 ? tile_max : hog_t / 4);
    const int64_t tile = hp->hog_tile > 0 ? std::min<int64_t>(hp->hog_tile, tile_max) : tile_default;
    ctx->hog_lanes = tensor_hog_lanes(N, ctx->JP, tile);
    // the BF16 form computes at rank 16 or 32 (the tensor cores' granularity), zero-extending
    // the context's layout
    const bool bf16_ok = N == 3 && ctx->JP <= 32;
    int jmax = 1;
    for (int n = 0; n < N; ++n) jmax = std::max(jmax, J[n]);
    // the non-negative form takes three quarters of the budget (see the staleness step below)
    const int64_t budget = hog_inflight_budget(jmax) * (hp->nonneg ? 3 : 4) / 4;
    ctx->bf_jp = ctx->JP <= 16 ? 16 : (ctx->JP == 20 ? 20 : 32);
    std::string msg = build_grouping(in, hord.data(), ctx->n_union, RULE_UNION, hp->batch, POS_SLOT, hmb, kShortSeg);
    if (msg.empty() && (rc_up = place(hmb, ctx->mb)) != S3_OK) return rc_up;
    if (msg.empty()) msg = build_grouping(in, hord.data(), ctx->n_union, RULE_TENSOR, tile, POS_SLOT, hhog);
    if (msg.empty() && (rc_up = place(hhog, ctx->hog)) != S3_OK) return rc_up;
    // HOGWILD concurrency of the FP32 form: CTAs resident at once, each on a tile of `tile`
    // entries
    if (msg.empty()) {
        int64_t ccap = 0;
        for (int m = 0; m < n_coupled; ++m) ccap += hhog.max_c[m];
        ctx->hog_ccap = ccap;
        ctx->hog_smem = tensor_hog_smem(N, ctx->JP, ctx->hog_lanes, hhog.max_ev, hhog.max_seg, ccap, nF);
        const int per_sm = ctx->hog_smem <= kMaxSmem
                               ? std::max(1, tensor_hog_blocks_per_sm(N, ctx->JP, ctx->hog_lanes,
                                                                      ctx->hog_smem))
                               : 1;
        int64_t cap = (int64_t)per_sm * ctx->num_sms;
        if (hp->hog_ctas > 0) cap = std::min<int64_t>(cap, hp->hog_ctas);
        else if (N == 3) cap = std::min<int64_t>(cap, std::max<int64_t>(1, budget / tile));
        ctx->hog_grid = std::max<int64_t>(1, std::min<int64_t>(cap, hhog.ngroups));
        ctx->hog_per_sm = per_sm;
        ctx->hog_tile = tile;
        if (hp->cp) {
            // S3CMTF-CP runs its own kernel on the same tiles and the same budget of entries in
            // flight
            ctx->cp_smem = tensor_cp_smem(ctx->JP, hhog.max_ev, hhog.max_seg, nF);
            const int cps = ctx->cp_smem <= kMaxSmem
                                ? std::max(1, tensor_cp_blocks_per_sm(N, ctx->JP, ctx->cp_smem)) : 1;
            int64_t ccap = (int64_t)cps * ctx->num_sms;
            if (hp->hog_ctas > 0) ccap = std::min<int64_t>(ccap, hp->hog_ctas);
            else ccap = std::min<int64_t>(ccap, std::max<int64_t>(1, budget / tile));
            ctx->hog_grid = std::max<int64_t>(1, std::min<int64_t>(ccap, hhog.ngroups));
            ctx->hog_per_sm = cps;
        }
    }
    // The BF16 form holds as many entries in flight as the FP32 form (the same lock-free
    // schedule: the two differ by their arithmetic only).  It takes full tiles of 128 entries
    // (the MMA's M) on as many CTAs as that makes, when they occupy at least 90% of the SMs;
    // else smaller tiles (multiples of 16, at least 32) on one CTA per SM.  With hog_ctas
    // given, that many CTAs of 128-entry tiles.  Smaller tiles also when a tile's row slots
    // and coupled entries would not fit in shared memory.
    int64_t bf_tile = tensor_hog_bf16_tile();
    if (msg.empty() && bf16_ok) {
        ctx->hog_bf_sync = hp->hog_core_sync > 0 ? hp->hog_core_sync : tensor_hog_bf16_core_sync(ctx->JP);
        const int64_t full = tensor_hog_bf16_tile();
        const int64_t inflight = ctx->hog_grid * ctx->hog_tile;
        int64_t want_ctas = 0, t0 = full;
        if (hp->hog_ctas > 0) {
            want_ctas = hp->hog_ctas;
        } else if (inflight >= full * ctx->num_sms * 9 / 10) {
            want_ctas = std::max<int64_t>(1, inflight / full);
        } else {
            t0 = std::max<int64_t>(32, std::min<int64_t>(full, inflight / ctx->num_sms / 16 * 16));
            want_ctas = std::max<int64_t>(1, inflight / t0);
        }
        for (int64_t t = t0; t >= 16; t -= 16) {
            bf_tile = t;
            hhog_bf = HostGrouping{};
            msg = build_grouping(in, hord.data(), ctx->n_union, RULE_TENSOR, bf_tile, POS_SLOT, hhog_bf);
            if (!msg.empty()) break;
            const size_t smem = tensor_hog_bf16_smem(ctx->bf_jp, hhog_bf.max_ev, hhog_bf.max_seg, nF);
            const int per_sm = smem <= kMaxSmem ? tensor_hog_bf16_blocks_per_sm(ctx->bf_jp, smem) : 0;
            if (per_sm >= 1 || t - 16 < 16) {
                const int64_t ctas = std::min<int64_t>((int64_t)std::max(per_sm, 1) * ctx->num_sms, want_ctas);
                ctx->hog_bf_grid = per_sm >= 1 ? ctas : 0;
                ctx->hog_bf_per_sm = std::max(per_sm, 1);
                ctx->hog_bf_tile = bf_tile;
                break;
            }
        }
        if (msg.empty() && (rc_up = place(hhog_bf, ctx->hog_bf)) != S3_OK) return rc_up;
    }
    // 2^22 items per gradient chunk by default: on cfg1 (14M items) a pass took 4.09 ms in
    // chunks of 2^20, 3.70 ms in chunks of 2^22 and 3.76 ms in one chunk (cfg3, 67M items:
    // 58.9, 54.8 ms at 2^23, 55.2 ms in one), while the slots stay a few hundred MB
    const int64_t grad_chunk = hp->grad_chunk > 0 ? hp->grad_chunk : 1 << 22;
    if (msg.empty()) msg = build_grouping(in, nullptr, ctx->n_union, RULE_UNION, grad_chunk, POS_SLOT, hgrad, kShortSeg,
                                             kHugeSeg);
    if (msg.empty() && (rc_up = place(hgrad, ctx->grad)) != S3_OK) return rc_up;
    if (!msg.empty()) return bail(S3_ERR_ARG, msg);
    // ---- device buffers
    for (int n = 0; n < N; ++n) {
        CK(dalloc(ctx, &ctx->P.U[n], (size_t)ctx->I[n] * ctx->JPR));
        CK(cudaMemsetAsync(ctx->P.U[n], 0, (size_t)ctx->I[n] * ctx->JPR * sizeof(float), ctx->stream));
    }
    for (int m = 0; m < n_coupled; ++m) {
        CK(dalloc(ctx, &ctx->P.V[m], (size_t)ctx->K[m] * ctx->JPR));
        CK(cudaMemsetAsync(ctx->P.V[m], 0, (size_t)ctx->K[m] * ctx->JPR * sizeof(float), ctx->stream));
    }
    {
        size_t q = 1;
        for (int n = 0; n < N - 1; ++n) q *= ctx->JP;
        CK(dalloc(ctx, &ctx->P.G, q * ctx->JPR));
        CK(cudaMemsetAsync(ctx->P.G, 0, q * ctx->JPR * sizeof(float), ctx->stream));
    }
    // per-row inverse counts from the train entries (|Omega^{n,i}|, |Omega_Y^{2,k}|), and
    // every row's occurrences per epoch (tensor entries plus coupled entries that touch it)
    std::vector<std::vector<int64_t>> occ((size_t)nF);
    for (int F = 0; F < nF; ++F) {
        const int64_t rows = factor_rows(ctx, F);
        std::vector<int64_t> cnt((size_t)rows, 0);
        if (F < N) for (int64_t e = 0; e < ctx->nnz; ++e) cnt[(size_t)hidx[F][(size_t)e]]++;
        else for (int64_t b = 0; b < ctx->ynnz[F - N]; ++b) cnt[(size_t)hyc[F - N][(size_t)b]]++;
        std::vector<float> inv((size_t)rows);
        for (int64_t i = 0; i < rows; ++i) inv[(size_t)i] = cnt[(size_t)i] ? (float)(1.0 / (double)cnt[(size_t)i]) : 0.f;
        CK(upload(ctx, &ctx->inv_cnt[F], inv));
        CK(cudaStreamSynchronize(ctx->stream));
        occ[(size_t)F] = cnt;
    }
    for (int m = 0; m < n_coupled; ++m)
        for (int64_t b = 0; b < ctx->ynnz[m]; ++b) occ[(size_t)ctx->cmode[m]][(size_t)hyr[m][(size_t)b]]++;
    fill_params(ctx);
    int rc;
    // scratch: contribution slots (minibatch and gradient groups), core partials
    for (int F = 0; F < nF; ++F) {
        const int64_t ev = std::max(ctx->mb.max_ev[F], ctx->grad.max_ev[F]);
        CK(dalloc(ctx, &ctx->contrib[F], (size_t)std::max<int64_t>(ev, 1) * ctx->JPR));
    }
    {
        int64_t pd = 1;
        for (int n = 0; n < N; ++n) pd *= ctx->JP;
        const int64_t parts = std::max<int64_t>({(ctx->mb.max_t + kTile - 1) / kTile,
                                                 (ctx->grad.max_t + kTile - 1) / kTile,
                                                 (int64_t)ctx->num_sms * 8, 1});
        ctx->core_part_n = parts;
        CK(dalloc(ctx, &ctx->core_part, (size_t)(parts * pd)));
    }
    {
        // the gradient pass's huge segments are summed in kHugeParts pieces each (k_segments):
        // room for the most huge segments of any gradient chunk
        int64_t hmax = 0;
        for (int64_t g = 0; g < ctx->grad.ngroups; ++g) {
            int64_t h = 0;
            for (int F = 0; F < nF; ++F) h += ctx->grad.seg_nhuge[F][(size_t)g];
            hmax = std::max(hmax, h);
        }
        CK(dalloc(ctx, &ctx->seg_parts, (size_t)std::max<int64_t>(hmax, 1) * kHugeParts * ctx->JPR));
        CK(dalloc(ctx, &ctx->seg_done, (size_t)std::max<int64_t>(hmax, 1)));
        CK(cudaMemsetAsync(ctx->seg_done, 0, (size_t)std::max<int64_t>(hmax, 1) * sizeof(int), ctx->stream));
    }
    CK(dalloc(ctx, &ctx->d_red, 64));
    CK(cudaMallocHost((void**)&ctx->h_red, 64 * sizeof(double)));
    CK(dalloc(ctx, &ctx->d_eta, 1));
    CK(cudaMallocHost((void**)&ctx->h_eta, sizeof(float)));
    CK(dalloc(ctx, &ctx->d_flag, 1));
    CK(dalloc(ctx, &ctx->d_tile_counter, 1));
    CK(dalloc(ctx, &ctx->d_kerr, 1));
    CK(dalloc(ctx, &ctx->d_idx_bad, 1));
    CK(cudaMallocHost((void**)&ctx->h_idx_bad, sizeof(int)));
    CK(dalloc(ctx, &ctx->d_bar, 1));
    CK(cudaMemsetAsync(ctx->d_bar, 0, sizeof(unsigned), ctx->stream));
    // one CTA per SM by default: the epoch's grid-wide barriers cost more with every CTA
    // than a second co-resident CTA gains in latency hiding
    ctx->mb_grid = std::min<int>({minibatch_epoch_grid(N, ctx->JP, ctx->num_sms), ctx->num_sms,
                                  (int)ctx->core_part_n});
    if (hp->mb_ctas > 0) ctx->mb_grid = std::min<int>(ctx->mb_grid, hp->mb_ctas);
    CK(cudaMemsetAsync(ctx->d_kerr, 0, sizeof(int), ctx->stream));
    CK(cudaMallocHost((void**)&ctx->h_flag, 2 * sizeof(int)));
    CK(tensor_prepare(N, ctx->JP));
    if (bf16_ok) {
        ctx->hog_bf_smem = tensor_hog_bf16_smem(ctx->bf_jp, ctx->hog_bf.max_ev, ctx->hog_bf.max_seg, nF);
        ctx->hog_bf_grid = std::min<int64_t>(ctx->hog_bf_grid, ctx->hog_bf.ngroups);
    }
    // staleness-aware step: a row with kappa updates expected in flight at once takes
    // gamma / kappa of its step when kappa > gamma (kappa = occurrences x entries in flight
    // / |Omega|); each HOGWILD grouping stores the scale of every row.  Default gamma =
    // 360 / (largest rank): 36 at rank 10, where the HOGWILD test-RMSE curve sits closest to
    // Algorithm 1's (larger gamma ends below it, smaller starts above it).  A coupled
    // entry's step has curvature eta * lambda_m * ||v||^2, which grows with the rank, and
    // gamma stale steps of it must stay well inside the stable range.
    {
        int jmax = 1;
        for (int n = 0; n < N; ++n) jmax = std::max(jmax, ctx->J[n]);
        // The non-negative form takes 2000 / (largest rank), 200 at rank 10, with three
        // quarters of the entries in flight: its projected steps do not pull the curve down
        // as the plain group steps do, so that the plain form's stronger damping of hot rows
        // leaves it 2-3% above projected Algorithm 1, while this setting keeps it within 1%
        // (cfg1, rank 10: 0.82%).
        double gamma = (hp->nonneg ? 2000.0 : 360.0) / jmax;
        if (hp->hog_staleness != 0.f) gamma = (double)hp->hog_staleness;
        auto row_scales = [&](DevGrouping& D, double inflight) -> int {
            for (int F = 0; F < nF; ++F) {
                std::vector<float> d(occ[(size_t)F].size(), 1.f);
                if (gamma > 0)
                    for (size_t i = 0; i < d.size(); ++i) {
                        const double kappa = (double)occ[(size_t)F][i] * inflight / (double)ctx->nnz;
                        if (kappa > gamma) d[i] = (float)(gamma / kappa);
                    }
                float* p = nullptr;
                CK(upload(ctx, &p, d));
                D.d.row_damp[F] = p;
                CK(cudaStreamSynchronize(ctx->stream));
            }
            return S3_OK;
        };
        if ((rc = row_scales(ctx->hog, (double)ctx->hog_grid * (double)tile)) != S3_OK) return rc;
        if (bf16_ok && (rc = row_scales(ctx->hog_bf,
                                        (double)std::max<int64_t>(ctx->hog_bf_grid, 1) *
                                            (double)bf_tile)) != S3_OK)
            return rc;
    }
    // initial parameters
    KL(launch_init_params(ctx->P, ctx->I, ctx->J, ctx->K, ctx->JP, seed, ctx->stream));
    if (ctx->hp.cp) KL(launch_cp_mask(ctx->P.G, N, ctx->JP, ctx->JPR, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return S3_OK;
}

static void free_coo(int32_t** idx, float** val) {
    for (int k = 0; k < kMaxN; ++k) {
        if (idx[k]) cudaFree(idx[k]);
        idx[k] = nullptr;
    }
    if (*val) cudaFree(*val);
    *val = nullptr;
}

static void prof_clear(s3_ctx* ctx) {
    for (auto& f : ctx->fam) {
        for (cudaEvent_t e : f.ev) cudaEventDestroy(e);
        f.ev.clear();
        f.launches = 0;
        f.entries = 0;
    }
    ctx->launches = 0;
}

extern "C" void s3_destroy(s3_ctx* ctx) {
    if (!ctx) return;
    prof_clear(ctx);
    free_coo(ctx->test_idx, &ctx->test_val);
    cudaStreamSynchronize(ctx->stream);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->h_red) cudaFreeHost(ctx->h_red);
    if (ctx->h_eta) cudaFreeHost(ctx->h_eta);
    if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
    if (ctx->h_idx_bad) cudaFreeHost(ctx->h_idx_bad);
    delete ctx;
}

extern "C" int s3_profile(s3_ctx* ctx, int enable) {
    if (!usable(ctx)) return S3_ERR_STATE;
    CK(cudaStreamSynchronize(ctx->stream));
    if (enable) prof_clear(ctx);
    ctx->prof = enable != 0;
    return S3_OK;
}

extern "C" int s3_profile_read(s3_ctx* ctx, int family, double* ms, int64_t* launches,
                               int64_t* entries) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (family < -1 || family > 3) return fail(ctx, S3_ERR_ARG, "unknown kernel family");
    CK(cudaStreamSynchronize(ctx->stream));
    if (family == -1) {
        if (ms) *ms = 0.0;
        if (launches) *launches = ctx->launches;
        if (entries) *entries = 0;
        return S3_OK;
    }
    auto& f = ctx->fam[family];
    double total = 0.0;
    for (size_t k = 0; k + 1 < f.ev.size(); k += 2) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, f.ev[k], f.ev[k + 1]));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = f.launches;
    if (entries) *entries = f.entries;
    return S3_OK;
}

extern "C" const char* s3_last_error(const s3_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "NULL context";
}

// ------------------------------------------------------------------ epoch
// gathers the values staged by s3_update_values into grouping k's order (0 minibatch,
// 1 HOGWILD, 2 gradient and loss, 3 BF16 HOGWILD) if they have not been yet
static int refresh_values(s3_ctx* ctx, int k) {
    DevGrouping* gs[4] = {&ctx->mb, &ctx->hog, &ctx->grad, &ctx->hog_bf};
    DevGrouping* D = gs[k];
    if (D->ngroups == 0) return S3_OK;   // not built for this context
    if (ctx->stale_t[k]) {
        KL(launch_gather_f32(D->tval, ctx->values_stage, D->t_src, D->t_off.back(), ctx->stream));
        ctx->stale_t[k] = 0;
    }
    int64_t o = ctx->nnz;
    for (int m = 0; m < ctx->M; ++m) {
        if (ctx->stale_c[k][m]) {
            KL(launch_gather_f32(D->cval[m], ctx->values_stage + o, D->c_src[m], ctx->ynnz[m], ctx->stream));
            ctx->stale_c[k][m] = 0;
        }
        o += ctx->ynnz[m];
    }
    return S3_OK;
}

static int enqueue_minibatch(s3_ctx* ctx) {
    const int nF = ctx->N + ctx->M;
    if (ctx->mb_grid <= 0) return fail(ctx, S3_ERR_ARG, "the minibatch kernel cannot be made co-resident");
    if (int rc = refresh_values(ctx, 0)) return rc;
    MbLaunch L{};
    for (int F = 0; F < nF; ++F) L.contrib[F] = ctx->contrib[F];
    L.core_part = ctx->core_part;
    L.bar_count = ctx->d_bar;
    L.err_flag = ctx->d_kerr;
    L.eta = ctx->d_eta;
    L.core_scale = ctx->hp.core_scale;
    L.row_mean = ctx->hp.row_rule == S3_ROW_MEAN;
    L.n_batches = ctx->mb.ngroups;
    L.grid = ctx->mb_grid;
    L.wait_ns = wait_ns(ctx);
    CK(cudaMemsetAsync(ctx->d_bar, 0, sizeof(unsigned), ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_MB));
    KL(launch_minibatch_epoch(ctx->N, ctx->JP, ctx->P, ctx->mb.d, L, ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_MB));
    prof_count(ctx, S3_K_TENSOR_MB, ctx->nnz);
    return S3_OK;
}

static int enqueue_hogwild(s3_ctx* ctx) {
    if (int rc = refresh_values(ctx, 1)) return rc;
    DevGrouping& D = ctx->hog;
    if (ctx->hog_smem > kMaxSmem)
        return fail(ctx, S3_ERR_ARG, "a HOGWILD tile needs " + std::to_string(ctx->hog_smem) +
                                         " bytes of shared memory; lower hog_tile");
    const int row_mean = ctx->hp.row_rule == S3_ROW_MEAN;
    CK(cudaMemsetAsync(ctx->d_tile_counter, 0, sizeof(int), ctx->stream));
    if (ctx->hp.cp) {
        if (ctx->cp_smem > kMaxSmem)
            return fail(ctx, S3_ERR_ARG, "a CP HOGWILD tile needs " + std::to_string(ctx->cp_smem) +
                                             " bytes of shared memory; lower hog_tile");
        CK(prof_mark(ctx, S3_K_TENSOR_HOG));
        KL(launch_tensor_cp_hog(ctx->N, ctx->JP, ctx->P, D.d, D.ngroups, ctx->d_tile_counter,
                                (int)ctx->hog_grid, ctx->d_eta, row_mean,
                                ctx->hp.core_scale / (float)ctx->hog_grid, D.max_ev, D.max_seg,
                                ctx->stream));
        CK(prof_mark(ctx, S3_K_TENSOR_HOG));
        prof_count(ctx, S3_K_TENSOR_HOG, ctx->nnz);
        return S3_OK;
    }
    CK(prof_mark(ctx, S3_K_TENSOR_HOG));
    KL(launch_tensor_hog(ctx->N, ctx->JP, ctx->hog_lanes, ctx->P, D.d, D.ngroups, ctx->d_tile_counter,
                         (int)ctx->hog_grid, ctx->d_eta, row_mean,
                         ctx->hp.core_scale / (float)ctx->hog_grid, D.max_ev, D.max_seg,
                         ctx->hog_ccap, ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_HOG));
    prof_count(ctx, S3_K_TENSOR_HOG, ctx->nnz);
    return S3_OK;
}

static int enqueue_hogwild_bf16(s3_ctx* ctx) {
    if (int rc = refresh_values(ctx, 3)) return rc;
    DevGrouping& D = ctx->hog_bf;
    if (ctx->N != 3 || ctx->JP > 32)
        return fail(ctx, S3_ERR_ARG, "the BF16 form is built for 3-way tensors with ranks up to 32");
    if (ctx->hp.cp) return fail(ctx, S3_ERR_ARG, "the BF16 form is built for the Tucker core, not S3CMTF-CP");
    if (ctx->hog_bf_smem > kMaxSmem)
        return fail(ctx, S3_ERR_ARG, "a BF16 HOGWILD tile needs " + std::to_string(ctx->hog_bf_smem) +
                                         " bytes of shared memory (too many coupled entries per tile)");
    if (ctx->hog_bf_grid < 1)
        return fail(ctx, S3_ERR_CUDA, "the BF16 HOGWILD kernel cannot be made resident");
    const int row_mean = ctx->hp.row_rule == S3_ROW_MEAN;
    const int grid = (int)ctx->hog_bf_grid;
    CK(cudaMemsetAsync(ctx->d_tile_counter, 0, sizeof(int), ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_HOG));
    KL(launch_tensor_hog_bf16(ctx->bf_jp, ctx->P, D.d, D.ngroups, ctx->d_tile_counter, grid,
                              ctx->d_eta, row_mean, ctx->hp.core_scale / (float)grid,
                              ctx->hog_bf_sync, D.max_ev, D.max_seg, ctx->d_kerr, wait_ns(ctx),
                              ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_HOG));
    prof_count(ctx, S3_K_TENSOR_HOG, ctx->nnz);
    return S3_OK;
}

static int check_params_finite(s3_ctx* ctx, bool* bad) {
    CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    size_t q = 1;
    for (int n = 0; n < ctx->N - 1; ++n) q *= ctx->JP;
    KL(launch_check_finite(ctx->P.G, (int64_t)(q * ctx->JPR), ctx->d_flag, ctx->stream));
    for (int F = 0; F < ctx->N + ctx->M; ++F)
        KL(launch_check_finite(factor_ptr(ctx, F), factor_rows(ctx, F) * ctx->JPR, ctx->d_flag, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_flag + 1, ctx->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_flag[1]) {
        ctx->failed = true;
        static const char* sites[] = {"?", "tile start (MMA warp)", "stage-1 buffer free (MMA warp)",
                                      "Khatri-Rao chunk (MMA warp)", "final commit (MMA warp)",
                                      "stage-1 buffer full", "Khatri-Rao buffer free", "P3 and core GEMM"};
        const int code = ctx->h_flag[1];
        const int site = (code >> 24) & 0x7f;
        return fail(ctx, S3_ERR_CUDA,
                    std::string("a bounded wait ran out in the epoch kernel: ") +
                        (site >= 1 && site <= 7 ? sites[site] : "grid barrier") + ", after " +
                        std::to_string(code & 0xFFFFFF) + " tiles of its CTA");
    }
    *bad = *ctx->h_flag != 0;
    return S3_OK;
}

extern "C" int s3_epoch(s3_ctx* ctx, int mode, int precision) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (mode != S3_MINIBATCH && mode != S3_HOGWILD) return fail(ctx, S3_ERR_ARG, "unknown mode");
    if (precision != S3_FP32 && precision != S3_BF16) return fail(ctx, S3_ERR_ARG, "unknown precision");
    if (precision == S3_BF16 && mode != S3_HOGWILD)
        return fail(ctx, S3_ERR_ARG, "the BF16 form is built for the HOGWILD epoch");
    *ctx->h_eta = eta_of(ctx, ctx->epoch);
    CK(cudaMemcpyAsync(ctx->d_eta, ctx->h_eta, sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    int rc = S3_OK;
    if (mode == S3_MINIBATCH) {
        if ((rc = enqueue_minibatch(ctx)) != S3_OK) return rc;
    } else if (precision == S3_BF16) {
        if ((rc = enqueue_hogwild_bf16(ctx)) != S3_OK) return rc;
    } else {
        if ((rc = enqueue_hogwild(ctx)) != S3_OK) return rc;
    }
    ctx->epoch += 1;
    bool bad = false;
    if ((rc = check_params_finite(ctx, &bad)) != S3_OK) return rc;
    if (bad) return fail(ctx, S3_ERR_DIVERGED, "non-finite parameter after the epoch");
    return S3_OK;
}

// ------------------------------------------------------------------ loss / rmse / predict
extern "C" int s3_loss(s3_ctx* ctx, double* f_out, double* rmse_out) {
    if (!usable(ctx)) return S3_ERR_STATE;
    const int N = ctx->N, M = ctx->M, nF = N + M;
    const int tb = tensor_fwd_blocks(ctx->nnz);
    const int nb_sq = 64;
    int64_t need = tb;
    for (int m = 0; m < M; ++m) need = std::max<int64_t>(need, coupled_fwd_blocks(ctx->ynnz[m]));
    need = std::max<int64_t>(need, (int64_t)(nF + 1) * nb_sq);
    int rc;
    if ((rc = refresh_values(ctx, 2)) != S3_OK) return rc;
    if ((rc = ensure_red(ctx, need * 2)) != S3_OK) return rc;
    float* parts_a = ctx->red_parts;
    // tensor squared errors over the train entries
    const int32_t* idx[kMaxN];
    for (int n = 0; n < N; ++n) idx[n] = ctx->grad.d.tidx[n];
    CK(prof_mark(ctx, S3_K_TENSOR_FWD));
    KL(launch_tensor_fwd(N, ctx->JP, ctx->P, idx, ctx->I, nullptr, ctx->grad.d.tval, ctx->nnz, nullptr,
                         parts_a, ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_FWD));
    prof_count(ctx, S3_K_TENSOR_FWD, ctx->nnz);
    KL(launch_reduce_f64(parts_a, tb, ctx->d_red + 0, ctx->stream));
    for (int m = 0; m < M; ++m) {
        KL(launch_coupled_fwd(ctx->P, m, ctx->grad.d.cr[m], ctx->grad.d.cc[m], ctx->grad.d.cval[m],
                              ctx->ynnz[m], parts_a, ctx->stream));
        KL(launch_reduce_f64(parts_a, coupled_fwd_blocks(ctx->ynnz[m]), ctx->d_red + 1 + m, ctx->stream));
    }
    int64_t rows[kMaxF + 1];
    {
        size_t q = 1;
        for (int n = 0; n < N - 1; ++n) q *= ctx->JP;
        rows[0] = (int64_t)(q * ctx->JPR);
    }
    for (int F = 0; F < nF; ++F) rows[F + 1] = factor_rows(ctx, F);
    KL(launch_sqnorms(ctx->P, nF, rows, ctx->JP, parts_a, nb_sq, ctx->stream));
    for (int k = 0; k <= nF; ++k)
        KL(launch_reduce_f64(parts_a + 2 * (int64_t)k * nb_sq, nb_sq, ctx->d_red + 1 + M + k, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_red, ctx->d_red, sizeof(double) * (2 + M + nF), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const double* r = ctx->h_red;
    const double lam = ctx->hp.lambda_reg, lm = ctx->hp.lambda_m;
    const double se = r[0];
    double f = 0.5 * se;
    double regU = r[1 + M + 0];  // ||G||^2
    for (int n = 0; n < N; ++n) regU += r[1 + M + 1 + n];
    f += 0.5 * lam * regU;
    for (int m = 0; m < M; ++m) f += 0.5 * lm * (r[1 + m] + lam * r[1 + M + 1 + N + m]);
    if (f_out) *f_out = f;
    if (rmse_out) *rmse_out = sqrt(se / (double)ctx->nnz);
    if (!std::isfinite(f)) return fail(ctx, S3_ERR_DIVERGED, "non-finite loss");
    return S3_OK;
}

// copies test entries to fresh device buffers owned by the caller of this helper
static int upload_coo(s3_ctx* ctx, const s3_coo_tensor* t, int device_ptrs, int32_t** idx, float** val,
                      int64_t* n_out) {
    if (!t || !t->idx || !t->val || t->n_modes != ctx->N || t->nnz < 0)
        return fail(ctx, S3_ERR_ARG, "invalid test tensor");
    std::vector<int32_t> h;
    const size_t n = (size_t)std::max<int64_t>(t->nnz, 1);
    for (int k = 0; k < ctx->N; ++k) {
        cudaError_t e = to_host(t->idx[k], t->nnz, device_ptrs, h);
        if (e != cudaSuccess) return fail(ctx, S3_ERR_ARG, "reading test indices");
        for (int64_t q = 0; q < t->nnz; ++q)
            if (h[(size_t)q] < 0 || h[(size_t)q] >= ctx->I[k]) return fail(ctx, S3_ERR_INDEX, "test index out of range");
        CK(cudaMalloc((void**)&idx[k], n * sizeof(int32_t)));
        if (t->nnz) CK(cudaMemcpy(idx[k], h.data(), (size_t)t->nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    std::vector<float> v;
    cudaError_t e = to_host(t->val, t->nnz, device_ptrs, v);
    if (e != cudaSuccess) return fail(ctx, S3_ERR_ARG, "reading test values");
    CK(cudaMalloc((void**)val, n * sizeof(float)));
    if (t->nnz) CK(cudaMemcpy(*val, v.data(), (size_t)t->nnz * sizeof(float), cudaMemcpyHostToDevice));
    *n_out = t->nnz;
    return S3_OK;
}

extern "C" int s3_set_test(s3_ctx* ctx, const s3_coo_tensor* test, int device_ptrs) {
    if (!usable(ctx)) return S3_ERR_STATE;
    CK(cudaStreamSynchronize(ctx->stream));
    int32_t* idx[kMaxN] = {};
    float* val = nullptr;
    int64_t n = 0;
    int rc = upload_coo(ctx, test, device_ptrs, idx, &val, &n);
    if (rc != S3_OK) {
        free_coo(idx, &val);
        return rc;
    }
    free_coo(ctx->test_idx, &ctx->test_val);
    for (int k = 0; k < kMaxN; ++k) ctx->test_idx[k] = idx[k];
    ctx->test_val = val;
    ctx->ntest = n;
    return S3_OK;
}

extern "C" int s3_rmse(s3_ctx* ctx, const s3_coo_tensor* test, int device_ptrs, double* rmse_out) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (!rmse_out) return fail(ctx, S3_ERR_ARG, "rmse_out is NULL");
    const int32_t* idx[kMaxN] = {};
    const float* val = nullptr;
    int64_t n = 0;
    int32_t* tmp_idx[kMaxN] = {};
    float* tmp_val = nullptr;
    struct Tmp {
        int32_t** i;
        float** v;
        ~Tmp() { free_coo(i, v); }
    } tmp{tmp_idx, &tmp_val};
    if (test) {
        if (!device_ptrs) {
            CK(cudaStreamSynchronize(ctx->stream));
            int rc = upload_coo(ctx, test, 0, tmp_idx, &tmp_val, &n);
            if (rc != S3_OK) return rc;
            for (int k = 0; k < ctx->N; ++k) idx[k] = tmp_idx[k];
            val = tmp_val;
        } else {
            if (test->n_modes != ctx->N || !test->idx || !test->val) return fail(ctx, S3_ERR_ARG, "invalid test tensor");
            for (int k = 0; k < ctx->N; ++k) idx[k] = test->idx[k];
            val = test->val;
            n = test->nnz;
        }
    } else {
        for (int k = 0; k < ctx->N; ++k) idx[k] = ctx->test_idx[k];
        val = ctx->test_val;
        n = ctx->ntest;
    }
    if (n <= 0) { *rmse_out = 0.0; return S3_OK; }
    const int tb = tensor_fwd_blocks(n);
    int rc;
    if ((rc = ensure_red(ctx, tb)) != S3_OK) return rc;
    // indices the library did not copy and check itself are checked by the kernel
    const bool unchecked = test && device_ptrs;
    if (unchecked) CK(cudaMemsetAsync(ctx->d_idx_bad, 0, sizeof(int), ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_FWD));
    KL(launch_tensor_fwd(ctx->N, ctx->JP, ctx->P, idx, ctx->I, unchecked ? ctx->d_idx_bad : nullptr,
                         val, n, nullptr, ctx->red_parts, ctx->stream));
    CK(prof_mark(ctx, S3_K_TENSOR_FWD));
    prof_count(ctx, S3_K_TENSOR_FWD, n);
    KL(launch_reduce_f64(ctx->red_parts, tb, ctx->d_red, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_red, ctx->d_red, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    *ctx->h_idx_bad = 0;
    if (unchecked)
        CK(cudaMemcpyAsync(ctx->h_idx_bad, ctx->d_idx_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (*ctx->h_idx_bad) return fail(ctx, S3_ERR_INDEX, "s3_rmse: a test index lies outside its mode's range");
    *rmse_out = sqrt(ctx->h_red[0] / (double)n);
    return S3_OK;
}

extern "C" int s3_predict(s3_ctx* ctx, const int32_t* const* idx, int64_t n, float* out) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (n < 0 || (n > 0 && (!idx || !out))) return fail(ctx, S3_ERR_ARG, "invalid predict arguments");
    if (n == 0) return S3_OK;
    for (int k = 0; k < ctx->N; ++k)
        if (!idx[k]) return fail(ctx, S3_ERR_ARG, "s3_predict: an index pointer is NULL");
    CK(cudaMemsetAsync(ctx->d_idx_bad, 0, sizeof(int), ctx->stream));
    KL(launch_tensor_fwd(ctx->N, ctx->JP, ctx->P, idx, ctx->I, ctx->d_idx_bad, nullptr, n, out, nullptr,
                         ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_idx_bad, ctx->d_idx_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (*ctx->h_idx_bad) return fail(ctx, S3_ERR_INDEX, "s3_predict: an index lies outside its mode's range");
    return S3_OK;
}

// ------------------------------------------------------------------ gradient
extern "C" int s3_gradient(s3_ctx* ctx, const float* w, float* dG, float* const* dU, float* const* dV) {
    if (!usable(ctx)) return S3_ERR_STATE;
    const int N = ctx->N, M = ctx->M, nF = N + M;
    if (!dG || !dU || (M > 0 && !dV)) return fail(ctx, S3_ERR_ARG, "gradient outputs missing");
    int64_t pd = 1;
    for (int n = 0; n < N; ++n) pd *= ctx->J[n];
    // compensation buffers: core then every factor, unpadded
    int64_t need = pd;
    int64_t off[kMaxF];
    for (int F = 0; F < nF; ++F) { off[F] = need; need += factor_rows(ctx, F) * factor_cols(ctx, F); }
    if (need > ctx->grad_comp_n) {
        CK(dalloc(ctx, &ctx->grad_comp, (size_t)need));
        ctx->grad_comp_n = need;
    }
    CK(cudaMemsetAsync(ctx->grad_comp, 0, (size_t)need * sizeof(float), ctx->stream));
    CK(cudaMemsetAsync(dG, 0, (size_t)pd * sizeof(float), ctx->stream));
    float* outs[kMaxF];
    for (int F = 0; F < nF; ++F) {
        outs[F] = F < N ? dU[F] : dV[F - N];
        if (!outs[F]) return fail(ctx, S3_ERR_ARG, "gradient output missing");
        CK(cudaMemsetAsync(outs[F], 0, (size_t)(factor_rows(ctx, F) * factor_cols(ctx, F)) * sizeof(float), ctx->stream));
    }
    DevGrouping& D = ctx->grad;
    if (int rc = refresh_values(ctx, 2)) return rc;
    if (w) {
        // the caller's weights, from the order given to s3_init into the grouping's order
        if (!ctx->grad_w) CK(dalloc(ctx, &ctx->grad_w, (size_t)ctx->nnz));
        KL(launch_gather_f32(ctx->grad_w, w, D.t_src, ctx->nnz, ctx->stream));
    }
    for (int64_t g = 0; g < D.ngroups; ++g) {
        TensorLaunch L{};
        L.w = w ? ctx->grad_w : nullptr;
        L.e_begin = D.t_off[(size_t)g];
        L.e_end = D.t_off[(size_t)g + 1];
        for (int n = 0; n < N; ++n) L.contrib[n] = ctx->contrib[n];
        L.core_part = ctx->core_part;
        CK(prof_mark(ctx, S3_K_TENSOR_GRAD));
        int nparts = 0;
        KL(launch_tensor_contrib(N, ctx->JP, ctx->P, D.d, L,
                                 (int)std::min<int64_t>(ctx->core_part_n, 2 * (int64_t)ctx->num_sms),
                                 &nparts, ctx->stream));
        CK(prof_mark(ctx, S3_K_TENSOR_GRAD));
        prof_count(ctx, S3_K_TENSOR_GRAD, L.e_end - L.e_begin);
        for (int m = 0; m < M; ++m)
            KL(launch_coupled_contrib(ctx->P, D.d, m, D.c_off[m][(size_t)g], D.c_off[m][(size_t)g + 1],
                                      ctx->contrib[ctx->cmode[m]], ctx->contrib[N + m], ctx->stream));
        SegmentLaunch S{};
        S.nF = nF;
        S.g = g;
        S.part_sums = ctx->seg_parts;
        S.part_done = ctx->seg_done;
        for (int F = 0; F < nF; ++F) {
            S.contrib[F] = ctx->contrib[F];
            S.out[F] = outs[F];
            S.comp[F] = ctx->grad_comp + off[F];
            S.Jf[F] = factor_cols(ctx, F);
            const int64_t ns = D.seg_off[F][(size_t)g + 1] - D.seg_off[F][(size_t)g];
            S.nlong[F] = D.seg_nlong[F][(size_t)g];
            S.nhuge[F] = D.seg_nhuge[F][(size_t)g];
            S.huge_begin[F + 1] = S.huge_begin[F] + S.nhuge[F];
            S.long_begin[F + 1] = S.long_begin[F] + (S.nlong[F] - S.nhuge[F]);
            S.short_begin[F + 1] = S.short_begin[F] + (ns - S.nlong[F]);
        }
        KL(launch_segments(ctx->P, D.d, S, ctx->d_eta, 0, 1, ctx->stream));
        const int64_t nt = L.e_end - L.e_begin;
        KL(launch_core(ctx->P, N, ctx->JP, ctx->J, ctx->core_part, nparts, nt,
                       ctx->d_eta, 1.f, 1, dG, ctx->grad_comp, ctx->stream));
    }
    KL(launch_add_comp(dG, ctx->grad_comp, pd, ctx->stream));
    for (int F = 0; F < nF; ++F)
        KL(launch_add_comp(outs[F], ctx->grad_comp + off[F], factor_rows(ctx, F) * factor_cols(ctx, F), ctx->stream));
    // the core regulariser lambda_reg / |Omega| G of every entry: this context's share of the
    // whole problem's lambda_reg G
    KL(launch_core_reg(dG, ctx->P.G, N, ctx->J, ctx->JP,
                       (float)((double)ctx->hp.lambda_reg * (double)ctx->nnz / (double)ctx->nnz_total),
                       ctx->stream));
    return S3_OK;
}

// ------------------------------------------------------------------ partitioned problems
extern "C" int s3_set_counts(s3_ctx* ctx, const int64_t* const* counts, int64_t nnz_total) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (!counts || nnz_total < ctx->nnz)
        return fail(ctx, S3_ERR_ARG, "s3_set_counts: counts missing or nnz_total below this context's entries");
    const int nF = ctx->N + ctx->M;
    std::vector<std::vector<float>> inv((size_t)nF);
    for (int F = 0; F < nF; ++F) {
        if (!counts[F]) return fail(ctx, S3_ERR_ARG, "s3_set_counts: a count array is NULL");
        const int64_t rows = factor_rows(ctx, F);
        std::vector<float> local((size_t)rows);
        CK(cudaMemcpyAsync(local.data(), ctx->inv_cnt[F], (size_t)rows * sizeof(float), cudaMemcpyDeviceToHost,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        inv[(size_t)F].resize((size_t)rows);
        for (int64_t i = 0; i < rows; ++i) {
            const int64_t c = counts[F][i];
            // the context's own count of the row (from 1 / count), which the whole problem's
            // count must cover
            const int64_t own = local[(size_t)i] > 0.f ? (int64_t)std::llround(1.0 / (double)local[(size_t)i]) : 0;
            if (c < own)
                return fail(ctx, S3_ERR_ARG, "s3_set_counts: factor " + std::to_string(F) + ", row " +
                                                 std::to_string(i) + ": count below this context's own");
            inv[(size_t)F][(size_t)i] = c > 0 ? (float)(1.0 / (double)c) : 0.f;
        }
    }
    for (int F = 0; F < nF; ++F)
        CK(cudaMemcpyAsync(ctx->inv_cnt[F], inv[(size_t)F].data(), inv[(size_t)F].size() * sizeof(float),
                           cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->nnz_total = nnz_total;
    ctx->P.inv_nnz = (float)(1.0 / (double)nnz_total);
    return S3_OK;
}

extern "C" int s3_apply_gradient(s3_ctx* ctx, const float* dG, const float* const* dU,
                                 const float* const* dV) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (ctx->hp.row_rule != S3_ROW_SUM)
        return fail(ctx, S3_ERR_ARG, "s3_apply_gradient: built for the row rule S3_ROW_SUM");
    if (!dG || !dU || (ctx->M > 0 && !dV)) return fail(ctx, S3_ERR_ARG, "s3_apply_gradient: gradient missing");
    for (int n = 0; n < ctx->N; ++n)
        if (!dU[n]) return fail(ctx, S3_ERR_ARG, "s3_apply_gradient: gradient missing");
    for (int m = 0; m < ctx->M; ++m)
        if (!dV[m]) return fail(ctx, S3_ERR_ARG, "s3_apply_gradient: gradient missing");
    const float eta = eta_of(ctx, ctx->epoch);
    const int nonneg = ctx->hp.nonneg;
    // the core: -eta core_scale (the mean of the whole epoch's core gradients)
    KL(launch_core_step(ctx->P.G, dG, ctx->N, ctx->J, ctx->JP,
                        (float)(-(double)eta * ctx->hp.core_scale / (double)ctx->nnz_total), nonneg,
                        ctx->hp.cp, ctx->stream));
    // the rows: -eta (the sum of their gradients)
    for (int F = 0; F < ctx->N + ctx->M; ++F)
        KL(launch_rows_step(factor_ptr(ctx, F), ctx->JPR, F < ctx->N ? dU[F] : dV[F - ctx->N],
                            factor_rows(ctx, F), factor_cols(ctx, F), -eta, nonneg, ctx->stream));
    ctx->epoch += 1;
    bool bad = false;
    int rc;
    if ((rc = check_params_finite(ctx, &bad)) != S3_OK) return rc;
    if (bad) return fail(ctx, S3_ERR_DIVERGED, "non-finite parameter after the step");
    return S3_OK;
}

// ------------------------------------------------------------------ params
// ------------------------------------------------------------------ final QR step
extern "C" int s3_finalize_qr(s3_ctx* ctx) {
    if (!usable(ctx)) return S3_ERR_STATE;
    const int N = ctx->N;
    for (int n = 0; n < N; ++n)
        if (ctx->I[n] < ctx->J[n])
            return fail(ctx, S3_ERR_ARG, "s3_finalize_qr: U^(" + std::to_string(n + 1) +
                                             ") has fewer rows than its rank");
    // scratch, allocated once: Gram partials, per-mode R and R^-1, pass-1 factors, the flag,
    // the out-of-place core
    int64_t grid = 1;
    for (int n = 0; n < N; ++n) grid = std::max<int64_t>(grid, qr_gram_ctas(ctx->I[n], ctx->num_sms));
    size_t q = 1;
    for (int n = 0; n < N - 1; ++n) q *= ctx->JP;
    const size_t core_n = q * ctx->JPR;
    if (!ctx->qr_parts) {
        CK(dalloc(ctx, &ctx->qr_parts, (size_t)grid * 32 * 32));
        CK(dalloc(ctx, &ctx->qr_R, (size_t)(2 * kMaxN + 2) * 32 * 32));
        CK(dalloc(ctx, &ctx->qr_bad, (size_t)kMaxN));
        CK(dalloc(ctx, &ctx->qr_core, core_n));
        ctx->qr_grid = grid;
    }
    double* Rn[kMaxN];
    double* Rin[kMaxN];
    for (int n = 0; n < N; ++n) {
        Rn[n] = ctx->qr_R + (size_t)(2 * n) * 32 * 32;
        Rin[n] = ctx->qr_R + (size_t)(2 * n + 1) * 32 * 32;
    }
    double* R1 = ctx->qr_R + (size_t)(2 * kMaxN) * 32 * 32;
    double* R1i = R1 + 32 * 32;
    CK(cudaMemsetAsync(ctx->qr_bad, 0, sizeof(int) * kMaxN, ctx->stream));
    // every factor first: nothing changes when one of them is rank deficient
    for (int n = 0; n < N; ++n) {
        const int g = qr_gram_ctas(ctx->I[n], ctx->num_sms);
        KL(launch_qr_factor(ctx->P.U[n], ctx->I[n], ctx->JPR, ctx->J[n], std::min<int>(g, (int)ctx->qr_grid),
                            ctx->qr_parts, Rn[n], Rin[n], R1, R1i, ctx->qr_bad + n, ctx->stream));
    }
    int bad[kMaxN] = {};
    CK(cudaMemcpyAsync(bad, ctx->qr_bad, sizeof(int) * kMaxN, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int n = 0; n < N; ++n)
        if (bad[n])
            return fail(ctx, S3_ERR_ARG, "s3_finalize_qr: U^(" + std::to_string(n + 1) +
                                             ") does not have full column rank");
    for (int n = 0; n < N; ++n) {
        KL(launch_qr_rows(ctx->P.U[n], ctx->I[n], ctx->JPR, ctx->J[n], Rin[n], 0, ctx->stream));
        KL(launch_qr_core(ctx->P.G, ctx->qr_core, N, ctx->JP, ctx->JPR, n, ctx->J[n], Rn[n], ctx->stream));
        CK(cudaMemcpyAsync(ctx->P.G, ctx->qr_core, core_n * sizeof(float), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        for (int m = 0; m < ctx->M; ++m)
            if (ctx->cmode[m] == n)
                KL(launch_qr_rows(ctx->P.V[m], ctx->K[m], ctx->JPR, ctx->J[n], Rn[n], 1, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return S3_OK;
}

extern "C" int s3_get_params(s3_ctx* ctx, float* G, float* const* U, float* const* V) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (G) KL(launch_unpack_core(G, ctx->P.G, ctx->N, ctx->J, ctx->JP, ctx->stream));
    for (int n = 0; n < ctx->N; ++n)
        if (U && U[n]) KL(launch_unpack_rows(U[n], ctx->P.U[n], ctx->JPR, ctx->I[n], ctx->J[n], ctx->stream));
    for (int m = 0; m < ctx->M; ++m)
        if (V && V[m]) KL(launch_unpack_rows(V[m], ctx->P.V[m], ctx->JPR, ctx->K[m], ctx->J[ctx->cmode[m]], ctx->stream));
    return S3_OK;
}

extern "C" int s3_set_params(s3_ctx* ctx, const float* G, const float* const* U, const float* const* V) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (G) KL(launch_pack_core(ctx->P.G, G, ctx->N, ctx->J, ctx->JP, ctx->stream));
    if (G && ctx->hp.cp) KL(launch_cp_mask(ctx->P.G, ctx->N, ctx->JP, ctx->JPR, ctx->stream));
    for (int n = 0; n < ctx->N; ++n)
        if (U && U[n]) KL(launch_pack_rows(ctx->P.U[n], ctx->JPR, U[n], ctx->I[n], ctx->J[n], ctx->stream));
    for (int m = 0; m < ctx->M; ++m)
        if (V && V[m]) KL(launch_pack_rows(ctx->P.V[m], ctx->JPR, V[m], ctx->K[m], ctx->J[ctx->cmode[m]], ctx->stream));
    return S3_OK;
}

extern "C" int s3_get_epoch(s3_ctx* ctx, int64_t* t) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (!t) return fail(ctx, S3_ERR_ARG, "t is NULL");
    *t = ctx->epoch;
    return S3_OK;
}

extern "C" int s3_set_epoch(s3_ctx* ctx, int64_t t) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (t < 0) return fail(ctx, S3_ERR_ARG, "negative epoch");
    ctx->epoch = t;
    return S3_OK;
}

extern "C" int s3_info(s3_ctx* ctx, int64_t* n_union, int64_t* n_batches, int64_t* n_tiles) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (n_union) *n_union = ctx->n_union;
    if (n_batches) *n_batches = ctx->mb.ngroups;
    if (n_tiles) *n_tiles = ctx->hog.ngroups;
    return S3_OK;
}

extern "C" int s3_hog_config(s3_ctx* ctx, int precision, int64_t* ctas, int64_t* tile,
                             int64_t* smem_bytes, int64_t* ctas_per_sm) {
    if (!usable(ctx)) return S3_ERR_STATE;
    int64_t c = 0, tl = 0, sm = 0, per = 0;
    if (precision == S3_FP32) {
        c = ctx->hog_grid;
        tl = ctx->hog_tile;
        sm = (int64_t)ctx->hog_smem;
        per = ctx->hog_per_sm;
    } else if (precision == S3_BF16) {
        c = ctx->hog_bf_grid;
        tl = ctx->hog_bf_grid > 0 ? ctx->hog_bf_tile : 0;
        sm = (int64_t)ctx->hog_bf_smem;
        per = ctx->hog_bf_per_sm;
    } else {
        return fail(ctx, S3_ERR_ARG, "precision must be S3_FP32 or S3_BF16");
    }
    if (ctas) *ctas = c;
    if (tile) *tile = tl;
    if (smem_bytes) *smem_bytes = sm;
    if (ctas_per_sm) *ctas_per_sm = per;
    return S3_OK;
}

// ------------------------------------------------------------------ values from the host
// The values go to one staging array; each grouping gathers them into its own order only when
// a call next reads that grouping (refresh_values), so an epoch after an update pays for the
// one layout it uses, not for all four.
extern "C" int s3_update_values(s3_ctx* ctx, const float* x_val, const float* const* y_val) {
    if (!usable(ctx)) return S3_ERR_STATE;
    if (!x_val) return fail(ctx, S3_ERR_ARG, "x_val is NULL");
    int64_t total = ctx->nnz;
    for (int m = 0; m < ctx->M; ++m) total += ctx->ynnz[m];
    if (!ctx->values_stage) CK(dalloc(ctx, &ctx->values_stage, (size_t)total));
    CK(cudaMemcpyAsync(ctx->values_stage, x_val, (size_t)ctx->nnz * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    for (int k = 0; k < 4; ++k) ctx->stale_t[k] = 1;
    int64_t o = ctx->nnz;
    for (int m = 0; m < ctx->M; ++m) {
        if (y_val && y_val[m]) {
            CK(cudaMemcpyAsync(ctx->values_stage + o, y_val[m], (size_t)ctx->ynnz[m] * sizeof(float),
                               cudaMemcpyHostToDevice, ctx->stream));
            for (int k = 0; k < 4; ++k) ctx->stale_c[k][m] = 1;
        }
        o += ctx->ynnz[m];
    }
    return S3_OK;
}

// ------------------------------------------------------------------ accessors for noalloc.cu
namespace s3 {
const DParams* ctx_params(const s3_ctx* ctx, int* N, int* JP, cudaStream_t* stream, int* device,
                          const int64_t** dims) {
    if (!usable(ctx)) return nullptr;
    *N = ctx->N;
    *JP = ctx->JP;
    *stream = ctx->stream;
    *device = ctx->device;
    *dims = ctx->I;
    return &ctx->P;
}
int ctx_fail(s3_ctx* ctx, int code, const char* msg) { return fail(ctx, code, msg); }
}  // namespace s3
