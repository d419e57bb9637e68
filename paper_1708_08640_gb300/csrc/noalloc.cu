// s3_rmse_noalloc: the test-RMSE reduction of s3_rmse for callers that must not allocate
// device memory (see include/s3cmtf.h).  Its only scratch is the file-scope array below.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "s3cmtf.h"

namespace s3 {
const DParams* ctx_params(const s3_ctx* ctx, int* N, int* JP, cudaStream_t* stream, int* device,
                          const int64_t** dims);
int ctx_fail(s3_ctx* ctx, int code, const char* msg);
}  // namespace s3

using namespace s3;

namespace {

// One partial pair (compensated FP32 sum) per CTA of 256 entries, then the FP64 total, and
// the flag the forward kernel raises on an index outside its mode's range.
constexpr int64_t kMaxPairs = 8192;                       // 64 KiB of partials
constexpr int64_t kMaxEntries = kMaxPairs * kTile;       // 2,097,152 test entries

struct Scratch {
    float pairs[2 * kMaxPairs];
    double total;
    int bad;
};

// Shared by every call on a device; holds the last call's contents.  Each call clears the
// index flag before its kernel runs; every other byte it reads is written earlier in the same
// call (each CTA writes its pair, the reduction writes the total).
static __device__ __align__(256) Scratch g_scratch;

// The device address of g_scratch, looked up once per device (and again if that device's
// current context is no longer the one it was looked up in, e.g. after a device reset).
struct Cached {
    CUcontext cu = nullptr;
    void* addr = nullptr;
};
std::mutex g_mu;
Cached g_addr[64];
using CtxGetCurrent = CUresult (*)(CUcontext*);
CtxGetCurrent g_get_current = nullptr;

// the current driver context, through the runtime's entry-point lookup (the library does not
// link the driver library itself); nullptr when it cannot be told
CUcontext current_context() {
    if (!g_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        g_get_current = reinterpret_cast<CtxGetCurrent>(fn);
    }
    CUcontext c = nullptr;
    return g_get_current(&c) == CUDA_SUCCESS ? c : nullptr;
}

}  // namespace

extern "C" int s3_rmse_noalloc(s3_ctx* ctx, const int32_t* const* idx, const float* val, int64_t n,
                               double* rmse_out) {
    int N = 0, JP = 0, dev = 0;
    cudaStream_t stream = nullptr;
    const int64_t* dims = nullptr;
    const DParams* P = ctx_params(ctx, &N, &JP, &stream, &dev, &dims);
    if (!P) return S3_ERR_STATE;
    if (!rmse_out || n < 0 || (n > 0 && (!idx || !val)))
        return ctx_fail(ctx, S3_ERR_ARG, "s3_rmse_noalloc: invalid arguments");
    for (int k = 0; k < N && n > 0; ++k)
        if (!idx[k]) return ctx_fail(ctx, S3_ERR_ARG, "s3_rmse_noalloc: index pointer is NULL");
    if (n > kMaxEntries)
        return ctx_fail(ctx, S3_ERR_ARG,
                        "s3_rmse_noalloc: more than 2,097,152 entries (the static scratch holds "
                        "8192 partial sums of 256 entries each); split the call or use s3_rmse");
    if (n == 0) {
        *rmse_out = 0.0;
        return S3_OK;
    }
    if (dev < 0 || dev >= 64) return ctx_fail(ctx, S3_ERR_ARG, "s3_rmse_noalloc: device id >= 64");
    // every call: the context's device must be the current one (the array's address is only
    // valid there)
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != dev)
        return ctx_fail(ctx, S3_ERR_ARG, "s3_rmse_noalloc: make the context's device current");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const CUcontext cu = current_context();
        Cached& c = g_addr[dev];
        if (!c.addr || cu != c.cu) {
            // set-up, once per device (and per context of it), with that device current
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return ctx_fail(ctx, S3_ERR_CUDA, cudaGetErrorString(e));
            c.addr = p;
            c.cu = cu;
        }
        base = c.addr;
    }
    Scratch* sc = static_cast<Scratch*>(base);
    cudaError_t e = cudaMemsetAsync(&sc->bad, 0, sizeof(int), stream);
    if (e == cudaSuccess)
        e = launch_tensor_fwd_one_pass(N, JP, *P, idx, dims, &sc->bad, val, n, sc->pairs, stream);
    if (e == cudaSuccess) e = launch_reduce_f64(sc->pairs, (n + kTile - 1) / kTile, &sc->total, stream);
    double total = 0.0;
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, &sc->total, sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &sc->bad, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return ctx_fail(ctx, S3_ERR_CUDA, cudaGetErrorString(e));
    if (bad) return ctx_fail(ctx, S3_ERR_INDEX, "s3_rmse_noalloc: an index lies outside its mode's range");
    *rmse_out = sqrt(total / (double)n);
    return S3_OK;
}
