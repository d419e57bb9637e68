// s3_rmse_noalloc: the test-RMSE reduction of s3_rmse for callers that must not allocate
// device memory (see include/s3cmtf.h).  Its only scratch is the file-scope array below.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"
#include "s3cmtf.h"

namespace s3 {
cudaError_t launch_tensor_fwd_one_pass(int N, int JP, const DParams& P, const int32_t* const* idx,
                                       const float* x, int64_t n, float* sq_part, cudaStream_t s);
const DParams* ctx_params(const s3_ctx* ctx, int* N, int* JP, cudaStream_t* stream, int* device);
int ctx_fail(s3_ctx* ctx, int code, const char* msg);
}  // namespace s3

using namespace s3;

namespace {

// One partial pair (compensated FP32 sum) per CTA of 256 entries, then the FP64 total.
constexpr int64_t kMaxPairs = 8192;                       // 64 KiB of partials
constexpr int64_t kMaxEntries = kMaxPairs * kTile;       // 2,097,152 test entries

struct Scratch {
    float pairs[2 * kMaxPairs];
    double total;
};

// Shared by every call on a device; holds the last call's contents.  Every byte a call reads
// is written earlier in the same call (each CTA writes its pair, the reduction writes the
// total), so nothing needs clearing between calls.
static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mu;
void* g_addr[64] = {};   // device address of g_scratch, per device

}  // namespace

extern "C" int s3_rmse_noalloc(s3_ctx* ctx, const int32_t* const* idx, const float* val, int64_t n,
                               double* rmse_out) {
    int N = 0, JP = 0, dev = 0;
    cudaStream_t stream = nullptr;
    const DParams* P = ctx_params(ctx, &N, &JP, &stream, &dev);
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
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            // once per device, with the context's device current (it is: contexts are bound to
            // the device that was current at s3_init, and the caller keeps it current)
            int cur = -1;
            if (cudaGetDevice(&cur) != cudaSuccess || cur != dev)
                return ctx_fail(ctx, S3_ERR_ARG, "s3_rmse_noalloc: make the context's device current");
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess) return ctx_fail(ctx, S3_ERR_CUDA, cudaGetErrorString(e));
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    Scratch* sc = static_cast<Scratch*>(base);
    cudaError_t e = launch_tensor_fwd_one_pass(N, JP, *P, idx, val, n, sc->pairs, stream);
    if (e == cudaSuccess) e = launch_reduce_f64(sc->pairs, (n + kTile - 1) / kTile, &sc->total, stream);
    double total = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, &sc->total, sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return ctx_fail(ctx, S3_ERR_CUDA, cudaGetErrorString(e));
    *rmse_out = sqrt(total / (double)n);
    return S3_OK;
}
