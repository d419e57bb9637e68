// The final QR step of Algorithm 1 (Section 3.4) on the GPU: for every mode n the thin QR
// U^(n) = Q^(n) R^(n), then U^(n) <- Q^(n), G <- G x_n R^(n), and every coupled factor of
// mode n  V_m <- V_m R^(n)^T.
//
// CholeskyQR2 in double precision: W = U^T U (FP64 sums of exact FP32 products, per-CTA
// partials added in CTA order), R1 = chol(W); W2 = (U R1^-1)^T (U R1^-1) computed on the
// fly, R2 = chol(W2); R = R2 R1 (upper triangular, positive diagonal: the unique thin QR of
// a full-column-rank U), Q = U R^-1.  The second pass restores orthogonality lost to
// cond(U)^2 in the first.  Deterministic: fixed partitions and summation orders.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.h"

namespace s3 {

constexpr int kQrRows = 128;      // rows of U staged in shared memory per step
constexpr int kQrThreads = 256;

// Per-CTA partial Gram matrices of Y = U (Rinv == nullptr) or Y = U Rinv (Rinv upper
// triangular J x J, FP64).  parts: [gridDim.x][J * J] (full symmetric matrix).
__global__ void __launch_bounds__(kQrThreads) k_qr_gram(const float* __restrict__ U, int64_t rows,
                                                        int ld, int J, const double* __restrict__ Rinv,
                                                        double* __restrict__ parts) {
    extern __shared__ double qsm[];
    double* ys = qsm;                     // [kQrRows][J]
    double* ri = qsm + kQrRows * J;       // [J][J]
    const int tid = threadIdx.x;
    if (Rinv)
        for (int l = tid; l < J * J; l += kQrThreads) ri[l] = Rinv[l];
    const int npair = J * (J + 1) / 2;
    double acc[3] = {0.0, 0.0, 0.0};      // pairs tid, tid + 256, tid + 512 (npair <= 528)
    int pa[3], pb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int p = tid + k * kQrThreads, a = 0;
        if (p >= npair) { pa[k] = -1; pb[k] = -1; continue; }
        while (p >= J - a) { p -= J - a; ++a; }
        pa[k] = a;
        pb[k] = a + p;
    }
    for (int64_t r0 = (int64_t)blockIdx.x * kQrRows; r0 < rows; r0 += (int64_t)gridDim.x * kQrRows) {
        const int nr = (int)min((int64_t)kQrRows, rows - r0);
        __syncthreads();
        if (tid < kQrRows) {
            const float* src = U + (r0 + tid) * ld;
            double* y = ys + tid * J;
            for (int j = 0; j < J; ++j) y[j] = tid < nr ? (double)src[j] : 0.0;
            if (Rinv)
                // y <- y Rinv in place, Rinv upper triangular: y_j = sum_{k <= j} y_k Rinv[k][j],
                // from the last column down, so that every y_k it reads is still the input
                for (int j = J - 1; j >= 0; --j) {
                    double s = 0.0;
                    for (int k = 0; k <= j; ++k) s += y[k] * ri[k * J + j];
                    y[j] = s;
                }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (pa[k] < 0) continue;
            double s = 0.0;
            for (int r = 0; r < nr; ++r) s += ys[r * J + pa[k]] * ys[r * J + pb[k]];
            acc[k] += s;
        }
    }
    double* out = parts + (int64_t)blockIdx.x * J * J;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (pa[k] < 0) continue;
        out[pa[k] * J + pb[k]] = acc[k];
        out[pb[k] * J + pa[k]] = acc[k];
    }
}

// One CTA: W = sum of the nparts partials in order (an element per thread); then thread 0:
// R = chol(W)^T (W = R^T R, R upper triangular), Rinv = R^-1 and, with Rprev (the previous
// pass's R and Rinv, or null), Rout = R Rprev and Rinv_out = Rprev_inv R^-1.  *bad = 1 (and
// the outputs are left unwritten) when W is not numerically positive definite: a pivot at
// most 1e-14 of the largest diagonal entry of W, i.e. a diagonal entry of R at most 1e-7 of
// the largest (pivots are R_ii^2, and FP64 rounding in the Gram matrix leaves ~1e-16 of
// noise in them).
__global__ void k_qr_chol(const double* __restrict__ parts, int nparts, int J,
                          const double* __restrict__ Rprev, const double* __restrict__ Rprev_inv,
                          double* __restrict__ Rout, double* __restrict__ Rinv_out, int* bad) {
    __shared__ double W[32 * 32], R[32 * 32], Ri[32 * 32];
    // the sum of the partials in partial order, one element per thread
    for (int l = threadIdx.x; l < J * J; l += blockDim.x) {
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += parts[(int64_t)p * J * J + l];
        W[l] = s;
        R[l] = 0.0;
        Ri[l] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double wmax = 0.0;
    for (int i = 0; i < J; ++i) wmax = fmax(wmax, W[i * J + i]);
    // Cholesky, upper form: R[i][i] = sqrt(W_ii - sum_k R_ki^2), R[i][j] = (W_ij - sum_k R_ki R_kj) / R_ii
    for (int i = 0; i < J; ++i) {
        double d = W[i * J + i];
        for (int k = 0; k < i; ++k) d -= R[k * J + i] * R[k * J + i];
        if (!(d > 1e-14 * wmax)) { *bad = 1; return; }
        const double rii = sqrt(d);
        R[i * J + i] = rii;
        for (int j = i + 1; j < J; ++j) {
            double s = W[i * J + j];
            for (int k = 0; k < i; ++k) s -= R[k * J + i] * R[k * J + j];
            R[i * J + j] = s / rii;
        }
    }
    // inverse of the upper triangular R, column by column: R Ri = I
    for (int c = 0; c < J; ++c)
        for (int i = c; i >= 0; --i) {
            double s = i == c ? 1.0 : 0.0;
            for (int k = i + 1; k <= c; ++k) s -= R[i * J + k] * Ri[k * J + c];
            Ri[i * J + c] = s / R[i * J + i];
        }
    for (int i = 0; i < J; ++i)
        for (int j = 0; j < J; ++j) {
            double a = 0.0, b = 0.0;
            if (Rprev) {
                for (int k = 0; k < J; ++k) {
                    a += R[i * J + k] * Rprev[k * J + j];        // R Rprev
                    b += Rprev_inv[i * J + k] * Ri[k * J + j];   // Rprev^-1 R^-1
                }
            } else {
                a = R[i * J + j];
                b = Ri[i * J + j];
            }
            Rout[i * J + j] = a;
            Rinv_out[i * J + j] = b;
        }
}

// U <- U Rinv (rows of J values, FP64 arithmetic, FP32 storage; padding untouched), or with
// transpose = 1, V <- V R^T
__global__ void __launch_bounds__(kQrThreads) k_qr_rows(float* __restrict__ X, int64_t rows, int ld,
                                                        int J, const double* __restrict__ M,
                                                        int transpose) {
    __shared__ double m[32 * 32];
    for (int l = threadIdx.x; l < J * J; l += kQrThreads) m[l] = M[l];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * kQrThreads + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * kQrThreads) {
        float* x = X + r * ld;
        if (!transpose) {
            // (u Rinv)_i = sum_{k <= i} u_k Rinv[k][i], in place from the last i down
            for (int i = J - 1; i >= 0; --i) {
                double s = 0.0;
                for (int k = 0; k <= i; ++k) s += (double)x[k] * m[k * J + i];
                x[i] = (float)s;
            }
        } else {
            // (v R^T)_i = sum_{k >= i} v_k R[i][k], in place from the first i up
            for (int i = 0; i < J; ++i) {
                double s = 0.0;
                for (int k = i; k < J; ++k) s += (double)x[k] * m[i * J + k];
                x[i] = (float)s;
            }
        }
    }
}

// G <- G x_n R on the padded core (JP in every mode, last mode padded to ldg): out-of-place
// into Gout, element by element: Gout[.., i, ..] = sum_{j < J} R[i][j] G[.., j, ..] for i < J,
// and 0 for the padded i >= J
__global__ void __launch_bounds__(kQrThreads) k_qr_core(const float* __restrict__ G, float* __restrict__ Gout,
                                                        int N, int JP, int ldg, int n, int J,
                                                        const double* __restrict__ R) {
    int64_t total = 1;
    for (int k = 0; k < N - 1; ++k) total *= JP;
    total *= ldg;
    int64_t stride = 1;   // distance between consecutive indices of mode n
    if (n < N - 1) {
        stride = ldg;
        for (int k = N - 2; k > n; --k) stride *= JP;
    }
    for (int64_t l = (int64_t)blockIdx.x * kQrThreads + threadIdx.x; l < total;
         l += (int64_t)gridDim.x * kQrThreads) {
        const int i = (int)((l / stride) % (n == N - 1 ? ldg : JP));
        const int64_t base = l - (int64_t)i * stride;
        double s = 0.0;
        if (i < J)
            for (int j = 0; j < J; ++j) s += R[i * J + j] * (double)G[base + (int64_t)j * stride];
        Gout[l] = i < J ? (float)s : 0.f;
    }
}

int qr_gram_ctas(int64_t rows, int num_sms) {
    const int64_t by_rows = (rows + kQrRows - 1) / kQrRows;
    const int64_t cap = (int64_t)num_sms * 4;
    return (int)(by_rows < cap ? (by_rows > 0 ? by_rows : 1) : cap);
}

cudaError_t launch_qr_factor(const float* U, int64_t rows, int ld, int J, int grid, double* parts,
                             double* R, double* Rinv, double* R1, double* R1inv, int* bad,
                             cudaStream_t s) {
    if (J < 1 || J > 32) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double) * ((size_t)kQrRows * J + (size_t)J * J);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_qr_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // pass 1: W = U^T U -> R1
    k_qr_gram<<<grid, kQrThreads, smem, s>>>(U, rows, ld, J, nullptr, parts);
    k_qr_chol<<<1, 256, 0, s>>>(parts, grid, J, nullptr, nullptr, R1, R1inv, bad);
    // pass 2: W2 = (U R1^-1)^T (U R1^-1) -> R2; R = R2 R1, Rinv = R1^-1 R2^-1
    k_qr_gram<<<grid, kQrThreads, smem, s>>>(U, rows, ld, J, R1inv, parts);
    k_qr_chol<<<1, 256, 0, s>>>(parts, grid, J, R1, R1inv, R, Rinv, bad);
    return cudaGetLastError();
}

cudaError_t launch_qr_rows(float* X, int64_t rows, int ld, int J, const double* M, int transpose,
                           cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>((rows + kQrThreads - 1) / kQrThreads, 4096);
    k_qr_rows<<<grid, kQrThreads, 0, s>>>(X, rows, ld, J, M, transpose);
    return cudaGetLastError();
}

cudaError_t launch_qr_core(const float* G, float* Gout, int N, int JP, int ldg, int n, int J,
                           const double* R, cudaStream_t s) {
    int64_t total = 1;
    for (int k = 0; k < N - 1; ++k) total *= JP;
    total *= ldg;
    const unsigned grid = (unsigned)std::min<int64_t>((total + kQrThreads - 1) / kQrThreads, 1024);
    k_qr_core<<<grid, kQrThreads, 0, s>>>(G, Gout, N, JP, ldg, n, J, R);
    return cudaGetLastError();
}

}  // namespace s3
