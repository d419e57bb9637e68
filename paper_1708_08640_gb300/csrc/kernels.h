// Host-side launch interface of the S3CMTF device kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace s3 {

// Sizes of one launch over a contiguous range of a grouping's tensor entries.
struct TensorLaunch {
    int64_t e_begin, e_end;      // tensor entries [e_begin, e_end) of the grouping
    float* contrib[kMaxN];       // per-mode contribution slots (minibatch / gradient)
    float* core_part;            // one partial core gradient per CTA, dense [prod JP]
};

// Shared-memory bytes of the FP32 tensor kernels (for cudaFuncSetAttribute / launch).
size_t tensor_contrib_smem(int N, int JP);
size_t tensor_hog_smem(int N, int JP, const int64_t* max_segs_per_factor, int n_factors);

// Minibatch / gradient: contributions of every tensor entry in [e_begin, e_end) written
// to their slots, and the CTA partials of sum e a1 o..o aN.  One CTA per kTile entries.
cudaError_t launch_tensor_contrib(int N, int JP, const DParams& P, const DGroup& G,
                                  const TensorLaunch& L, cudaStream_t s);

// HOGWILD epoch: n_tiles tiles claimed from *tile_counter (zeroed by the caller) by `grid`
// persistent CTAs; rows updated atomically with step -eta * damp * (sum or mean per tile);
// each tile adds core_step_scale * eta * (its mean core step) to G atomically.
// max_segs[F]: the largest number of segments of factor F in any tile (sizes the row
// accumulators in shared memory; see tensor_hog_smem).
cudaError_t launch_tensor_hog(int N, int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                              int* tile_counter, int grid, const float* eta, int row_mean,
                              float core_step_scale, const int64_t* max_segs, cudaStream_t s);

// BF16 tensor-core HOGWILD epoch (N = 3, JP = 16): as launch_tensor_hog, one CTA per SM;
// sets *err_flag when a bounded wait on the tensor cores ran out.
size_t tensor_hog_bf16_smem(int JP, const int64_t* max_segs, int nF);
cudaError_t launch_tensor_hog_bf16(int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                   int* tile_counter, int grid, const float* eta, int row_mean,
                                   float core_step_scale, const int64_t* max_segs, int* err_flag,
                                   cudaStream_t s);

// Deterministic minibatch epoch as one cooperative launch of `grid` CTAs (see k_minibatch.cu).
struct MbLaunch {
    float* contrib[kMaxF];
    float* core_part;        // >= grid partials of JP^N floats
    unsigned* bar_count;     // zero before the launch
    unsigned* bar_gen;
    int* err_flag;
    const float* eta;
    float core_scale;
    int row_mean;
    int64_t n_batches;
    int grid;
};
int minibatch_epoch_grid(int N, int JP, int num_sms);   // co-resident CTAs, 0 if none
cudaError_t launch_minibatch_epoch(int N, int JP, const DParams& P, const DGroup& G,
                                   const MbLaunch& L, cudaStream_t s);

// Forward: x~ of n entries given as SoA index arrays; optional predictions out, optional
// per-CTA compensated partial sums of (x - x~)^2 (2 floats per CTA).
cudaError_t launch_tensor_fwd(int N, int JP, const DParams& P, const int32_t* const* idx,
                              const float* x, int64_t n, float* pred, float* sq_part,
                              cudaStream_t s);

int tensor_supported_jp(int N, int J);   // smallest instantiated JP >= J, or 0
// sets the dynamic shared-memory limits of this shape's kernels (before any graph capture)
cudaError_t tensor_prepare(int N, int JP, size_t hog_smem);
int tensor_fwd_blocks(int64_t n);        // CTAs (and partial pairs) of launch_tensor_fwd

// Coupled-matrix entries of group range [c_begin, c_end) of matrix m: contributions to
// the u-side (factor cmode[m]) and v-side (factor N+m) slots.
cudaError_t launch_coupled_contrib(const DParams& P, const DGroup& G, int m, int64_t c_begin,
                                   int64_t c_end, float* contrib_u, float* contrib_v,
                                   cudaStream_t s);
// Coupled forward: per-CTA compensated partials of (y - y~)^2 (2 floats per CTA).
cudaError_t launch_coupled_fwd(const DParams& P, int m, const int32_t* r, const int32_t* c,
                               const float* y, int64_t n, float* sq_part, cudaStream_t s);
int coupled_fwd_blocks(int64_t n);

// Segment pass of one group: for every factor F in [0, nF) and every segment of group g,
// sum the contributions of its events in slot order (compensated) and either
//   mode 0: apply  row <- row - eta * sum / (row_mean ? count : 1)
//   mode 1: accumulate into out[F] (dense unpadded, row stride Jf[F]) with compensation
//           buffer comp[F] of the same shape.
struct SegmentLaunch {
    int nF;
    int64_t g;
    const float* contrib[kMaxF];
    float* out[kMaxF];
    float* comp[kMaxF];
    int Jf[kMaxF];
    int64_t total_segs;     // number of segments of group g over all factors
    int64_t seg_begin[kMaxF + 1];  // prefix of per-factor segment counts within group g
};
cudaError_t launch_segments(const DParams& P, const DGroup& G, const SegmentLaunch& S,
                            const float* eta, int row_mean, int mode, cudaStream_t s);

// Core pass: sums nparts partials [prod JP dense] in order and either
//   mode 0: G <- G + eta*cs*sum/n_t - eta*cs*lambda_reg/|Omega| * G   (n_t > 0)
//   mode 1: accumulate -sum into out (dense unpadded [prod J]) with compensation comp.
cudaError_t launch_core(const DParams& P, int N, int JP, const int* J, const float* parts,
                        int64_t nparts, int64_t n_t, const float* eta, float core_scale,
                        int mode, float* out, float* comp, cudaStream_t s);

// Regulariser sums: per factor F (rows with inv_cnt > 0) sum ||row||^2, and ||G||^2;
// writes compensated partials (2 floats per CTA) for each of the 1 + nF sums.
cudaError_t launch_sqnorms(const DParams& P, int nF, const int64_t* rows, int JP,
                           float* parts, int blocks_per_sum, cudaStream_t s);

// FP64 final reduction of `count` (s, c) float pairs into out[0] (device double).
cudaError_t launch_reduce_f64(const float* parts, int64_t count, double* out, cudaStream_t s);

// Parameter initialisation with the counter-based generator.
cudaError_t launch_init_params(const DParams& P, const int64_t* I, const int* J, const int64_t* K,
                               int JP, uint64_t seed, cudaStream_t s);

// Sets *flag = 1 if any of the n floats is not finite.
cudaError_t launch_check_finite(const float* p, int64_t n, int* flag, cudaStream_t s);

// Dense unpadded <-> padded copies of factor matrices / core.
cudaError_t launch_pack_rows(float* dst, int ld, const float* src, int64_t rows, int J,
                             cudaStream_t s);
cudaError_t launch_unpack_rows(float* dst, const float* src, int ld, int64_t rows, int J,
                               cudaStream_t s);
cudaError_t launch_pack_core(float* dst, const float* src, int N, const int* J, int JP,
                             cudaStream_t s);
cudaError_t launch_unpack_core(float* dst, const float* src, int N, const int* J, int JP,
                               cudaStream_t s);
// out[l] += comp[l] (folds a compensation buffer into its sum)
cudaError_t launch_add_comp(float* out, const float* comp, int64_t n, cudaStream_t s);
// dG (dense unpadded) += lam * G (G padded)
cudaError_t launch_core_reg(float* out, const float* G, int N, const int* J, int JP, float lam,
                            cudaStream_t s);
// dst[k] = src[idx[k]] (values into the library's layout)
cudaError_t launch_gather_f32(float* dst, const float* src, const int64_t* idx, int64_t n,
                              cudaStream_t s);
// resident CTAs per SM of the HOGWILD kernel with `smem` dynamic shared memory
int tensor_hog_blocks_per_sm(int N, int JP, size_t smem);

}  // namespace s3
