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
    const float* w;              // gradient pass: per-entry weights in grouping order that
                                 // take the place of -(x - x~) in the data terms; null = -e
};

// Shared-memory bytes of the FP32 tensor kernels (for cudaFuncSetAttribute / launch).
size_t tensor_contrib_smem(int N, int JP);
size_t tensor_hog_smem(int N, int JP, int L, const int64_t* max_events, const int64_t* max_segs,
                       int64_t ccap, int n_factors);

// Gradient: contributions of every tensor entry in [e_begin, e_end) written to their slots,
// and one partial of sum e a1 o..o aN per CTA (at most max_grid CTAs, grid-stride over
// tiles); *grid_out = the number of partials written.
cudaError_t launch_tensor_contrib(int N, int JP, const DParams& P, const DGroup& G,
                                  const TensorLaunch& L, int max_grid, int* grid_out,
                                  cudaStream_t s);

// HOGWILD epoch: n_tiles tiles claimed from *tile_counter (zeroed by the caller) by `grid`
// persistent CTAs; rows updated atomically with step -eta * (the row's step scale,
// row_damp) * (sum or mean per tile);
// each tile adds core_step_scale * eta * (its mean core step) to G atomically.
// The grouping numbers events by slot (POS_SLOT); max_events[F]: the largest number of events
// of factor F in any tile (sizes the gradient slots in shared memory; see tensor_hog_smem).
// L: lanes per entry (tensor_hog_lanes).
// ccap: the most coupled entries (all matrices) of any tile.
cudaError_t launch_tensor_hog(int N, int JP, int L, const DParams& P, const DGroup& G,
                              int64_t n_tiles, int* tile_counter, int grid, const float* eta,
                              int row_mean, float core_step_scale, const int64_t* max_events,
                              const int64_t* max_segs, int64_t ccap, cudaStream_t s);

// BF16 tensor-core HOGWILD epoch (N = 3, JP = 16, 20 or 32): as launch_tensor_hog with tiles
// of at most tensor_hog_bf16_tile() entries, at most two CTAs per SM at rank 16 and one above
// (tensor_hog_bf16_blocks_per_sm); each CTA adds its accumulated core steps to G every
// core_sync tiles (and re-reads the core then); sets *err_flag when a bounded wait on the
// tensor cores ran out.
int tensor_hog_bf16_tile();
int tensor_hog_bf16_core_sync(int JP);   // the default core_sync of a rank
int tensor_hog_bf16_blocks_per_sm(int JP, size_t smem);
size_t tensor_hog_bf16_smem(int JP, const int64_t* max_events, const int64_t* max_segs, int nF);
cudaError_t launch_tensor_hog_bf16(int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                   int* tile_counter, int grid, const float* eta, int row_mean,
                                   float core_step_scale, int core_sync, const int64_t* max_events,
                                   const int64_t* max_segs, int* err_flag, uint64_t wait_ns,
                                   cudaStream_t s);

// Deterministic minibatch epoch as one cooperative launch of `grid` CTAs (see k_minibatch.cu).
struct MbLaunch {
    float* contrib[kMaxF];
    float* core_part;        // >= grid partials of JP^N floats
    unsigned* bar_count;     // cumulative grid-barrier arrivals: zero before the launch
    int* err_flag;
    const float* eta;
    float core_scale;
    int row_mean;
    int64_t n_batches;
    int grid;
    uint64_t wait_ns;        // bound of a grid-barrier wait
};
int minibatch_epoch_grid(int N, int JP, int num_sms);   // co-resident CTAs, 0 if none
cudaError_t launch_minibatch_epoch(int N, int JP, const DParams& P, const DGroup& G,
                                   const MbLaunch& L, cudaStream_t s);

// Forward: x~ of n entries given as SoA index arrays; optional predictions out, optional
// per-CTA compensated partial sums of (x - x~)^2 (2 floats per CTA).  dims: host [N] mode
// extents; an entry with an index outside [0, dims[m]) reads nothing, gets a NaN
// prediction, adds nothing to the sums and sets *bad = 1 (bad may be null).
cudaError_t launch_tensor_fwd(int N, int JP, const DParams& P, const int32_t* const* idx,
                              const int64_t* dims, int* bad, const float* x, int64_t n,
                              float* pred, float* sq_part, cudaStream_t s);
// the same with one CTA per 256 entries (no grid-stride loop): ceil(n / 256) pairs
cudaError_t launch_tensor_fwd_one_pass(int N, int JP, const DParams& P, const int32_t* const* idx,
                                       const int64_t* dims, int* bad, const float* x, int64_t n,
                                       float* sq_part, cudaStream_t s);

int tensor_supported_jp(int N, int J);   // smallest instantiated JP >= J, or 0
// Compute threads of a CTA of the FP32 HOGWILD kernel (it adds one prefetch warp): 384
// for 3-way tensors up to padded rank 16 (one CTA per SM, tiles of up to 192 entries on
// two lanes), else 256.  A tile's phases are latency-bound; larger tiles on fewer CTAs
// hold the same number of entries in flight with fewer tile latencies per entry.
__host__ __device__ constexpr int hog_compute_threads(int N, int JP) {
    return N == 3 && JP <= 16 ? 384 : 256;
}
// lanes per entry of the FP32 HOGWILD kernel for tiles of `tile` entries (tiles hold at
// most hog_compute_threads / lanes entries)
int tensor_hog_lanes(int N, int JP, int64_t tile);
// sets the dynamic shared-memory limits of this shape's gradient and forward kernels
cudaError_t tensor_prepare(int N, int JP);
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
    // group g's segments of each factor: the first nhuge[F] have more than kHugeSeg events,
    // the first nlong[F] (huge included) more than kShortSeg, the rest are short; prefixes
    // over the factors of the three class sizes
    int64_t nhuge[kMaxF];
    int64_t nlong[kMaxF];
    int64_t huge_begin[kMaxF + 1];
    int64_t long_begin[kMaxF + 1];    // long, not huge
    int64_t short_begin[kMaxF + 1];
    // a huge segment is summed in kHugeParts contiguous pieces by as many CTAs; each piece's
    // sums go to part_sums[huge index][piece][4 * C4] and the CTA that completes the segment
    // (part_done[huge index], zero between launches) adds them in piece order
    float* part_sums;
    int* part_done;
};
constexpr int kHugeParts = 16;
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
// a step from a given gradient: P (rows padded to ld) += alpha * g (dense, rows of J), and the
// core G (padded) += alpha * dG (dense; cp: the hyper-diagonal only); then max(0, .) with
// nonneg
cudaError_t launch_rows_step(float* P, int ld, const float* g, int64_t rows, int J, float alpha,
                             int nonneg, cudaStream_t s);
cudaError_t launch_core_step(float* G, const float* dG, int N, const int* J, int JP, float alpha,
                             int nonneg, int cp, cudaStream_t s);
// dst[k] = src[idx[k]] (values into the library's layout)
cudaError_t launch_gather_f32(float* dst, const float* src, const int64_t* idx, int64_t n,
                              cudaStream_t s);
// resident CTAs per SM of the HOGWILD kernel with `smem` dynamic shared memory
int tensor_hog_blocks_per_sm(int N, int JP, int L, size_t smem);
// the per-variant halves of launch_tensor_hog / tensor_hog_blocks_per_sm (k_tensor_hog2.cu:
// L = 2; k_tensor_hog4.cu: L = 4 and the 4-way L = 1)
cudaError_t launch_tensor_hog_l2(int N, int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                 int* tile_counter, int grid, const float* eta, int row_mean,
                                 float core_step_scale, const int64_t* max_events,
                                 const int64_t* max_segs, int64_t ccap, cudaStream_t s);
int tensor_hog_blocks_l2(int N, int JP, size_t smem);
cudaError_t launch_tensor_hog_l41(int N, int JP, int L, const DParams& P, const DGroup& G,
                                  int64_t n_tiles, int* tile_counter, int grid, const float* eta,
                                  int row_mean, float core_step_scale, const int64_t* max_events,
                                  const int64_t* max_segs, int64_t ccap, cudaStream_t s);
int tensor_hog_blocks_l41(int N, int JP, int L, size_t smem);

// S3CMTF-CP (k_cp.cu): the HOGWILD epoch of the hyper-diagonal core model (FP32, one thread
// per entry, tiles of at most 256 entries; tile bookkeeping as launch_tensor_hog), and the
// mask that zeroes the padded core's off-diagonal elements.
size_t tensor_cp_smem(int JP, const int64_t* max_events, const int64_t* max_segs, int nF);
int tensor_cp_blocks_per_sm(int N, int JP, size_t smem);
cudaError_t launch_tensor_cp_hog(int N, int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                 int* tile_counter, int grid, const float* eta, int row_mean,
                                 float core_step_scale, const int64_t* max_events,
                                 const int64_t* max_segs, cudaStream_t s);
cudaError_t launch_cp_mask(float* G, int N, int JP, int ldg, cudaStream_t s);

// Final QR step (k_qr.cu).  launch_qr_factor: CholeskyQR2 of U (rows x J of a row-major
// matrix with leading dimension ld, J <= 32) into R, Rinv (J x J FP64, upper triangular),
// with scratch parts ([grid][J * J] FP64), R1 and R1inv (J x J); *bad = 1 if U is
// numerically rank deficient.  launch_qr_rows: X <- X M (transpose 0: M = Rinv) or
// X <- X M^T (transpose 1: M = R) on rows of J values.  launch_qr_core: Gout = G x_n R on the
// padded core.
int qr_gram_ctas(int64_t rows, int num_sms);
cudaError_t launch_qr_factor(const float* U, int64_t rows, int ld, int J, int grid, double* parts,
                             double* R, double* Rinv, double* R1, double* R1inv, int* bad,
                             cudaStream_t s);
cudaError_t launch_qr_rows(float* X, int64_t rows, int ld, int J, const double* M, int transpose,
                           cudaStream_t s);
cudaError_t launch_qr_core(const float* G, float* Gout, int N, int JP, int ldg, int n, int J,
                           const double* R, cudaStream_t s);

}  // namespace s3
