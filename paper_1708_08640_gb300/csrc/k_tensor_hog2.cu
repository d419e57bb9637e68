// FP32 HOGWILD kernel variants with two lanes per tensor entry (3-way tensors, tiles of up
// to 128 entries).
#include "tensor_hog.cuh"

namespace s3 {

#define S3_HOG_SHAPES_L2(X) \
    X(3, 2, 2) X(3, 4, 2) X(3, 5, 2) X(3, 8, 2) X(3, 10, 2) X(3, 16, 2) X(3, 20, 2) X(3, 32, 2)

S3_DEFINE_HOG_VARIANTS(S3_HOG_SHAPES_L2, launch_tensor_hog_l2_all, tensor_hog_blocks_l2_all)

cudaError_t launch_tensor_hog_l2(int N, int JP, const DParams& P, const DGroup& G, int64_t n_tiles,
                                 int* tile_counter, int grid, const float* eta, int row_mean,
                                 float core_step_scale, const int64_t* max_events,
                                 const int64_t* max_segs, int64_t ccap, cudaStream_t s) {
    return launch_tensor_hog_l2_all(N, JP, 2, P, G, n_tiles, tile_counter, grid, eta, row_mean,
                                    core_step_scale, max_events, max_segs, ccap, s);
}

int tensor_hog_blocks_l2(int N, int JP, size_t smem) { return tensor_hog_blocks_l2_all(N, JP, 2, smem); }

}  // namespace s3
