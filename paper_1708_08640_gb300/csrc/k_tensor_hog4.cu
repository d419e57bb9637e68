// FP32 HOGWILD kernel variants with four lanes per tensor entry (3-way tensors, tiles of up
// to 64 entries) and the one-lane 4-way form (tiles of up to 256).
#include "tensor_hog.cuh"

namespace s3 {

#define S3_HOG_SHAPES_L41(X)                                                               \
    X(3, 2, 4) X(3, 4, 4) X(3, 5, 4) X(3, 8, 4) X(3, 10, 4) X(3, 16, 4) X(3, 20, 4)       \
    X(3, 32, 4) X(4, 2, 1) X(4, 4, 1) X(4, 8, 1)

S3_DEFINE_HOG_VARIANTS(S3_HOG_SHAPES_L41, launch_tensor_hog_l41, tensor_hog_blocks_l41)

}  // namespace s3
