// Per-tile features for the learned variant picker (see features.cu).
#pragma once

#include "common.cuh"

namespace rtk {

constexpr int kNumFeatures = 24;
constexpr int kMaxFeatImgs = 32;

struct FeatImage {
    const uint8_t *img;
    int64_t ld;
    int H, W;
    uint32_t *hist;   // workspace: 256 bins
    uint8_t *dark;    // workspace: dark pixels per 8 x 8 block
    uint8_t *bmax;    // workspace: maximum per 8 x 8 block
    unsigned long long *acc;   // workspace: full-block sums of dark, dark^2, blocks > 10 %, frontier count
};

struct FeatBatch {
    int n;
    FeatImage img[kMaxFeatImgs];
};

size_t feat_workspace_bytes(int H, int W);
// out: n x kNumFeatures float32, row-major
cudaError_t launch_features(const FeatBatch &fb, float *out, cudaStream_t s);

}  // namespace rtk
