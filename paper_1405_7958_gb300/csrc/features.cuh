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
// the features, then the picker network on each image's features in the same
// launch as their last pass (picks as the network's forward gives them)
cudaError_t launch_features_pick(const FeatBatch &fb, float *out, const uint16_t *wb, const float *norm,
                                 int32_t *pick, float min_prob, int fallback, cudaStream_t s);

}  // namespace rtk
