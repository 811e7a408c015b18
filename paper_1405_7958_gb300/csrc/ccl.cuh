// Union-find connected components on the GPU (labeling and hole filling).
#pragma once

#include "common.cuh"

namespace rtk {

// How the binary input is read: foreground = (byte != 0), or the complement
// (background components, used by hole filling).
enum UfSource { kFgNonzero = 0, kFgZero = 1 };

struct UfArgs {
    const uint8_t *in;   // binary input, H x W, stride ld_in
    int64_t ld_in;
    int H, W;
    int32_t *U;          // parent forest, H*W int32, index r*W + c (workspace)
    int32_t *A;          // per-root accumulator (area or border flag), H*W int32 (workspace)
};

cudaError_t uf_build(const UfArgs &a, int conn, int source, bool count_area, bool flag_border,
                     cudaStream_t s);
// labels = root if fg and min_area <= area(root) <= max_area, else -1
cudaError_t uf_labels_out(const UfArgs &a, int32_t *labels, int64_t ld_lab, int32_t min_area,
                          int32_t max_area, int32_t *n_kept, cudaStream_t s);
// out = 1 where in != 0 or the background component does not touch the border
cudaError_t uf_fill_out(const UfArgs &a, uint8_t *out, int64_t ld_out, cudaStream_t s);

}  // namespace rtk
