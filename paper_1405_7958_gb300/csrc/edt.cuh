// Exact squared Euclidean distance transform on the GPU.
#pragma once

#include "common.cuh"

namespace rtk {

// One image, byte input (fg = byte != 0) or label input (fg = label >= 0).
struct EdtArgs {
    const uint8_t *fg8;     // one of fg8 / lab32 is set
    const int32_t *lab32;
    int64_t ld_in;
    int H, W;
    int32_t *d2;            // output
    int64_t ld_d2;
    uint16_t *g;            // workspace: vertical distance, H x W (stride W)
    int32_t *seg;           // workspace: 2 x nseg x W, first / last background row of each segment
    uint32_t *any_bg;       // workspace word
};

size_t edt_workspace_bytes(int H, int W);
cudaError_t launch_edt(const EdtArgs &a, cudaStream_t s);

// A batch of images given as bit planes of their foreground (fg = bit set;
// ceil(W / 32) words per row), one launch per stage for the whole batch.
constexpr int kEdtMaxImgs = 32;
struct EdtBitsImage {
    const uint32_t *bits;
    int H, W;
    int32_t *d2;            // output
    int64_t ld_d2;
    uint32_t *cmask;        // workspace: per segment s and column c, bit i set where row 32 s + i is
                            // background (nseg x W)
    int32_t *seg;           // workspace: 2 x nseg x W, the last background row above and the first
                            // below each segment (-1: none)
    int64_t mask_base, col_base, row_base;   // first CTA of the image in each stage's grid
};
struct EdtBitsBatch {
    int n;
    int maxW;
    int64_t mask_ctas, col_ctas, rows;
    EdtBitsImage img[kEdtMaxImgs];
};
// Workspace bytes of one H x W image (cmask and seg, 256-byte aligned pieces).
size_t edt_bits_workspace_bytes(int H, int W);
// Carves cmask and seg from base and appends the image.
void edt_bits_add(EdtBitsBatch &b, const uint32_t *bits, int H, int W, int32_t *d2, int64_t ld_d2, char *base);
cudaError_t launch_edt_bits_batch(const EdtBitsBatch &b, cudaStream_t s);

}  // namespace rtk
