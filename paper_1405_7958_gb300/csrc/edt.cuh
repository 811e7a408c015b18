// Exact squared Euclidean distance transform on the GPU.
#pragma once

#include "common.cuh"

namespace rtk {

// Foreground source: a binary byte image (fg = byte != 0), a label image
// (fg = label >= 0) or a bit plane (fg = bit set; ceil(W / 32) words per row).
struct EdtArgs {
    const uint8_t *fg8;     // one of fg8 / lab32 / bits is set
    const int32_t *lab32;
    const uint32_t *bits;
    int64_t ld_in;
    int H, W;
    int32_t *d2;            // output
    int64_t ld_d2;
    uint16_t *g;            // workspace (byte / label input): vertical distance, H x W (stride W)
    uint32_t *cmask;        // workspace (bit-plane input): per segment s and column c, bit i set
                            // where row 32 s + i is background (nseg x W)
    int32_t *seg;           // workspace: 2 x nseg x W; byte / label input: first / last background
                            // row of each segment; bit-plane input: last background row above and
                            // first below each segment (-1: none)
    uint32_t *any_bg;       // workspace word
};

size_t edt_workspace_bytes(int H, int W);
cudaError_t launch_edt(const EdtArgs &a, cudaStream_t s);

}  // namespace rtk
