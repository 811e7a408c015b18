// Union-find connected components on the GPU (BWLabel).
#pragma once

#include "common.cuh"

namespace rtk {

// How the binary input is read: foreground = (byte != 0), or the complement
// (the components of the background).
enum UfSource { kFgNonzero = 0, kFgZero = 1 };

constexpr int kUfBlock = 32;       // block side
constexpr int kUfEdge = 4 * kUfBlock;

struct UfArgs {
    const uint8_t *in;   // binary input, H x W, stride ld_in
    int64_t ld_in;
    int H, W;
    int32_t *U;          // forest over block-local roots, indexed by pixel index r*W + c (sparse use)
    int32_t *A;          // per local root: area or border flag (sparse use)
    int32_t *edge;       // per block, kUfEdge entries: local root of the top row, bottom row,
                         // left column, right column pixels (-1 = not in a component)
    int32_t *list;       // the local roots
    uint32_t *nlist;     // their number
    uint16_t *lroot;     // per pixel (stride W): its local root inside its block (lr * 32 + lc), 0xFFFF = none;
                         // not written for blocks without foreground
    uint8_t *bempty;     // per block: 1 = no foreground
};

// Workspace bytes the arrays need for an H x W image.
size_t uf_workspace_bytes(int H, int W);

// Builds the forest: block-local components, merges across block edges, and
// the final root of every local root with its aggregated area (count_area)
// or border-contact flag (flag_border).
cudaError_t uf_build(const UfArgs &a, int conn, int source, bool count_area, bool flag_border,
                     cudaStream_t s);
// labels = root if fg and min_area <= area(root) <= max_area, else -1; with
// fgbits, also the bit plane of labels >= 0 (ceil(W / 32) words per row)
cudaError_t uf_labels_out(const UfArgs &a, int conn, int32_t *labels, int64_t ld_lab, int32_t min_area,
                          int32_t max_area, int32_t *n_kept, uint32_t *fgbits, cudaStream_t s);

}  // namespace rtk
