// Union-find connected components on the GPU (BWLabel + AreaThreshold), for
// a batch of images in one launch per stage.
#pragma once

#include "common.cuh"

namespace rtk {

constexpr int kUfBlock = 32;                   // block side
constexpr int kUfEdge = 4 * kUfBlock;
constexpr int kUfMaxRoots = kUfBlock * kUfBlock / 2;   // local components of a block (4-conn checkerboard)
constexpr int kUfMaxImgs = 32;

// One image of a labeling batch: the binary input, the workspace arrays
// (carved by the caller, uf_workspace_bytes long in total) and the outputs.
struct UfImage {
    const uint8_t *in;   // binary input (nonzero = foreground), H x W, stride ld_in
    int64_t ld_in;
    int H, W;
    int nbx, nby;        // 32 x 32 blocks per row / column
    int64_t blk_base;    // first block of this image in the batch's block numbering
    int32_t *U;          // forest over block-local roots, indexed by pixel index r*W + c (sparse use)
    int32_t *A;          // per local root: its area, then the component's (sparse use)
    int32_t *edge;       // per block, kUfEdge entries: local root of the top row, bottom row,
                         // left column, right column pixels (-1 = not in a component)
    int32_t *list;       // per block, kUfMaxRoots slots: the block's local roots
    uint16_t *cnt;       // per block: number of local roots
    uint16_t *lroot;     // per pixel (stride W): its local root inside its block (lr * 32 + lc), 0xFFFF = none;
                         // not written for blocks without foreground
    uint8_t *bempty;     // per block: 1 = no foreground
    int32_t *labels;     // output, H x W, stride ld_lab
    int64_t ld_lab;
    int32_t *n_kept;     // nullable: number of components kept (zeroed by the first stage)
    uint32_t *fgbits;    // nullable: kept pixels as a bit plane, ceil(W / 32) words per row
};

struct UfBatch {
    int n;
    int64_t nblk;        // blocks over all images
    int32_t amin, amax;  // area range kept, inclusive
    UfImage img[kUfMaxImgs];
};

// Workspace bytes of one H x W image (every array above, 256-byte aligned pieces).
size_t uf_workspace_bytes(int H, int W);
// Carves the workspace arrays of `d` from base (uf_workspace_bytes(H, W) bytes, 256-byte aligned) and sets
// the block counts; in, labels, n_kept and fgbits are left to the caller.
void uf_carve(UfImage &d, char *base, int H, int W);
// Appends image `d` to the batch (sets its blk_base).
void uf_add(UfBatch &b, const UfImage &d);
// Labels with the area filter for every image of the batch: block-local
// components, merges across block edges, final roots with their areas, and
// the output pass (four launches).
cudaError_t launch_label_batch(const UfBatch &b, int conn, cudaStream_t s);

}  // namespace rtk
