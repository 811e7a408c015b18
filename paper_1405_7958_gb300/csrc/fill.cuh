// Hole filling as a binary reconstruction on bit planes (FillHoles,
// Sections 3.2.1 and 5.1).
#pragma once

#include "common.cuh"

namespace rtk {

// Bit tiles: 32 rows x 32 words (1024 columns); a warp holds one tile, lane
// = word column, one register per row.
constexpr int kFillTH = 32;
constexpr int kFillTW = 1024;

constexpr int kFillMaxImgs = 32;

// One image of a fill batch.
struct FillImage {
    const uint8_t *in;    // binary image (nonzero = foreground), H x W, stride ld_in
    int64_t ld_in;
    uint8_t *out;         // F, H x W, stride ld_out (may be in itself, with the same stride)
    int64_t ld_out;
    int H, W;
    int ny, nx;           // tiles per column / per row
    int wq;               // words per bit-plane row (nx * 32)
    int tile_base;        // first tile of the image in the batch (tiles column-major per image)
    uint32_t *m;          // background mask, (ny * 32) rows x wq words
    uint32_t *x;          // background reached from the border, same layout
};

// Up to kFillMaxImgs images, passed by value.
struct FillBatch {
    int n, ntiles;
    int conn;             // 4 or 8 (connectivity of the background)
    int maxW, maxH, maxHp, maxWq;
    FillImage img[kFillMaxImgs];
    uint32_t *flags;      // per tile of the batch
    uint32_t *pending;    // flagged + in-progress visits
    int32_t *err;         // device status
    uint64_t timeout_ns;
};

// Workspace of one H x W image: its two bit planes.
size_t fill_image_bytes(int H, int W);
// Appends an image whose planes start at base (256-byte aligned, fill_image_bytes long).
void fill_add(FillBatch &b, const uint8_t *in, int64_t ld_in, uint8_t *out, int64_t ld_out, int H, int W,
              char *base);
// pack -> propagate (persistent, cooperative) -> output; flags needs b.ntiles words
cudaError_t launch_fill(const FillBatch &b, int num_sms, cudaStream_t s);

}  // namespace rtk
