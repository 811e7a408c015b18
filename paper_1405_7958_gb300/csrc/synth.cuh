// Seeded synthetic nuclei tiles generated on the GPU (inputs only).
#pragma once

#include "common.cuh"

namespace rtk {

struct SynthArgs {
    int H, W;
    uint32_t k0, k1;          // Philox key = (seed mod 2^32, seed div 2^32)
    int n_shapes;
    int kind;                 // 0 ellipses, 1 disks
    int vlo, vhi;             // shape intensities
    int rmin, rmax;           // disk radii (px)
    int amin, amax;           // ellipse semi-axes (px)
    int flat;                 // 1: constant 200 background
    int noise;                // 1: add the Irwin-Hall noise
};

size_t synth_workspace_bytes(int H, int W);
cudaError_t launch_synth(const SynthArgs &a, void *ws, uint8_t *out, int64_t ld, cudaStream_t s);

}  // namespace rtk
