// Per-object steps after the labels: enumeration of the objects of a label
// image, their features (feature computation stage) and the watershed of
// the distance map inside them (objects.cu).
#pragma once

#include "common.cuh"

namespace rtk {

constexpr int kObjFeat = 20;         // features per object
constexpr int kObjChunk = 1024;      // pixels per enumeration chunk (raster order)
constexpr int kWsSmemPx = 4096;      // largest bounding box a watershed block holds in shared memory

// Per-object intermediate results of the feature computation (one block
// per object writes them, one thread per object turns them into features).
struct ObjInter {
    int64_t area, per, sr, sc, srr, scc, src, si, sii;
    uint32_t hist[256];
    uint32_t glcm[64];
};

struct ObjArgs {
    const int32_t *L;      // labels (>= 0: object; the label is the linear index r * W + c of the
    int64_t ld_L;          // object's first pixel in raster order, as rt_label_area writes them)
    const uint8_t *I;      // intensities (features)
    int64_t ld_I;
    const int32_t *D;      // distance map (watershed)
    int64_t ld_D;
    int H, W;
    // workspace
    uint32_t *chunk_cnt;   // per chunk: objects whose first pixel lies in it, then their prefix sum
    uint32_t *ctl;         // [0] objects, [1] next object of the per-object blocks, [2] basins,
                           // [3] objects with a large box, [4] the others (watershed)
    int32_t *order;        // watershed: objects by box size class (large first from the front, small
                           // from the back)
    int32_t *idx_of;       // per pixel index (sparse): object index of the label it is the first pixel of
    int32_t *olabel;       // per object: label
    int32_t *box;          // per object: r0, c0, r1, c1
    int64_t max_obj;       // capacity of olabel / box
    ObjInter *inter;       // per written object (features)
    int32_t *R;            // watershed, image-sized (stride W): large objects' working copies
    unsigned long long *st;
    uint8_t *nm;
    // outputs
    int32_t *out_labels;   // features: labels of the written objects
    double *feat;          // features: cap x kObjFeat
    int cap;
    int32_t *basins;       // watershed: basin per pixel (-1 outside objects)
    int64_t ld_B;
    int h;                 // watershed: h of the h-maxima markers
    int32_t *n_obj;        // nullable (device)
    int32_t *n_basins;     // nullable (device)
    int32_t *err;          // device status
};

size_t obj_workspace_bytes(int H, int W, bool features, bool watershed, int cap);
// Carves the workspace arrays of `a` (features / watershed parts as asked) from base.
void obj_carve(ObjArgs &a, char *base, bool features, bool watershed);
// Enumeration, per-object blocks and the per-object threads; returns the
// number of kernels launched in *launches.
cudaError_t launch_object_features(const ObjArgs &a, int num_sms, cudaStream_t s, int *launches);
cudaError_t launch_watershed(const ObjArgs &a, int num_sms, cudaStream_t s, int *launches);

}  // namespace rtk
