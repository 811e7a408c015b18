/*
 * rt.h -- C ABI of the GB300 (sm_103a) segmentation hot path.
 *
 * The operations are the per-tile segmentation functions of the microscopy
 * pipeline in Teodoro et al., "Region Templates: Data Representation and
 * Management for Large-Scale Image Analysis": ReconToNuclei, FillHoles,
 * Pre-Watershed and BWLabel (Section 5.1, "Example Application") and
 * AreaThreshold (Section 3.2.1, "PATS"). The paper states that a
 * segmentation stage takes an image tile and produces a mask array
 * (Section 4, "Global Storage Implementations for Data Regions"). It names
 * the functions but does not define them; each entry point below states the
 * textbook definition it computes, and all results are unique, so every
 * variant returns identical bytes.
 *
 * Conventions for every entry point:
 *  - Image pointers are DEVICE pointers owned by the caller; the library
 *    never frees or retains them. Images are row-major; `ld_*` is the row
 *    stride in ELEMENTS (bytes for uint8 images, int32 elements for int32
 *    images) and must be >= W.
 *  - 1 <= H, W <= 32768. conn is 4 or 8 (neighbourhood of a pixel: its 4
 *    edge neighbours, or those plus the 4 diagonal ones). Out-of-image
 *    neighbours do not exist.
 *  - Binary inputs: any nonzero byte is foreground. Binary outputs are 0/1.
 *  - All work is enqueued asynchronously on `stream` (a cudaStream_t; NULL
 *    means the legacy default stream). Inputs must stay valid and unchanged
 *    until the work completes.
 *  - The return value reports synchronous failures only: invalid arguments
 *    (RT_EINVAL), workspace allocation failure (RT_ENOMEM) or a launch error
 *    (RT_ECUDA). Outcomes known only on the device (an iteration bound hit,
 *    a marker above the mask) are written to `dev_status`, a device int32
 *    the caller may pass (NULL = not reported) and read after synchronising;
 *    it holds RT_OK or the first error code raised.
 *  - A context owns its workspace (device scratch), reserves it at creation
 *    (rt_create's workspace_bytes; rt_segment_workspace_bytes gives the
 *    exact need of a batch), grows it on demand with cudaMalloc (which
 *    synchronises the device) when a call needs more, and reuses it across
 *    calls. Calls on one context must be serialised by the caller (one
 *    stream at a time); use one context per concurrent stream.
 *  - Iterative steps are bounded: the reconstruction's propagation by a
 *    number of tile visits (max_iters, see rt_set_limits), and every
 *    propagation (reconstruction and hole filling) by device time (20 s
 *    unless set otherwise). A bound that is reached stops the step short of
 *    its fixed point, reports RT_ETIMEOUT in the device status, and leaves
 *    the context usable for the next call.
 *  - Strides are in elements, not bytes (a reading of the boundary: every
 *    image has one element type, so an element stride cannot be misaligned).
 */
#ifndef RT_SEG_H
#define RT_SEG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RT_API __attribute__((visibility("default")))
#else
#define RT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0,
    RT_EINVAL = 1,    /* bad argument (null pointer, size, stride, conn, alias) */
    RT_ENOMEM = 2,    /* workspace allocation failed */
    RT_ECUDA = 3,     /* CUDA runtime error at launch */
    RT_ETIMEOUT = 4,  /* device-side iteration or wait bound reached */
    RT_EMARKER = 5,   /* marker above the mask somewhere (output still defined) */
    RT_EQUEUE = 6,    /* frontier queue overflow; never raised here: every queue of the
                         RT_QUEUE / RT_HYBRID visits has one slot per pixel of its tile and
                         a pixel is queued at most once at a time, and a full RT_FRONTIER
                         queue hands the propagation to the directional sweeps (same
                         output) */
    RT_EUNAVAIL = 7,  /* requested variant or feature not available */
    RT_ESIZE = 8      /* image larger than the fixed scratch of rt_edt_noalloc */
} rt_status;

/* Propagation variants of rt_reconstruct; all give identical output. */
enum {
    RT_AUTO = 0,    /* library choice (RT_RASTER) */
    RT_RASTER = 1,  /* directional sweeps of 32 x 64 tiles, revisiting flagged tiles */
    RT_QUEUE = 2,   /* per-tile pixel FIFOs (irregular wavefront propagation) */
    RT_HYBRID = 3,  /* one sweep visit of every tile, then pixel FIFOs for what remains */
    RT_FRONTIER = 4 /* one sweep visit of every tile, then global frontier queues of the
                       pixels that can still grow: warp-ballot compacted seeding, persistent
                       CTAs cascading through shared-memory queues with warp-aggregated
                       appends, one grid barrier per global round. A full queue (or more than
                       1022 rounds) hands over to the directional sweeps; batches of 2^21
                       tiles of 32 x 64 or more run RT_HYBRID instead */
};

typedef struct rt_ctx rt_ctx;

/* Create a context bound to CUDA device `device`, reserving
 * `workspace_bytes` of device workspace at once (0: none until a call needs
 * it). Returns RT_OK and sets *ctx, or an error (RT_ECUDA: the device is not
 * usable; RT_ENOMEM: the reservation failed). */
RT_API rt_status rt_create(rt_ctx **ctx, int device, size_t workspace_bytes);

/* Bounds of the iterative steps of the single-operation entry points
 * (rt_reconstruct, rt_fill_holes) on this context, and the defaults of
 * rt_segment_batch: max_iters > 0 lets one reconstruction propagation make
 * at most max_iters tile visits per 32 x 64 tile of its images on average (0: no
 * bound; how many visits a propagation needs depends on the schedule, so a
 * bound close to the need may or may not be reached); timeout_ms > 0 bounds
 * each propagation's device time (0: 20 s). Negative values: RT_EINVAL. */
RT_API rt_status rt_set_limits(rt_ctx *ctx, int max_iters, int timeout_ms);

/* Entries of each of the two global frontier queues of RT_FRONTIER on this
 * context (4 bytes each, part of the workspace); 0 = one per pixel of the
 * call's images padded to 32 x 64 tiles (the default). A smaller capacity
 * bounds the workspace: a propagation whose queue fills up is finished by
 * the directional sweeps, with the same output. Negative or above
 * 2^32 - 1: RT_EINVAL. */
RT_API rt_status rt_set_queue_capacity(rt_ctx *ctx, int64_t entries);

/* Free a context and its workspace. Waits for the device first. NULL is a
 * no-op. */
RT_API void rt_destroy(rt_ctx *ctx);

/* Static, human-readable name of a status code. */
RT_API const char *rt_status_str(int status);

/* ABI version (major * 100 + minor). */
RT_API int rt_version(void);

/* Bytes of device workspace the context currently holds. */
RT_API size_t rt_workspace_bytes(const rt_ctx *ctx);

/*
 * Marker of the ReconToNuclei step for nuclei tiles:
 *     J = max(I - h_offset, 0) inside the tile, J = I on the one-pixel border.
 * mask: uint8 H x W (ld_mask); marker: uint8 H x W output (ld_marker).
 * 0 <= h_offset <= 255. The two buffers may not overlap.
 */
RT_API rt_status rt_marker(rt_ctx *ctx, const uint8_t *mask, int64_t ld_mask,
                    uint8_t *marker, int64_t ld_marker, int H, int W, int h_offset,
                    void *stream);

/*
 * ReconToNuclei (Section 5.1): grayscale morphological reconstruction by
 * dilation of `marker` (J) under `mask` (I), the limit of
 *     R_0 = min(J, I),  R_{k+1} = min(delta_conn(R_k), I)
 * where delta_conn is the maximum over a pixel and its conn-neighbours
 * (Vincent 1993). The paper runs it as an irregular wavefront propagation
 * (IWPP) over active elements; `variant` picks how the GPU propagates
 * (RT_RASTER, RT_QUEUE, RT_HYBRID, RT_FRONTIER, or RT_AUTO), with identical
 * results.
 *
 * marker: uint8 H x W (ld_marker), or NULL: then the marker is derived on
 *         the fly as in rt_marker with `h_offset`.
 * mask:   uint8 H x W (ld_mask).
 * out:    uint8 H x W (ld_out); may alias `marker` exactly (same pointer and
 *         stride), must not overlap `mask`.
 * A marker above the mask is clamped (R_0 = min(J, I)) and reported as
 * RT_EMARKER in dev_status; the output is still the reconstruction of the
 * clamped marker. An iteration bound hit is reported as RT_ETIMEOUT.
 */
RT_API rt_status rt_reconstruct(rt_ctx *ctx, const uint8_t *marker, int64_t ld_marker,
                         const uint8_t *mask, int64_t ld_mask, uint8_t *out, int64_t ld_out,
                         int H, int W, int conn, int variant, int h_offset,
                         int32_t *dev_status, void *stream);

/*
 * FillHoles (Sections 3.2.1 and 5.1): out = 1 on the foreground of `in` and
 * on every background pixel that no conn-connected path of background pixels
 * links to the tile border (a hole); 0 on background reachable from the
 * border. Equivalently 1 - R(M, C) with C = 1 - in and M = C on the border, 0
 * elsewhere (reconstruction from the tile border).
 * in: uint8 H x W (ld_in); out: uint8 H x W (ld_out), may alias `in` exactly.
 */
RT_API rt_status rt_fill_holes(rt_ctx *ctx, const uint8_t *in, int64_t ld_in, uint8_t *out,
                        int64_t ld_out, int H, int W, int conn, int32_t *dev_status,
                        void *stream);

/*
 * BWLabel (Section 5.1) + AreaThreshold (Section 3.2.1): labels of the
 * conn-connected components of the foreground of `bin`. The label of a
 * component is the smallest linear index r * W + c of its pixels (W, not the
 * stride). Components whose pixel count lies outside [min_area, max_area]
 * (both ends kept) and background pixels get -1. The GPU follows the
 * union-find pattern the paper cites (a forest of pixel trees merged across
 * neighbours, then flattened).
 * bin: uint8 H x W (ld_bin); labels: int32 H x W (ld_lab), must not overlap bin.
 * dev_n_kept (device int32, nullable) receives the number of components kept.
 */
RT_API rt_status rt_label_area(rt_ctx *ctx, const uint8_t *bin, int64_t ld_bin, int32_t *labels,
                        int64_t ld_lab, int H, int W, int conn, int32_t min_area,
                        int32_t max_area, int32_t *dev_n_kept, int32_t *dev_status,
                        void *stream);

/*
 * Exact squared Euclidean distance transform, the input of the
 * Pre-Watershed step (Section 5.1):
 *     d2(p) = min over background pixels q of (r_p - r_q)^2 + (c_p - c_q)^2,
 * background = (fg == 0); only in-image pixels count; 0 on the background;
 * -1 everywhere if the image has no background pixel. Integer-exact.
 * fg: uint8 H x W (ld_fg); d2: int32 H x W (ld_d2), must not overlap fg.
 */
RT_API rt_status rt_edt(rt_ctx *ctx, const uint8_t *fg, int64_t ld_fg, int32_t *d2, int64_t ld_d2,
                 int H, int W, int32_t *dev_status, void *stream);

/* Phases of the library's launches, for the timing diagnostics below. */
enum {
    RT_PHASE_RECON_INIT = 0,   /* marker / padded copies of the mask */
    RT_PHASE_RECON_SWEEP = 1,  /* propagation to the fixed point */
    RT_PHASE_RECON_OUT = 2,    /* R output and threshold */
    RT_PHASE_FILL = 3,         /* hole filling */
    RT_PHASE_LABEL = 4,        /* labeling and area filter */
    RT_PHASE_EDT = 5,          /* distance transform */
    RT_PHASE_PICK = 6,         /* features and picker network */
    RT_PHASE_OBJECTS = 7,      /* per-object features */
    RT_PHASE_WATERSHED = 8,    /* watershed */
    RT_NPHASES = 9
};

/*
 * Timing diagnostics. With enable != 0 every phase of every later call is
 * bracketed by CUDA events recorded on the call's stream. rt_timing_read
 * waits for the recorded events, adds each phase's elapsed milliseconds to
 * ms[phase] and its number of bracketed intervals to count[phase] (arrays of
 * RT_NPHASES, either may be NULL), and forgets the records if reset != 0.
 * rt_kernel_launches returns how many kernels the context has launched.
 * rt_recon_stats waits for the device and reports how many tile visits,
 * dense sweep iterations and queue pops the last reconstruction made
 * (statistics; 0 if none); any pointer may be NULL.
 */
RT_API rt_status rt_timing_enable(rt_ctx *ctx, int enable);
RT_API rt_status rt_timing_read(rt_ctx *ctx, double *ms, int64_t *count, int reset);
RT_API int64_t rt_kernel_launches(const rt_ctx *ctx);
RT_API rt_status rt_recon_stats(rt_ctx *ctx, int64_t *visits, int64_t *iterations, int64_t *pops);

/*
 * Watershed (Section 5.1: the step after Pre-Watershed that splits touching
 * nuclei), marker-controlled flooding of the squared distance map `d2`
 * inside every object of `labels`; objects never exchange pixels, and
 * pixels are 8-connected within their object. Per object:
 *   1. markers: the regional maxima of the h-maxima transform of d2 (the
 *      reconstruction by dilation of max(d2 - h, 0) under d2, inside the
 *      object): 8-connected plateaus of equal value without a higher
 *      neighbour, each labelled by its smallest linear index r * W + c;
 *   2. flooding by levels (Vincent-Soille geodesic influence zones): for
 *      every distinct d2 value t of the object, highest first, the basins
 *      grow in synchronous breadth-first layers into the pixels with
 *      d2 >= t that have no basin yet; a pixel takes the smallest basin
 *      label among its neighbours labelled in earlier layers.
 * labels: int32 H x W (ld_lab) as rt_label_area writes them (-1 outside
 * objects; an object's label is the linear index of its first pixel in
 * raster order; other label images report RT_EINVAL in dev_status).
 * d2: int32 H x W (ld_d2). h >= 0. basins: int32 H x W (ld_b), the basin
 * label of every object pixel, -1 elsewhere; must not overlap the inputs.
 * dev_n_basins (device int32, nullable) receives the number of markers.
 * The workspace holds about 37 bytes per pixel.
 */
RT_API rt_status rt_watershed(rt_ctx *ctx, const int32_t *labels, int64_t ld_lab, const int32_t *d2,
                              int64_t ld_d2, int H, int W, int h, int32_t *basins, int64_t ld_b,
                              int32_t *dev_n_basins, int32_t *dev_status, void *stream);

/*
 * Feature computation stage (Section 5.1): per object of `labels` (as for
 * rt_watershed), over the intensities `img`, RT_NOBJFEAT features, computed
 * as the paper organises it: one thread block per object's minimum bounding
 * box accumulates the intermediate results (pixel count, perimeter,
 * coordinate and intensity moments, the 256-bin histogram, the 8-level
 * co-occurrence matrix of horizontally adjacent pixels), then one thread
 * per object computes the features. In order: area; perimeter (pixel edges
 * between the object and a 4-neighbour outside it, the image border
 * included); bounding box height, width; centroid row, column; major and
 * minor axis 4 sqrt(l1), 4 sqrt(l2) (l1 >= l2 >= 0 the eigenvalues of the
 * coordinates' population covariance); eccentricity sqrt(1 - l2 / l1) (0
 * when l1 = 0); compactness 4 pi area / perimeter^2; intensity mean,
 * population standard deviation, minimum, maximum, median (the smallest v
 * with 2 #{I <= v} >= area), entropy of the histogram in bits;
 * co-occurrence pairs n2 ((r, c), (r, c + 1) both in the object, levels
 * I >> 5), contrast sum (a - b)^2 g / n2, energy sum g^2 / n2^2,
 * homogeneity sum g / (1 + |a - b|) / n2 (0 for the last three if n2 = 0).
 * obj_labels: int32[cap], feat: double[cap][RT_NOBJFEAT], both device,
 * written for the first min(cap, number of objects) objects in increasing
 * label order; dev_n_obj (device int32, nullable) receives the number of
 * objects. The workspace holds about 28 bytes per pixel plus 1.4 KB per
 * output slot.
 */
#define RT_NOBJFEAT 20
RT_API rt_status rt_object_features(rt_ctx *ctx, const int32_t *labels, int64_t ld_lab, const uint8_t *img,
                                    int64_t ld_img, int H, int W, int32_t *obj_labels, double *feat, int cap,
                                    int32_t *dev_n_obj, int32_t *dev_status, void *stream);

/*
 * The same squared EDT as rt_edt, for callers that must not allocate device
 * memory while they run: for instance a serving loop that reserved its whole
 * memory budget at start-up, or a plug-in inside a host application that
 * owns every device allocation. For them a cudaMalloc can fail at the worst
 * moment and it synchronises the whole device. This entry point has no
 * counterpart in the paper; it exists only for such callers.
 *
 * No context and no allocation: the scratch is a fixed array built into the
 * library (about 2.5 MiB, held on every GPU that loads the library until
 * the process exits), so images are limited to H * W <= 1,048,576 pixels
 * (and W <= 32768); larger ones return RT_ESIZE. It runs on the current
 * device. The first call on a device looks the array's address up once;
 * that first call may also load the library's module onto the device,
 * which places the array there and may synchronise the device. So make
 * one warm-up call at start-up, before reserving a memory budget and
 * before any stream capture. All calls share the one
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. Arguments,
 * output and status are as for rt_edt.
 */
RT_API rt_status rt_edt_noalloc(const uint8_t *fg, int64_t ld_fg, int32_t *d2, int64_t ld_d2,
                                int H, int W, int32_t *dev_status, void *stream);

/*
 * Seeded synthetic nuclei tile, drawn on the GPU (input generation, not an
 * operation of the paper). The paper evaluates on 4K x 4K tiles of
 * brain-tumour slides (Section 5); this generator makes stand-ins of the
 * same size: dark ellipses (kind 0; semi-axes amin..amax px) or disks
 * (kind 1; radii rmin..rmax px) with intensities vlo..vhi on a 200 +- 15
 * lattice-noise background (flat = 1: constant 200), plus integer noise of
 * standard deviation ~8 (noise = 1). Every draw comes from Philox4x32-10 and
 * all geometry is integer, so the bytes equal those of the project's Python
 * generator for the same parameters. out: uint8 H x W (ld).
 */
RT_API rt_status rt_synth_tile(rt_ctx *ctx, uint8_t *out, int64_t ld, int H, int W, uint64_t seed,
                               int n_shapes, int kind, int vlo, int vhi, int rmin, int rmax,
                               int amin, int amax, int flat, int noise, void *stream);

/*
 * Learned schedule picker. The paper's PATS scheduler (Section 3.2.1) orders
 * tasks by estimated speedup because the run time of its irregular
 * operations cannot be estimated in advance; here a small network reads 24
 * cheap statistics of a tile and picks one of three schedules for its
 * reconstruction: a propagation variant and its sweep iterations per dense
 * tile visit (rt_set_picker_classes; by default RT_RASTER with 4, 12 and 24
 * iterations: short visits win on small tiles, longer ones on large tiles).
 * The budgets are learned on lone tiles; in a chunk of several tiles the
 * shared launch's throughput sets the time, and raster budgets below the
 * call's plain one are raised to it.
 *
 * rt_tile_features: features of n tiles (host arrays of device pointers,
 * strides and sizes; n <= 32) into out, a device float array n x
 * RT_NFEATURES, row-major. The features, in order: H, W, ln(H W); mean,
 * variance, skewness, kurtosis of the histogram; the lower 1, 5, 10, 25, 50,
 * 75, 90, 95, 99 percentiles; the fractions below 80 and below 110; the
 * histogram entropy (bits); mean and population standard deviation over 8 x 8
 * blocks of the fraction of pixels below 80, and the fraction of blocks above
 * 0.1; on the 8 x 8 block maximum D with marker max(D - 30, 0) (D on its
 * border), the fraction of pixels a raster-order neighbour could raise, and
 * ln(1 + their count).
 */
#define RT_NFEATURES 24
#define RT_MLP_NPARAM 5955
RT_API rt_status rt_tile_features(rt_ctx *ctx, const uint8_t *const *imgs, const int64_t *lds,
                                  const int *Hs, const int *Ws, int n, float *out, void *stream);

/*
 * The network: 24 -> 64 -> 64 -> 3, ReLU, bf16 parameters, fp32
 * accumulation. Parameters are one flat vector of RT_MLP_NPARAM values,
 * W1[64][24] b1[64] W2[64][64] b2[64] W3[3][64] b3[3] (row-major), as bf16
 * bit patterns (wb) for compute and fp32 (master) for the optimizer. norm
 * holds mu[24] then sd[24]; the input is normalised as (x - mu) / sd. All
 * pointers are device pointers.
 *
 * rt_mlp_forward: logits (B x 3, nullable), saved activations act (B x 128:
 * h1 then h2 after ReLU, nullable, needed by the backward pass) and the
 * argmax pick (B int32, nullable). Confidence fall-back: where the argmax's
 * softmax probability 1 / sum_k exp(z_k - z_max) (fp32) is below min_prob,
 * pick is `fallback` instead (min_prob <= 0: never).
 * rt_mlp_backward: gradient of the mean cross-entropy loss with respect to
 * every parameter into grad (RT_MLP_NPARAM fp32, overwritten), and the loss
 * into *loss (device float, nullable); label holds class indices 0..2. The
 * batch sums run in a fixed order, so the result is deterministic.
 * rt_mlp_adamw: one AdamW step (step counts from 1) on master, then wb =
 * bf16(master) with round-to-nearest-even; m and v are the moment buffers.
 */
RT_API rt_status rt_mlp_forward(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x, int B,
                                float *logits, float *act, int32_t *pick, float min_prob, int fallback,
                                void *stream);
/*
 * rt_mlp_forward_tc: the forward of rt_mlp_forward on the tensor cores, for
 * training batches (the paper's PATS scheduler needs an estimate per task,
 * Section 3.2.1; the network and its training are this library's). Three
 * products of 128 samples per thread block with fp32 accumulators in tensor
 * memory; their operands are bf16: the parameters, and the normalised input
 * and both hidden layers rounded to nearest even. Outputs as in
 * rt_mlp_forward; act holds the hidden layers in fp32 before that rounding.
 * The rounding makes logits differ from rt_mlp_forward's by about 2^-8
 * relative. dev_status (device int32, nullable) gets RT_ETIMEOUT if a
 * product does not complete within its wait bound.
 */
RT_API rt_status rt_mlp_forward_tc(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x, int B,
                                   float *logits, float *act, int32_t *pick, float min_prob, int fallback,
                                   int32_t *dev_status, void *stream);
/*
 * rt_mlp_backward_tc: the gradient of rt_mlp_backward on the tensor cores,
 * from the act and logits of rt_mlp_forward_tc. Per block of 128 samples,
 * dh1 = (dh2 W2) * [h1 > 0] and the W1, b1, W2, b2 gradients are bf16
 * products with fp32 accumulators (dh2, dh1, h1 and the normalised input
 * rounded to bf16); dz, dh2 and the W3, b3 gradients stay fp32. The blocks'
 * partial sums are added in a fixed order, so the result is deterministic.
 * Uses the context's workspace; dev_status as for rt_mlp_forward_tc.
 */
RT_API rt_status rt_mlp_backward_tc(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x,
                                    const float *act, const float *logits, const int32_t *label, int B,
                                    float *grad, float *loss, int32_t *dev_status, void *stream);
RT_API rt_status rt_mlp_backward(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x,
                                 const float *act, const float *logits, const int32_t *label, int B,
                                 float *grad, float *loss, void *stream);
/* Normalisation of the network's input from a training set x (B x 24,
 * device, row-major): norm[0..23] = the column means, norm[24..47] = the
 * column standard deviations with divisor B - 1 (0 when B = 1), raised to
 * at least 1e-6; sums in double in a fixed order, so the result is
 * deterministic. */
RT_API rt_status rt_feature_norm(rt_ctx *ctx, const float *x, int B, float *norm, void *stream);
RT_API rt_status rt_mlp_adamw(rt_ctx *ctx, float *master, uint16_t *wb, const float *grad, float *m,
                              float *v, int step, float lr, float beta1, float beta2, float eps,
                              float weight_decay, void *stream);

/*
 * Attach a trained picker (device pointers, owned by the caller and read
 * during later calls) to the context for rt_segment_batch with
 * policy = RT_POLICY_LEARNED; NULL detaches it.
 */
RT_API rt_status rt_set_picker(rt_ctx *ctx, const uint16_t *wb, const float *norm);

/* The picker's three schedules on this context: class c runs variants[c]
 * (RT_AUTO = RT_RASTER) with max_locals[c] sweep iterations per dense tile
 * visit (0 = the variant's default). Default: RT_RASTER with 4, 12, 24. */
RT_API rt_status rt_set_picker_classes(rt_ctx *ctx, const int *variants, const int *max_locals);

/* Classes the picker chose for the tiles of the last chunk (up to 32 tiles)
 * of the last learned rt_segment_batch call: 0..2, or 3 where the tile ran
 * the call's plain schedule: the pick fell back (confidence below
 * pick_min_prob), or the picker was not run because no pick could change
 * the schedule (a chunk of several tiles, where raster classes run at the
 * plain budget, with a raster plain schedule and raster classes only). Copies
 * up to cap of them into classes (nullable) and returns how many there
 * were. The choices stay on the device during the call (the propagation
 * reads them there) and are copied to pinned host memory at its end; this
 * call waits for that copy. After the replay of a captured graph the caller
 * synchronizes the stream first. Returns 0 on a CUDA error. */
RT_API int rt_last_picks(const rt_ctx *ctx, int *classes, int cap);

/* One tile of a batch. Every pointer is a device pointer. */
typedef struct {
    const uint8_t *img;   /* input tile I, uint8 H x W */
    int64_t ld_img;
    int H, W;
    uint8_t *recon;       /* R, uint8 H x W; NULL = not returned */
    int64_t ld_recon;
    uint8_t *filled;      /* F, uint8 H x W; NULL = not returned */
    int64_t ld_filled;
    int32_t *labels;      /* L', int32 H x W (required) */
    int64_t ld_labels;
    int32_t *d2;          /* D, int32 H x W (required) */
    int64_t ld_d2;
    int32_t *n_kept;      /* device int32, nullable: components kept */
    int32_t *status;      /* device int32, nullable: per-tile rt_status */
} rt_tile;

/* Parameters of the segmentation chain. */
typedef struct {
    int h_offset;    /* marker offset (30) */
    int threshold;   /* B = (R < threshold) (80) */
    int min_area;    /* area range kept, inclusive (20) */
    int max_area;    /* (1000) */
    int conn_recon;  /* connectivity of the reconstruction (8) */
    int conn_fill;   /* connectivity of the background flood in fill-holes (4) */
    int variant;     /* reconstruction variant for every tile (RT_AUTO) */
    int max_local;   /* sweep iterations per dense tile visit; 0 = default (12; RT_HYBRID and
                        RT_FRONTIER 64) */
    int policy;      /* RT_POLICY_PLAIN: `variant` and `max_local` for every tile;
                        RT_POLICY_LEARNED: the attached picker chooses a schedule per tile
                        (rt_set_picker_classes), and the plain schedule is kept whenever no
                        picker is attached. In a chunk of several tiles a raster class runs
                        at the plain budget (`max_local`): there the tiles share one launch,
                        whose throughput, not a tile's latency, sets the time */
    int max_iters;   /* tile visits per 32 x 64 tile allowed to the propagation, as in
                        rt_set_limits; 0 = the context's bound */
    int timeout_ms;  /* device-time bound of each propagation; 0 = the context's (20 s) */
    int pick_min_prob; /* learned policy: the network's pick stands only when its softmax
                          probability is at least pick_min_prob / 1000; below, the tile runs
                          the plain schedule (`variant`, `max_local`). 0 = always the pick */
    int strip_tiles; /* raster propagation: tiles of 32 x 64 per strip, the block of
                        vertically adjacent tiles one warp owns (1..32; strips are dealt to
                        the warps in turn); 0 = the library's choice (up to 8, about the
                        tiles per warp). Any value gives the same output */
} rt_seg_params;

enum { RT_POLICY_PLAIN = 0, RT_POLICY_LEARNED = 1 };

/* Fill `p` with the defaults listed above (policy RT_POLICY_PLAIN). */
RT_API void rt_seg_params_default(rt_seg_params *p);

/*
 * The segmentation chain of the nuclei tiles on a batch of `n` tiles of
 * possibly different sizes:
 *   J = marker(I, h_offset); R = reconstruct(J, I, conn_recon);
 *   B = (R < threshold); F = fill_holes(B, conn_fill);
 *   L' = label_area(F, 8, [min_area, max_area]); D = edt(L' >= 0).
 * `tiles` is a HOST array (copied before return); all outputs are device
 * buffers. The per-tile outputs are identical to running the single-tile
 * entry points one tile at a time. Tiles run in chunks of up to 32; every
 * stage of the chain is one launch for the whole chunk. A single tile may be
 * a whole slide (up to 32768 x 32768): the propagations cross the seams of
 * their internal tiles and the labels join across block edges, so the
 * result is that of the slide as one image.
 */
RT_API rt_status rt_segment_batch(rt_ctx *ctx, const rt_tile *tiles, int n, const rt_seg_params *params,
                           void *stream);

/* Device workspace bytes rt_segment_batch needs for these tiles and
 * parameters (its largest chunk of up to 32 tiles) on context `ctx`, whose
 * picker classes and frontier-queue capacity count (NULL: the defaults): a
 * context created with at least this much never allocates during such a
 * call. 0 on invalid arguments. Host-only; the tiles' pointers are not
 * read. */
RT_API size_t rt_segment_workspace_bytes(const rt_ctx *ctx, const rt_tile *tiles, int n,
                                         const rt_seg_params *params);

#ifdef __cplusplus
}
#endif
#endif /* RT_SEG_H */
