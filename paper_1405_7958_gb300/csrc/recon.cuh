// Reconstruction by dilation on the GPU: data structures shared by the
// kernels (recon.cu) and the host entry points (api.cu).
#pragma once

#include "common.cuh"

namespace rtk {

constexpr int kTH = 32;       // warp tile: 32 rows
constexpr int kTW = 64;       //            x 64 columns (2 per lane)
// The first and last column of every tile are also kept contiguously (32
// bytes each) so that a visit reads its left and right halo in one sector
// each instead of one sector per row.
constexpr int kEdgeBytes = 2 * kTH;

// One image of a reconstruction batch. The kernels work on padded copies
// (Iw = mask, Rw = running reconstruction) of Hp x Wp pixels (multiples of
// the 32 x 64 tile) with row stride Wp; padding holds 0 in both, which never
// changes and is neutral for the maximum, so every tile is full-sized.
struct ReconImage {
    const uint8_t *marker;  // NULL: derived from the mask with h_offset
    int64_t ld_marker;
    const uint8_t *mask;
    int64_t ld_mask;
    uint8_t *Rw;
    uint8_t *Iw;
    uint8_t *Cw;            // per tile (local index), kEdgeBytes: its first and last column of Rw
    int H, W, Hp, Wp;
    int tiles_x, tiles_y;
    int tile_base;          // index of this image's first tile in the batch
    int h_offset;
    uint8_t *out;           // nullable: R, H x W, stride ld_out (output pass)
    int64_t ld_out;
    uint8_t *bin;           // nullable: B = (R < threshold), H x W, stride ld_bin (output pass)
    int64_t ld_bin;
};

constexpr int kMaxImgs = 32;

// Up to kMaxImgs images, passed by value as a kernel parameter.
struct ReconBatch {
    int n;
    int ntiles;
    int64_t max_words;        // largest Hp * Wp / 4 over the images
    ReconImage img[kMaxImgs];
};

// Schedules the picker chooses between: entry c (c < kPickClasses) is class
// c of the network, entry kPickClasses the plain schedule of the call (the
// fall-back). group = variant - 1 (0 raster, 1 queue, 2 hybrid, 3 frontier);
// max_local = that schedule's sweep iterations per dense visit.
constexpr int kPickClasses = 3;
constexpr int kPickEntries = kPickClasses + 1;
struct PickTable {
    int group[kPickEntries];
    int max_local[kPickEntries];
};

struct SweepParams {
    ReconBatch b;
    int ntiles;
    uint32_t *flags;          // per tile: nonzero = must be visited
    uint32_t *pending;        // flagged + in-progress visits
    int32_t *err;             // device status word
    uint32_t *visits;         // [0] tile visits, [1] dense iterations, [2] queue pops (statistics)
    int max_local;            // local iterations per visit before revisiting
    int seg_max;              // tiles per warp strip (0: up to kSegMax, about the tiles per warp)
    uint64_t timeout_ns;      // bound on the whole propagation (device time)
    uint32_t max_visits;      // bound on the tile visits of the propagation (0 = none)
    uint32_t *spent;          // visits started so far (device word, zeroed with the control words)
    uint32_t *abort;          // nonzero: a bound was reached, every warp leaves
    const int32_t *map;       // NULL: the launch covers tiles 0..ntiles-1; else its k-th tile is map[k]
    const uint32_t *nvirt;    // with map: number of tiles the launch covers (device word)
    const int32_t *pick;      // NULL: max_local for every tile; else image i runs table.max_local of pick[i]
    PickTable table;
    // RT_FRONTIER: the two global frontier queues (entries tile << 11 | row << 6
    // | column, row and column within the 32 x 64 tile), their capacity in
    // entries, and their control words (kFq* offsets)
    uint32_t *fq[2];
    uint32_t fq_cap;
    uint32_t *fctl;
};

// Control words of the global frontier queues. Round r drains the queue
// fq[r & 1] of fctl[kFqTail + r] entries (CTAs take them in chunks through
// fctl[kFqHead + r]) and spills into fq[(r + 1) & 1]; a grid barrier
// separates the rounds. Past kFqRounds rounds, or once an entry finds its
// queue full, the overflow word is set and the directional sweeps finish
// the propagation.
constexpr int kFqRounds = 1024;
constexpr int kFqTail = 0;
constexpr int kFqHead = kFqRounds;
constexpr int kFqBar = 2 * kFqRounds;
constexpr int kFqOver = 2 * kFqRounds + 2;
constexpr int kFqPops = 2 * kFqRounds + 4;         // 64-bit count of the drain's pops so far
constexpr int kFqCtlWords = 2 * kFqRounds + 6;
constexpr int kFqPopsPerVisit = kTH * kTW;          // pops counted as one tile visit against max_visits
constexpr int64_t kFqMaxTiles = int64_t(1) << 21;   // tiles an entry can name

// Control words of a propagation (device, zeroed before the init kernel):
// kCtlPending: pending count of an ungrouped launch; kCtlVisits..+2: the
// statistics; kCtlGroupPending + g / kCtlGroupCount + g: pending count and
// number of tiles of variant group g when the variant is chosen per image.
constexpr int kCtlPending = 0;
constexpr int kCtlVisits = 1;
constexpr int kCtlGroupPending = 4;
constexpr int kCtlGroupCount = 8;
constexpr int kCtlSpent = 12;
constexpr int kCtlAbort = 13;
constexpr int kCtlWords = 16;
constexpr int kGroups = 4;    // RT_RASTER, RT_QUEUE, RT_HYBRID, RT_FRONTIER

void plan_recon_image(ReconImage &d, int H, int W);
cudaError_t launch_marker(const uint8_t *mask, int64_t ld_mask, uint8_t *marker, int64_t ld_marker, int H,
                          int W, int h_offset, cudaStream_t s);
// pick == NULL: every tile starts with flag0, ctl[kCtlPending] counts them.
// pick != NULL (device, one table entry per image; out-of-range entries are
// the plain schedule): an image propagates in group table.group[entry];
// tiles of raster and queue images start flagged, hybrid and frontier ones
// not;
// map[g * ntiles + k] lists the tiles of group g in batch order, with their
// count and pending count in ctl.
cudaError_t launch_recon_init(const ReconBatch &b, uint32_t *flags, uint32_t *ctl, uint32_t flag0,
                              const int32_t *pick, const PickTable &table, int32_t *map, int32_t *err,
                              cudaStream_t s);
// one dense visit of every tile (non-persistent)
cudaError_t launch_recon_dense(const SweepParams &p, int conn, cudaStream_t s);
// RT_FRONTIER after the dense visits: every flagged tile (flag cleared) raises
// the pixels its neighbours allow and appends them to fq[0]
cudaError_t launch_recon_seed(const SweepParams &p, int conn, cudaStream_t s);
// RT_FRONTIER: persistent CTAs drain the global frontier queues; then the
// group's pending count is 0, or, after an overflow, every tile is flagged
// for the directional sweeps that must follow (launch_recon_persistent)
cudaError_t launch_recon_frontier(const SweepParams &p, int conn, int num_sms, cudaStream_t s, int *grid_used);
// persistent visits of flagged tiles until quiescence; queue = 1: queue visits
cudaError_t launch_recon_persistent(const SweepParams &p, int conn, int queue, int num_sms, cudaStream_t s,
                                    int *grid_used);
// R and B = (R < threshold) of every image of the batch into its out / bin
// (either may be NULL), one launch
cudaError_t launch_recon_out(const ReconBatch &b, int threshold, cudaStream_t s);

}  // namespace rtk
