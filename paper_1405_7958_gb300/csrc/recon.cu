// ReconToNuclei (Section 5.1 of the Region Templates paper): grayscale
// morphological reconstruction by dilation,
//     R = lim R_k,  R_0 = min(J, I),  R_{k+1} = min(delta(R_k), I).
//
// Every update here has the form R(p) <- min(I(p), max(R(p), R(q))) for a
// neighbour q, so the running image never exceeds the reconstruction and
// only grows; any schedule of such updates that stops at a fixed point of
// the 8- (or 4-) neighbourhood ends exactly at the reconstruction. The paper
// runs the operation as an irregular wavefront propagation (IWPP) over
// active elements held in a hierarchical queue. Here the image is cut into
// 32 x 64 tiles and the active elements are tiles (global level) and pixels
// inside a tile (shared-memory level). Three schedules, same bytes:
//   * dense visit: a warp loads the tile into registers as packed 16-bit
//     pairs (lane = two columns, one register per row) and sweeps it (down,
//     up, then along every row through shared memory) to its local fixed
//     point;
//   * queue visit: the warp loads the tile with its one-pixel halo into
//     shared memory, seeds a FIFO with the pixels the halo can raise (or
//     with every pixel), and propagates pixel by pixel with atomicMax,
//     queueing each pixel that increases;
//   * after a visit the warp writes the tile back and flags the neighbouring
//     tiles whose halo changed. Persistent kernels keep visiting flagged
//     tiles until no tile is flagged or being visited (no grid barrier).
// RT_RASTER = dense visits only; RT_QUEUE = queue visits only, every tile
// seeded with all its pixels; RT_HYBRID = one dense visit of every tile,
// then queue visits for the tiles whose halo changed; RT_FRONTIER = one
// dense visit of every tile, then the active pixels of the whole batch in
// global frontier queues: seeded with warp-ballot compaction, drained by
// persistent CTAs that cascade through shared-memory queues with
// warp-aggregated appends and spill to the global queue of the next round.
#include "recon.cuh"

namespace rtk {

constexpr int kWarpsPerCta = 4;
constexpr int kTS = 33;                                  // transposed row stride (words)
constexpr int kWarpWords = 2 * kTH * kTS + 2 * (kTH + 2) + kTH * 32 / 2;


// ---------------------------------------------------------------- init
// Iw = mask (0 in the padding), Rw = min(J, I). One thread per 4 pixels.
__device__ __forceinline__ int pick_entry(const int32_t *pick, int i)
{
    const int c = pick[i];
    return (c >= 0 && c < kPickEntries) ? c : kPickClasses;
}
__device__ __forceinline__ int pick_group(const int32_t *pick, const PickTable &t, int i)
{
    const int g = t.group[pick_entry(pick, i)];
    return (g >= 0 && g < kGroups) ? g : 0;
}

// Stores 16 bytes at p: one 16-byte store when p is 16-byte aligned, else bytes.
__device__ __forceinline__ void store16(uint8_t *p, uint4 v, int n)
{
    if (n == 16 && ((uintptr_t)p & 15u) == 0) {
        *reinterpret_cast<uint4 *>(p) = v;
        return;
    }
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < n; ++k) p[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
}

// Loads n <= 16 bytes at p (zeros past n), with one 16-byte load when aligned.
__device__ __forceinline__ uint4 load16(const uint8_t *p, int n)
{
    if (n == 16 && ((uintptr_t)p & 15u) == 0) return __ldg(reinterpret_cast<const uint4 *>(p));
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (int k = 0; k < n; ++k) w[k >> 2] |= (uint32_t)__ldg(p + k) << (8 * (k & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// One row of the batch per blockIdx.y, 16 padded columns per thread:
// Iw = mask (0 in the padding), Rw = min(J, I); blocks of row 0 also set the
// image's tile flags (and queue nothing: the propagation starts from them).
__global__ void recon_init_kernel(const ReconBatch b, uint32_t *flags, uint32_t *ctl, uint32_t flag0,
                                  const int32_t *pick, const PickTable table, int32_t *map, int32_t *err)
{
    const int i = blockIdx.z;
    const ReconImage &d = b.img[i];
    if (blockIdx.y == 0) {
        const int nt = d.tiles_x * d.tiles_y;
        const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
        if (!pick) {
            for (int k = tid; k < nt; k += nth) flags[d.tile_base + k] = flag0;
            if (i == 0 && tid == 0) ctl[kCtlPending] = flag0 ? (uint32_t)b.ntiles : 0u;
        } else {
            const int g = pick_group(pick, table, i);
            int off = 0;   // tiles of group g in the images before this one
            for (int j = 0; j < i; ++j)
                if (pick_group(pick, table, j) == g) off += b.img[j].tiles_x * b.img[j].tiles_y;
            int32_t *mg = map + (int64_t)g * b.ntiles + off;
            const uint32_t f0 = g >= 2 ? 0u : 2u;   // hybrid, frontier: the dense pass flags
            for (int k = tid; k < nt; k += nth) {
                flags[d.tile_base + k] = f0;
                mg[k] = d.tile_base + k;
            }
            if (i == 0 && tid == 0) {
                uint32_t cnt[kGroups] = {0u, 0u, 0u, 0u};
                for (int j = 0; j < b.n; ++j) cnt[pick_group(pick, table, j)] += b.img[j].tiles_x * b.img[j].tiles_y;
                for (int q = 0; q < kGroups; ++q) {
                    ctl[kCtlGroupCount + q] = cnt[q];
                    ctl[kCtlGroupPending + q] = q >= 2 ? 0u : cnt[q];
                }
            }
        }
    }
    const int r = blockIdx.y;
    const int c0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (r >= d.Hp || c0 >= d.Wp) return;
    uint4 iv = make_uint4(0u, 0u, 0u, 0u), rv = iv;
    if (r < d.H && c0 < d.W) {
        const int n = min(16, d.W - c0);
        iv = load16(d.mask + (int64_t)r * d.ld_mask + c0, n);
        uint32_t I[4] = {iv.x, iv.y, iv.z, iv.w}, J[4];
        if (d.marker) {
            const uint4 jv = load16(d.marker + (int64_t)r * d.ld_marker + c0, n);
            J[0] = jv.x, J[1] = jv.y, J[2] = jv.z, J[3] = jv.w;
        }
        const bool border_row = r == 0 || r == d.H - 1;
        bool bad = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t rw = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c0 + 4 * q + k;
                const int ib = (I[q] >> (8 * k)) & 0xffu;
                int jb;
                if (d.marker) jb = (J[q] >> (8 * k)) & 0xffu;
                else jb = (border_row || c == 0 || c == d.W - 1) ? ib : max(ib - d.h_offset, 0);
                if (c < d.W) {
                    bad |= jb > ib;
                    rw |= (uint32_t)min(jb, ib) << (8 * k);
                }
            }
            J[q] = rw;
        }
        rv = make_uint4(J[0], J[1], J[2], J[3]);
        if (bad) raise_status(err, RT_EMARKER);
    }
    const int64_t o = (int64_t)r * d.Wp + c0;   // Wp is a multiple of 64 and the buffers 256-byte aligned
    *reinterpret_cast<uint4 *>(d.Iw + o) = iv;
    *reinterpret_cast<uint4 *>(d.Rw + o) = rv;
    // a tile's first column starts a 16-column chunk, its last column ends one
    const int lt = (c0 / kTW) * d.tiles_y + r / kTH;
    if (c0 % kTW == 0) d.Cw[(int64_t)lt * kEdgeBytes + r % kTH] = (uint8_t)rv.x;
    if (c0 % kTW == kTW - 16) d.Cw[(int64_t)lt * kEdgeBytes + kTH + r % kTH] = (uint8_t)(rv.w >> 24);
}

cudaError_t launch_recon_init(const ReconBatch &b, uint32_t *flags, uint32_t *ctl, uint32_t flag0,
                              const int32_t *pick, const PickTable &table, int32_t *map, int32_t *err,
                              cudaStream_t s)
{
    if (pick && !map) return cudaErrorInvalidValue;
    int maxHp = 1, maxWp = 16;
    for (int i = 0; i < b.n; ++i) {
        maxHp = b.img[i].Hp > maxHp ? b.img[i].Hp : maxHp;
        maxWp = b.img[i].Wp > maxWp ? b.img[i].Wp : maxWp;
    }
    const int threads = 128;
    const dim3 grid((unsigned)ceil_div(maxWp / 16, threads), (unsigned)maxHp, (unsigned)b.n);
    recon_init_kernel<<<grid, threads, 0, s>>>(b, flags, ctl, flag0, pick, table, map, err);
    return cudaGetLastError();
}

void plan_recon_image(ReconImage &d, int H, int W)
{
    d.H = H;
    d.W = W;
    d.Hp = (int)round_up(H, kTH);
    d.Wp = (int)round_up(W, kTW);
    d.tiles_x = d.Wp / kTW;
    d.tiles_y = d.Hp / kTH;
}

// Marker of the nuclei tiles: J = max(I - h, 0) inside, J = I on the border.
__global__ void marker_kernel(const uint8_t *mask, int64_t ld_mask, uint8_t *marker, int64_t ld_marker, int H,
                              int W, int h)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W; c += gridDim.x * blockDim.x) {
        const int iv = mask[(int64_t)r * ld_mask + c];
        const bool border = r == 0 || r == H - 1 || c == 0 || c == W - 1;
        marker[(int64_t)r * ld_marker + c] = (uint8_t)(border ? iv : max(iv - h, 0));
    }
}

cudaError_t launch_marker(const uint8_t *mask, int64_t ld_mask, uint8_t *marker, int64_t ld_marker, int H,
                          int W, int h_offset, cudaStream_t s)
{
    marker_kernel<<<dim3((unsigned)ceil_div(W, 256), (unsigned)H), 256, 0, s>>>(mask, ld_mask, marker,
                                                                                ld_marker, H, W, h_offset);
    return cudaGetLastError();
}

// --------------------------------------------------------------- sweeps
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// two bytes (low 16 bits) -> two 16-bit lanes, and back
__device__ __forceinline__ uint32_t widen2(uint32_t v) { return __byte_perm(v, 0u, 0x4140); }
__device__ __forceinline__ uint32_t narrow2(uint32_t w) { return __byte_perm(w, 0u, 0x4420); }

// Flag bits of a tile: it needs a dense visit (kDense), or one side of its
// halo changed: the row above it (read by the down sweep, kTopHalo), the row
// below it (read by the up sweep, kBotHalo), or a side column or corner
// (read by the row pass, kSideHalo). kHalo: any of the three.
constexpr uint32_t kTopHalo = 1u, kDense = 2u, kBotHalo = 4u, kSideHalo = 8u;
constexpr uint32_t kHalo = kTopHalo | kBotHalo | kSideHalo;
// Set while a warp visits the tile: no other warp may take it then, since
// two visits of one tile at once would write its pixels from different
// states. Flag bits set meanwhile stay for a later visit.
constexpr uint32_t kBusy = 0x80000000u;

// Sets a tile's flag; returns 1 if the tile was already flagged (its visit
// was counted before).
__device__ __forceinline__ uint32_t mark_tile(uint32_t *flags, int t, uint32_t bits)
{
    return (atomicOr(flags + t, bits) & ~kBusy) != 0u ? 1u : 0u;
}

// Flags the neighbouring tiles that see a changed halo (and the tile itself
// with `self_bits` when nonzero). Lane 0 only, the lane that ends the visit.
template <int CONN>
__device__ __forceinline__ void mark_neighbours(const SweepParams &p, const ReconImage &d, int t, int ty, int tx,
                                                bool top, bool bot, bool left, bool right, bool tl, bool tr,
                                                bool bl, bool br, uint32_t self_bits)
{
    const int nx = d.tiles_x, ny = d.tiles_y;
    const bool c[9] = {self_bits != 0, top && ty > 0, bot && ty + 1 < ny, left && tx > 0, right && tx + 1 < nx,
                       CONN == 8 && tl && ty > 0 && tx > 0, CONN == 8 && tr && ty > 0 && tx + 1 < nx,
                       CONN == 8 && bl && ty + 1 < ny && tx > 0, CONN == 8 && br && ty + 1 < ny && tx + 1 < nx};
    const int u[9] = {t, t - 1, t + 1, t - ny, t + ny, t - ny - 1, t + ny - 1, t - ny + 1, t + ny + 1};
    uint32_t nc = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) nc += c[k];
    if (nc == 0) return;
    // Count the tiles before any warp can see their flags, then take back the
    // ones already flagged: `pending` never undercounts, even if a flagged
    // tile's visit ends before this lane gets to its next instruction. The
    // returned count is checked for wrap-around, which also makes the
    // increment complete before the flags are set.
    const uint32_t before = atomicAdd(p.pending, nc);
    if (before + nc < before) {
        raise_status(p.err, RT_ETIMEOUT);
        return;
    }
    uint32_t stale = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        if (c[k]) stale += mark_tile(p.flags, u[k], k == 0 ? self_bits : k == 1 ? kBotHalo : k == 2 ? kTopHalo : kSideHalo);
    if (stale) atomicSub(p.pending, stale);
}

__device__ __forceinline__ int find_image(const SweepParams &p, int t)
{
    int k = 0;
    while (k + 1 < p.b.n && t >= p.b.img[k + 1].tile_base) ++k;
    return k;
}

// sweep iterations a dense visit of image k may make before it is revisited
__device__ __forceinline__ int visit_budget(const SweepParams &p, int k)
{
    return p.pick ? p.table.max_local[pick_entry(p.pick, k)] : p.max_local;
}

// Halo columns of tile (tx, ty) from the neighbours' edge columns: hl for
// lane i = pixel (row i, column -1), hr = (row i, column kTW); the corners
// (rows -1 and kTH) come from the diagonal neighbours. Zero outside the
// padded image, like the padding itself.
struct Halo {
    uint32_t hl, hr, corner;   // corner: lane 0 (-1,-1), 1 (kTH,-1), 2 (-1,kTW), 3 (kTH,kTW)
};
__device__ __forceinline__ Halo load_halo(const ReconImage &d, int lt, int ty, int tx, int lane)
{
    const int ny = d.tiles_y, nx = d.tiles_x;
    const uint8_t *C = d.Cw;
    Halo h;
    h.hl = tx > 0 ? __ldcg(C + (int64_t)(lt - ny) * kEdgeBytes + kTH + lane) : 0u;
    h.hr = tx + 1 < nx ? __ldcg(C + (int64_t)(lt + ny) * kEdgeBytes + lane) : 0u;
    h.corner = 0u;
    if (lane == 0 && tx > 0 && ty > 0) h.corner = __ldcg(C + (int64_t)(lt - ny - 1) * kEdgeBytes + 2 * kTH - 1);
    if (lane == 1 && tx > 0 && ty + 1 < ny) h.corner = __ldcg(C + (int64_t)(lt - ny + 1) * kEdgeBytes + kTH);
    if (lane == 2 && tx + 1 < nx && ty > 0) h.corner = __ldcg(C + (int64_t)(lt + ny - 1) * kEdgeBytes + kTH - 1);
    if (lane == 3 && tx + 1 < nx && ty + 1 < ny) h.corner = __ldcg(C + (int64_t)(lt + ny + 1) * kEdgeBytes);
    return h;
}

struct WarpBuf {
    uint32_t *sRT, *sIT;   // kTH rows x kTS words: transposed R, I (u16x2 per word)
    uint32_t *sHL, *sHR;   // halo columns, index i <-> tile row i - 1
    uint16_t *sR0;         // the tile as loaded (kTH rows x 32 lanes), for the write-back
};

// One visit of tile t by a warp. Returns after marking the tiles to visit.
template <int CONN>
__device__ __forceinline__ uint32_t visit_tile(const SweepParams &p, int t, uint32_t bits, const WarpBuf &wb, int lane)
{
    const int img = find_image(p, t);
    const ReconImage &d = p.b.img[img];
    const int max_local = visit_budget(p, img);
    const int lt = t - d.tile_base;          // column-major: lt = tx * tiles_y + ty
    const int ty = lt % d.tiles_y, tx = lt / d.tiles_y;
    const int r0 = ty * kTH, c0 = tx * kTW;
    const int64_t Wp = d.Wp;
    const uint16_t *Rg = reinterpret_cast<const uint16_t *>(d.Rw + (int64_t)r0 * Wp + c0) + lane;
    const uint16_t *Ig = reinterpret_cast<const uint16_t *>(d.Iw + (int64_t)r0 * Wp + c0) + lane;
    const int64_t ws = Wp / 2;   // row stride in 16-bit units

    uint32_t R[kTH];
    const uint32_t *Is = wb.sIT + lane;   // mask, row r at Is[r * kTS]
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
        const uint16_t raw = __ldcg(Rg + r * ws);
        wb.sR0[r * 32 + lane] = raw;
        R[r] = widen2(raw);
        wb.sIT[r * kTS + lane] = widen2(__ldg(Ig + r * ws));
    }
    const uint32_t topw = r0 > 0 ? widen2(__ldcg(Rg - ws)) : 0u;
    const uint32_t botw = r0 + kTH < d.Hp ? widen2(__ldcg(Rg + kTH * ws)) : 0u;
    {
        const Halo h = load_halo(d, lt, ty, tx, lane);
        wb.sHL[lane + 1] = h.hl;
        wb.sHR[lane + 1] = h.hr;
        if (lane < 4) ((lane & 2) ? wb.sHR : wb.sHL)[(lane & 1) ? kTH + 1 : 0] = h.corner;
    }
    __syncwarp();

    // Passes run in the cycle down, up, rows; each pass is idempotent. `need`
    // holds the pass kinds (1 down, 2 up, 4 rows) that must still run without
    // a change: a pass that changes something requires the other two again, a
    // clean one drops itself, and the tile is at its fixed point when none is
    // left. A dense visit needs all three. A tile flagged only because part of
    // its halo moved was at the fixed point for its old halo (a visit that
    // stops short flags its own tile dense), so only the passes that read the
    // moved part can change it: the visit starts with the first of those.
    uint32_t need = (bits & kDense) || !(bits & kHalo)
                        ? 7u
                        : ((bits & kTopHalo) ? 1u : 0u) | ((bits & kBotHalo) ? 2u : 0u) | ((bits & kSideHalo) ? 4u : 0u);
    const int start = (need & 1u) ? 0 : (need & 2u) ? 1 : 2;
    int it = 0;
    for (; it < max_local && need; ++it) {
        bool ch = false;
        uint32_t prev;
        if (it > 0 || start == 0) {
            // down sweep
            prev = topw;
#pragma unroll
            for (int r = 0; r < kTH; ++r) {
                uint32_t m = vmax2(R[r], prev);
                if (CONN == 8) {
                    // lanes 0 and 31 get their own word back from the shuffles:
                    // the extra terms are in-tile neighbours anyway; the halo
                    // columns enter through the row pass
                    const uint32_t sl = __shfl_up_sync(0xffffffffu, prev, 1);
                    const uint32_t sr = __shfl_down_sync(0xffffffffu, prev, 1);
                    m = vmax2(m, vmax2(__byte_perm(sl, prev, 0x5432), __byte_perm(prev, sr, 0x5432)));
                }
                const uint32_t nv = vmin2(m, Is[r * kTS]);
                ch |= nv != R[r];
                R[r] = nv;
                prev = nv;
            }
            need = __any_sync(0xffffffffu, ch) ? 6u : need & ~1u;
            if (!need) break;
        }
        if (it > 0 || start <= 1) {
            ch = false;
            // up sweep
            prev = botw;
#pragma unroll
            for (int r = kTH - 1; r >= 0; --r) {
                uint32_t m = vmax2(R[r], prev);
                if (CONN == 8) {
                    const uint32_t sl = __shfl_up_sync(0xffffffffu, prev, 1);
                    const uint32_t sr = __shfl_down_sync(0xffffffffu, prev, 1);
                    m = vmax2(m, vmax2(__byte_perm(sl, prev, 0x5432), __byte_perm(prev, sr, 0x5432)));
                }
                const uint32_t nv = vmin2(m, Is[r * kTS]);
                ch |= nv != R[r];
                R[r] = nv;
                prev = nv;
            }
            need = __any_sync(0xffffffffu, ch) ? 5u : need & ~2u;
            if (!need) break;
        }
        ch = false;
        // left-to-right and right-to-left along every row (lane = row)
#pragma unroll
        for (int r = 0; r < kTH; ++r) wb.sRT[r * kTS + lane] = R[r];
        __syncwarp();
        {
            uint32_t *row = wb.sRT + lane * kTS;
            const uint32_t *irow = wb.sIT + lane * kTS;
            // x2 holds the incoming value in both halves. Left to right:
            // t's low half is the new left pixel a (t's high half is not
            // used); with a in both halves the same clamp gives the new word
            // (its low half stays a, because a already absorbed w_lo and is
            // at most i_lo). Right to left mirrors it.
            // the halo pixels next to the row's ends: the same row's, and for
            // 8-connectivity also the rows above and below it
            uint32_t hl = wb.sHL[lane + 1], hr = wb.sHR[lane + 1];
            if (CONN == 8) {
                hl = max(hl, max(wb.sHL[lane], wb.sHL[lane + 2]));
                hr = max(hr, max(wb.sHR[lane], wb.sHR[lane + 2]));
            }
            uint32_t x2 = __byte_perm(hl, 0u, 0x1010), hd = 0;
#pragma unroll 8
            for (int j = 0; j < kTW / 2; ++j) {
                const uint32_t w = row[j], iw = irow[j];
                const uint32_t t = vmin2(vmax2(w, x2), iw);
                const uint32_t nw = vmin2(vmax2(w, __byte_perm(t, 0u, 0x1010)), iw);
                x2 = __byte_perm(nw, 0u, 0x3232);
                row[j] = nw;
                hd |= nw ^ w;
            }
            x2 = __byte_perm(hr, 0u, 0x1010);
#pragma unroll 8
            for (int j = kTW / 2 - 1; j >= 0; --j) {
                const uint32_t w = row[j], iw = irow[j];
                const uint32_t t = vmin2(vmax2(w, x2), iw);
                const uint32_t nw = vmin2(vmax2(w, __byte_perm(t, 0u, 0x3232)), iw);
                x2 = __byte_perm(nw, 0u, 0x1010);
                row[j] = nw;
                hd |= nw ^ w;
            }
            ch = hd != 0;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kTH; ++r) R[r] = wb.sRT[r * kTS + lane];
        __syncwarp();
        need = __any_sync(0xffffffffu, ch) ? 3u : need & ~4u;
    }
    const bool converged = need == 0;

    // write back, and find which borders moved
    uint16_t *Rs = reinterpret_cast<uint16_t *>(d.Rw + (int64_t)r0 * Wp + c0) + lane;
    uint32_t dl = 0, dr = 0, dtop = 0, dbot = 0, any = 0;
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
        const uint32_t orig = widen2(wb.sR0[r * 32 + lane]);
        const uint32_t diff = orig ^ R[r];
        if (diff) __stcg(Rs + r * ws, (uint16_t)narrow2(R[r]));
        dl |= diff & 0xffffu;
        dr |= diff >> 16;
        any |= diff;
        if (r == 0) dtop = diff;
        if (r == kTH - 1) dbot = diff;
    }
    if (!__any_sync(0xffffffffu, any != 0)) return (uint32_t)it;
    // edge columns: lane 0 holds column 0 (low halves), lane 31 column kTW - 1
    if ((lane == 0 && dl) || (lane == 31 && dr)) {
        uint32_t *ce = reinterpret_cast<uint32_t *>(d.Cw + (int64_t)lt * kEdgeBytes + (lane ? kTH : 0));
#pragma unroll
        for (int q = 0; q < kTH / 4; ++q) {
            uint32_t wv = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) wv |= ((lane ? R[4 * q + k] >> 16 : R[4 * q + k]) & 0xffu) << (8 * k);
            __stcg(ce + q, wv);
        }
    }
    const bool top = __any_sync(0xffffffffu, dtop != 0);
    const bool bot = __any_sync(0xffffffffu, dbot != 0);
    const bool left = __shfl_sync(0xffffffffu, dl, 0) != 0;
    const bool right = __shfl_sync(0xffffffffu, dr, 31) != 0;
    const bool tl = __shfl_sync(0xffffffffu, dtop & 0xffffu, 0) != 0;
    const bool tr = __shfl_sync(0xffffffffu, dtop >> 16, 31) != 0;
    const bool bl = __shfl_sync(0xffffffffu, dbot & 0xffffu, 0) != 0;
    const bool br = __shfl_sync(0xffffffffu, dbot >> 16, 31) != 0;
    __threadfence();
    if (lane == 0)
        mark_neighbours<CONN>(p, d, t, ty, tx, top, bot, left, right, tl, tr, bl, br, converged ? 0u : kDense);
    return (uint32_t)it;
}

// ------------------------------------------------------------ queue visit
constexpr int kQW = kTW + 2;           // padded row (halo columns included)
constexpr int kQCap = kTH * kTW;       // one slot per pixel of the tile
constexpr int kQWords = (kTH + 2) * kQW + kTH * kTW / 4 + kQCap / 2 + kQCap / 32 + 1;
constexpr uint32_t kMaxPops = 64u * kQCap;   // bound on one queue visit

struct QBuf {
    uint32_t *R;     // (kTH + 2) x kQW, one pixel per word, halo included
    uint8_t *I;      // kTH x kTW mask
    uint16_t *q;     // FIFO of pixel indices r * kTW + c
    uint32_t *inq;   // one bit per pixel: queued
    uint32_t *tail;  // FIFO tail
};

__device__ __forceinline__ void q_push(const QBuf &qb, int idx)
{
    const uint32_t bit = 1u << (idx & 31);
    if (!(atomicOr(qb.inq + (idx >> 5), bit) & bit)) {
        const uint32_t pos = atomicAdd(qb.tail, 1u);
        qb.q[pos & (kQCap - 1)] = (uint16_t)idx;
    }
}

// Raise pixel (r, c) of the tile to min(v, I) if that is larger; queue it if
// it grew.
__device__ __forceinline__ void q_relax(const QBuf &qb, int r, int c, uint32_t v)
{
    const uint32_t cand = min(v, (uint32_t)qb.I[r * kTW + c]);
    uint32_t *a = qb.R + (r + 1) * kQW + c + 1;
    if (cand > *reinterpret_cast<volatile uint32_t *>(a)) {
        if (atomicMax(a, cand) < cand) q_push(qb, r * kTW + c);
    }
}

template <int CONN>
__device__ __forceinline__ uint32_t visit_queue(const SweepParams &p, int t, uint32_t bits, const QBuf &qb, int lane)
{
    const ReconImage &d = p.b.img[find_image(p, t)];
    const int lt = t - d.tile_base;
    const int ty = lt % d.tiles_y, tx = lt / d.tiles_y;
    const int r0 = ty * kTH, c0 = tx * kTW;
    const int64_t Wp = d.Wp;
    volatile uint32_t *vR = qb.R;

    // stage R with its halo (rows r0-1 .. r0+kTH) and the mask
    for (int i = 0; i < kTH + 2; ++i) {
        const int r = r0 - 1 + i;
        uint32_t w = 0;
        if (r >= 0 && r < d.Hp) w = __ldcg(reinterpret_cast<const uint16_t *>(d.Rw + (int64_t)r * Wp + c0) + lane);
        qb.R[i * kQW + 1 + 2 * lane] = w & 0xffu;
        qb.R[i * kQW + 2 + 2 * lane] = w >> 8;
    }
    {
        const Halo h = load_halo(d, lt, ty, tx, lane);
        qb.R[(lane + 1) * kQW] = h.hl;
        qb.R[(lane + 1) * kQW + kQW - 1] = h.hr;
        if (lane < 4) qb.R[((lane & 1) ? kTH + 1 : 0) * kQW + ((lane & 2) ? kQW - 1 : 0)] = h.corner;
    }
    for (int r = 0; r < kTH; ++r)
        reinterpret_cast<uint16_t *>(qb.I + r * kTW)[lane] =
            __ldg(reinterpret_cast<const uint16_t *>(d.Iw + (int64_t)(r0 + r) * Wp + c0) + lane);
    for (int i = lane; i < kQCap / 32; i += 32) qb.inq[i] = 0u;
    if (lane == 0) *qb.tail = 0u;
    __syncwarp();

    if (bits & kDense) {
        // every pixel is active
        for (int i = lane; i < kQCap / 32; i += 32) qb.inq[i] = 0xffffffffu;
        for (int i = lane; i < kQCap; i += 32) qb.q[i] = (uint16_t)i;
        if (lane == 0) *qb.tail = kQCap;
        __syncwarp();
    }
    // the border pixels the halo can raise: top and bottom rows, then the
    // left and right columns (values flow into the tile only here)
    for (int pos = lane; pos < 2 * kTW + 2 * kTH; pos += 32) {
        int r, c;
        if (pos < kTW) { r = 0; c = pos; }
        else if (pos < 2 * kTW) { r = kTH - 1; c = pos - kTW; }
        else if (pos < 2 * kTW + kTH) { r = pos - 2 * kTW; c = 0; }
        else { r = pos - 2 * kTW - kTH; c = kTW - 1; }
        const int a = (r + 1) * kQW + c + 1;
        uint32_t m = max(max(vR[a - kQW], vR[a + kQW]), max(vR[a - 1], vR[a + 1]));
        if (CONN == 8) m = max(m, max(max(vR[a - kQW - 1], vR[a - kQW + 1]), max(vR[a + kQW - 1], vR[a + kQW + 1])));
        const uint32_t cand = min(m, (uint32_t)qb.I[r * kTW + c]);
        if (cand > vR[a] && atomicMax(qb.R + a, cand) < cand) q_push(qb, r * kTW + c);
    }
    __syncwarp();

    // FIFO propagation, up to 32 pixels per step
    uint32_t head = 0, pops = 0;
    uint32_t tail = *reinterpret_cast<volatile uint32_t *>(qb.tail);
    while (head < tail && pops < kMaxPops) {
        const uint32_t n = min(32u, tail - head);
        int idx = -1;
        if ((uint32_t)lane < n) idx = qb.q[(head + lane) & (kQCap - 1)];
        __syncwarp();   // every slot of this step is read before any push of it
        if (idx >= 0) {
            atomicAnd(qb.inq + (idx >> 5), ~(1u << (idx & 31)));
            __threadfence_block();
            const int r = idx / kTW, c = idx % kTW;
            const uint32_t v = vR[(r + 1) * kQW + c + 1];
            if (r > 0) q_relax(qb, r - 1, c, v);
            if (r + 1 < kTH) q_relax(qb, r + 1, c, v);
            if (c > 0) q_relax(qb, r, c - 1, v);
            if (c + 1 < kTW) q_relax(qb, r, c + 1, v);
            if (CONN == 8) {
                if (r > 0 && c > 0) q_relax(qb, r - 1, c - 1, v);
                if (r > 0 && c + 1 < kTW) q_relax(qb, r - 1, c + 1, v);
                if (r + 1 < kTH && c > 0) q_relax(qb, r + 1, c - 1, v);
                if (r + 1 < kTH && c + 1 < kTW) q_relax(qb, r + 1, c + 1, v);
            }
        }
        head += n;
        pops += n;
        __syncwarp();
        tail = *reinterpret_cast<volatile uint32_t *>(qb.tail);
    }
    if (head < tail && lane == 0) raise_status(p.err, RT_ETIMEOUT);

    // write back, and find which borders moved
    uint16_t *Rs = reinterpret_cast<uint16_t *>(d.Rw + (int64_t)r0 * Wp + c0) + lane;
    const int64_t ws = Wp / 2;
    uint32_t dl = 0, dr = 0, dtop = 0, dbot = 0, any = 0;
    for (int r = 0; r < kTH; ++r) {
        const uint32_t orig = __ldcg(Rs + r * ws);
        const uint32_t nv = vR[(r + 1) * kQW + 1 + 2 * lane] | (vR[(r + 1) * kQW + 2 + 2 * lane] << 8);
        const uint32_t diff = orig ^ nv;
        if (diff) __stcg(Rs + r * ws, (uint16_t)nv);
        dl |= diff & 0xffu;
        dr |= diff >> 8;
        any |= diff;
        if (r == 0) dtop = diff;
        if (r == kTH - 1) dbot = diff;
    }
    if (!__any_sync(0xffffffffu, any != 0)) return pops;
    // edge columns, lane = row
    if (__shfl_sync(0xffffffffu, dl, 0)) d.Cw[(int64_t)lt * kEdgeBytes + lane] = (uint8_t)vR[(lane + 1) * kQW + 1];
    if (__shfl_sync(0xffffffffu, dr, 31))
        d.Cw[(int64_t)lt * kEdgeBytes + kTH + lane] = (uint8_t)vR[(lane + 1) * kQW + kTW];
    const bool top = __any_sync(0xffffffffu, dtop != 0);
    const bool bot = __any_sync(0xffffffffu, dbot != 0);
    const bool left = __shfl_sync(0xffffffffu, dl, 0) != 0;
    const bool right = __shfl_sync(0xffffffffu, dr, 31) != 0;
    const bool tl = __shfl_sync(0xffffffffu, dtop & 0xffu, 0) != 0;
    const bool tr = __shfl_sync(0xffffffffu, dtop >> 8, 31) != 0;
    const bool bl = __shfl_sync(0xffffffffu, dbot & 0xffu, 0) != 0;
    const bool br = __shfl_sync(0xffffffffu, dbot >> 8, 31) != 0;
    __threadfence();
    if (lane == 0) mark_neighbours<CONN>(p, d, t, ty, tx, top, bot, left, right, tl, tr, bl, br, 0u);
    return pops;
}

// ------------------------------------------------------------- kernels
// One dense visit of every tile (first phase of RT_HYBRID).
template <int CONN>
__global__ void __launch_bounds__(kWarpsPerCta * 32) recon_dense_kernel(SweepParams p)
{
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = blockIdx.x * kWarpsPerCta + warp;
    const int n = p.nvirt ? (int)*p.nvirt : p.ntiles;
    if (v >= n) return;
    const int t = p.map ? p.map[v] : v;
    WarpBuf wb;
    wb.sRT = smem + warp * kWarpWords;
    wb.sIT = wb.sRT + kTH * kTS;
    wb.sHL = wb.sIT + kTH * kTS;
    wb.sHR = wb.sHL + (kTH + 2);
    wb.sR0 = reinterpret_cast<uint16_t *>(wb.sHR + (kTH + 2));
    const uint32_t it = visit_tile<CONN>(p, t, kDense, wb, lane);
    if (lane == 0 && p.max_visits) atomicAdd(p.spent, 1u);   // one visit per tile: within any bound
    if (lane == 0 && p.visits) {
        atomicAdd(p.visits, 1u);
        atomicAdd(p.visits + 1, it);
    }
}

// Persistent propagation. The tiles (numbered column by column) are cut into
// segments of `seg` tiles (a vertical strip each; up to kSegMax, and about
// the tiles per warp when there are fewer), dealt to the warps in turn:
// segment s belongs to warp s mod nw. A warp visits the flagged tiles of its
// segments in order, so a change flows down a strip within one pass over
// it; a warp with nothing flagged in its own segments takes flagged tiles
// of another warp's (a different one each idle round), which keeps the
// warps busy while the flagged tiles gather in a few regions. A tile is
// taken by swapping its flag bits for kBusy and released after the visit.
// A visit is counted in `pending` from the moment its tile is flagged until
// after the visit has flagged its neighbours, so pending = 0 means the image
// is at the fixed point, and every warp leaves. The launch is cooperative
// only to guarantee that every warp is resident.
// QUEUE = 0: dense visits; QUEUE = 1: queue visits.
constexpr int kSegMax = 8;
template <int CONN, int QUEUE>
__global__ void __launch_bounds__(kWarpsPerCta * 32, QUEUE ? 3 : 4) recon_persistent_kernel(SweepParams p)
{
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpBuf wb;
    QBuf qb;
    if (QUEUE) {
        uint32_t *base = smem + warp * kQWords;
        qb.R = base;
        qb.I = reinterpret_cast<uint8_t *>(base + (kTH + 2) * kQW);
        qb.q = reinterpret_cast<uint16_t *>(base + (kTH + 2) * kQW + kTH * kTW / 4);
        qb.inq = base + (kTH + 2) * kQW + kTH * kTW / 4 + kQCap / 2;
        qb.tail = qb.inq + kQCap / 32;
    } else {
        wb.sRT = smem + warp * kWarpWords;
        wb.sIT = wb.sRT + kTH * kTS;
        wb.sHL = wb.sIT + kTH * kTS;
        wb.sHR = wb.sHL + (kTH + 2);
    wb.sR0 = reinterpret_cast<uint16_t *>(wb.sHR + (kTH + 2));
    }
    const int gw = blockIdx.x * kWarpsPerCta + warp;
    const int nw = gridDim.x * kWarpsPerCta;
    const int n = p.nvirt ? (int)*p.nvirt : p.ntiles;
    const int seg = p.seg_max > 0 ? min(p.seg_max, 32) : max(1, min(kSegMax, n / nw));
    const int spb = 32 / seg;                     // segments per ballot
    const int nseg = (n + seg - 1) / seg;
    const uint64_t t_start = globaltimer_ns();
    uint32_t nvisits = 0, work = 0;
    int idle = 0;
    bool stop = false;
    for (;;) {
        bool did = false;
        // the own segments, spb per ballot; with nothing flagged there,
        // another warp's
        for (int attempt = 0; attempt < 2 && !did && !stop; ++attempt) {
            int owner = gw;
            if (attempt == 1) {
                if (nw == 1) break;
                // the next warp first, then pseudo-random others (a hash of
                // the warp and the idle round, so every warp gets probed
                // whatever the warp count)
                const uint32_t h = idle ? ((uint32_t)gw * 0x9E3779B1u) ^ ((uint32_t)idle * 0x85EBCA77u) : 0u;
                owner = (int)(((uint32_t)gw + 1u + (h >> 8)) % (uint32_t)nw);
                if (owner == gw) owner = (owner + 1) % nw;
            }
            for (int s0 = owner; s0 < nseg && !stop; s0 += spb * nw) {
                const int sl = lane / seg;
                const int sg = s0 + sl * nw;
                const int vl = sg * seg + lane % seg;
                const bool in = sl < spb && sg < nseg && vl < n;
                const int tl = in ? (p.map ? p.map[vl] : vl) : 0;
                const uint32_t fv = in ? *reinterpret_cast<volatile uint32_t *>(p.flags + tl) : 0u;
                uint32_t mask = __ballot_sync(0xffffffffu, (fv & ~kBusy) != 0u && !(fv & kBusy));
                while (mask) {
                    const int i = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int t = __shfl_sync(0xffffffffu, tl, i);
                    uint32_t cur = __shfl_sync(0xffffffffu, fv, i);
                    uint32_t got = 0;
                    if (lane == 0) {
                        if (*reinterpret_cast<volatile uint32_t *>(p.abort)) {
                            got = 0xffffffffu;
                        } else {
                            // the flag bits for kBusy, unless another warp is
                            // visiting the tile or took its flag (then skip it)
                            for (int k = 0; k < 16; ++k) {
                                if ((cur & kBusy) || !(cur & ~kBusy)) break;
                                const uint32_t prev = atomicCAS(p.flags + t, cur, kBusy);
                                if (prev == cur) {
                                    got = cur;
                                    break;
                                }
                                cur = prev;
                            }
                            // a visit starts only within the visit bound; past
                            // it the tile gets its flag back and the
                            // propagation stops short of the fixed point and
                            // says so
                            if (got && p.max_visits && atomicAdd(p.spent, 1u) >= p.max_visits) {
                                atomicOr(p.flags + t, got);
                                atomicAnd(p.flags + t, ~kBusy);
                                raise_status(p.err, RT_ETIMEOUT);
                                atomicExch(p.abort, 1u);
                                got = 0xffffffffu;
                            }
                        }
                    }
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (got == 0xffffffffu) {
                        stop = true;
                        break;
                    }
                    if (!got) continue;
                    __threadfence();
                    if (QUEUE) work += visit_queue<CONN>(p, t, got, qb, lane);
                    else work += visit_tile<CONN>(p, t, got, wb, lane);
                    if (lane == 0) {
                        atomicAnd(p.flags + t, ~kBusy);
                        atomicSub(p.pending, 1u);
                    }
                    did = true;
                    ++nvisits;
                }
            }
        }
        if (stop) break;
        if (did) {
            idle = 0;
            continue;
        }
        uint32_t pend = 0;
        if (lane == 0) pend = ld_acquire(p.abort) ? 0u : ld_acquire(p.pending);
        pend = __shfl_sync(0xffffffffu, pend, 0);
        if (pend == 0) break;
        if (++idle > 4) __nanosleep(1500);
        int late = 0;
        if (lane == 0 && (idle & 63) == 0) late = globaltimer_ns() - t_start > p.timeout_ns;
        if (__shfl_sync(0xffffffffu, late, 0)) {
            if (lane == 0) {
                raise_status(p.err, RT_ETIMEOUT);
                atomicExch(p.abort, 1u);
            }
            break;
        }
    }
    if (lane == 0 && p.visits && nvisits) {
        atomicAdd(p.visits, nvisits);
        atomicAdd(p.visits + (QUEUE ? 2 : 1), work);
    }
}

size_t recon_smem_bytes(int queue) { return sizeof(uint32_t) * (queue ? kQWords : kWarpWords) * kWarpsPerCta; }

cudaError_t launch_recon_dense(const SweepParams &p, int conn, cudaStream_t s)
{
    const size_t smem = recon_smem_bytes(0);
    const void *fn = conn == 8 ? (const void *)recon_dense_kernel<8> : (const void *)recon_dense_kernel<4>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SweepParams pp = p;
    void *args[] = {&pp};
    return cudaLaunchKernel(fn, dim3((unsigned)ceil_div(p.ntiles, kWarpsPerCta)), dim3(kWarpsPerCta * 32), args,
                            smem, s);
}

cudaError_t launch_recon_persistent(const SweepParams &p, int conn, int queue, int num_sms, cudaStream_t s,
                                    int *grid_used)
{
    const size_t smem = recon_smem_bytes(queue);
    const void *fn;
    if (queue) fn = conn == 8 ? (const void *)recon_persistent_kernel<8, 1> : (const void *)recon_persistent_kernel<4, 1>;
    else fn = conn == 8 ? (const void *)recon_persistent_kernel<8, 0> : (const void *)recon_persistent_kernel<4, 0>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWarpsPerCta * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * num_sms;
    const int need = (int)ceil_div(p.ntiles, kWarpsPerCta);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (grid_used) *grid_used = grid;
    SweepParams pp = p;
    void *args[] = {&pp};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kWarpsPerCta * 32), args, smem, s);
}

// ------------------------------------------------------ global frontier
// Entry of the frontier queues: tile << 11 | row << 6 | column (row, column
// within the 32 x 64 tile).
__device__ __forceinline__ uint32_t fq_entry(int t, int r, int c)
{
    return ((uint32_t)t << 11) | ((uint32_t)r << 6) | (uint32_t)c;
}

// Image, padded row and column of tile t's pixel (r, c).
struct FqPixel {
    int img, row, col;
};
__device__ __forceinline__ FqPixel fq_decode(const SweepParams &p, uint32_t e)
{
    const int t = (int)(e >> 11);
    FqPixel q;
    q.img = find_image(p, t);
    const ReconImage &d = p.b.img[q.img];
    const int lt = t - d.tile_base;
    const int tx = lt / d.tiles_y, ty = lt - tx * d.tiles_y;
    q.row = ty * kTH + (int)((e >> 6) & 31u);
    q.col = tx * kTW + (int)(e & 63u);
    return q;
}

// Raises byte *a to v if that is larger (a 32-bit compare-and-swap on the
// word holding it; every other writer of the word during the drain does the
// same). Returns true if this call raised it. Bytes only grow, so the loop
// retries at most once per increase of one of the word's four bytes.
__device__ __forceinline__ bool fq_raise(uint8_t *a, uint32_t v)
{
    uint32_t *w = reinterpret_cast<uint32_t *>(reinterpret_cast<uintptr_t>(a) & ~uintptr_t(3));
    const uint32_t sh = 8u * (uint32_t)(reinterpret_cast<uintptr_t>(a) & 3u);
    uint32_t old = __ldcg(w);
    while (((old >> sh) & 0xffu) < v) {
        const uint32_t nw = (old & ~(0xffu << sh)) | (v << sh);
        const uint32_t prev = atomicCAS(w, old, nw);
        if (prev == old) return true;
        old = prev;
    }
    return false;
}

__device__ __forceinline__ uint32_t lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Seeding: one warp per tile of the launch that the dense visits left
// flagged. The tile and its one-pixel halo are read into shared memory; every
// pixel is raised once to min(I, maximum of its neighbours) where that is
// larger, and the raised pixels are appended to fq[0] (one atomic per warp).
// Unflagged tiles need nothing: their visit reached the local fixed point and
// no neighbour changed their halo since, so the only pixels that can still
// grow lie in flagged tiles or next to pixels raised here, which the queue
// holds.
constexpr int kSeedWarps = 4;
constexpr int kSeedW = kTW + 4;   // shared row: column c at index c + 1
template <int CONN>
__global__ void __launch_bounds__(kSeedWarps * 32) recon_seed_kernel(SweepParams p)
{
    __shared__ uint8_t sR[kSeedWarps][kTH + 2][kSeedW];
    __shared__ uint8_t sI[kSeedWarps][kTH][kTW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = blockIdx.x * kSeedWarps + warp;
    const int n = p.nvirt ? (int)*p.nvirt : p.ntiles;
    if (v >= n) return;
    const int t = p.map ? p.map[v] : v;
    uint32_t f = 0;
    if (lane == 0) f = atomicExch(p.flags + t, 0u);
    if (__shfl_sync(0xffffffffu, f, 0) == 0u) return;
    const int img = find_image(p, t);
    const ReconImage &d = p.b.img[img];
    const int lt = t - d.tile_base;
    const int tx = lt / d.tiles_y, ty = lt - tx * d.tiles_y;
    const int r0 = ty * kTH, c0 = tx * kTW;
    const int64_t Wp = d.Wp;
    uint8_t (*R)[kSeedW] = sR[warp];
    uint8_t (*I)[kTW] = sI[warp];
    for (int rr = -1; rr <= kTH; ++rr) {
        const int gr = r0 + rr;
        const bool in = gr >= 0 && gr < d.Hp;
        uint32_t pr = 0;
        if (in) pr = __ldcg(reinterpret_cast<const uint16_t *>(d.Rw + gr * Wp + c0) + lane);
        R[rr + 1][2 * lane + 1] = (uint8_t)pr;
        R[rr + 1][2 * lane + 2] = (uint8_t)(pr >> 8);
        if (lane < 2) {
            const int gc = lane ? c0 + kTW : c0 - 1;
            R[rr + 1][lane ? kTW + 1 : 0] = (in && gc >= 0 && gc < d.Wp) ? __ldcg(d.Rw + gr * Wp + gc) : (uint8_t)0;
        }
        if (rr >= 0 && rr < kTH) {
            const uint32_t pi = __ldg(reinterpret_cast<const uint16_t *>(d.Iw + gr * Wp + c0) + lane);
            I[rr][2 * lane] = (uint8_t)pi;
            I[rr][2 * lane + 1] = (uint8_t)(pi >> 8);
        }
    }
    __syncwarp();
    uint64_t bits = 0;   // bit 2 r + k: pixel (r, 2 lane + k) was raised
    for (int r = 0; r < kTH; ++r) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int c = 2 * lane + k;       // shared column c + 1
            uint32_t m = max(max((uint32_t)R[r][c + 1], (uint32_t)R[r + 2][c + 1]),
                             max((uint32_t)R[r + 1][c], (uint32_t)R[r + 1][c + 2]));
            if (CONN == 8)
                m = max(m, max(max((uint32_t)R[r][c], (uint32_t)R[r][c + 2]),
                               max((uint32_t)R[r + 2][c], (uint32_t)R[r + 2][c + 2])));
            const uint32_t nv = min(m, (uint32_t)I[r][c]);
            if (nv > R[r + 1][c + 1]) {
                d.Rw[(int64_t)(r0 + r) * Wp + c0 + c] = (uint8_t)nv;
                bits |= 1ull << (2 * r + k);
            }
        }
    }
    // append: an inclusive warp scan of the counts, one atomic per warp
    const uint32_t cnt = (uint32_t)__popcll(bits);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0u) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(p.fctl + kFqTail, total);
    base = __shfl_sync(0xffffffffu, base, 0);
    uint32_t pos = base + incl - cnt;
    bool over = false;
    while (bits) {
        const int b = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        if (pos < p.fq_cap) p.fq[0][pos] = fq_entry(t, b >> 1, 2 * lane + (b & 1));
        else over = true;
        ++pos;
    }
    if (over) atomicExch(p.fctl + kFqOver, 1u);
}

cudaError_t launch_recon_seed(const SweepParams &p, int conn, cudaStream_t s)
{
    const dim3 grid((unsigned)ceil_div(p.ntiles, kSeedWarps));
    if (conn == 8) recon_seed_kernel<8><<<grid, kSeedWarps * 32, 0, s>>>(p);
    else recon_seed_kernel<4><<<grid, kSeedWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

constexpr int kFqThreads = 256;
constexpr int kFqLocal = 2048;   // entries per shared-memory queue
constexpr int kFqGrab = 1024;    // entries a CTA takes from a global queue at a time

// Appends the lanes' raised pixels: into the CTA's next shared queue through
// one shared atomic per warp, and what does not fit into the global queue of
// the next round through one global atomic per warp. Called by all 32 lanes.
__device__ __forceinline__ void fq_push(const SweepParams &p, bool raised, uint32_t e, uint32_t *next,
                                        uint32_t *cnt, uint32_t *out, uint32_t *out_tail, int lane)
{
    const uint32_t m = __ballot_sync(0xffffffffu, raised);
    if (m == 0u) return;
    const int lead = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == lead) base = atomicAdd(cnt, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, lead);
    const uint32_t slot = base + (uint32_t)__popc(m & lanemask_lt(lane));
    const bool spill = raised && slot >= (uint32_t)kFqLocal;
    if (raised && !spill) next[slot] = e;
    const uint32_t sm = __ballot_sync(0xffffffffu, spill);
    if (sm == 0u) return;
    const int l2 = __ffs(sm) - 1;
    uint32_t gb = 0;
    if (lane == l2) gb = atomicAdd(out_tail, (uint32_t)__popc(sm));
    gb = __shfl_sync(0xffffffffu, gb, l2);
    if (spill) {
        const uint32_t g = gb + (uint32_t)__popc(sm & lanemask_lt(lane));
        if (g < p.fq_cap) out[g] = e;
        else atomicExch(p.fctl + kFqOver, 1u);
    }
}

// Pops one entry per lane (valid lanes): reads the pixel's current value v
// and raises each neighbour q to min(v, I(q)) where that is larger, queueing
// the neighbours it raised. The pixel's value and all neighbours' I and R are
// loaded together (one round trip to L2), then the raises (compare-and-swap),
// then the appends. Called by all 32 lanes.
template <int CONN>
__device__ __forceinline__ void fq_relax(const SweepParams &p, bool valid, uint32_t e, uint32_t *next,
                                         uint32_t *cnt, uint32_t *out, uint32_t *out_tail, int lane)
{
    constexpr int kN = CONN == 8 ? 8 : 4;
    FqPixel q{0, 0, 0};
    if (valid) q = fq_decode(p, e);
    const ReconImage &d = p.b.img[q.img];
    const int64_t o0 = (int64_t)q.row * d.Wp + q.col;
    const uint32_t v = valid ? (uint32_t)__ldcg(d.Rw + o0) : 0u;
    uint32_t iq[kN], rq[kN];
    uint32_t inside = 0;   // bit k: neighbour k lies in the padded image
#pragma unroll
    for (int k = 0; k < kN; ++k) {
        const int dr = k == 0 ? -1 : k == 1 ? 1 : k < 4 ? 0 : (k & 1 ? 1 : -1);
        const int dc = k < 2 ? 0 : k == 2 ? -1 : k == 3 ? 1 : (k < 6 ? -1 : 1);
        const int rr = q.row + dr, cc = q.col + dc;
        iq[k] = rq[k] = 0u;
        if (valid && rr >= 0 && rr < d.Hp && cc >= 0 && cc < d.Wp) {
            const int64_t o = o0 + (int64_t)dr * d.Wp + dc;
            iq[k] = __ldg(d.Iw + o);
            rq[k] = __ldcg(d.Rw + o);
            inside |= 1u << k;
        }
    }
    uint32_t raised = 0;
#pragma unroll
    for (int k = 0; k < kN; ++k) {
        const int dr = k == 0 ? -1 : k == 1 ? 1 : k < 4 ? 0 : (k & 1 ? 1 : -1);
        const int dc = k < 2 ? 0 : k == 2 ? -1 : k == 3 ? 1 : (k < 6 ? -1 : 1);
        const uint32_t nv = min(v, iq[k]);
        if (((inside >> k) & 1u) && nv > rq[k] && fq_raise(d.Rw + o0 + (int64_t)dr * d.Wp + dc, nv))
            raised |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < kN; ++k) {
        const int dr = k == 0 ? -1 : k == 1 ? 1 : k < 4 ? 0 : (k & 1 ? 1 : -1);
        const int dc = k < 2 ? 0 : k == 2 ? -1 : k == 3 ? 1 : (k < 6 ? -1 : 1);
        const int rr = q.row + dr, cc = q.col + dc;
        const bool r_k = (raised >> k) & 1u;
        const uint32_t eq = r_k ? fq_entry(d.tile_base + (cc / kTW) * d.tiles_y + rr / kTH, rr % kTH, cc % kTW) : 0u;
        fq_push(p, r_k, eq, next, cnt, out, out_tail, lane);
    }
}

// Grid barrier between the drain's rounds: bar[0] arrivals, bar[1]
// generation. The wait ends when every CTA has arrived, or early once the
// abort or the overflow word is set (both are sticky and stop every CTA at
// its next check, so none waits for a CTA that has left) or the time bound
// passes. Returns false when it ended early.
__device__ __forceinline__ bool fq_barrier(const SweepParams &p, uint32_t *bar, uint64_t t0)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        const uint32_t gen = ld_acquire(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            uint32_t spins = 0;
            while (ld_acquire(bar + 1) == gen) {
                if (++spins > 64) __nanosleep(64);
                if ((spins & 63u) == 0u) {
                    if (ld_acquire(p.abort) || ld_acquire(p.fctl + kFqOver)) {
                        s_ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > p.timeout_ns) {
                        raise_status(p.err, RT_ETIMEOUT);
                        atomicExch(p.abort, 1u);
                        s_ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

// The drain. Round r: CTAs take chunks of the round's global queue into a
// shared-memory queue and cascade locally (each step pops the whole local
// queue, __syncthreads, the pushes become the next local queue) until the
// chunk's cascade dies out, then take another chunk; pushes that overflow
// the local queue go to the next round's global queue. A grid barrier ends
// the round (the launch is cooperative, so every CTA is resident). The
// abort word, the time bound, the visit bound (kFqPopsPerVisit pops count as
// one tile visit, after the visits already spent) and the overflow word are
// checked at every chunk and every 64 local steps.
template <int CONN>
__global__ void __launch_bounds__(kFqThreads) recon_frontier_kernel(SweepParams p)
{
    __shared__ uint32_t sq[2][kFqLocal];
    __shared__ uint32_t s_cnt[3];
    __shared__ uint32_t s_lo, s_hi, s_stop;
    __shared__ uint32_t s_pops, s_told;   // pops of this CTA; the part added to the global count
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t *ctl = p.fctl;
    unsigned long long *pops_all = reinterpret_cast<unsigned long long *>(ctl + kFqPops);
    const unsigned long long bound = (unsigned long long)p.max_visits * kFqPopsPerVisit;
    const uint64_t t0 = globaltimer_ns();
    if (tid == 0) s_pops = s_told = 0u;
    bool go = ld_acquire(ctl + kFqOver) == 0u && ld_acquire(p.abort) == 0u;
    for (int round = 0; go; ++round) {
        const uint32_t *in = p.fq[round & 1];
        uint32_t *out = p.fq[(round + 1) & 1];
        uint32_t *out_tail = ctl + kFqTail + round + 1;
        const uint32_t n_in = min(ld_acquire(ctl + kFqTail + round), p.fq_cap);
        if (tid == 0) s_cnt[0] = s_cnt[1] = s_cnt[2] = 0u;
        __syncthreads();
        uint32_t n = 0, step = 0;
        int cur = 0;
        for (;;) {
            if (n == 0u || (step & 63u) == 63u) {
                if (tid == 0) {
                    uint32_t stop = ld_acquire(p.abort) | ld_acquire(ctl + kFqOver);
                    const uint32_t add = s_pops - s_told;
                    s_told = s_pops;
                    const unsigned long long done = add ? atomicAdd(pops_all, (unsigned long long)add) + add : 0ull;
                    const bool spent = bound && (unsigned long long)ld_acquire(p.spent) * kFqPopsPerVisit + done > bound;
                    if (!stop && (spent || globaltimer_ns() - t0 > p.timeout_ns)) {
                        raise_status(p.err, RT_ETIMEOUT);
                        atomicExch(p.abort, 1u);
                        stop = 1u;
                    }
                    uint32_t lo = 0, hi = 0;
                    if (!stop && n == 0u) {
                        lo = atomicAdd(ctl + kFqHead + round, (uint32_t)kFqGrab);
                        hi = min(lo + (uint32_t)kFqGrab, n_in);
                    }
                    s_lo = lo;
                    s_hi = hi;
                    s_stop = stop;
                }
                __syncthreads();
                if (s_stop) break;
                if (n == 0u) {
                    const uint32_t lo = s_lo, hi = s_hi;
                    if (lo >= hi) break;
                    n = hi - lo;
                    for (uint32_t i = tid; i < n; i += kFqThreads) sq[cur][i] = __ldcg(in + lo + i);
                    __syncthreads();
                }
            }
            // step s pushes into s_cnt[s % 3]; the counter of step s + 1 was
            // last read at the start of step s - 1, before the barrier that
            // began this step, so it can be cleared now
            uint32_t *cnt = &s_cnt[step % 3u];
            if (tid == 0) s_cnt[(step + 1u) % 3u] = 0u;
            for (uint32_t base = (uint32_t)warp * 32u; base < n; base += kFqThreads) {
                const uint32_t i = base + (uint32_t)lane;
                const bool valid = i < n;
                fq_relax<CONN>(p, valid, valid ? sq[cur][i] : 0u, sq[cur ^ 1], cnt, out, out_tail, lane);
                if (lane == 0) atomicAdd(&s_pops, min(n - base, 32u));
            }
            __syncthreads();
            n = min(*cnt, (uint32_t)kFqLocal);
            cur ^= 1;
            ++step;
        }
        if (!fq_barrier(p, ctl + kFqBar, t0)) break;
        // the round's spill count is final here (the next round spills into
        // the next counter), so every CTA takes the same decision; the abort
        // and overflow words may be set later by a CTA already in the next
        // round, which the early exits of its checks and barrier absorb
        if (ld_acquire(p.abort) || ld_acquire(ctl + kFqOver)) break;
        if (ld_acquire(out_tail) == 0u) break;
        if (round + 2 >= kFqRounds) {   // the next round would have no spill counter
            if (tid == 0) atomicExch(ctl + kFqOver, 1u);
            break;
        }
    }
    __syncthreads();
    if (tid == 0 && s_pops && p.visits) atomicAdd(p.visits + 2, s_pops);
    // Hand over to the directional sweeps: nothing to do (pending 0), or,
    // after an overflow, every tile flagged for a dense visit with its edge
    // columns refreshed from the drained image.
    if (ld_acquire(p.abort)) return;
    const bool over = ld_acquire(ctl + kFqOver) != 0u;
    const int n = p.nvirt ? (int)*p.nvirt : p.ntiles;
    if (over) {
        for (int v = blockIdx.x * kFqThreads + tid; v < n; v += gridDim.x * kFqThreads) {
            const int t = p.map ? p.map[v] : v;
            const ReconImage &d = p.b.img[find_image(p, t)];
            const int lt = t - d.tile_base;
            const int tx = lt / d.tiles_y, ty = lt - tx * d.tiles_y;
            const uint8_t *src = d.Rw + (int64_t)ty * kTH * d.Wp + tx * kTW;
            uint8_t *ce = d.Cw + (int64_t)lt * kEdgeBytes;
            for (int r = 0; r < kTH; ++r) {
                ce[r] = __ldcg(src + (int64_t)r * d.Wp);
                ce[kTH + r] = __ldcg(src + (int64_t)r * d.Wp + kTW - 1);
            }
            p.flags[t] = kDense;
        }
    }
    if (blockIdx.x == 0 && tid == 0) *p.pending = over ? (uint32_t)n : 0u;
}

cudaError_t launch_recon_frontier(const SweepParams &p, int conn, int num_sms, cudaStream_t s, int *grid_used)
{
    const void *fn = conn == 8 ? (const void *)recon_frontier_kernel<8> : (const void *)recon_frontier_kernel<4>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFqThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * num_sms;
    if (grid > p.ntiles) grid = p.ntiles;   // small batches: fewer CTAs at the barriers
    if (grid < 1) grid = 1;
    if (grid_used) *grid_used = grid;
    SweepParams pp = p;
    void *args[] = {&pp};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kFqThreads), args, 0, s);
}

// --------------------------------------------------------------- output
// out = R (cropped to H x W) and bin = (R < threshold), either optional,
// for image blockIdx.z; one row per blockIdx.y, 16 columns per thread.
__global__ void recon_out_kernel(const ReconBatch b, int threshold)
{
    const ReconImage &d = b.img[blockIdx.z];
    const int r = blockIdx.y;
    const int c0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (r >= d.H || c0 >= d.W) return;
    const int n = min(16, d.W - c0);
    const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(d.Rw + (int64_t)r * d.Wp + c0));
    if (d.out) store16(d.out + (int64_t)r * d.ld_out + c0, v, n);
    if (d.bin) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t x = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) x |= (uint32_t)((int)((w[q] >> (8 * k)) & 0xffu) < threshold) << (8 * k);
            o[q] = x;
        }
        store16(d.bin + (int64_t)r * d.ld_bin + c0, make_uint4(o[0], o[1], o[2], o[3]), n);
    }
}

cudaError_t launch_recon_out(const ReconBatch &b, int threshold, cudaStream_t s)
{
    int maxH = 1, maxW = 1;
    for (int i = 0; i < b.n; ++i) {
        maxH = b.img[i].H > maxH ? b.img[i].H : maxH;
        maxW = b.img[i].W > maxW ? b.img[i].W : maxW;
    }
    const int threads = 128;
    recon_out_kernel<<<dim3((unsigned)ceil_div(ceil_div(maxW, 16), threads), (unsigned)maxH, (unsigned)b.n), threads, 0,
                       s>>>(b, threshold);
    return cudaGetLastError();
}

}  // namespace rtk
