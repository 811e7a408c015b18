// ReconToNuclei (Section 5.1 of the Region Templates paper): grayscale
// morphological reconstruction by dilation,
//     R = lim R_k,  R_0 = min(J, I),  R_{k+1} = min(delta(R_k), I).
//
// Every update here has the form R(p) <- min(I(p), max(R(p), R(q))) for a
// neighbour q, so the running image never exceeds the reconstruction and
// only grows; any schedule of such updates that stops at a fixed point of
// the 8- (or 4-) neighbourhood ends exactly at the reconstruction. The paper
// runs the operation as an irregular wavefront propagation over active
// elements; here the active elements are 32 x 64 tiles:
//   * a warp visits a tile by loading it into registers as packed 16-bit
//     pairs (lane = two columns, one register per row for R and for I),
//     with a one-pixel halo from the current image;
//   * it sweeps the tile until nothing changes: a down and an up sweep (each
//     row takes the maximum of itself and the neighbouring pixels of the row
//     just done), then a left-to-right and a right-to-left sweep along every
//     row (rows transposed through shared memory so each lane walks one row);
//   * it writes the tile back and flags the neighbouring tiles whose halo
//     changed. A persistent kernel keeps visiting flagged tiles until no tile
//     is flagged or being visited; there is no grid-wide barrier.
#include "recon.cuh"

namespace rtk {

constexpr int kWarpsPerCta = 4;
constexpr int kTS = 33;                                  // transposed row stride (words)
constexpr int kWarpWords = 2 * kTH * kTS + 2 * (kTH + 2);

size_t sweep_smem_bytes() { return sizeof(uint32_t) * kWarpWords * kWarpsPerCta; }

// ---------------------------------------------------------------- init
// Iw = mask (0 in the padding), Rw = min(J, I). One thread per 4 pixels.
__global__ void recon_init_kernel(const ReconBatch b, uint32_t *flags, uint32_t *pending, int32_t *err)
{
    if (blockIdx.y == 0) {
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < b.ntiles; t += gridDim.x * blockDim.x) flags[t] = 1u;
        if (blockIdx.x == 0 && threadIdx.x == 0) *pending = (uint32_t)b.ntiles;
    }
    const ReconImage &d = b.img[blockIdx.y];
    const int64_t wpr = d.Wp / 4;
    const int64_t nwords = (int64_t)d.Hp * wpr;
    bool bad = false;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(w / wpr);
        const int c0 = (int)(w % wpr) * 4;
        uint32_t iw = 0, rw = 0;
        if (r < d.H) {
            const bool border_row = (r == 0 || r == d.H - 1);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = c0 + b;
                if (c < d.W) {
                    const int iv = d.mask[(int64_t)r * d.ld_mask + c];
                    int jv;
                    if (d.marker) {
                        jv = d.marker[(int64_t)r * d.ld_marker + c];
                    } else {
                        jv = (border_row || c == 0 || c == d.W - 1) ? iv : max(iv - d.h_offset, 0);
                    }
                    if (jv > iv) bad = true;
                    iw |= (uint32_t)iv << (8 * b);
                    rw |= (uint32_t)min(jv, iv) << (8 * b);
                }
            }
        }
        reinterpret_cast<uint32_t *>(d.Iw)[w] = iw;
        reinterpret_cast<uint32_t *>(d.Rw)[w] = rw;
    }
    if (bad) raise_status(err, RT_EMARKER);
}

cudaError_t launch_recon_init(const ReconBatch &b, uint32_t *flags, uint32_t *pending, int32_t *err,
                              cudaStream_t s)
{
    const int threads = 256;
    int64_t blocks = ceil_div(b.max_words, threads);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    recon_init_kernel<<<dim3((unsigned)blocks, (unsigned)b.n), threads, 0, s>>>(b, flags, pending, err);
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

__device__ __forceinline__ void mark_tile(uint32_t *flags, uint32_t *pending, int t)
{
    if (atomicExch(flags + t, 1u) == 0u) atomicAdd(pending, 1u);
}

struct WarpBuf {
    uint32_t *sRT, *sIT;   // kTH rows x kTS words: transposed R, I (u16x2 per word)
    uint32_t *sHL, *sHR;   // halo columns, index i <-> tile row i - 1
};

// One visit of tile t by a warp. Returns after marking the tiles to visit.
template <int CONN>
__device__ __forceinline__ uint32_t visit_tile(const SweepParams &p, int t, const WarpBuf &wb, int lane)
{
    int k = 0;
    while (k + 1 < p.b.n && t >= p.b.img[k + 1].tile_base) ++k;
    const ReconImage &d = p.b.img[k];
    const int lt = t - d.tile_base;
    const int ty = lt / d.tiles_x, tx = lt % d.tiles_x;
    const int r0 = ty * kTH, c0 = tx * kTW;
    const int64_t Wp = d.Wp;
    const uint16_t *Rg = reinterpret_cast<const uint16_t *>(d.Rw + (int64_t)r0 * Wp + c0) + lane;
    const uint16_t *Ig = reinterpret_cast<const uint16_t *>(d.Iw + (int64_t)r0 * Wp + c0) + lane;
    const int64_t ws = Wp / 2;   // row stride in 16-bit units

    uint32_t R[kTH], I[kTH];
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
        R[r] = widen2(__ldcg(Rg + r * ws));
        I[r] = widen2(__ldg(Ig + r * ws));
        wb.sIT[r * kTS + lane] = I[r];
    }
    const uint32_t topw = r0 > 0 ? widen2(__ldcg(Rg - ws)) : 0u;
    const uint32_t botw = r0 + kTH < d.Hp ? widen2(__ldcg(Rg + kTH * ws)) : 0u;
    for (int i = lane; i < kTH + 2; i += 32) {
        const int r = r0 - 1 + i;
        uint32_t hl = 0, hr = 0;
        if (r >= 0 && r < d.Hp) {
            if (c0 > 0) hl = __ldcg(d.Rw + (int64_t)r * Wp + c0 - 1);
            if (c0 + kTW < Wp) hr = __ldcg(d.Rw + (int64_t)r * Wp + c0 + kTW);
        }
        wb.sHL[i] = hl;
        wb.sHR[i] = hr;
    }
    __syncwarp();

    bool converged = false;
    int it = 0;
    for (; it < p.max_local; ++it) {
        bool ch = false;
        // down sweep
        uint32_t prev = topw;
#pragma unroll
        for (int r = 0; r < kTH; ++r) {
            uint32_t m = vmax2(R[r], prev);
            if (CONN == 8) {
                uint32_t sl = __shfl_up_sync(0xffffffffu, prev, 1);
                uint32_t sr = __shfl_down_sync(0xffffffffu, prev, 1);
                if (lane == 0) sl = wb.sHL[r] << 16;
                if (lane == 31) sr = wb.sHR[r];
                m = vmax2(m, vmax2(__byte_perm(sl, prev, 0x5432), __byte_perm(prev, sr, 0x5432)));
            }
            const uint32_t nv = vmin2(m, I[r]);
            ch |= nv != R[r];
            R[r] = nv;
            prev = nv;
        }
        // up sweep
        prev = botw;
#pragma unroll
        for (int r = kTH - 1; r >= 0; --r) {
            uint32_t m = vmax2(R[r], prev);
            if (CONN == 8) {
                uint32_t sl = __shfl_up_sync(0xffffffffu, prev, 1);
                uint32_t sr = __shfl_down_sync(0xffffffffu, prev, 1);
                if (lane == 0) sl = wb.sHL[r + 2] << 16;
                if (lane == 31) sr = wb.sHR[r + 2];
                m = vmax2(m, vmax2(__byte_perm(sl, prev, 0x5432), __byte_perm(prev, sr, 0x5432)));
            }
            const uint32_t nv = vmin2(m, I[r]);
            ch |= nv != R[r];
            R[r] = nv;
            prev = nv;
        }
        // left-to-right and right-to-left along every row (lane = row)
#pragma unroll
        for (int r = 0; r < kTH; ++r) wb.sRT[r * kTS + lane] = R[r];
        __syncwarp();
        {
            uint32_t *row = wb.sRT + lane * kTS;
            const uint32_t *irow = wb.sIT + lane * kTS;
            uint32_t x = wb.sHL[lane + 1];
#pragma unroll 8
            for (int j = 0; j < kTW / 2; ++j) {
                const uint32_t w = row[j], iw = irow[j];
                const uint32_t a = min(max(w & 0xffffu, x), iw & 0xffffu);
                x = min(max(w >> 16, a), iw >> 16);
                const uint32_t nw = a | (x << 16);
                if (nw != w) {
                    row[j] = nw;
                    ch = true;
                }
            }
            x = wb.sHR[lane + 1];
#pragma unroll 8
            for (int j = kTW / 2 - 1; j >= 0; --j) {
                const uint32_t w = row[j], iw = irow[j];
                const uint32_t b = min(max(w >> 16, x), iw >> 16);
                x = min(max(w & 0xffffu, b), iw & 0xffffu);
                const uint32_t nw = x | (b << 16);
                if (nw != w) {
                    row[j] = nw;
                    ch = true;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kTH; ++r) R[r] = wb.sRT[r * kTS + lane];
        __syncwarp();
        if (!__any_sync(0xffffffffu, ch)) {
            converged = true;
            ++it;
            break;
        }
    }

    // write back, and find which borders moved
    uint16_t *Rs = reinterpret_cast<uint16_t *>(d.Rw + (int64_t)r0 * Wp + c0) + lane;
    uint32_t dl = 0, dr = 0, dtop = 0, dbot = 0, any = 0;
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
        const uint32_t orig = widen2(__ldcg(Rs + r * ws));
        const uint32_t diff = orig ^ R[r];
        if (diff) __stcg(Rs + r * ws, (uint16_t)narrow2(R[r]));
        dl |= diff & 0xffffu;
        dr |= diff >> 16;
        any |= diff;
        if (r == 0) dtop = diff;
        if (r == kTH - 1) dbot = diff;
    }
    if (!__any_sync(0xffffffffu, any != 0)) return (uint32_t)it;
    const bool top = __any_sync(0xffffffffu, dtop != 0);
    const bool bot = __any_sync(0xffffffffu, dbot != 0);
    const bool left = __shfl_sync(0xffffffffu, dl, 0) != 0;
    const bool right = __shfl_sync(0xffffffffu, dr, 31) != 0;
    const bool tl = __shfl_sync(0xffffffffu, dtop & 0xffffu, 0) != 0;
    const bool tr = __shfl_sync(0xffffffffu, dtop >> 16, 31) != 0;
    const bool bl = __shfl_sync(0xffffffffu, dbot & 0xffffu, 0) != 0;
    const bool br = __shfl_sync(0xffffffffu, dbot >> 16, 31) != 0;
    __threadfence();
    if (lane == 0) {
        const int nx = d.tiles_x, ny = d.tiles_y, base = d.tile_base;
        if (!converged) mark_tile(p.flags, p.pending, t);
        if (top && ty > 0) mark_tile(p.flags, p.pending, base + lt - nx);
        if (bot && ty + 1 < ny) mark_tile(p.flags, p.pending, base + lt + nx);
        if (left && tx > 0) mark_tile(p.flags, p.pending, base + lt - 1);
        if (right && tx + 1 < nx) mark_tile(p.flags, p.pending, base + lt + 1);
        if (CONN == 8) {
            if (tl && ty > 0 && tx > 0) mark_tile(p.flags, p.pending, base + lt - nx - 1);
            if (tr && ty > 0 && tx + 1 < nx) mark_tile(p.flags, p.pending, base + lt - nx + 1);
            if (bl && ty + 1 < ny && tx > 0) mark_tile(p.flags, p.pending, base + lt + nx - 1);
            if (br && ty + 1 < ny && tx + 1 < nx) mark_tile(p.flags, p.pending, base + lt + nx + 1);
        }
    }
    return (uint32_t)it;
}

// Persistent propagation. Warp w owns tiles w, w + nwarps, ...; it visits
// those flagged, and leaves when nothing is flagged or being visited
// anywhere. A visit is counted in `pending` from the moment its tile is
// flagged until after the visit has flagged its neighbours, so pending = 0
// means the image is at the fixed point. The launch is cooperative only to
// guarantee that every warp is resident (a flagged tile's owner always runs).
template <int CONN>
__global__ void __launch_bounds__(kWarpsPerCta * 32) recon_sweep_kernel(SweepParams p)
{
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpBuf wb;
    wb.sRT = smem + warp * kWarpWords;
    wb.sIT = wb.sRT + kTH * kTS;
    wb.sHL = wb.sIT + kTH * kTS;
    wb.sHR = wb.sHL + (kTH + 2);
    const int gw = blockIdx.x * kWarpsPerCta + warp;
    const int nw = gridDim.x * kWarpsPerCta;
    const uint64_t t_start = globaltimer_ns();
    uint32_t nvisits = 0, niters = 0;
    int idle = 0;
    for (;;) {
        bool did = false;
        // the warp's tiles, 32 flags per load
        for (int base = gw; base < p.ntiles; base += nw * 32) {
            const int tl = base + lane * nw;
            const bool f = tl < p.ntiles && *reinterpret_cast<volatile uint32_t *>(p.flags + tl) != 0u;
            uint32_t mask = __ballot_sync(0xffffffffu, f);
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                const int t = base + i * nw;
                uint32_t got = 0;
                if (lane == 0) got = atomicExch(p.flags + t, 0u);
                if (!__shfl_sync(0xffffffffu, got, 0)) continue;
                __threadfence();
                niters += visit_tile<CONN>(p, t, wb, lane);
                if (lane == 0) atomicSub(p.pending, 1u);
                did = true;
                ++nvisits;
            }
        }
        if (did) {
            idle = 0;
            continue;
        }
        uint32_t pend = 0;
        if (lane == 0) pend = ld_acquire(p.pending);
        pend = __shfl_sync(0xffffffffu, pend, 0);
        if (pend == 0) break;
        if (++idle > 4) __nanosleep(100);
        int late = 0;
        if (lane == 0 && (idle & 63) == 0) late = globaltimer_ns() - t_start > p.timeout_ns;
        if (__shfl_sync(0xffffffffu, late, 0)) {
            if (lane == 0) raise_status(p.err, RT_ETIMEOUT);
            break;
        }
    }
    if (lane == 0 && p.visits && nvisits) {
        atomicAdd(p.visits, nvisits);
        atomicAdd(p.visits + 1, niters);
    }
}

cudaError_t launch_recon_sweep(const SweepParams &p, int conn, int num_sms, cudaStream_t s, int *grid_used)
{
    const size_t smem = sweep_smem_bytes();
    const void *fn = conn == 8 ? (const void *)recon_sweep_kernel<8> : (const void *)recon_sweep_kernel<4>;
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

// --------------------------------------------------------------- output
// out = R (cropped to H x W); optionally bin = (R < threshold).
__global__ void recon_out_kernel(const uint8_t *Rw, int Wp, uint8_t *out, int64_t ld_out, int H, int W,
                                 uint8_t *bin, int64_t ld_bin, int threshold)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W; c += gridDim.x * blockDim.x) {
        const uint8_t v = Rw[(int64_t)r * Wp + c];
        if (out) out[(int64_t)r * ld_out + c] = v;
        if (bin) bin[(int64_t)r * ld_bin + c] = v < threshold ? 1 : 0;
    }
}

cudaError_t launch_recon_out(const uint8_t *Rw, int Wp, uint8_t *out, int64_t ld_out, int H, int W,
                             uint8_t *bin, int64_t ld_bin, int threshold, cudaStream_t s)
{
    recon_out_kernel<<<dim3((unsigned)ceil_div(W, 256), (unsigned)H), 256, 0, s>>>(Rw, Wp, out, ld_out, H, W,
                                                                                  bin, ld_bin, threshold);
    return cudaGetLastError();
}

}  // namespace rtk
