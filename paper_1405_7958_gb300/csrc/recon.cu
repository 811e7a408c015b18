// ReconToNuclei (Section 5.1 of the Region Templates paper): grayscale
// morphological reconstruction by dilation,
//     R = lim R_k,  R_0 = min(J, I),  R_{k+1} = min(delta(R_k), I),
// computed by tile-resident directional sweeps.
//
// Every update has the form R(p) <- min(I(p), max(R(p), R(q))) for a
// neighbour q, so the running image never exceeds the reconstruction and
// only grows; any schedule of such updates that stops at a fixed point of
// the 8- (or 4-) neighbourhood ends exactly at the reconstruction. The
// schedule here:
//   * the image is cut into 64 x 128 tiles; one warp owns one tile and stages
//     it in shared memory with a one-pixel halo read from the current image;
//   * per visit the warp runs a down and an up sweep (row by row, each row
//     taking the maximum of the three pixels above / below it) and a
//     left-to-right and right-to-left sweep (pixel by pixel along every
//     row), then writes the tile back;
//   * a persistent cooperative kernel repeats rounds of visits separated by
//     a grid barrier; a tile is visited again only when it changed or a
//     neighbour changed the pixels of its halo, and the kernel stops after
//     the first round without any change.
// The paper implements this operation as an irregular wavefront propagation
// over active elements; here the active elements are whole tiles.
#include "recon.cuh"

namespace rtk {

constexpr int kTH = 64;                  // tile height
constexpr int kWarpsPerCta = 4;
constexpr int kWarpWords = (kTH + 2) * kRStride + kTH * kRStride + 2 * (kTH + 2);

int sweep_tile_rows() { return kTH; }
size_t sweep_smem_bytes() { return sizeof(uint32_t) * kWarpWords * kWarpsPerCta; }

// ---------------------------------------------------------------- init
// Iw = mask (0 in the padding), Rw = min(J, I). One thread per 4 pixels.
__global__ void recon_init_kernel(const ReconBatch b, int32_t *err)
{
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

cudaError_t launch_recon_init(const ReconBatch &b, int32_t *err, cudaStream_t s)
{
    const int threads = 256;
    int64_t blocks = ceil_div(b.max_words, threads);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    recon_init_kernel<<<dim3((unsigned)blocks, (unsigned)b.n), threads, 0, s>>>(b, err);
    return cudaGetLastError();
}

void plan_recon_image(ReconImage &d, int H, int W)
{
    d.H = H;
    d.W = W;
    d.Hp = (int)round_up(H, kTH);
    d.Wp = (int)round_up(W, kRTW);
    d.tiles_x = d.Wp / kRTW;
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
__device__ __forceinline__ uint32_t vmax4(uint32_t a, uint32_t b) { return __vmaxu4(a, b); }
__device__ __forceinline__ uint32_t vmin4(uint32_t a, uint32_t b) { return __vminu4(a, b); }

// Per-warp shared-memory layout (32-bit words):
//   sR[(kTH + 2) * kRStride]: rows 0..kTH+1 = image rows r0-1 .. r0+kTH;
//                              word j of a row = columns c0+4j .. c0+4j+3
//   sI[kTH * kRStride]      : mask rows r0 .. r0+kTH-1
//   sHL[kTH + 2], sHR[kTH + 2]: halo columns c0-1 and c0+128 (low byte)
struct WarpTile {
    uint32_t *sR, *sI, *sHL, *sHR;
};

// Down (dir = +1) or up (dir = -1) sweep: each row takes the maximum of its
// own value and the (conn = 8: three, conn = 4: one) pixels of the row just
// processed, capped by the mask. Returns true if a pixel changed.
template <int CONN, int DIR>
__device__ __forceinline__ bool sweep_vertical(const WarpTile &t, int lane)
{
    const int first = DIR > 0 ? 0 : kTH + 1;
    uint32_t prev = t.sR[first * kRStride + lane];
    uint32_t prevL = 0, prevR = 0;
    if (CONN == 8) {
        prevL = lane == 0 ? (t.sHL[first] << 24) : t.sR[first * kRStride + lane - 1];
        prevR = lane == 31 ? t.sHR[first] : t.sR[first * kRStride + lane + 1];
    }
    bool ch = false;
#pragma unroll 4
    for (int k = 1; k <= kTH; ++k) {
        const int i = DIR > 0 ? k : kTH + 1 - k;
        uint32_t up = prev;
        if (CONN == 8) {
            const uint32_t left = __byte_perm(prevL, prev, 0x6543);
            const uint32_t right = __byte_perm(prev, prevR, 0x4321);
            up = vmax4(prev, vmax4(left, right));
        }
        const uint32_t cur = t.sR[i * kRStride + lane];
        const uint32_t nw = vmin4(vmax4(cur, up), t.sI[(i - 1) * kRStride + lane]);
        if (nw != cur) {
            t.sR[i * kRStride + lane] = nw;
            ch = true;
        }
        prev = nw;
        if (CONN == 8) {
            prevL = __shfl_up_sync(0xffffffffu, nw, 1);
            prevR = __shfl_down_sync(0xffffffffu, nw, 1);
            if (lane == 0) prevL = t.sHL[i] << 24;
            if (lane == 31) prevR = t.sHR[i];
        }
    }
    return ch;
}

// Left-to-right (DIR = +1) or right-to-left (DIR = -1) sweep along every
// row: lane = row. Inside a word the carried value is pushed through the
// four bytes by four shift-max-min steps (byte k is exact after step k+1).
template <int DIR>
__device__ __forceinline__ bool sweep_horizontal(const WarpTile &t, int lane)
{
    bool ch = false;
#pragma unroll 1
    for (int g = 0; g < kTH / 32; ++g) {
        const int i = 1 + lane + 32 * g;       // sR row
        uint32_t x = DIR > 0 ? t.sHL[i] : t.sHR[i];
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const int j = DIR > 0 ? k : 31 - k;
            const uint32_t w0 = t.sR[i * kRStride + j];
            const uint32_t iw = t.sI[(i - 1) * kRStride + j];
            uint32_t w = w0;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const uint32_t sh = DIR > 0 ? ((w << 8) | x) : ((w >> 8) | (x << 24));
                w = vmin4(vmax4(w, sh), iw);
            }
            x = DIR > 0 ? (w >> 24) : (w & 0xffu);
            if (w != w0) {
                t.sR[i * kRStride + j] = w;
                ch = true;
            }
        }
    }
    return ch;
}

template <int CONN>
__device__ void visit_tile(const SweepParams &p, int t, const WarpTile &wt, int lane, uint8_t *next_active,
                           uint32_t *counter)
{
    int k = 0;
    while (k + 1 < p.b.n && t >= p.b.img[k + 1].tile_base) ++k;
    const ReconImage &d = p.b.img[k];
    const int lt = t - d.tile_base;
    const int ty = lt / d.tiles_x, tx = lt % d.tiles_x;
    const int r0 = ty * kTH, c0 = tx * kRTW;
    const int Wp = d.Wp, Hp = d.Hp;

    // stage rows r0-1 .. r0+kTH of R, and the mask
#pragma unroll 4
    for (int i = 0; i < kTH + 2; ++i) {
        const int r = r0 - 1 + i;
        uint32_t w = 0;
        if (r >= 0 && r < Hp) w = __ldcg(reinterpret_cast<const uint32_t *>(d.Rw + (int64_t)r * Wp + c0) + lane);
        wt.sR[i * kRStride + lane] = w;
    }
#pragma unroll 4
    for (int i = 0; i < kTH; ++i)
        wt.sI[i * kRStride + lane] =
            __ldg(reinterpret_cast<const uint32_t *>(d.Iw + (int64_t)(r0 + i) * Wp + c0) + lane);
    for (int i = lane; i < kTH + 2; i += 32) {
        const int r = r0 - 1 + i;
        uint32_t hl = 0, hr = 0;
        if (r >= 0 && r < Hp) {
            if (c0 > 0) hl = __ldcg(d.Rw + (int64_t)r * Wp + c0 - 1);
            if (c0 + kRTW < Wp) hr = __ldcg(d.Rw + (int64_t)r * Wp + c0 + kRTW);
        }
        wt.sHL[i] = hl;
        wt.sHR[i] = hr;
    }
    __syncwarp();
    const uint32_t top0 = wt.sR[1 * kRStride + lane];
    const uint32_t bot0 = wt.sR[kTH * kRStride + lane];
    uint32_t left0[kTH / 32], right0[kTH / 32];
#pragma unroll
    for (int g = 0; g < kTH / 32; ++g) {
        left0[g] = wt.sR[(1 + lane + 32 * g) * kRStride + 0] & 0xffu;
        right0[g] = wt.sR[(1 + lane + 32 * g) * kRStride + 31] >> 24;
    }

    bool ch = sweep_vertical<CONN, +1>(wt, lane);
    __syncwarp();
    ch |= sweep_vertical<CONN, -1>(wt, lane);
    __syncwarp();
    ch |= sweep_horizontal<+1>(wt, lane);
    __syncwarp();
    ch |= sweep_horizontal<-1>(wt, lane);
    __syncwarp();

    if (!__any_sync(0xffffffffu, ch)) return;

    // write back and work out which neighbours see a changed halo
    const uint32_t top1 = wt.sR[1 * kRStride + lane];
    const uint32_t bot1 = wt.sR[kTH * kRStride + lane];
#pragma unroll 4
    for (int i = 1; i <= kTH; ++i)
        __stcg(reinterpret_cast<uint32_t *>(d.Rw + (int64_t)(r0 + i - 1) * Wp + c0) + lane,
               wt.sR[i * kRStride + lane]);
    bool lch = false, rch = false;
#pragma unroll
    for (int g = 0; g < kTH / 32; ++g) {
        lch |= (wt.sR[(1 + lane + 32 * g) * kRStride + 0] & 0xffu) != left0[g];
        rch |= (wt.sR[(1 + lane + 32 * g) * kRStride + 31] >> 24) != right0[g];
    }
    const bool top = __any_sync(0xffffffffu, top1 != top0);
    const bool bot = __any_sync(0xffffffffu, bot1 != bot0);
    const bool left = __any_sync(0xffffffffu, lch);
    const bool right = __any_sync(0xffffffffu, rch);
    const bool tl = __shfl_sync(0xffffffffu, (top1 ^ top0) & 0xffu, 0) != 0;
    const bool tr = __shfl_sync(0xffffffffu, (top1 ^ top0) >> 24, 31) != 0;
    const bool bl = __shfl_sync(0xffffffffu, (bot1 ^ bot0) & 0xffu, 0) != 0;
    const bool br = __shfl_sync(0xffffffffu, (bot1 ^ bot0) >> 24, 31) != 0;
    if (lane == 0) {
        uint8_t *na = next_active + d.tile_base;
        const int nx = d.tiles_x, ny = d.tiles_y;
        na[lt] = 1;   // not yet at a local fixed point: visit again
        if (top && ty > 0) na[lt - nx] = 1;
        if (bot && ty + 1 < ny) na[lt + nx] = 1;
        if (left && tx > 0) na[lt - 1] = 1;
        if (right && tx + 1 < nx) na[lt + 1] = 1;
        if (CONN == 8) {
            if (tl && ty > 0 && tx > 0) na[lt - nx - 1] = 1;
            if (tr && ty > 0 && tx + 1 < nx) na[lt - nx + 1] = 1;
            if (bl && ty + 1 < ny && tx > 0) na[lt + nx - 1] = 1;
            if (br && ty + 1 < ny && tx + 1 < nx) na[lt + nx + 1] = 1;
        }
        atomicAdd(counter, 1u);
    }
}

template <int CONN>
__global__ void __launch_bounds__(kWarpsPerCta * 32) recon_sweep_kernel(SweepParams p)
{
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile wt;
    wt.sR = smem + warp * kWarpWords;
    wt.sI = wt.sR + (kTH + 2) * kRStride;
    wt.sHL = wt.sI + kTH * kRStride;
    wt.sHR = wt.sHL + (kTH + 2);
    const int gw = blockIdx.x * kWarpsPerCta + warp;
    const int nw = gridDim.x * kWarpsPerCta;
    int round = 0;
    for (; round < p.max_rounds; ++round) {
        uint8_t *act = p.active + (size_t)(round & 1) * p.ntiles;
        uint8_t *nxt = p.active + (size_t)((round + 1) & 1) * p.ntiles;
        uint32_t *cnt = p.counters + (round % 3);
        for (int t = gw; t < p.ntiles; t += nw) {
            if (!__ldcg(act + t)) continue;
            if (lane == 0) act[t] = 0;
            visit_tile<CONN>(p, t, wt, lane, nxt, cnt);
        }
        if (!grid_barrier(p.bar, gridDim.x, p.err, p.timeout_ns)) return;
        const uint32_t changed = ld_acquire(cnt);
        if (blockIdx.x == 0 && threadIdx.x == 0) p.counters[(round + 2) % 3] = 0;
        if (changed == 0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (p.rounds_out) *p.rounds_out = round + 1;
        if (round >= p.max_rounds) raise_status(p.err, RT_ETIMEOUT);
    }
}

cudaError_t launch_recon_sweep(const SweepParams &p, int conn, int num_sms, cudaStream_t s,
                               int *grid_used)
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
