// FillHoles (Sections 3.2.1 and 5.1): the holes of a binary image are the
// background pixels that no background path connects to the image border.
// The paper computes them by morphological reconstruction: the background
// reached from the border is the reconstruction by dilation of the border
// background under the background mask, and the filled image is its
// complement. Here that binary reconstruction runs on bit planes, 32 pixels
// per word:
//   * pack: background mask m, and the seed x = m on the image border;
//   * propagate: warp tiles of 32 rows x 1024 columns (lane = word column,
//     one register per row) are swept down and up. A row takes what the row
//     before it reached (4-connectivity: the same column; 8-connectivity:
//     that row widened by one pixel), then is flooded along its runs of
//     background in both directions. The flood is an addition: adding the
//     seeds to the mask turns every mask bit from a seed to the end of its
//     run, so ((m + s) ^ m) & m | s is the rightward flood, and the carry
//     crosses words like in a 1024-bit addition (carries resolved from two
//     ballots, generate and propagate). The leftward flood is the same on
//     the bit-reversed row. Tiles that see a changed halo are flagged and
//     revisited, with the same pending count and termination as the grayscale
//     propagation;
//   * output: F = 1 for foreground pixels and for background not reached.
// The result is the unique fixed point, so it does not depend on the order
// of the visits.
#include "fill.cuh"

namespace rtk {

namespace {

constexpr int kFillWarps = 4;          // warps per CTA of the propagation
constexpr int kFillMaxPasses = 16;     // sweeps per visit before it is revisited

size_t plane_words(int H, int W)
{
    const int64_t ny = ceil_div(H, kFillTH), nx = ceil_div(W, kFillTW);
    return (size_t)(ny * kFillTH) * (size_t)(nx * 32);
}

}  // namespace

size_t fill_image_bytes(int H, int W) { return 2 * (size_t)round_up((int64_t)plane_words(H, W) * 4, 256); }

void fill_add(FillBatch &b, const uint8_t *in, int64_t ld_in, uint8_t *out, int64_t ld_out, int H, int W,
              char *base)
{
    if (b.n == 0) {
        b.ntiles = 0;
        b.maxW = b.maxH = b.maxHp = b.maxWq = 0;
    }
    FillImage &d = b.img[b.n++];
    d.in = in;
    d.ld_in = ld_in;
    d.out = out;
    d.ld_out = ld_out;
    d.H = H;
    d.W = W;
    d.ny = (int)ceil_div(H, kFillTH);
    d.nx = (int)ceil_div(W, kFillTW);
    d.wq = d.nx * 32;
    d.tile_base = b.ntiles;
    b.ntiles += d.ny * d.nx;
    const size_t pb = (size_t)round_up((int64_t)plane_words(H, W) * 4, 256);
    d.m = reinterpret_cast<uint32_t *>(base);
    d.x = reinterpret_cast<uint32_t *>(base + pb);
    b.maxW = W > b.maxW ? W : b.maxW;
    b.maxH = H > b.maxH ? H : b.maxH;
    b.maxHp = d.ny * kFillTH > b.maxHp ? d.ny * kFillTH : b.maxHp;
    b.maxWq = d.wq > b.maxWq ? d.wq : b.maxWq;
}

// ------------------------------------------------------------------- pack
// Thread per bit-plane word (32 columns of one row); blockIdx.z = image.
__global__ void fill_pack_kernel(FillBatch b)
{
    const FillImage &a = b.img[blockIdx.z];
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (r == 0) {
        const int nt = a.ny * a.nx;
        for (int t = w; t < nt; t += gridDim.x * blockDim.x) b.flags[a.tile_base + t] = 1u;
        if (w == 0 && blockIdx.z == 0) *b.pending = (uint32_t)b.ntiles;
    }
    if (w >= a.wq || r >= a.ny * kFillTH) return;
    const int c0 = w * 32;
    uint32_t m = 0;
    if (r < a.H && c0 < a.W) {
        const uint8_t *p = a.in + (int64_t)r * a.ld_in + c0;
        const int n = min(32, a.W - c0);
        if (n == 32 && (((uintptr_t)p) & 15u) == 0) {
            const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(p));
            const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
            const uint32_t v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) m |= (uint32_t)(((v[q] >> (8 * k)) & 0xffu) == 0u) << (4 * q + k);
        } else {
            for (int k = 0; k < n; ++k) m |= (uint32_t)(p[k] == 0) << k;
        }
    }
    // seeds: the background on the image border
    uint32_t x = 0;
    if (r == 0 || r == a.H - 1) {
        x = m;
    } else {
        if (c0 == 0) x |= m & 1u;
        const int cl = a.W - 1 - c0;
        if (cl >= 0 && cl < 32) x |= m & (1u << cl);
    }
    a.m[(int64_t)r * a.wq + w] = m;
    a.x[(int64_t)r * a.wq + w] = x;
}

// -------------------------------------------------------------- propagate
// Rightward flood of the seeds s (a subset of m) along the runs of m over
// the warp's 1024-bit row (bit k of lane l = column 32 l + k).
__device__ __forceinline__ uint32_t flood_up(uint32_t m, uint32_t s, int lane)
{
    const uint32_t a = m + s;
    const uint32_t G = __ballot_sync(0xffffffffu, a < m);              // carries out on its own
    const uint32_t P = __ballot_sync(0xffffffffu, a == 0xffffffffu);   // passes a carry through
    // carry into lane i = bit i of (G + (G | P)) ^ P (the carry chain of that sum)
    const uint32_t cin = (((G + (G | P)) ^ P) >> lane) & 1u;
    return (((a + cin) ^ m) & m) | s;
}

// Both directions: the leftward flood is the rightward one on the reversed row.
__device__ __forceinline__ uint32_t flood_row(uint32_t m, uint32_t s, int lane)
{
    const uint32_t right = flood_up(m, s, lane);
    const uint32_t mr = __brev(__shfl_sync(0xffffffffu, m, 31 - lane));
    const uint32_t sr = __brev(__shfl_sync(0xffffffffu, s, 31 - lane));
    const uint32_t left = __shfl_sync(0xffffffffu, __brev(flood_up(mr, sr, lane)), 31 - lane);
    return right | left;
}

// Flags tile t. `pending` is raised first (the returned count is checked,
// which makes the increment complete before the flag is set) and lowered
// again if the tile was already flagged, so it never undercounts.
__device__ __forceinline__ void fill_mark(const FillBatch &b, int t)
{
    if (atomicAdd(b.pending, 1u) == 0xffffffffu) {
        raise_status(b.err, RT_ETIMEOUT);
        return;
    }
    if (atomicOr(b.flags + t, 1u) != 0u) atomicSub(b.pending, 1u);
}

// One visit of batch tile tg by a warp.
template <int CONN>
__device__ __forceinline__ void fill_visit(const FillBatch &b, int tg, int lane)
{
    int k = 0;
    while (k + 1 < b.n && tg >= b.img[k + 1].tile_base) ++k;
    const FillImage &a = b.img[k];
    const int t = tg - a.tile_base;
    const int ty = t % a.ny, tx = t / a.ny;
    const int r0 = ty * kFillTH, w = tx * 32 + lane;
    const int hp = a.ny * kFillTH;
    const int64_t wq = a.wq;
    uint32_t m[kFillTH], x[kFillTH];
#pragma unroll
    for (int r = 0; r < kFillTH; ++r) {
        m[r] = __ldg(a.m + (r0 + r) * wq + w);
        x[r] = __ldcg(a.x + (r0 + r) * wq + w);
    }
    const uint32_t top = r0 > 0 ? __ldcg(a.x + (r0 - 1) * wq + w) : 0u;
    const uint32_t bot = r0 + kFillTH < hp ? __ldcg(a.x + (r0 + kFillTH) * wq + w) : 0u;
    // side halos as row bit masks: bit i = row r0 + i; plus the corner rows
    uint32_t hl = 0, hr = 0;
    if (tx > 0) hl = __ballot_sync(0xffffffffu, (__ldcg(a.x + (r0 + lane) * wq + tx * 32 - 1) >> 31) & 1u);
    if (tx + 1 < a.nx) hr = __ballot_sync(0xffffffffu, __ldcg(a.x + (r0 + lane) * wq + tx * 32 + 32) & 1u);
    uint32_t hl_top = 0, hl_bot = 0, hr_top = 0, hr_bot = 0;
    if (CONN == 8) {
        if (tx > 0 && r0 > 0) hl_top = __ldcg(a.x + (r0 - 1) * wq + tx * 32 - 1) >> 31;
        if (tx > 0 && r0 + kFillTH < hp) hl_bot = __ldcg(a.x + (r0 + kFillTH) * wq + tx * 32 - 1) >> 31;
        if (tx + 1 < a.nx && r0 > 0) hr_top = __ldcg(a.x + (r0 - 1) * wq + tx * 32 + 32) & 1u;
        if (tx + 1 < a.nx && r0 + kFillTH < hp) hr_bot = __ldcg(a.x + (r0 + kFillTH) * wq + tx * 32 + 32) & 1u;
    }
    // seed a row: from the row before it (prev, whose side halo bits are
    // pl / pr), and from its own side halo pixels
    auto step = [&](uint32_t mr_, uint32_t xr, uint32_t prev, uint32_t pl, uint32_t pr, uint32_t sl, uint32_t sr) {
        uint32_t v = prev;
        if (CONN == 8) {
            uint32_t lo = __shfl_up_sync(0xffffffffu, prev, 1) >> 31;
            uint32_t hi = __shfl_down_sync(0xffffffffu, prev, 1) & 1u;
            lo = lane == 0 ? pl : lo;
            hi = lane == 31 ? pr : hi;
            v |= (prev << 1) | lo | (prev >> 1) | (hi << 31);
        }
        uint32_t s = xr | (mr_ & v);
        s |= mr_ & ((lane == 0 ? sl : 0u) | (lane == 31 ? sr << 31 : 0u));
        return flood_row(mr_, s, lane);
    };
    uint32_t diff = 0;
    int pass = 0;
    bool converged = false;
    for (; pass < kFillMaxPasses; ++pass) {
        uint32_t ch = 0;
        if ((pass & 1) == 0) {
            uint32_t prev = top, pl = hl_top, pr = hr_top;
#pragma unroll
            for (int r = 0; r < kFillTH; ++r) {
                const uint32_t nv = step(m[r], x[r], prev, pl, pr, (hl >> r) & 1u, (hr >> r) & 1u);
                ch |= nv ^ x[r];
                x[r] = nv;
                prev = nv;
                pl = (hl >> r) & 1u;
                pr = (hr >> r) & 1u;
            }
        } else {
            uint32_t prev = bot, pl = hl_bot, pr = hr_bot;
#pragma unroll
            for (int r = kFillTH - 1; r >= 0; --r) {
                const uint32_t nv = step(m[r], x[r], prev, pl, pr, (hl >> r) & 1u, (hr >> r) & 1u);
                ch |= nv ^ x[r];
                x[r] = nv;
                prev = nv;
                pl = (hl >> r) & 1u;
                pr = (hr >> r) & 1u;
            }
        }
        diff |= ch;
        // both sweeps are idempotent: a clean sweep after at least one other
        // leaves both clean
        if (!__any_sync(0xffffffffu, ch != 0) && pass > 0) {
            converged = true;
            break;
        }
    }
    if (!__any_sync(0xffffffffu, diff != 0) && converged) return;
    // write back and find the borders that moved
    uint32_t dtop = 0, dbot = 0, dl = 0, dr = 0;
#pragma unroll
    for (int r = 0; r < kFillTH; ++r) {
        uint32_t *p = a.x + (r0 + r) * wq + w;
        const uint32_t d = __ldcg(p) ^ x[r];
        if (d) __stcg(p, x[r]);
        if (r == 0) dtop = d;
        if (r == kFillTH - 1) dbot = d;
        dl |= (d & 1u) << r;
        dr |= (d >> 31) << r;
    }
    const bool top_ch = __any_sync(0xffffffffu, dtop != 0);
    const bool bot_ch = __any_sync(0xffffffffu, dbot != 0);
    const uint32_t left_ch = __shfl_sync(0xffffffffu, dl, 0);
    const uint32_t right_ch = __shfl_sync(0xffffffffu, dr, 31);
    __threadfence();
    if (lane == 0) {
        const int ny = a.ny;
        if (!converged) fill_mark(b, tg);
        if (top_ch && ty > 0) fill_mark(b, tg - 1);
        if (bot_ch && ty + 1 < ny) fill_mark(b, tg + 1);
        if (left_ch && tx > 0) fill_mark(b, tg - ny);
        if (right_ch && tx + 1 < a.nx) fill_mark(b, tg + ny);
        if (CONN == 8) {
            if ((left_ch & 1u) && tx > 0 && ty > 0) fill_mark(b, tg - ny - 1);
            if ((left_ch >> 31) && tx > 0 && ty + 1 < ny) fill_mark(b, tg - ny + 1);
            if ((right_ch & 1u) && tx + 1 < a.nx && ty > 0) fill_mark(b, tg + ny - 1);
            if ((right_ch >> 31) && tx + 1 < a.nx && ty + 1 < ny) fill_mark(b, tg + ny + 1);
        }
    }
}

// Persistent propagation: warp w owns a contiguous run of tiles (column by
// column) and visits those flagged until nothing is flagged or being
// visited. Cooperative launch only to make every owner resident.
template <int CONN>
__global__ void __launch_bounds__(kFillWarps * 32, 4) fill_prop_kernel(FillBatch a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = a.ntiles;
    const int gw = blockIdx.x * kFillWarps + warp, nw = gridDim.x * kFillWarps;
    const int chunk = (ntiles + nw - 1) / nw;
    const int own0 = gw * chunk, own1 = min(ntiles, own0 + chunk);
    const uint64_t t_start = globaltimer_ns();
    int idle = 0;
    for (;;) {
        bool did = false;
        for (int base = own0; base < own1; base += 32) {
            const int tl = base + lane;
            const bool f = tl < own1 && *reinterpret_cast<volatile uint32_t *>(a.flags + tl) != 0u;
            uint32_t mask = __ballot_sync(0xffffffffu, f);
            while (mask) {
                const int i = __ffs(mask) - 1;
                mask &= mask - 1;
                const int t = base + i;
                uint32_t got = 0;
                if (lane == 0) got = atomicExch(a.flags + t, 0u);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) continue;
                __threadfence();
                fill_visit<CONN>(a, t, lane);
                if (lane == 0) atomicSub(a.pending, 1u);
                did = true;
            }
        }
        if (did) {
            idle = 0;
            continue;
        }
        uint32_t pend = 0;
        if (lane == 0) pend = ld_acquire(a.pending);
        pend = __shfl_sync(0xffffffffu, pend, 0);
        if (pend == 0) break;
        if (++idle > 4) __nanosleep(500);
        int late = 0;
        if (lane == 0 && (idle & 63) == 0) late = globaltimer_ns() - t_start > a.timeout_ns;
        if (__shfl_sync(0xffffffffu, late, 0)) {
            if (lane == 0) raise_status(a.err, RT_ETIMEOUT);
            break;
        }
    }
}

// ------------------------------------------------------------------ output
// 16 columns per thread: F = 1 unless the pixel is background reached from
// the border; blockIdx.z = image.
__global__ void fill_out_kernel(FillBatch b)
{
    const FillImage &a = b.img[blockIdx.z];
    const int r = blockIdx.y;
    const int c0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16;
    if (c0 >= a.W || r >= a.H) return;
    const int n = min(16, a.W - c0);
    const uint32_t xw = __ldcs(a.x + (int64_t)r * a.wq + c0 / 32) >> (c0 & 31);
    const uint8_t *ip = a.in + (int64_t)r * a.ld_in + c0;
    uint8_t *op = a.out + (int64_t)r * a.ld_out + c0;
    if (n == 16 && ((((uintptr_t)ip) | ((uintptr_t)op)) & 15u) == 0) {
        const uint4 v = *reinterpret_cast<const uint4 *>(ip);
        const uint32_t iv[4] = {v.x, v.y, v.z, v.w};
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t wv = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool fg = ((iv[q] >> (8 * k)) & 0xffu) != 0u;
                const bool reached = (xw >> (4 * q + k)) & 1u;
                wv |= (uint32_t)(fg || !reached) << (8 * k);
            }
            o[q] = wv;
        }
        *reinterpret_cast<uint4 *>(op) = make_uint4(o[0], o[1], o[2], o[3]);
    } else {
        uint8_t o[16];
        for (int k = 0; k < n; ++k) o[k] = (uint8_t)(ip[k] != 0 || !((xw >> k) & 1u));
        for (int k = 0; k < n; ++k) op[k] = o[k];
    }
}

cudaError_t launch_fill(const FillBatch &b, int num_sms, cudaStream_t s)
{
    if ((b.conn != 4 && b.conn != 8) || b.n < 1 || b.n > kFillMaxImgs) return cudaErrorInvalidValue;
    const int threads = 128;
    fill_pack_kernel<<<dim3((unsigned)ceil_div(b.maxWq, threads), (unsigned)b.maxHp, (unsigned)b.n), threads, 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const void *fn = b.conn == 8 ? (const void *)fill_prop_kernel<8> : (const void *)fill_prop_kernel<4>;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFillWarps * 32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = per_sm * num_sms;
    const int need = (int)ceil_div(b.ntiles, kFillWarps);
    if (grid > need) grid = need;
    FillBatch bb = b;
    void *args[] = {&bb};
    e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kFillWarps * 32), args, 0, s);
    if (e != cudaSuccess) return e;
    fill_out_kernel<<<dim3((unsigned)ceil_div(ceil_div(b.maxW, 16), threads), (unsigned)b.maxH, (unsigned)b.n), threads,
                      0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace rtk
