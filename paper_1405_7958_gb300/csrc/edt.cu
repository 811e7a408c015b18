// Exact squared Euclidean distance transform (input of the Pre-Watershed
// step, Section 5.1):
//     d2(p) = min over background q of (r_p - r_q)^2 + (c_p - c_q)^2.
// Separable form (the same decomposition as Meijster et al. 2000):
//     g(r, c)  = distance from (r, c) to the nearest background pixel of
//                column c (vertical pass),
//     d2(r, c) = min over c' of (c - c')^2 + g(r, c')^2 (horizontal pass).
// Vertical pass: columns are cut into 32-row segments; a first kernel
// records each segment's first and last background row, a second one walks
// every segment with the carries from the segments above and below.
// With a bit-plane input (the segmentation chain, a batch of images per
// launch) g is never stored: a first kernel turns each 32 x 32 block's row
// words into column masks (ballots), a second records for every segment and
// column the nearest background row above and below the segment, and the
// horizontal pass computes the g values of its row from those (bit scans of
// the column's mask) while staging them.
// Horizontal pass: a CTA per row stages g in shared memory. For pixel c the
// candidate c' = c gives g(r,c)^2, and any c' with |c - c'| >= sqrt(best)
// cannot win, so the search runs outward from c and stops as soon as
// (c - c')^2 reaches the best value found. The result is exact for any
// input; the work per pixel grows with its distance, which is small on
// nuclei masks.
#include "edt.cuh"

namespace rtk {

constexpr int kSeg = 32;
constexpr uint16_t kInf = 0xFFFFu;

size_t edt_workspace_bytes(int H, int W)
{
    const int64_t nseg = ceil_div(H, kSeg);
    return (size_t)H * W * sizeof(uint16_t) + (size_t)3 * nseg * W * sizeof(int32_t) + 512;
}

__device__ __forceinline__ bool edt_is_bg(const EdtArgs &a, int r, int c)
{
    if (a.lab32) return a.lab32[(int64_t)r * a.ld_in + c] < 0;
    return a.fg8[(int64_t)r * a.ld_in + c] == 0;
}

// thread per (column, segment): first / last background row in the segment
__global__ void edt_seg_kernel(EdtArgs a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (c >= a.W) return;
    const int nseg = (int)ceil_div(a.H, kSeg);
    const int rb = s * kSeg, re = min(a.H, rb + kSeg);
    int first = -1, last = -1;
    for (int r = rb; r < re; ++r) {
        if (edt_is_bg(a, r, c)) {
            if (first < 0) first = r;
            last = r;
        }
    }
    a.seg[(int64_t)s * a.W + c] = first;
    a.seg[(int64_t)(nseg + s) * a.W + c] = last;
    if (first >= 0 && *a.any_bg == 0) atomicOr(a.any_bg, 1u);
}

// thread per (column, segment): g for the rows of the segment
__global__ void edt_col_kernel(EdtArgs a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (c >= a.W) return;
    const int nseg = (int)ceil_div(a.H, kSeg);
    const int rb = s * kSeg, re = min(a.H, rb + kSeg);
    int above = -1;                      // last background row < rb
    for (int t = s - 1; t >= 0; --t) {
        const int v = a.seg[(int64_t)(nseg + t) * a.W + c];
        if (v >= 0) { above = v; break; }
    }
    int below = -1;                      // first background row >= re
    for (int t = s + 1; t < nseg; ++t) {
        const int v = a.seg[(int64_t)t * a.W + c];
        if (v >= 0) { below = v; break; }
    }
    int up[kSeg];
    int last = above;
    for (int r = rb; r < re; ++r) {
        if (edt_is_bg(a, r, c)) last = r;
        up[r - rb] = last;
    }
    int next = below;
    for (int r = re - 1; r >= rb; --r) {
        if (up[r - rb] == r) next = r;
        int d = 0x7fffffff;
        if (up[r - rb] >= 0) d = r - up[r - rb];
        if (next >= 0 && next - r < d) d = next - r;
        a.g[(int64_t)r * a.W + c] = d == 0x7fffffff ? kInf : (uint16_t)d;
    }
}

// d2 of one row from its g values in shared memory: for pixel c the search
// runs outward from c and stops once (c - c')^2 reaches the best value. A
// pixel that finds no background in any column gets -1 (the image has no
// background: a column with background gives every row a finite g there).
__device__ __forceinline__ void edt_row_search(const uint16_t *sg, int W, bool any, int32_t *out)
{
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        if (!any) {
            out[c] = -1;
            continue;
        }
        const int gc = sg[c];
        constexpr long long kNone = 0x7fffffffffffLL;
        long long best = gc == kInf ? kNone : (long long)gc * gc;
        for (int d = 1; (long long)d * d < best; ++d) {
            const int cl = c - d, cr = c + d;
            if (cl < 0 && cr >= W) break;
            if (cl >= 0) {
                const int g = sg[cl];
                if (g != kInf) {
                    const long long v = (long long)d * d + (long long)g * g;
                    if (v < best) best = v;
                }
            }
            if (cr < W) {
                const int g = sg[cr];
                if (g != kInf) {
                    const long long v = (long long)d * d + (long long)g * g;
                    if (v < best) best = v;
                }
            }
        }
        out[c] = best == kNone ? -1 : (int32_t)best;
    }
}

// The same search in 32-bit arithmetic (bit-plane path): sides are at most
// 32768, so d^2 + g^2 < 2^31 is exact in unsigned 32 bits. Consecutive lanes
// take consecutive columns (conflict-free 16-bit shared reads).
__device__ __forceinline__ void edt_row_search32(const uint16_t *sg, int W, int32_t *out)
{
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        const uint32_t gc = sg[c];
        uint32_t best = gc == kInf ? 0xffffffffu : gc * gc;
        for (uint32_t d = 1; d * d < best; ++d) {
            const int cl = c - (int)d, cr = c + (int)d;
            if (cl < 0 && cr >= W) break;
            if (cl >= 0) {
                const uint32_t g = sg[cl];
                if (g != kInf) best = min(best, d * d + g * g);
            }
            if (cr < W) {
                const uint32_t g = sg[cr];
                if (g != kInf) best = min(best, d * d + g * g);
            }
        }
        out[c] = best == 0xffffffffu ? -1 : (int32_t)best;
    }
}

// CTA per row: exact minimum over columns with early termination
__global__ void edt_row_kernel(EdtArgs a)
{
    extern __shared__ uint16_t sg[];
    const int r = blockIdx.x;
    const uint16_t *grow = a.g + (int64_t)r * a.W;
    if ((a.W & 7) == 0) {   // rows 16-byte aligned: 8 values per load
        const uint4 *src = reinterpret_cast<const uint4 *>(grow);
        uint4 *dst = reinterpret_cast<uint4 *>(sg);
        for (int k = threadIdx.x; k < a.W / 8; k += blockDim.x) dst[k] = __ldcs(src + k);
    } else {
        for (int c = threadIdx.x; c < a.W; c += blockDim.x) sg[c] = grow[c];
    }
    __syncthreads();
    edt_row_search(sg, a.W, *a.any_bg != 0, a.d2 + (int64_t)r * a.ld_d2);
}

cudaError_t launch_edt(const EdtArgs &a, cudaStream_t s)
{
    const int nseg = (int)ceil_div(a.H, kSeg);
    cudaError_t e = cudaMemsetAsync(a.any_bg, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)a.W * sizeof(uint16_t);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(edt_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const dim3 g1((unsigned)ceil_div(a.W, 128), (unsigned)nseg);
    edt_seg_kernel<<<g1, 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    edt_col_kernel<<<g1, 128, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    edt_row_kernel<<<(unsigned)a.H, 256, smem, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------- bit-plane batch
namespace {
size_t piece(size_t bytes) { return (size_t)round_up((int64_t)bytes, 256); }
}  // namespace

size_t edt_bits_workspace_bytes(int H, int W)
{
    const size_t nseg = (size_t)ceil_div(H, kSeg);
    return piece(nseg * W * sizeof(uint32_t)) + piece(2 * nseg * W * sizeof(int32_t));
}

constexpr int kMaskWarps = 4;   // plane word columns per CTA of the mask stage
constexpr int kColThreads = 128;

void edt_bits_add(EdtBitsBatch &b, const uint32_t *bits, int H, int W, int32_t *d2, int64_t ld_d2, char *base)
{
    if (b.n == 0) {
        b.maxW = 0;
        b.mask_ctas = b.col_ctas = b.rows = 0;
    }
    EdtBitsImage &d = b.img[b.n++];
    const int64_t nseg = ceil_div(H, kSeg);
    d.bits = bits;
    d.H = H;
    d.W = W;
    d.d2 = d2;
    d.ld_d2 = ld_d2;
    d.cmask = reinterpret_cast<uint32_t *>(base);
    d.seg = reinterpret_cast<int32_t *>(base + piece((size_t)nseg * W * sizeof(uint32_t)));
    d.mask_base = b.mask_ctas;
    d.col_base = b.col_ctas;
    d.row_base = b.rows;
    b.mask_ctas += ceil_div(ceil_div(W, 32), kMaskWarps) * nseg;
    b.col_ctas += ceil_div(W, kColThreads) * nseg;
    b.rows += H;
    b.maxW = W > b.maxW ? W : b.maxW;
}

// the image whose CTA range [base, next base) holds CTA g of a stage
template <int64_t EdtBitsImage::*BASE>
__device__ __forceinline__ const EdtBitsImage &edt_image(const EdtBitsBatch &b, int64_t g)
{
    int k = 0;
    while (k + 1 < b.n && g >= b.img[k + 1].*BASE) ++k;
    return b.img[k];
}

// Lane i loads the plane word (32 columns starting at 32 * wc) of row
// rb + i; 32 ballots turn the rows' words into the columns' masks, lane j
// getting column 32 * wc + j with bit i set where row rb + i is background.
// Rows past the end count as foreground.
__device__ __forceinline__ uint32_t seg_bg_mask(const EdtBitsImage &a, int64_t wpr, int wc, int rb, int lane)
{
    const int r = rb + lane;
    const uint32_t w = r < a.H ? __ldg(a.bits + (int64_t)r * wpr + wc) : 0xffffffffu;
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t b = __ballot_sync(0xffffffffu, !((w >> j) & 1u));
        m = lane == j ? b : m;
    }
    return m;
}

// warp per (plane word column, segment): the segment's column masks
__global__ void __launch_bounds__(kMaskWarps * 32) edt_mask_bits_kernel(EdtBitsBatch b)
{
    const EdtBitsImage &a = edt_image<&EdtBitsImage::mask_base>(b, blockIdx.x);
    const int wpr = (a.W + 31) / 32;
    const int local = (int)(blockIdx.x - a.mask_base);
    const int gx = (wpr + kMaskWarps - 1) / kMaskWarps;
    const int s = local / gx;
    const int wc = (local - s * gx) * kMaskWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (wc >= wpr) return;
    const int rb = s * kSeg;
    const uint32_t bg = seg_bg_mask(a, wpr, wc, rb, lane);
    const int c = wc * 32 + lane;
    if (c >= a.W) return;
    a.cmask[(int64_t)s * a.W + c] = bg;
}

// thread per (column, segment): the last background row above the segment
// and the first one below it (-1: none)
__global__ void __launch_bounds__(kColThreads) edt_chase_bits_kernel(EdtBitsBatch b)
{
    const EdtBitsImage &a = edt_image<&EdtBitsImage::col_base>(b, blockIdx.x);
    const int local = (int)(blockIdx.x - a.col_base);
    const int gx = (a.W + kColThreads - 1) / kColThreads;
    const int s = local / gx;
    const int c = (local - s * gx) * kColThreads + threadIdx.x;
    if (c >= a.W) return;
    const int nseg = (int)ceil_div(a.H, kSeg);
    int above = -1;
    for (int t = s - 1; t >= 0; --t) {
        const uint32_t m = a.cmask[(int64_t)t * a.W + c];
        if (m) { above = t * kSeg + 31 - __clz(m); break; }
    }
    int below = -1;
    for (int t = s + 1; t < nseg; ++t) {
        const uint32_t m = a.cmask[(int64_t)t * a.W + c];
        if (m) { below = t * kSeg + __ffs(m) - 1; break; }
    }
    a.seg[(int64_t)s * a.W + c] = above;
    a.seg[(int64_t)(nseg + s) * a.W + c] = below;
}

// CTA per row: g of the row from the column masks of its segment (and,
// where the segment has no background on one side of the row, the nearest
// background beyond it), then the search. A row that finds no background
// anywhere belongs to an image without background (every column's g is
// infinite then), whose distances are -1.
__global__ void edt_row_bits_kernel(EdtBitsBatch b)
{
    extern __shared__ uint16_t sg[];
    const EdtBitsImage &a = edt_image<&EdtBitsImage::row_base>(b, blockIdx.x);
    const int r = (int)(blockIdx.x - a.row_base), s = r / kSeg, i = r % kSeg, rb = s * kSeg;
    const int nseg = (int)ceil_div(a.H, kSeg);
    const uint32_t *cm = a.cmask + (int64_t)s * a.W;
    // four columns per thread at a time: their mask loads are issued together
    for (int c0 = threadIdx.x; c0 < a.W; c0 += 4 * blockDim.x) {
        uint32_t mm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * blockDim.x;
            mm[u] = c < a.W ? __ldg(cm + c) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * blockDim.x;
            if (c >= a.W) break;
            const uint32_t m = mm[u];
            uint16_t g = 0;
            if (!((m >> i) & 1u)) {
                const uint32_t upto = m & (0xffffffffu >> (31 - i));   // rows rb .. r
                const uint32_t from = m & (0xffffffffu << i);          // rows r .. rb + 31
                const int up = upto ? rb + 31 - __clz(upto) : a.seg[(int64_t)s * a.W + c];
                const int dn = from ? rb + __ffs(from) - 1 : a.seg[(int64_t)(nseg + s) * a.W + c];
                int d = 0x7fffffff;
                if (up >= 0) d = r - up;
                if (dn >= 0 && dn - r < d) d = dn - r;
                g = d == 0x7fffffff ? kInf : (uint16_t)d;
            }
            sg[c] = g;
        }
    }
    __syncthreads();
    edt_row_search32(sg, a.W, a.d2 + (int64_t)r * a.ld_d2);
}

cudaError_t launch_edt_bits_batch(const EdtBitsBatch &b, cudaStream_t s)
{
    if (b.n < 1 || b.n > kEdtMaxImgs) return cudaErrorInvalidValue;
    const size_t smem = (size_t)b.maxW * sizeof(uint16_t);
    cudaError_t e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(edt_row_bits_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    edt_mask_bits_kernel<<<(unsigned)b.mask_ctas, kMaskWarps * 32, 0, s>>>(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    edt_chase_bits_kernel<<<(unsigned)b.col_ctas, kColThreads, 0, s>>>(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    edt_row_bits_kernel<<<(unsigned)b.rows, 256, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace rtk
