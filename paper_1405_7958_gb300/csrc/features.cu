// Per-tile features for the learned variant picker.
//
// The paper's PATS scheduler (Section 3.2.1) orders tasks by estimated GPU
// speedup because the run time of the irregular operations cannot be
// predicted in advance. Here a small network reads 24 cheap statistics of a
// tile and picks the propagation variant of its reconstruction. The
// features (in order): H, W, ln(H W); mean, variance, skewness, kurtosis of
// the 256-bin histogram; the lower 1/5/10/25/50/75/90/95/99 percentiles;
// the fractions of pixels below 80 and below 110; the histogram entropy in
// bits; mean and population standard deviation of the dark fraction
// (pixels < 80) over 8 x 8 blocks and the fraction of blocks whose dark
// fraction exceeds 0.1; and a frontier estimate on the 8 x 8 block maximum
// D with marker Jd = max(D - 30, 0) (Jd = D on D's border): the fraction of
// pixels p of D whose raster-order neighbours q (up-left, up, up-right,
// left) give max min(Jd(q), D(p)) > Jd(p), and ln(1 + their count).
// Counts are exact integers; the statistics are finished in double.
#include "features.cuh"
#include "mlp.cuh"

namespace rtk {

// pass 1, CTA = 64 rows x 1024 columns, thread = 4 adjacent columns (one
// 32-bit load per row where the row start allows it): histogram (per warp in
// shared memory, then global), and per 8 x 8 block the dark count and the
// maximum (a block's two threads are neighbouring lanes)
constexpr int kFeatCols = 4;
constexpr int kFeatSpan = 256 * kFeatCols;

__global__ void __launch_bounds__(256) feat_block_kernel(FeatBatch fb)
{
    // one 256-bin histogram per warp (values of neighbouring pixels cluster,
    // so a single shared histogram would serialise on a few bins)
    __shared__ uint32_t sh[8][256];
    const FeatImage &d = fb.img[blockIdx.z];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[k][threadIdx.x] = 0;
    __syncthreads();
    const int c0 = blockIdx.x * kFeatSpan + threadIdx.x * kFeatCols;
    const int r0 = blockIdx.y * 64;
    if (r0 < d.H && blockIdx.x * kFeatSpan < d.W) {
        const int bw = (d.W + 7) / 8;
        const int nc = max(0, min(kFeatCols, d.W - c0));   // this thread's columns inside the image
        const bool word = nc == kFeatCols && ((((uintptr_t)d.img) | (uintptr_t)d.ld) & 3u) == 0;
        for (int g = 0; g < 8; ++g) {
            const int rb = r0 + 8 * g;
            if (rb >= d.H) break;
            int dark = 0, mx = 0;
            const int re = min(d.H, rb + 8);
            for (int r = rb; r < re; ++r) {
                const uint8_t *row = d.img + (int64_t)r * d.ld + c0;
                uint32_t v4 = 0;
                if (word) {
                    v4 = *reinterpret_cast<const uint32_t *>(row);
                } else {
                    for (int k = 0; k < nc; ++k) v4 |= (uint32_t)row[k] << (8 * k);
                }
                for (int k = 0; k < nc; ++k) {
                    const int v = (v4 >> (8 * k)) & 0xff;
                    atomicAdd(&sh[warp][v], 1u);
                    dark += v < 80;
                    mx = max(mx, v);
                }
            }
            dark += __shfl_xor_sync(0xffffffffu, dark, 1);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            if ((threadIdx.x & 1) == 0 && c0 < d.W) {
                const int b = (rb / 8) * bw + c0 / 8;
                d.dark[b] = (uint8_t)dark;
                d.bmax[b] = (uint8_t)mx;
            }
        }
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += sh[k][threadIdx.x];
    if (tot) atomicAdd(d.hist + threadIdx.x, tot);
}

// clears the per-image accumulators of a call (one launch for the batch)
__global__ void feat_zero_kernel(FeatBatch fb)
{
    const FeatImage &d = fb.img[blockIdx.x];
    d.hist[threadIdx.x] = 0;
    if (threadIdx.x < 4) d.acc[threadIdx.x] = 0;
}

__device__ __forceinline__ int marker_of(const uint8_t *D, int bh, int bw, int r, int c)
{
    const int v = D[r * bw + c];
    return (r == 0 || c == 0 || r == bh - 1 || c == bw - 1) ? v : max(v - 30, 0);
}

// pass 2, thread per 8 x 8 block: integer sums over the full blocks (dark
// count, its square, blocks above 10 %) and the frontier count
__global__ void feat_count_kernel(FeatBatch fb)
{
    const FeatImage &d = fb.img[blockIdx.y];
    const int bh = (d.H + 7) / 8, bw = (d.W + 7) / 8;
    const int fbh = d.H / 8, fbw = d.W / 8;       // full blocks
    const int nb = bh * bw;
    unsigned long long s1 = 0, s2 = 0, over = 0, front = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int br = b / bw, bc = b % bw;
        if (br < fbh && bc < fbw) {
            const int k = d.dark[b];
            s1 += k;
            s2 += k * k;
            over += 10 * k > 64;
        }
        const int Dp = d.bmax[b], Jp = marker_of(d.bmax, bh, bw, br, bc);
        int best = -1;
        if (br > 0) {
            if (bc > 0) best = max(best, min(marker_of(d.bmax, bh, bw, br - 1, bc - 1), Dp));
            best = max(best, min(marker_of(d.bmax, bh, bw, br - 1, bc), Dp));
            if (bc + 1 < bw) best = max(best, min(marker_of(d.bmax, bh, bw, br - 1, bc + 1), Dp));
        }
        if (bc > 0) best = max(best, min(marker_of(d.bmax, bh, bw, br, bc - 1), Dp));
        front += best > Jp;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        over += __shfl_down_sync(0xffffffffu, over, o);
        front += __shfl_down_sync(0xffffffffu, front, o);
    }
    // one set of atomics per CTA (per-warp atomics on the four counters of
    // an image serialise)
    __shared__ unsigned long long part[4][32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        part[0][w] = s1;
        part[1][w] = s2;
        part[2][w] = over;
        part[3][w] = front;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[threadIdx.x][k];
        if (t) atomicAdd(d.acc + threadIdx.x, t);
    }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;   // valid in thread 0
}

// pass 3, CTA of 256 threads per image (thread = histogram bin): moments,
// entropy and percentiles from the histogram; the partial edge blocks; the
// 24 features into f
__device__ __forceinline__ void feat_final_image(const FeatImage &d, float *f)
{
    __shared__ double redd[8];
    __shared__ uint32_t cum[256];
    const int v = threadIdx.x;
    const double N = (double)d.H * d.W;
    const uint32_t h = d.hist[v];
    const double p = h / N;
    const double mean_all = block_sum(p * v, redd);
    __shared__ double s_mean;
    if (v == 0) s_mean = mean_all;
    __syncthreads();
    const double mean = s_mean, x = v - mean;
    const double m2 = block_sum(p * x * x, redd);
    const double m3 = block_sum(p * x * x * x, redd);
    const double m4 = block_sum(p * x * x * x * x, redd);
    const double ent = block_sum(p > 0 ? -p * log2(p) : 0.0, redd);
    // inclusive prefix sum of the histogram (Hillis-Steele in shared memory)
    cum[v] = h;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const uint32_t add = v >= o ? cum[v - o] : 0u;
        __syncthreads();
        cum[v] += add;
        __syncthreads();
    }
    const int pct[9] = {1, 5, 10, 25, 50, 75, 90, 95, 99};
    for (int k = 0; k < 9; ++k) {
        const double need = pct[k] / 100.0 * N;
        if ((double)cum[v] >= need && (v == 0 || (double)cum[v - 1] < need)) f[7 + k] = (float)v;
    }
    // partial blocks on the right column and the bottom row
    const int bh = (d.H + 7) / 8, bw = (d.W + 7) / 8;
    const int fbh = d.H / 8, fbw = d.W / 8;
    double ps1 = 0.0, ps2 = 0.0, pov = 0.0;
    const int npart = (bw > fbw ? bh : 0) + (bh > fbh ? fbw : 0);
    for (int i = v; i < npart; i += blockDim.x) {
        int br, bc;
        if (bw > fbw && i < bh) { br = i; bc = bw - 1; }
        else { br = bh - 1; bc = i - (bw > fbw ? bh : 0); }
        const int npx = (min(d.H, br * 8 + 8) - br * 8) * (min(d.W, bc * 8 + 8) - bc * 8);
        const int k = d.dark[br * bw + bc];
        const double fr = (double)k / npx;
        ps1 += fr;
        ps2 += fr * fr;
        pov += 10 * k > npx;
    }
    ps1 = block_sum(ps1, redd);
    ps2 = block_sum(ps2, redd);
    pov = block_sum(pov, redd);
    if (v != 0) return;
    const double nb = (double)bh * bw;
    f[0] = (float)d.H;
    f[1] = (float)d.W;
    f[2] = (float)log(N);
    f[3] = (float)mean;
    f[4] = (float)m2;
    f[5] = m2 > 0 ? (float)(m3 / (m2 * sqrt(m2))) : 0.f;
    f[6] = m2 > 0 ? (float)(m4 / (m2 * m2)) : 0.f;
    f[16] = (float)(cum[79] / N);
    f[17] = (float)(cum[109] / N);
    f[18] = (float)ent;
    const double s1 = d.acc[0] / 64.0 + ps1, s2 = d.acc[1] / 4096.0 + ps2;
    const double mfr = s1 / nb;
    f[19] = (float)mfr;
    f[20] = (float)sqrt(fmax(s2 / nb - mfr * mfr, 0.0));
    f[21] = (float)(((double)d.acc[2] + pov) / nb);
    f[22] = (float)((double)d.acc[3] / nb);
    f[23] = (float)log1p((double)d.acc[3]);
}

__global__ void __launch_bounds__(256) feat_final_kernel(FeatBatch fb, float *out)
{
    feat_final_image(fb.img[blockIdx.x], out + (int64_t)blockIdx.x * kNumFeatures);
}

// pass 3 and the picker's network on the image's features, in one CTA per
// image: warp 0 runs the same per-sample network (same order of operations,
// same bits) as the network's forward for a chunk of tiles
__global__ void __launch_bounds__(256) feat_final_pick_kernel(FeatBatch fb, float *out, const uint16_t *wb,
                                                              const float *norm, int32_t *pick, float min_prob,
                                                              int fallback)
{
    __shared__ float P[kMlpParams];
    __shared__ float xn[kMlpIn];
    __shared__ float h[2][kMlpH];
    float *f = out + (int64_t)blockIdx.x * kNumFeatures;
    feat_final_image(fb.img[blockIdx.x], f);
    mlp_stage_params(wb, P);
    __syncthreads();   // the features (written by several threads) and P
    if (threadIdx.x < kMlpIn) xn[threadIdx.x] = (f[threadIdx.x] - norm[threadIdx.x]) / norm[kMlpIn + threadIdx.x];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    mlp_warp_hidden(P, xn, h, threadIdx.x);
    if (threadIdx.x != 0) return;
    float z[kMlpOut];
    pick[blockIdx.x] = mlp_logits_pick(P, h[1], z, min_prob, fallback);
}

size_t feat_workspace_bytes(int H, int W)
{
    const size_t nb = (size_t)((H + 7) / 8) * ((W + 7) / 8);
    return 256 * sizeof(uint32_t) + 4 * sizeof(unsigned long long) + 2 * nb + 4 * 256;
}

cudaError_t launch_features(const FeatBatch &fb, float *out, cudaStream_t s)
{
    int maxH = 1, maxW = 1, maxnb = 1;
    for (int i = 0; i < fb.n; ++i) {
        const FeatImage &d = fb.img[i];
        maxH = d.H > maxH ? d.H : maxH;
        maxW = d.W > maxW ? d.W : maxW;
        const int nb = ((d.H + 7) / 8) * ((d.W + 7) / 8);
        maxnb = nb > maxnb ? nb : maxnb;
    }
    feat_zero_kernel<<<(unsigned)fb.n, 256, 0, s>>>(fb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    feat_block_kernel<<<dim3((unsigned)ceil_div(maxW, kFeatSpan), (unsigned)ceil_div(maxH, 64), (unsigned)fb.n), 256, 0,
                        s>>>(fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int gx = (int)ceil_div(maxnb, 256);
    if (gx > 512) gx = 512;
    feat_count_kernel<<<dim3((unsigned)gx, (unsigned)fb.n), 256, 0, s>>>(fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    feat_final_kernel<<<(unsigned)fb.n, 256, 0, s>>>(fb, out);
    return cudaGetLastError();
}

cudaError_t launch_features_pick(const FeatBatch &fb, float *out, const uint16_t *wb, const float *norm,
                                 int32_t *pick, float min_prob, int fallback, cudaStream_t s)
{
    int maxH = 1, maxW = 1, maxnb = 1;
    for (int i = 0; i < fb.n; ++i) {
        const FeatImage &d = fb.img[i];
        maxH = d.H > maxH ? d.H : maxH;
        maxW = d.W > maxW ? d.W : maxW;
        const int nb = ((d.H + 7) / 8) * ((d.W + 7) / 8);
        maxnb = nb > maxnb ? nb : maxnb;
    }
    feat_zero_kernel<<<(unsigned)fb.n, 256, 0, s>>>(fb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    feat_block_kernel<<<dim3((unsigned)ceil_div(maxW, kFeatSpan), (unsigned)ceil_div(maxH, 64), (unsigned)fb.n), 256, 0,
                        s>>>(fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int gx = (int)ceil_div(maxnb, 256);
    if (gx > 512) gx = 512;
    feat_count_kernel<<<dim3((unsigned)gx, (unsigned)fb.n), 256, 0, s>>>(fb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    feat_final_pick_kernel<<<(unsigned)fb.n, 256, 0, s>>>(fb, out, wb, norm, pick, min_prob, fallback);
    return cudaGetLastError();
}

}  // namespace rtk
