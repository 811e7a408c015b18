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

namespace rtk {

// one thread per 8 x 8 block: histogram (shared, then global), dark count,
// block maximum
__global__ void feat_block_kernel(FeatBatch fb)
{
    __shared__ uint32_t sh[256];
    const FeatImage &d = fb.img[blockIdx.y];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const int bh = (d.H + 7) / 8, bw = (d.W + 7) / 8;
    const int nb = bh * bw;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int br = b / bw, bc = b % bw;
        const int r1 = min(d.H, br * 8 + 8), c1 = min(d.W, bc * 8 + 8);
        int dark = 0, mx = 0;
        for (int r = br * 8; r < r1; ++r) {
            const uint8_t *row = d.img + (int64_t)r * d.ld;
            for (int c = bc * 8; c < c1; ++c) {
                const int v = row[c];
                atomicAdd(sh + v, 1u);
                dark += v < 80;
                mx = max(mx, v);
            }
        }
        d.dark[b] = (uint8_t)dark;
        d.bmax[b] = (uint8_t)mx;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (sh[i]) atomicAdd(d.hist + i, sh[i]);
}

__device__ __forceinline__ int marker_of(const uint8_t *D, int bh, int bw, int r, int c)
{
    const int v = D[r * bw + c];
    return (r == 0 || c == 0 || r == bh - 1 || c == bw - 1) ? v : max(v - 30, 0);
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

// one CTA per image: block statistics, frontier count, histogram statistics
__global__ void __launch_bounds__(1024) feat_final_kernel(FeatBatch fb, float *out)
{
    __shared__ double redd[32];
    __shared__ long long redl[32];
    const FeatImage &d = fb.img[blockIdx.x];
    const int bh = (d.H + 7) / 8, bw = (d.W + 7) / 8;
    const int nb = bh * bw;
    double s1 = 0.0, s2 = 0.0;
    long long over = 0, front = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int br = b / bw, bc = b % bw;
        const int npx = (min(d.H, br * 8 + 8) - br * 8) * (min(d.W, bc * 8 + 8) - bc * 8);
        const double fr = (double)d.dark[b] / npx;
        s1 += fr;
        s2 += fr * fr;
        over += fr > 0.1;
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
    s1 = block_sum(s1, redd);
    s2 = block_sum(s2, redd);
    over = block_sum(over, redl);
    front = block_sum(front, redl);
    if (threadIdx.x != 0) return;
    float *f = out + (int64_t)blockIdx.x * kNumFeatures;
    const double N = (double)d.H * d.W;
    f[0] = (float)d.H;
    f[1] = (float)d.W;
    f[2] = (float)log(N);
    double mean = 0.0;
    for (int v = 0; v < 256; ++v) mean += (d.hist[v] / N) * v;
    double m2 = 0.0, m3 = 0.0, m4 = 0.0, ent = 0.0;
    for (int v = 0; v < 256; ++v) {
        const double p = d.hist[v] / N, x = v - mean;
        m2 += p * x * x;
        m3 += p * x * x * x;
        m4 += p * x * x * x * x;
        if (p > 0) ent -= p * log2(p);
    }
    f[3] = (float)mean;
    f[4] = (float)m2;
    f[5] = m2 > 0 ? (float)(m3 / (m2 * sqrt(m2))) : 0.f;
    f[6] = m2 > 0 ? (float)(m4 / (m2 * m2)) : 0.f;
    const int pct[9] = {1, 5, 10, 25, 50, 75, 90, 95, 99};
    for (int k = 0; k < 9; ++k) {
        const double need = pct[k] / 100.0 * N;
        uint64_t cum = 0;
        int v = 0;
        for (; v < 256; ++v) {
            cum += d.hist[v];
            if ((double)cum >= need) break;
        }
        f[7 + k] = (float)v;
    }
    uint64_t lo80 = 0, lo110 = 0;
    for (int v = 0; v < 110; ++v) {
        if (v < 80) lo80 += d.hist[v];
        lo110 += d.hist[v];
    }
    f[16] = (float)(lo80 / N);
    f[17] = (float)(lo110 / N);
    f[18] = (float)ent;
    const double mfr = s1 / nb;
    f[19] = (float)mfr;
    f[20] = (float)sqrt(fmax(s2 / nb - mfr * mfr, 0.0));
    f[21] = (float)((double)over / nb);
    f[22] = (float)((double)front / nb);
    f[23] = (float)log1p((double)front);
}

size_t feat_workspace_bytes(int H, int W)
{
    const size_t nb = (size_t)((H + 7) / 8) * ((W + 7) / 8);
    return 256 * sizeof(uint32_t) + 2 * nb + 3 * 256;
}

cudaError_t launch_features(const FeatBatch &fb, float *out, cudaStream_t s)
{
    int maxnb = 1;
    for (int i = 0; i < fb.n; ++i) {
        const int nb = ((fb.img[i].H + 7) / 8) * ((fb.img[i].W + 7) / 8);
        maxnb = nb > maxnb ? nb : maxnb;
        cudaError_t e = cudaMemsetAsync(fb.img[i].hist, 0, 256 * sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
    }
    int gx = (int)ceil_div(maxnb, 256);
    if (gx > 1024) gx = 1024;
    feat_block_kernel<<<dim3((unsigned)gx, (unsigned)fb.n), 256, 0, s>>>(fb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    feat_final_kernel<<<(unsigned)fb.n, 1024, 0, s>>>(fb, out);
    return cudaGetLastError();
}

}  // namespace rtk
