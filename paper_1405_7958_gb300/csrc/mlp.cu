// The learned variant picker: an MLP 24 -> 64 -> 64 -> 3 with bf16
// parameters, fp32 accumulation and ReLU, trained on the GPU.
//
// Parameters form one flat vector (row-major weights, then biases):
//   W1[64][24] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]   (5955 values)
// kept as bf16 for compute and as an fp32 master copy for the optimizer.
// The input is normalised first: xn = (x - mu) / sd, elementwise.
//   h1 = relu(W1 xn + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3,
//   loss = mean over the batch of logsumexp(z) - z[label].
// The network is ~5.9 thousand multiply-adds per sample, so plain FMA
// loops are used; the work is negligible next to the segmentation.
#include <cuda_bf16.h>

#include "mlp.cuh"

namespace rtk {

__device__ __forceinline__ float bf(uint16_t h)
{
    return __uint_as_float((uint32_t)h << 16);   // bf16 -> fp32 is exact
}

// one thread per sample; parameters staged in shared memory as fp32
__global__ void __launch_bounds__(256) mlp_forward_kernel(const uint16_t *wb, const float *norm, const float *x, int B,
                                                          float *logits, float *act, int32_t *pick, float min_prob,
                                                          int fallback)
{
    __shared__ float P[kMlpParams];
    __shared__ float mu[kMlpIn], sd[kMlpIn];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) P[i] = bf(wb[i]);
    for (int i = threadIdx.x; i < kMlpIn; i += blockDim.x) {
        mu[i] = norm[i];
        sd[i] = norm[kMlpIn + i];
    }
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float xn[kMlpIn];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) xn[i] = (x[(int64_t)b * kMlpIn + i] - mu[i]) / sd[i];
    float h1[kMlpH];
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        float s = P[kB1 + j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) s = fmaf(P[kW1 + j * kMlpIn + i], xn[i], s);
        h1[j] = fmaxf(s, 0.f);
    }
    float z[kMlpOut];
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) z[k] = P[kB3 + k];
    for (int j = 0; j < kMlpH; ++j) {
        float s = P[kB2 + j];
#pragma unroll
        for (int i = 0; i < kMlpH; ++i) s = fmaf(P[kW2 + j * kMlpH + i], h1[i], s);
        const float h2 = fmaxf(s, 0.f);
        if (act) act[(int64_t)b * kMlpAct + kMlpH + j] = h2;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) z[k] = fmaf(P[kW3 + k * kMlpH + j], h2, z[k]);
    }
    if (act) {
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) act[(int64_t)b * kMlpAct + j] = h1[j];
    }
    int best = 0;
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) {
        if (logits) logits[(int64_t)b * kMlpOut + k] = z[k];
        if (z[k] > z[best]) best = k;
    }
    // confidence fall-back: the pick stands only when its softmax
    // probability 1 / sum_k exp(z_k - z_best) reaches min_prob
    if (min_prob > 0.f) {
        float se = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) se += expf(z[k] - z[best]);
        if (1.f / se < min_prob) best = fallback;
    }
    if (pick) pick[b] = best;
}

// per-sample deltas: dz = (softmax(z) - onehot(label)) / B, dh2, dh1 (after
// the ReLU masks), the normalised input, and the per-sample loss
__global__ void __launch_bounds__(256) mlp_delta_kernel(const uint16_t *wb, const float *norm, const float *x,
                                                        const float *act, const float *logits, const int32_t *label,
                                                        int B, float *ws)
{
    __shared__ float P[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) P[i] = bf(wb[i]);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float *dz = ws + (int64_t)b * kMlpDelta;
    float *dh2 = dz + kMlpOut;
    float *dh1 = dh2 + kMlpH;
    float *xn = dh1 + kMlpH;
    float *lossb = xn + kMlpIn;
    const float *z = logits + (int64_t)b * kMlpOut;
    const float *h1 = act + (int64_t)b * kMlpAct;
    const float *h2 = h1 + kMlpH;
    float m = z[0];
    for (int k = 1; k < kMlpOut; ++k) m = fmaxf(m, z[k]);
    float se = 0.f;
    for (int k = 0; k < kMlpOut; ++k) se += expf(z[k] - m);
    const int y = label[b];
    lossb[0] = logf(se) + m - z[y];
    float g[kMlpOut];
    for (int k = 0; k < kMlpOut; ++k) {
        g[k] = (expf(z[k] - m) / se - (k == y ? 1.f : 0.f)) / (float)B;
        dz[k] = g[k];
    }
    float d2[kMlpH];
    for (int j = 0; j < kMlpH; ++j) {
        float s = 0.f;
        for (int k = 0; k < kMlpOut; ++k) s = fmaf(P[kW3 + k * kMlpH + j], g[k], s);
        d2[j] = h2[j] > 0.f ? s : 0.f;
        dh2[j] = d2[j];
    }
    for (int i = 0; i < kMlpH; ++i) {
        float s = 0.f;
        for (int j = 0; j < kMlpH; ++j) s = fmaf(P[kW2 + j * kMlpH + i], d2[j], s);
        dh1[i] = h1[i] > 0.f ? s : 0.f;
    }
    for (int i = 0; i < kMlpIn; ++i) xn[i] = (x[(int64_t)b * kMlpIn + i] - norm[i]) / norm[kMlpIn + i];
}

// one thread per parameter: its gradient summed over the batch (fixed
// order, so results do not depend on scheduling); thread kMlpParams sums the
// loss
__global__ void mlp_grad_kernel(const float *ws, const float *act, int B, float *grad, float *loss)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > kMlpParams) return;
    float s = 0.f;
    if (t == kMlpParams) {
        for (int b = 0; b < B; ++b) s += ws[(int64_t)b * kMlpDelta + kMlpOut + 2 * kMlpH + kMlpIn];
        if (loss) *loss = s / (float)B;
        return;
    }
    // locate (delta column, input column) of parameter t
    int dcol, icol;   // icol < 0: bias (input = 1)
    int src;          // 0: input = xn, 1: input = h1 (act), 2: input = h2 (act)
    if (t < kB1) { dcol = kMlpOut + kMlpH + t / kMlpIn; icol = t % kMlpIn; src = 0; }
    else if (t < kW2) { dcol = kMlpOut + kMlpH + (t - kB1); icol = -1; src = 0; }
    else if (t < kB2) { dcol = kMlpOut + (t - kW2) / kMlpH; icol = (t - kW2) % kMlpH; src = 1; }
    else if (t < kW3) { dcol = kMlpOut + (t - kB2); icol = -1; src = 1; }
    else if (t < kB3) { dcol = (t - kW3) / kMlpH; icol = (t - kW3) % kMlpH; src = 2; }
    else { dcol = t - kB3; icol = -1; src = 2; }
    for (int b = 0; b < B; ++b) {
        const float d = ws[(int64_t)b * kMlpDelta + dcol];
        float in = 1.f;
        if (icol >= 0) {
            if (src == 0) in = ws[(int64_t)b * kMlpDelta + kMlpOut + 2 * kMlpH + icol];
            else in = act[(int64_t)b * kMlpAct + (src == 2 ? kMlpH : 0) + icol];
        }
        s = fmaf(d, in, s);
    }
    grad[t] = s;
}

__global__ void mlp_adamw_kernel(float *master, uint16_t *wb, const float *grad, float *m, float *v, int step,
                                 float lr, float b1, float b2, float eps, float wd)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kMlpParams) return;
    const float g = grad[t];
    const float mt = b1 * m[t] + (1.f - b1) * g;
    const float vt = b2 * v[t] + (1.f - b2) * g * g;
    m[t] = mt;
    v[t] = vt;
    const float mh = mt / (1.f - powf(b1, (float)step));
    const float vh = vt / (1.f - powf(b2, (float)step));
    float p = master[t];
    p -= lr * (mh / (sqrtf(vh) + eps) + wd * p);
    master[t] = p;
    wb[t] = __bfloat16_as_ushort(__float2bfloat16_rn(p));
}

// The same forward with one warp per sample, for the few samples of a
// segmentation chunk (thread per sample would leave a CTA nearly idle for the
// whole 5.9 k multiply-add chain). Lanes own hidden units j and j + 32; each
// unit's sum runs over its inputs in the same order, from the same bias, as
// in mlp_forward_kernel, and lane 0 forms the logits in the same order, so
// both kernels give the same bits.
constexpr int kFwdWarps = 8;
__global__ void __launch_bounds__(kFwdWarps * 32) mlp_forward_warp_kernel(const uint16_t *wb, const float *norm,
                                                                          const float *x, int B, float *logits,
                                                                          float *act, int32_t *pick, float min_prob,
                                                                          int fallback)
{
    __shared__ float P[kMlpParams];
    __shared__ float h[kFwdWarps][2][kMlpH];
    __shared__ float xn[kFwdWarps][kMlpIn];
    mlp_stage_params(wb, P);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kFwdWarps + w;
    if (b < B && lane < kMlpIn) xn[w][lane] = (x[(int64_t)b * kMlpIn + lane] - norm[lane]) / norm[kMlpIn + lane];
    __syncthreads();
    if (b >= B) return;
    mlp_warp_hidden(P, xn[w], h[w], lane);
    if (act) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            act[(int64_t)b * kMlpAct + lane + 32 * q] = h[w][0][lane + 32 * q];
            act[(int64_t)b * kMlpAct + kMlpH + lane + 32 * q] = h[w][1][lane + 32 * q];
        }
    }
    if (lane != 0) return;
    float z[kMlpOut];
    const int best = mlp_logits_pick(P, h[w][1], z, min_prob, fallback);
    if (logits) {
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) logits[(int64_t)b * kMlpOut + k] = z[k];
    }
    if (pick) pick[b] = best;
}

cudaError_t launch_mlp_forward(const uint16_t *wb, const float *norm, const float *x, int B, float *logits, float *act,
                               int32_t *pick, float min_prob, int fallback, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    if (B <= 64) {
        mlp_forward_warp_kernel<<<(unsigned)ceil_div(B, kFwdWarps), kFwdWarps * 32, 0, s>>>(wb, norm, x, B, logits, act,
                                                                                            pick, min_prob, fallback);
        return cudaGetLastError();
    }
    mlp_forward_kernel<<<(unsigned)ceil_div(B, 256), 256, 0, s>>>(wb, norm, x, B, logits, act, pick, min_prob,
                                                                  fallback);
    return cudaGetLastError();
}

size_t mlp_backward_workspace_bytes(int B) { return (size_t)B * kMlpDelta * sizeof(float); }

cudaError_t launch_mlp_backward(const uint16_t *wb, const float *norm, const float *x, const float *act,
                                const float *logits, const int32_t *label, int B, float *grad, float *loss, float *ws,
                                cudaStream_t s)
{
    if (B <= 0) return cudaErrorInvalidValue;
    mlp_delta_kernel<<<(unsigned)ceil_div(B, 256), 256, 0, s>>>(wb, norm, x, act, logits, label, B, ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp_grad_kernel<<<(unsigned)ceil_div(kMlpParams + 1, 128), 128, 0, s>>>(ws, act, B, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adamw(float *master, uint16_t *wb, const float *grad, float *m, float *v, int step, float lr,
                             float b1, float b2, float eps, float wd, cudaStream_t s)
{
    mlp_adamw_kernel<<<(unsigned)ceil_div(kMlpParams, 256), 256, 0, s>>>(master, wb, grad, m, v, step, lr, b1, b2,
                                                                         eps, wd);
    return cudaGetLastError();
}

// ---------------------------------------------------- input normalisation
// One CTA per feature column: each thread sums a fixed stride of rows in
// double, then a fixed-shape tree adds the partial sums; two passes (mean,
// then squared deviations).
constexpr int kNormThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int k = kNormThreads / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kNormThreads) feature_norm_kernel(const float *x, int B, float *norm)
{
    __shared__ double sh[kNormThreads];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += kNormThreads) s += (double)x[(int64_t)b * kMlpIn + f];
    const double mean = block_sum(s, sh) / B;
    double q = 0.0;
    for (int b = threadIdx.x; b < B; b += kNormThreads) {
        const double d = (double)x[(int64_t)b * kMlpIn + f] - mean;
        q += d * d;
    }
    const double ss = block_sum(q, sh);
    if (threadIdx.x == 0) {
        const double sd = B > 1 ? sqrt(ss / (B - 1)) : 0.0;
        norm[f] = (float)mean;
        norm[kMlpIn + f] = (float)(sd > 1e-6 ? sd : 1e-6);
    }
}

cudaError_t launch_feature_norm(const float *x, int B, float *norm, cudaStream_t s)
{
    feature_norm_kernel<<<kMlpIn, kNormThreads, 0, s>>>(x, B, norm);
    return cudaGetLastError();
}

}  // namespace rtk
