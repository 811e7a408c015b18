// The learned variant picker's MLP (see mlp.cu).
#pragma once

#include "common.cuh"

namespace rtk {

constexpr int kMlpIn = 24, kMlpH = 64, kMlpOut = 3;
// flat parameter vector: W1[64][24] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]
constexpr int kW1 = 0;
constexpr int kB1 = kW1 + kMlpH * kMlpIn;
constexpr int kW2 = kB1 + kMlpH;
constexpr int kB2 = kW2 + kMlpH * kMlpH;
constexpr int kW3 = kB2 + kMlpH;
constexpr int kB3 = kW3 + kMlpOut * kMlpH;
constexpr int kMlpParams = kB3 + kMlpOut;                 // 5955
constexpr int kMlpAct = 2 * kMlpH;                        // saved h1, h2 per sample
constexpr int kMlpDelta = kMlpOut + 2 * kMlpH + kMlpIn + 1;   // dz, dh2, dh1, xn, loss per sample

// The network on one sample by one warp, in a fixed order of operations
// (every caller gets the same bits): the parameters staged as fp32 in shared
// memory P (bf16 -> fp32 is exact), the normalised input xn; lanes own the
// hidden units j and j + 32 (h[0] = h1, h[1] = h2, shared); lane 0 forms the
// logits and the pick.
__device__ __forceinline__ void mlp_stage_params(const uint16_t *wb, float *P)
{
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) P[i] = __uint_as_float((uint32_t)wb[i] << 16);
}

__device__ __forceinline__ void mlp_warp_hidden(const float *P, const float *xn, float (*h)[kMlpH], int lane)
{
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = lane + 32 * q;
        float s = P[kB1 + j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) s = fmaf(P[kW1 + j * kMlpIn + i], xn[i], s);
        h[0][j] = fmaxf(s, 0.f);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = lane + 32 * q;
        float s = P[kB2 + j];
#pragma unroll 8
        for (int i = 0; i < kMlpH; ++i) s = fmaf(P[kW2 + j * kMlpH + i], h[0][i], s);
        h[1][j] = fmaxf(s, 0.f);
    }
    __syncwarp();
}

// lane 0: logits z from h2, and the argmax or `fallback` where its softmax
// probability is below min_prob
__device__ __forceinline__ int mlp_logits_pick(const float *P, const float *h2, float *z, float min_prob, int fallback)
{
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) z[k] = P[kB3 + k];
    for (int j = 0; j < kMlpH; ++j) {
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) z[k] = fmaf(P[kW3 + k * kMlpH + j], h2[j], z[k]);
    }
    int best = 0;
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k)
        if (z[k] > z[best]) best = k;
    if (min_prob > 0.f) {
        float se = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) se += expf(z[k] - z[best]);
        if (1.f / se < min_prob) best = fallback;
    }
    return best;
}

// pick = argmax of the logits, or `fallback` where the argmax's softmax
// probability is below min_prob (min_prob <= 0: never)
cudaError_t launch_mlp_forward(const uint16_t *wb, const float *norm, const float *x, int B, float *logits, float *act,
                               int32_t *pick, float min_prob, int fallback, cudaStream_t s);
// the same forward on the tensor cores (mlp_tc.cu): bf16 operands (the
// normalised input and the hidden layers rounded to bf16), fp32 accumulation
// in tensor memory, 128 samples per CTA; err (nullable) gets RT_ETIMEOUT if a
// product does not complete within its wait bound
cudaError_t launch_mlp_forward_tc(const uint16_t *wb, const float *norm, const float *x, int B, float *logits,
                                  float *act, int32_t *pick, float min_prob, int fallback, int32_t *err,
                                  cudaStream_t s);
size_t mlp_backward_workspace_bytes(int B);
// the backward on the tensor cores (mlp_tc.cu): dh1 and the W1, b1, W2, b2
// gradients as bf16 products with fp32 accumulation, W3 and b3 in fp32;
// deterministic (fixed-order sums of per-CTA partials)
size_t mlp_backward_tc_workspace_bytes(int B);
cudaError_t launch_mlp_backward_tc(const uint16_t *wb, const float *norm, const float *x, const float *act,
                                   const float *logits, const int32_t *label, int B, float *grad, float *loss,
                                   float *ws, int32_t *err, cudaStream_t s);
cudaError_t launch_mlp_backward(const uint16_t *wb, const float *norm, const float *x, const float *act,
                                const float *logits, const int32_t *label, int B, float *grad, float *loss, float *ws,
                                cudaStream_t s);
// norm = (mean[24], std[24]) of the columns of x (B x 24): the mean, and the
// sample standard deviation (divisor B - 1; 0 for B = 1) clamped below at
// 1e-6; sums in double in a fixed order (deterministic)
cudaError_t launch_feature_norm(const float *x, int B, float *norm, cudaStream_t s);
cudaError_t launch_mlp_adamw(float *master, uint16_t *wb, const float *grad, float *m, float *v, int step, float lr,
                             float b1, float b2, float eps, float wd, cudaStream_t s);

}  // namespace rtk
