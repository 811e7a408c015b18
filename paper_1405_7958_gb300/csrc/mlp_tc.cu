// The picker network's forward pass on the 5th-generation tensor cores
// (tcgen05), for training batches.
//
// One CTA of 128 threads takes 128 samples: the M = 128 rows of three
// products whose accumulators live in tensor memory,
//   H1 = Xn W1^T (K = 24, padded to 32),  H2 = relu(H1 + b1) W2^T (K = 64),
//   Z  = relu(H2 + b2) W3^T (N = 3, padded to 16),
// with bf16 operands (the parameters are bf16 already; the normalised input
// and the two hidden layers are rounded to bf16 to enter a product) and fp32
// accumulation. Thread t owns sample t: it writes row t of each A operand
// and reads row t (tensor-memory lane t) of each accumulator. One thread
// issues the products; their completion arrives on an mbarrier.
//
// Operands sit in shared memory in the no-swizzle K-major layout of 8-row x
// 16-byte core matrices: element (r, k) of a K-wide operand is at
//   (r / 8) * (K / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// bytes, so core matrices are 128 bytes apart along K (leading byte offset)
// and K * 16 bytes apart along M or N (stride byte offset).
#include <cuda_bf16.h>

#include "mlp.cuh"

namespace rtk {
namespace {

constexpr int kTcM = 128;       // samples per CTA = tensor-memory lanes
constexpr int kK1 = 32;         // layer 1 K: 24 inputs, zero-padded
constexpr int kN3 = 16;         // layer 3 N: 3 outputs, zero-padded
constexpr int kTmemCols = 256;  // H1 at columns 0..63, H2 at 64..127, Z at 128..143

// shared memory (bytes): the three A operands share one buffer in turn
constexpr int kOffA = 0;                          // 128 x 64 bf16 (layer 1 uses 128 x 32)
constexpr int kOffB1 = kOffA + kTcM * kMlpH * 2;  // 64 x 32
constexpr int kOffB2 = kOffB1 + kMlpH * kK1 * 2;  // 64 x 64
constexpr int kOffB3 = kOffB2 + kMlpH * kMlpH * 2;   // 16 x 64
constexpr int kOffEnd = kOffB3 + kN3 * kMlpH * 2;
constexpr int kTcSmem = kOffEnd;

__device__ __forceinline__ uint32_t core_off(int r, int k, int K)
{
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading byte offset (128:
// next core matrix along K), stride byte offset (K * 16: next 8 rows), the
// descriptor version bit of this architecture, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int K)
{
    const uint64_t lbo = 128, sbo = (uint64_t)K * 16;
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N and M
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// waits for the mbarrier phase `parity` to complete; false after the bound
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (uint32_t k = 0; k < (1u << 22); ++k) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (k > 64) __nanosleep(32);
    }
    return false;
}

// 16 consecutive fp32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint16_t to_bf16(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }

// ReLU(acc + bias) of 64 accumulator columns starting at `col`: saved in fp32
// (act) and written as this thread's bf16 row of the next A operand
__device__ __forceinline__ void hidden_row(uint32_t tbase, int col, const uint16_t *wb, int bias, uint8_t *A, int row,
                                           float *act_row)
{
#pragma unroll
    for (int q = 0; q < kMlpH / 16; ++q) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)(col + 16 * q), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = 16 * q + i;
            const float h = fmaxf(v[i] + __uint_as_float((uint32_t)wb[bias + j] << 16), 0.f);
            if (act_row) act_row[j] = h;
            *reinterpret_cast<uint16_t *>(A + core_off(row, j, kMlpH)) = to_bf16(h);
        }
    }
}

__global__ void __launch_bounds__(kTcM) mlp_forward_tc_kernel(const uint16_t *wb, const float *norm, const float *x,
                                                              int B, float *logits, float *act, int32_t *pick,
                                                              float min_prob, int fallback, int32_t *err)
{
    __shared__ __align__(1024) uint8_t sm[kTcSmem];
    __shared__ __align__(8) uint64_t mbar_store;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    const int b = blockIdx.x * kTcM + t;
    const bool live = b < B;
    uint8_t *A = sm + kOffA;
    const uint32_t mbar = smem_u32(&mbar_store);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B operands (the parameters, zero-padded) and this thread's row of the
    // layer-1 A operand (the normalised input, zero-padded)
    for (int i = t; i < kMlpH * kK1; i += kTcM) {
        const int n = i / kK1, k = i % kK1;
        *reinterpret_cast<uint16_t *>(sm + kOffB1 + core_off(n, k, kK1)) = k < kMlpIn ? wb[kW1 + n * kMlpIn + k] : 0;
    }
    for (int i = t; i < kMlpH * kMlpH; i += kTcM) {
        const int n = i / kMlpH, k = i % kMlpH;
        *reinterpret_cast<uint16_t *>(sm + kOffB2 + core_off(n, k, kMlpH)) = wb[kW2 + n * kMlpH + k];
    }
    for (int i = t; i < kN3 * kMlpH; i += kTcM) {
        const int n = i / kMlpH, k = i % kMlpH;
        *reinterpret_cast<uint16_t *>(sm + kOffB3 + core_off(n, k, kMlpH)) = n < kMlpOut ? wb[kW3 + n * kMlpH + k] : 0;
    }
#pragma unroll
    for (int k = 0; k < kK1; ++k) {
        float v = 0.f;
        if (live && k < kMlpIn) v = (x[(int64_t)b * kMlpIn + k] - norm[k]) / norm[kMlpIn + k];
        *reinterpret_cast<uint16_t *>(A + core_off(t, k, kK1)) = to_bf16(v);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's 32 lanes
    const uint32_t aaddr = smem_u32(A);
    bool ok = true;

    // layer 1: H1 = Xn W1^T, two K = 16 steps
    if (t == 0) {
        for (int s = 0; s < kK1 / 16; ++s)
            mma_bf16(tmem, smem_desc(aaddr + 256 * s, kK1), smem_desc(smem_u32(sm + kOffB1) + 256 * s, kK1),
                     instr_desc(kTcM, kMlpH), s > 0);
        mma_commit(mbar);
    }
    ok = mbar_wait(mbar, 0) && ok;
    tc_after_sync();
    hidden_row(tlane, 0, wb, kB1, A, t, live && act ? act + (int64_t)b * kMlpAct : nullptr);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();

    // layer 2: H2 = relu(H1 + b1) W2^T, four K = 16 steps
    if (t == 0 && ok) {
        for (int s = 0; s < kMlpH / 16; ++s)
            mma_bf16(tmem + kMlpH, smem_desc(aaddr + 256 * s, kMlpH), smem_desc(smem_u32(sm + kOffB2) + 256 * s, kMlpH),
                     instr_desc(kTcM, kMlpH), s > 0);
        mma_commit(mbar);
    }
    ok = ok && mbar_wait(mbar, 1);
    tc_after_sync();
    hidden_row(tlane, kMlpH, wb, kB2, A, t, live && act ? act + (int64_t)b * kMlpAct + kMlpH : nullptr);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();

    // layer 3: Z = relu(H2 + b2) W3^T, N padded to 16
    if (t == 0 && ok) {
        for (int s = 0; s < kMlpH / 16; ++s)
            mma_bf16(tmem + 2 * kMlpH, smem_desc(aaddr + 256 * s, kMlpH),
                     smem_desc(smem_u32(sm + kOffB3) + 256 * s, kMlpH), instr_desc(kTcM, kN3), s > 0);
        mma_commit(mbar);
    }
    ok = ok && mbar_wait(mbar, 0);
    tc_after_sync();
    float zv[16];
    tmem_ld16(tlane + 2 * kMlpH, zv);
    tc_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (!ok) {
        if (t == 0) raise_status(err, RT_ETIMEOUT);
        return;
    }
    if (!live) return;
    float z[kMlpOut];
    int best = 0;
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) {
        z[k] = zv[k] + __uint_as_float((uint32_t)wb[kB3 + k] << 16);
        if (logits) logits[(int64_t)b * kMlpOut + k] = z[k];
        if (z[k] > z[best]) best = k;
    }
    if (min_prob > 0.f) {
        float se = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) se += expf(z[k] - z[best]);
        if (1.f / se < min_prob) best = fallback;
    }
    if (pick) pick[b] = best;
}

// Backward on the tensor cores, 128 samples per CTA (thread t: sample t).
//   dz  = (softmax(z) - onehot(label)) / B               (fp32, per thread)
//   dh2 = (dz W3) * [h2 > 0]                              (fp32, per thread: K = 3)
//   dh1 = (dh2 W2) * [h1 > 0]                             (product 1: 128 x 64, K = 64)
//   [dW2 db2; dW1 db1] from [dh2 | dh1]^T [h1 | xn | 1]   (product 2: M = 128
//                                                          features, N = 96, K = 128 samples)
// Product 2 stacks both weight gradients in one M = 128 accumulator: rows
// 0..63 are dh2's features against h1 (dW2) and a column of ones (db2), rows
// 64..127 dh1's features against xn (dW1) and the ones (db1); the two mixed
// blocks are not read. Each CTA writes its partial sums of W1, b1, W2, b2
// and its samples' dz and loss; a second kernel adds the partials of the
// CTAs in a fixed order and forms W3 and b3 from dz and h2 (fp32), so the
// result is deterministic.
constexpr int kBwN2 = 96;                           // product 2 N: h1 (64) | xn (24) | ones | pad
constexpr int kBwOne = kMlpH + kMlpIn;              // the ones column (88)
constexpr int kBwA1 = 0;                            // 128 x 64: dh2 (product 1 A)
constexpr int kBwB1 = kBwA1 + kTcM * kMlpH * 2;     // 64 x 64: W2^T
constexpr int kBwA2 = kBwB1 + kMlpH * kMlpH * 2;    // 128 x 128: [dh2 | dh1]^T
constexpr int kBwB2 = kBwA2 + kTcM * kTcM * 2;      // 96 x 128: [h1 | xn | 1]^T
constexpr int kBwSmem = kBwB2 + kBwN2 * kTcM * 2;   // 73728 bytes (dynamic)
constexpr int kBwPart = kW3;                        // partial sums per CTA: W1 b1 W2 b2

__global__ void __launch_bounds__(kTcM) mlp_backward_tc_kernel(const uint16_t *wb, const float *norm, const float *x,
                                                               const float *act, const float *logits,
                                                               const int32_t *label, int B, float *part, float *dz_out,
                                                               float *loss_out, int32_t *err)
{
    extern __shared__ __align__(1024) uint8_t smb[];
    __shared__ __align__(8) uint64_t mbar_store;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    const int b = blockIdx.x * kTcM + t;
    const bool live = b < B;
    const uint32_t mbar = smem_u32(&mbar_store);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // W2^T as product 1's B: B[n][k] = W2[k][n]
    for (int i = t; i < kMlpH * kMlpH; i += kTcM) {
        const int n = i % kMlpH, k = i / kMlpH;
        *reinterpret_cast<uint16_t *>(smb + kBwB1 + core_off(n, k, kMlpH)) = wb[kW2 + k * kMlpH + n];
    }
    // this sample's deltas of the output and the second hidden layer (fp32)
    float h2[kMlpH], dz[kMlpOut];
    float lossb = 0.f;
    if (live) {
        const float *z = logits + (int64_t)b * kMlpOut;
        float m = z[0];
#pragma unroll
        for (int k = 1; k < kMlpOut; ++k) m = fmaxf(m, z[k]);
        float se = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) se += expf(z[k] - m);
        const int y = label[b];
        lossb = logf(se) + m - z[y];
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) {
            dz[k] = (expf(z[k] - m) / se - (k == y ? 1.f : 0.f)) / (float)B;
            dz_out[(int64_t)b * kMlpOut + k] = dz[k];
        }
        loss_out[b] = lossb;
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) h2[j] = act[(int64_t)b * kMlpAct + kMlpH + j];
    } else {
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) dz[k] = 0.f;
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) h2[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) s = fmaf(__uint_as_float((uint32_t)wb[kW3 + k * kMlpH + j] << 16), dz[k], s);
        const uint16_t d = to_bf16(h2[j] > 0.f ? s : 0.f);
        *reinterpret_cast<uint16_t *>(smb + kBwA1 + core_off(t, j, kMlpH)) = d;     // row t of product 1's A
        *reinterpret_cast<uint16_t *>(smb + kBwA2 + core_off(j, t, kTcM)) = d;      // column t of product 2's A
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
    bool ok = true;
    if (t == 0) {
        for (int s = 0; s < kMlpH / 16; ++s)
            mma_bf16(tmem, smem_desc(smem_u32(smb + kBwA1) + 256 * s, kMlpH),
                     smem_desc(smem_u32(smb + kBwB1) + 256 * s, kMlpH), instr_desc(kTcM, kMlpH), s > 0);
        mma_commit(mbar);
    }
    // meanwhile: column t of product 2's B (h1, xn and a one, as bf16)
    {
        float xn[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) xn[k] = live ? (x[(int64_t)b * kMlpIn + k] - norm[k]) / norm[kMlpIn + k] : 0.f;
#pragma unroll
        for (int n = 0; n < kBwN2; ++n) {
            float v = 0.f;
            if (live) {
                if (n < kMlpH) v = act[(int64_t)b * kMlpAct + n];
                else if (n < kBwOne) v = xn[n - kMlpH];
                else if (n == kBwOne) v = 1.f;
            }
            *reinterpret_cast<uint16_t *>(smb + kBwB2 + core_off(n, t, kTcM)) = to_bf16(v);
        }
    }
    ok = mbar_wait(mbar, 0) && ok;
    tc_after_sync();
    // dh1 = (dh2 W2) * [h1 > 0]: column t of product 2's A, rows 64..127
#pragma unroll
    for (int q = 0; q < kMlpH / 16; ++q) {
        float v[16];
        tmem_ld16(tlane + (uint32_t)(16 * q), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = 16 * q + i;
            const bool on = live && act[(int64_t)b * kMlpAct + j] > 0.f;
            *reinterpret_cast<uint16_t *>(smb + kBwA2 + core_off(kMlpH + j, t, kTcM)) = to_bf16(on ? v[i] : 0.f);
        }
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (t == 0 && ok) {
        for (int s = 0; s < kTcM / 16; ++s)
            mma_bf16(tmem + kMlpH, smem_desc(smem_u32(smb + kBwA2) + 256 * s, kTcM),
                     smem_desc(smem_u32(smb + kBwB2) + 256 * s, kTcM), instr_desc(kTcM, kBwN2), s > 0);
        mma_commit(mbar);
    }
    ok = ok && mbar_wait(mbar, 1);
    tc_after_sync();
    // row t of product 2: feature t of dh2 (t < 64) or of dh1 (t >= 64)
    float *pc = part + (int64_t)blockIdx.x * kBwPart;
    if (warp < 2) {
#pragma unroll
        for (int q = 0; q < kMlpH / 16; ++q) {
            float v[16];
            tmem_ld16(tlane + kMlpH + (uint32_t)(16 * q), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) pc[kW2 + t * kMlpH + 16 * q + i] = v[i];
        }
        float v[16];
        tmem_ld16(tlane + kMlpH + 80, v);
        pc[kB2 + t] = v[kBwOne - 80];
    } else {
        const int i1 = t - kMlpH;
        float v[16];
        tmem_ld16(tlane + kMlpH + 64, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) pc[kW1 + i1 * kMlpIn + i] = v[i];
        tmem_ld16(tlane + kMlpH + 80, v);
#pragma unroll
        for (int i = 0; i < kMlpIn - 16; ++i) pc[kW1 + i1 * kMlpIn + 16 + i] = v[i];
        pc[kB1 + i1] = v[kBwOne - 80];
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (!ok && t == 0) raise_status(err, RT_ETIMEOUT);
}

// the gradient, one warp per parameter: W1, b1, W2, b2 as the sum of the
// CTAs' partials, W3 and b3 over the samples from dz and h2 (fp32); the last
// warp sums the loss. Lane l adds the terms l, l + 32, ... in order, then a
// fixed butterfly adds the lanes, so the result does not depend on
// scheduling.
__global__ void mlp_grad_tc_kernel(const float *part, int nblk, const float *dz, const float *act, const float *lossb,
                                   int B, float *grad, float *loss)
{
    const int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (p > kMlpParams) return;
    float s = 0.f;
    if (p == kMlpParams) {
        for (int b = lane; b < B; b += 32) s += lossb[b];
    } else if (p < kW3) {
        for (int k = lane; k < nblk; k += 32) s += part[(int64_t)k * kBwPart + p];
    } else if (p < kB3) {
        const int k = (p - kW3) / kMlpH, j = (p - kW3) % kMlpH;
        for (int b = lane; b < B; b += 32)
            s = fmaf(dz[(int64_t)b * kMlpOut + k], act[(int64_t)b * kMlpAct + kMlpH + j], s);
    } else {
        for (int b = lane; b < B; b += 32) s += dz[(int64_t)b * kMlpOut + (p - kB3)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0) return;
    if (p == kMlpParams) {
        if (loss) *loss = s / (float)B;
    } else {
        grad[p] = s;
    }
}

}  // namespace

size_t mlp_backward_tc_workspace_bytes(int B)
{
    const int64_t nblk = ceil_div(B, kTcM);
    return sizeof(float) * (size_t)(nblk * kBwPart + (int64_t)B * (kMlpOut + 1));
}

cudaError_t launch_mlp_backward_tc(const uint16_t *wb, const float *norm, const float *x, const float *act,
                                   const float *logits, const int32_t *label, int B, float *grad, float *loss,
                                   float *ws, int32_t *err, cudaStream_t s)
{
    if (B <= 0) return cudaErrorInvalidValue;
    const int nblk = (int)ceil_div(B, kTcM);
    float *part = ws;
    float *dz = part + (int64_t)nblk * kBwPart;
    float *lossb = dz + (int64_t)B * kMlpOut;
    cudaError_t e = cudaFuncSetAttribute(mlp_backward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwSmem);
    if (e != cudaSuccess) return e;
    mlp_backward_tc_kernel<<<nblk, kTcM, kBwSmem, s>>>(wb, norm, x, act, logits, label, B, part, dz, lossb, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    mlp_grad_tc_kernel<<<(unsigned)ceil_div((int64_t)(kMlpParams + 1) * 32, 256), 256, 0, s>>>(part, nblk, dz, act,
                                                                                               lossb, B, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward_tc(const uint16_t *wb, const float *norm, const float *x, int B, float *logits,
                                  float *act, int32_t *pick, float min_prob, int fallback, int32_t *err,
                                  cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    mlp_forward_tc_kernel<<<(unsigned)ceil_div(B, kTcM), kTcM, 0, s>>>(wb, norm, x, B, logits, act, pick, min_prob,
                                                                       fallback, err);
    return cudaGetLastError();
}

}  // namespace rtk
