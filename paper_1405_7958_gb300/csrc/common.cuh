// Shared device helpers of the segmentation kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"

#define RT_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return RT_ECUDA;             \
    } while (0)

namespace rtk {

constexpr int kMaxSide = 32768;

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int32_t ld_relaxed_i32(const int32_t *p)
{
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Record the first error code raised on the device (0 = RT_OK stays until an
// error arrives). Never traps.
__device__ __forceinline__ void raise_status(int32_t *st, int code)
{
    if (st) atomicCAS(st, 0, code);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// bar[0] = arrival count, bar[1] = generation. The wait is bounded by
// `timeout_ns`; on expiry the CTA records RT_ETIMEOUT in *err and returns
// false so the caller can leave the loop.
__device__ __forceinline__ bool grid_barrier(uint32_t *bar, uint32_t nblocks, int32_t *err,
                                             uint64_t timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        uint32_t gen = ld_acquire(bar + 1);
        __threadfence();
        uint32_t arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            while (ld_acquire(bar + 1) == gen) {
                if (++spins > 64) __nanosleep(64);
                if ((spins & 255u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
                    raise_status(err, RT_ETIMEOUT);
                    s_ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

}  // namespace rtk
