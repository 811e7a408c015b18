// Allocation-free entry point for the squared EDT (rt_edt_noalloc in rt.h).
//
// The regular entry points keep their scratch in a context workspace that
// grows with cudaMalloc. This one keeps it in a fixed array compiled into
// the library, so a call never allocates device memory. The array lives in
// every GPU that loads the library until the process exits.
#include <mutex>

#include "edt.cuh"

namespace {

constexpr int64_t kNoAllocMaxPixels = int64_t(1) << 20;      // H * W limit
constexpr size_t kDistBytes = (size_t)kNoAllocMaxPixels * sizeof(uint16_t);
// segment summaries: 2 * ceil(H / 32) * W int32 values take at most
// H*W/4 + 8*W bytes, which is at most 512 KiB for H * W <= 2^20, W <= 32768
constexpr size_t kSegBytes = size_t(512) << 10;
constexpr size_t kScratchBytes = kDistBytes + kSegBytes + 256;
constexpr int kMaxDevices = 64;

// Shared by every call on a device: contents persist between calls.
static __device__ __align__(256) unsigned char g_edt_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
void *scratch_on_current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_edt_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" rt_status rt_edt_noalloc(const uint8_t *fg, int64_t ld_fg, int32_t *d2, int64_t ld_d2, int H, int W,
                                    int32_t *dev_status, void *stream)
{
    if (!fg || !d2 || H < 1 || W < 1 || H > rtk::kMaxSide || W > rtk::kMaxSide || ld_fg < W || ld_d2 < W)
        return RT_EINVAL;
    if (overlaps(fg, ((size_t)(H - 1) * ld_fg + W), d2, ((size_t)(H - 1) * ld_d2 + W) * 4)) return RT_EINVAL;
    if ((int64_t)H * W > kNoAllocMaxPixels) return RT_ESIZE;
    const size_t seg_bytes = (size_t)2 * rtk::ceil_div(H, 32) * W * sizeof(int32_t);
    if (seg_bytes > kSegBytes) return RT_ESIZE;
    char *base = static_cast<char *>(scratch_on_current_device());
    if (!base) return RT_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    rtk::EdtArgs a;
    a.fg8 = fg;
    a.lab32 = nullptr;
    a.ld_in = ld_fg;
    a.H = H;
    a.W = W;
    a.d2 = d2;
    a.ld_d2 = ld_d2;
    a.g = reinterpret_cast<uint16_t *>(base);
    a.seg = reinterpret_cast<int32_t *>(base + kDistBytes);
    a.any_bg = reinterpret_cast<uint32_t *>(base + kDistBytes + kSegBytes);   // cleared by launch_edt
    if (dev_status && cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return RT_ECUDA;
    }
    if (rtk::launch_edt(a, s) != cudaSuccess) {
        cudaGetLastError();
        return RT_ECUDA;
    }
    return RT_OK;
}
