// Seeded synthetic nuclei tiles generated on the GPU.
//
// The same integer definition as the Python generator (synth/__init__.py):
// Philox4x32-10 draws (Salmon, Moraes, Dror, Shaw, SC 2011), integer
// lattice-noise background, integer ellipse / disk inclusion tests, and an
// Irwin-Hall noise of twelve 3-bit fields. Every step is exact integer
// arithmetic, so both produce identical bytes for the same parameters. This
// file holds no arithmetic of the segmentation method; it only makes inputs
// (so large training and serving workloads need not be drawn on the host).
#include "common.cuh"
#include "synth.cuh"

namespace rtk {

struct Philox4 {
    uint32_t x[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    Philox4 o;
    o.x[0] = c0;
    o.x[1] = c1;
    o.x[2] = c2;
    o.x[3] = c3;
    return o;
}

__device__ __forceinline__ int64_t umul(uint32_t x, int64_t n) { return (int64_t)(((uint64_t)x * (uint64_t)n) >> 32); }

// lattice nodes of the three octaves: value (x0 >> 21) - 1024 of counter (i, j, octave, 1)
__global__ void synth_lattice_kernel(SynthArgs a, int32_t *lat, int ny0, int nx0, int ny1, int nx1, int ny2, int nx2)
{
    const int tot = ny0 * nx0 + ny1 * nx1 + ny2 * nx2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        int o, i, j;
        if (t < ny0 * nx0) { o = 0; i = t / nx0; j = t % nx0; }
        else if (t < ny0 * nx0 + ny1 * nx1) { const int u = t - ny0 * nx0; o = 1; i = u / nx1; j = u % nx1; }
        else { const int u = t - ny0 * nx0 - ny1 * nx1; o = 2; i = u / nx2; j = u % nx2; }
        const Philox4 x = philox4x32_10((uint32_t)i, (uint32_t)j, (uint32_t)o, 1u, a.k0, a.k1);
        lat[t] = (int32_t)(x.x[0] >> 21) - 1024;
    }
}

// shape layer: minimum intensity over the shapes covering each pixel
__global__ void synth_shape_kernel(SynthArgs a, uint32_t *layer)
{
    for (int k = blockIdx.x; k < a.n_shapes; k += gridDim.x) {
        const Philox4 pa = philox4x32_10((uint32_t)k, 0u, 0u, 0u, a.k0, a.k1);
        const Philox4 pb = philox4x32_10((uint32_t)k, 1u, 0u, 0u, a.k0, a.k1);
        const int64_t cy = umul(pa.x[0], (int64_t)a.H * 16), cx = umul(pa.x[1], (int64_t)a.W * 16);
        const int64_t val = a.vlo + umul(pa.x[2], a.vhi - a.vlo + 1);
        int64_t s2, sa = 0, sb = 0, u = 0, v = 0;
        if (a.kind == 1) {
            s2 = a.rmin * 16 + umul(pa.x[3], (int64_t)(a.rmax - a.rmin) * 16 + 1);
        } else {
            sa = a.amin * 16 + umul(pa.x[3], (int64_t)(a.amax - a.amin) * 16 + 1);
            sb = a.amin * 16 + umul(pb.x[0], (int64_t)(a.amax - a.amin) * 16 + 1);
            u = umul(pb.x[1], 129) - 64;
            v = umul(pb.x[2], 129) - 64;
            if (u == 0 && v == 0) u = 1;
            s2 = sa > sb ? sa : sb;
        }
        const int64_t reach = s2 / 16 + 2;
        const int64_t r0 = max((int64_t)0, cy / 16 - reach), r1 = min((int64_t)a.H, cy / 16 + reach + 1);
        const int64_t c0 = max((int64_t)0, cx / 16 - reach), c1 = min((int64_t)a.W, cx / 16 + reach + 1);
        if (r0 >= r1 || c0 >= c1) continue;
        const int64_t bw = c1 - c0, npx = (r1 - r0) * bw;
        for (int64_t t = threadIdx.x; t < npx; t += blockDim.x) {
            const int64_t r = r0 + t / bw, c = c0 + t % bw;
            const int64_t dy = r * 16 - cy, dx = c * 16 - cx;
            bool inside;
            if (a.kind == 1) {
                inside = dx * dx + dy * dy <= s2 * s2;
            } else {
                const int64_t p = u * dx + v * dy, q = -v * dx + u * dy;
                inside = p * p * (sb * sb) + q * q * (sa * sa) <= (sa * sa) * (sb * sb) * (u * u + v * v);
            }
            if (inside) atomicMin(layer + r * a.W + c, (uint32_t)val);
        }
    }
}

// background + shapes + noise, clipped to uint8
__global__ void synth_pixel_kernel(SynthArgs a, const int32_t *lat, int nx0, int nx1, int nx2, int off1, int off2,
                                   const uint32_t *layer, uint8_t *out, int64_t ld)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.W; c += gridDim.x * blockDim.x) {
        int64_t base;
        if (a.flat) {
            base = 200;
        } else {
            int64_t total = 0;
            const int cells[3] = {512, 256, 128}, weights[3] = {4, 2, 1};
            const int nxs[3] = {nx0, nx1, nx2}, offs[3] = {0, off1, off2};
            for (int o = 0; o < 3; ++o) {
                const int cell = cells[o], nx = nxs[o];
                const int i0 = r / cell, ty = r % cell, j0 = c / cell, tx = c % cell;
                const int32_t *L = lat + offs[o];
                const int64_t row0 = (int64_t)L[i0 * nx + j0] * (cell - tx) + (int64_t)L[i0 * nx + j0 + 1] * tx;
                const int64_t row1 = (int64_t)L[(i0 + 1) * nx + j0] * (cell - tx) + (int64_t)L[(i0 + 1) * nx + j0 + 1] * tx;
                const int64_t val = row0 * (cell - ty) + row1 * ty;
                const int64_t scale = (int64_t)(512 / cell) * (512 / cell);
                total += weights[o] * scale * val;
            }
            const int64_t den = (int64_t)7 * 1024 * 512 * 512, num = 15 * total;
            const int64_t q = num >= 0 ? (num + den / 2) / den : -((-num + den / 2) / den);
            base = 200 + q;
        }
        int64_t v = min(base, (int64_t)layer[(int64_t)r * a.W + c]);
        if (a.noise) {
            const int64_t p = (int64_t)r * a.W + c;
            const Philox4 x = philox4x32_10((uint32_t)(p >> 1), 0u, 0u, 2u, a.k0, a.k1);
            const uint32_t lo = (p & 1) ? x.x[2] : x.x[0];
            const uint32_t hi = (p & 1) ? x.x[3] : x.x[1];
            int acc = 0;
#pragma unroll
            for (int f = 0; f < 10; ++f) acc += (lo >> (3 * f)) & 7u;
            acc += (hi & 7u) + ((hi >> 3) & 7u);
            v += acc - 42;
        }
        out[(int64_t)r * ld + c] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
    }
}

size_t synth_workspace_bytes(int H, int W)
{
    const int n0 = (H / 512 + 2) * (W / 512 + 2), n1 = (H / 256 + 2) * (W / 256 + 2), n2 = (H / 128 + 2) * (W / 128 + 2);
    return (size_t)H * W * sizeof(uint32_t) + (size_t)(n0 + n1 + n2) * sizeof(int32_t) + 512;
}

cudaError_t launch_synth(const SynthArgs &a, void *ws, uint8_t *out, int64_t ld, cudaStream_t s)
{
    uint32_t *layer = static_cast<uint32_t *>(ws);
    int32_t *lat = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + round_up((int64_t)a.H * a.W * 4, 256));
    const int ny0 = a.H / 512 + 2, nx0 = a.W / 512 + 2, ny1 = a.H / 256 + 2, nx1 = a.W / 256 + 2;
    const int ny2 = a.H / 128 + 2, nx2 = a.W / 128 + 2;
    cudaError_t e = cudaMemsetAsync(layer, 0xFF, (size_t)a.H * a.W * sizeof(uint32_t), s);   // >= 255
    if (e != cudaSuccess) return e;
    if (!a.flat) {
        synth_lattice_kernel<<<64, 256, 0, s>>>(a, lat, ny0, nx0, ny1, nx1, ny2, nx2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.n_shapes > 0) {
        synth_shape_kernel<<<(unsigned)(a.n_shapes < 4096 ? a.n_shapes : 4096), 256, 0, s>>>(a, layer);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    synth_pixel_kernel<<<dim3((unsigned)ceil_div(a.W, 256), (unsigned)a.H), 256, 0, s>>>(
        a, lat, nx0, nx1, nx2, ny0 * nx0, ny0 * nx0 + ny1 * nx1, layer, out, ld);
    return cudaGetLastError();
}

}  // namespace rtk
