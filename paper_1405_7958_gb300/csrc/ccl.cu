// BWLabel (Section 5.1) and FillHoles (Sections 3.2.1, 5.1) by union-find.
//
// The paper's BWLabel follows the union-find pattern: every pixel starts as
// its own tree, trees of adjacent foreground pixels are merged, and labels
// are read off by flattening the trees. Merging always hooks the root with
// the larger linear index under the smaller one (atomicMin on the parent),
// so the root of a finished tree is the smallest index of its component:
// the canonical label. The forest is built in two levels:
//   1. each 32 x 32 block merges its own pixels in shared memory and writes
//      for every pixel the (global) index of its block-local root;
//   2. pixel pairs that straddle a block edge are merged in global memory;
//   3. flattening points every pixel at its final root and accumulates, per
//      root, the component area (labeling) or whether the component touches
//      the image border (hole filling: the background components are built
//      and the ones that do not touch the border are holes).
#include "ccl.cuh"

namespace rtk {

constexpr int kB = 32;          // block side
constexpr int kRowsPerThread = 4;

__device__ __forceinline__ bool is_fg(const uint8_t *in, int64_t ld, int r, int c, int source)
{
    const uint8_t v = in[(int64_t)r * ld + c];
    return source == kFgNonzero ? v != 0 : v == 0;
}

// --------------------------------------------------- shared-memory forest
// Finds that run while unions are still hooking roots only read; path
// halving (every visited node pointed at its grandparent) is used only
// after all unions of the forest have finished.
__device__ __forceinline__ int find_s(volatile int *P, int x)
{
    int p = P[x];
    while (p != x) {
        x = p;
        p = P[x];
    }
    return x;
}

__device__ __forceinline__ int find_s_halve(volatile int *P, int x)
{
    int p = P[x];
    while (p != x) {
        const int gp = P[p];
        if (gp != p) P[x] = gp;
        x = gp;
        p = P[x];
    }
    return x;
}

__device__ __forceinline__ void union_s(int *P, int a, int b)
{
    volatile int *VP = P;
    for (;;) {
        a = find_s(VP, a);
        b = find_s(VP, b);
        if (a == b) return;
        if (a < b) {
            const int t = a; a = b; b = t;
        }
        // a > b: hook a under b
        const int old = atomicMin(P + a, b);
        if (old == a) return;
        a = old;
    }
}

// ---------------------------------------------------- global forest
__device__ __forceinline__ int32_t find_g(const int32_t *U, int32_t x)
{
    int32_t p = ld_relaxed_i32(U + x);
    while (p != x) {
        x = p;
        p = ld_relaxed_i32(U + x);
    }
    return x;
}

// Path halving for the flatten pass (after every union is done). Other
// threads store final roots into the same nodes meanwhile; since every
// ancestor has a smaller index than its descendants and the root is the
// smallest of all, the halving store is an atomicMin, so no node can move
// back from its root to a lower ancestor.
__device__ __forceinline__ int32_t find_g_halve(int32_t *U, int32_t x)
{
    int32_t p = ld_relaxed_i32(U + x);
    while (p != x) {
        const int32_t gp = ld_relaxed_i32(U + p);
        if (gp != p) atomicMin(U + x, gp);
        x = gp;
        p = ld_relaxed_i32(U + x);
    }
    return x;
}

__device__ __forceinline__ void union_g(int32_t *U, int32_t a, int32_t b)
{
    for (;;) {
        a = find_g(U, a);
        b = find_g(U, b);
        if (a == b) return;
        if (a < b) {
            const int32_t t = a; a = b; b = t;
        }
        const int32_t old = atomicMin(U + a, b);
        if (old == a) return;
        a = old;
    }
}

// 1. block-local forests. Block of 32 x 32 pixels, 8 warps; warp w owns rows
// 4w .. 4w+3 and lane = column. Inside a row, a run of foreground pixels
// is one tree from the start: every pixel points at the run's first pixel
// (found from the row's ballot mask). Rows are then joined with one union per
// pair of touching runs: for 4-connectivity at the first column where the
// runs overlap; for 8-connectivity the first pixel of a run joins each run of
// the row above that starts within its three upper neighbours, and any other
// pixel joins only a run of the row above that starts at its upper-right
// neighbour.
template <int CONN>
__global__ void __launch_bounds__(256) uf_local_kernel(UfArgs a, int source, bool zero_acc)
{
    __shared__ int P[kB * kB];
    __shared__ uint32_t M[kB];
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = blockIdx.y * kB, c0 = blockIdx.x * kB;
    const int c = c0 + tx;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int lr = w * kRowsPerThread + k;
        const int r = r0 + lr;
        const bool f = (r < a.H && c < a.W) && is_fg(a.in, a.ld_in, r, c, source);
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        const uint32_t starts = m & ~(m << 1);
        if (tx == 0) M[lr] = m;
        int v = -1;
        if (f) v = lr * kB + (31 - __clz(starts & (0xffffffffu >> (31 - tx))));
        P[lr * kB + tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int lr = w * kRowsPerThread + k;
        if (lr == 0) continue;
        const uint32_t m = M[lr], up = M[lr - 1];
        if (!((m >> tx) & 1u)) continue;
        const int i = lr * kB + tx;
        const bool fl = tx > 0 && ((m >> (tx - 1)) & 1u);
        const bool uc = (up >> tx) & 1u;
        const bool ul = tx > 0 && ((up >> (tx - 1)) & 1u);
        if (CONN == 4) {
            if (uc && !(fl && ul)) union_s(P, i, i - kB);
        } else {
            const bool ur = tx < kB - 1 && ((up >> (tx + 1)) & 1u);
            if (!fl) {
                if (ul) union_s(P, i, i - kB - 1);
                if (uc && !ul) union_s(P, i, i - kB);
                if (ur && !uc) union_s(P, i, i - kB + 1);
            } else if (ur && !uc) {
                union_s(P, i, i - kB + 1);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int lr = w * kRowsPerThread + k;
        const int r = r0 + lr;
        const int i = lr * kB + tx;
        const int root = P[i] >= 0 ? find_s_halve(P, i) : -1;
        if (r >= a.H || c >= a.W) continue;
        const int64_t p = (int64_t)r * a.W + c;
        int32_t g = -1;
        if (root >= 0) {
            g = (int32_t)((int64_t)(r0 + root / kB) * a.W + (c0 + root % kB));
            if (zero_acc && root == i) a.A[p] = 0;
        }
        a.U[p] = g;
    }
}

// 2. merges across block edges, one CTA of 96 threads per block: threads
// 0..31 the top row (with the row above), 32..63 the left column (with the
// column to the left), 64..95 the right column (up-right neighbours, 8 only).
// Pixels adjacent along the same block row or column are already in one
// block-local tree, so along an edge only the first pixel pair of each pair
// of touching runs needs a union; the others are skipped.
template <int CONN>
__global__ void __launch_bounds__(96) uf_border_kernel(UfArgs a, int source)
{
    const int r0 = blockIdx.y * kB, c0 = blockIdx.x * kB;
    const int pos = threadIdx.x;
    auto fg = [&](int r, int c) { return r >= 0 && c >= 0 && r < a.H && c < a.W && is_fg(a.in, a.ld_in, r, c, source); };
    if (pos < 32) {
        const int r = r0, c = c0 + pos;
        if (r == 0 || c >= a.W || !fg(r, c)) return;
        const int32_t p = (int32_t)((int64_t)r * a.W + c);
        const bool left_in = pos > 0 && fg(r, c - 1);          // same block row
        const bool right_in = pos < 31 && fg(r, c + 1);
        if (fg(r - 1, c) && !(left_in && fg(r - 1, c - 1))) union_g(a.U, p, p - a.W);
        if (CONN == 8) {
            if (c > 0 && fg(r - 1, c - 1) && !left_in) union_g(a.U, p, p - a.W - 1);
            if (fg(r - 1, c + 1) && !right_in) union_g(a.U, p, p - a.W + 1);
        }
    } else if (pos < 64) {
        const int r = r0 + pos - 32, c = c0;
        if (c == 0 || r >= a.H || !fg(r, c)) return;
        const int32_t p = (int32_t)((int64_t)r * a.W + c);
        const bool up_in = r > r0 && fg(r - 1, c);              // same block column
        if (fg(r, c - 1) && !(up_in && fg(r - 1, c - 1))) union_g(a.U, p, p - 1);
        if (CONN == 8 && r > r0 && fg(r - 1, c - 1) && !up_in) union_g(a.U, p, p - a.W - 1);
    } else {
        if (CONN != 8) return;
        const int r = r0 + pos - 64, c = c0 + kB - 1;
        if (r == r0 || r >= a.H || c + 1 >= a.W || !fg(r, c)) return;
        const int32_t p = (int32_t)((int64_t)r * a.W + c);
        if (fg(r - 1, c + 1) && !fg(r - 1, c)) union_g(a.U, p, p - a.W + 1);
    }
}

// 3. flatten: U[p] = root(p); accumulate area (warp-aggregated) or the
// border flag at the root.
__global__ void uf_flatten_kernel(UfArgs a, bool count_area, bool flag_border)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c - (int)threadIdx.x < a.W; c += gridDim.x * blockDim.x) {
        const bool in = c < a.W;
        const int64_t p = (int64_t)r * a.W + c;
        int32_t root = -1;
        const int32_t u = in ? a.U[p] : -1;
        // lanes holding the same value share one find
        const unsigned has = __ballot_sync(0xffffffffu, u >= 0);
        if (u >= 0) {
            const unsigned same = __match_any_sync(has, u);
            const int leader = __ffs(same) - 1;
            if ((int)(threadIdx.x & 31) == leader) root = find_g_halve(a.U, u);
            root = __shfl_sync(same, root, leader);
            // plain store: the root is the smallest value any concurrent
            // halving (atomicMin) could write here
            if (root != u) a.U[p] = root;
        }
        if (count_area) {
            const unsigned act = __ballot_sync(0xffffffffu, root >= 0);
            if (root >= 0) {
                const unsigned peers = __match_any_sync(act, root);
                if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(a.A + root, __popc(peers));
            }
        }
        if (flag_border && root >= 0 && (r == 0 || r == a.H - 1 || c == 0 || c == a.W - 1)) a.A[root] = 1;
    }
}

cudaError_t uf_build(const UfArgs &a, int conn, int source, bool count_area, bool flag_border, cudaStream_t s)
{
    const dim3 grid_blk((unsigned)ceil_div(a.W, kB), (unsigned)ceil_div(a.H, kB));
    const bool zero = count_area || flag_border;
    if (conn == 8) uf_local_kernel<8><<<grid_blk, 256, 0, s>>>(a, source, zero);
    else uf_local_kernel<4><<<grid_blk, 256, 0, s>>>(a, source, zero);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (conn == 8) uf_border_kernel<8><<<grid_blk, 96, 0, s>>>(a, source);
    else uf_border_kernel<4><<<grid_blk, 96, 0, s>>>(a, source);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int bx = (int)ceil_div(a.W, 256);
    uf_flatten_kernel<<<dim3((unsigned)bx, (unsigned)a.H), 256, 0, s>>>(a, count_area, flag_border);
    return cudaGetLastError();
}

// 4a. labels with the area filter
__global__ void uf_labels_kernel(UfArgs a, int32_t *labels, int64_t ld_lab, int32_t amin, int32_t amax,
                                 int32_t *n_kept)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.W; c += gridDim.x * blockDim.x) {
        const int64_t p = (int64_t)r * a.W + c;
        const int32_t root = a.U[p];
        int32_t out = -1;
        if (root >= 0) {
            const int32_t area = a.A[root];
            if (area >= amin && area <= amax) {
                out = root;
                if (root == p && n_kept) atomicAdd(n_kept, 1);
            }
        }
        labels[(int64_t)r * ld_lab + c] = out;
    }
}

cudaError_t uf_labels_out(const UfArgs &a, int32_t *labels, int64_t ld_lab, int32_t min_area,
                          int32_t max_area, int32_t *n_kept, cudaStream_t s)
{
    const int bx = (int)ceil_div(a.W, 256);
    uf_labels_kernel<<<dim3((unsigned)bx, (unsigned)a.H), 256, 0, s>>>(a, labels, ld_lab, min_area, max_area,
                                                                       n_kept);
    return cudaGetLastError();
}

// 4b. hole filling from the background components
__global__ void uf_fill_kernel(UfArgs a, uint8_t *out, int64_t ld_out)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.W; c += gridDim.x * blockDim.x) {
        const int64_t p = (int64_t)r * a.W + c;
        const int32_t root = a.U[p];     // background pixels have a root
        const uint8_t v = (root < 0) ? 1 : (a.A[root] ? 0 : 1);
        out[(int64_t)r * ld_out + c] = v;
    }
}

cudaError_t uf_fill_out(const UfArgs &a, uint8_t *out, int64_t ld_out, cudaStream_t s)
{
    const int bx = (int)ceil_div(a.W, 256);
    uf_fill_kernel<<<dim3((unsigned)bx, (unsigned)a.H), 256, 0, s>>>(a, out, ld_out);
    return cudaGetLastError();
}

}  // namespace rtk
