// BWLabel (Section 5.1) by union-find.
//
// The paper's BWLabel follows the union-find pattern: every pixel starts as
// its own tree, trees of adjacent foreground pixels are merged, and labels
// are read off by flattening the trees. Merging always hooks the root with
// the larger linear index under the smaller one (atomicMin on the parent),
// so the root of a finished tree is the smallest index of its component:
// the canonical label. The forest is built in two levels so that global
// memory only ever holds the roots of block-local components:
//   1. each 32 x 32 block labels its own pixels in shared memory; for every
//      local root it records the local area (or whether the local component
//      touches the image border) and appends the root to a list; for the
//      pixels on the block's four edges it records their local root;
//   2. local roots of pixels that touch across a block edge are merged in
//      global memory (only those roots are nodes of the global forest);
//   3. every listed local root is pointed at its final root, to which it adds
//      its area (or its border-contact flag, for the components of the
//      complement);
//   4. the output pass maps every pixel through its local root (recorded by
//      pass 1) to its final root.
#include "ccl.cuh"

namespace rtk {

constexpr int kB = kUfBlock;
constexpr int kRowsPerThread = 4;                     // warp w owns rows kRowsPerThread * w + 0, 1, ...
constexpr int kThreads = 32 * kB / kRowsPerThread;    // threads per block CTA

size_t uf_workspace_bytes(int H, int W)
{
    const size_t N = (size_t)H * W;
    const size_t nblk = (size_t)ceil_div(W, kB) * ceil_div(H, kB);
    return 2 * N * sizeof(int32_t) + nblk * kUfEdge * sizeof(int32_t) + (N / 2 + 2) * sizeof(int32_t) +
           N * sizeof(uint16_t) + nblk + 8 * 256;
}

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
// Path halving. Every ancestor has a smaller index than its descendants, so
// the halving store is an atomicMin: no node ever moves back from a higher
// ancestor (or, once unions are over, from its final root, which other
// threads store with plain writes) to a lower one.
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

// Hooking and halving are both atomicMin, so every parent only moves to a
// smaller index in the same (growing) tree while unions run concurrently.
__device__ __forceinline__ void union_g(int32_t *U, int32_t a, int32_t b)
{
    for (;;) {
        a = find_g_halve(U, a);
        b = find_g_halve(U, b);
        if (a == b) return;
        if (a < b) {
            const int32_t t = a; a = b; b = t;
        }
        const int32_t old = atomicMin(U + a, b);
        if (old == a) return;
        a = old;
    }
}

// ---------------------------------------------------- block-local labeling
// Labels block (blockIdx.x, blockIdx.y) in shared memory. Inside a row, a run
// of foreground pixels is one tree from the start: every pixel points at the
// run's first pixel (found from the row's ballot mask). Rows are then joined
// with one union per pair of touching runs: for 4-connectivity at the first
// column where the runs overlap; for 8-connectivity the first pixel of a run
// joins each run of the row above that starts within its three upper
// neighbours, and any other pixel joins only a run of the row above that
// starts at its upper-right neighbour. On return roots[k] holds the local
// index (lr * 32 + c) of the root of the thread's k-th pixel, or -1.
template <int CONN>
__device__ __forceinline__ bool local_labels(const UfArgs &a, int source, int *P, uint32_t *M,
                                             int roots[kRowsPerThread])
{
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = blockIdx.y * kB, c0 = blockIdx.x * kB;
    const int c = c0 + tx;
    uint32_t any = 0;
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
        any |= m;
    }
    // a block without foreground (most of a sparse mask) has nothing to join
    if (!__syncthreads_or(any != 0)) {
#pragma unroll
        for (int k = 0; k < kRowsPerThread; ++k) roots[k] = -1;
        return false;
    }
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
        const int i = (w * kRowsPerThread + k) * kB + tx;
        roots[k] = P[i] >= 0 ? find_s_halve(P, i) : -1;
    }
    return true;
}

__device__ __forceinline__ int32_t global_index(const UfArgs &a, int local)
{
    const int r = blockIdx.y * kB + local / kB, c = blockIdx.x * kB + local % kB;
    return (int32_t)((int64_t)r * a.W + c);
}

// 1. block-local components, their roots, areas / border flags and edges
template <int CONN>
__global__ void __launch_bounds__(kThreads) uf_local_kernel(UfArgs a, int source, bool count_area)
{
    __shared__ int P[kB * kB];
    __shared__ int cnt[kB * kB];
    __shared__ uint32_t M[kB];
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    int roots[kRowsPerThread];
    const bool nonempty = local_labels<CONN>(a, source, P, M, roots);
    const int r0 = blockIdx.y * kB, c0 = blockIdx.x * kB;
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    int32_t *edge = a.edge + blk * kUfEdge;
    if (!nonempty) {   // no roots, no edge roots; the output pass skips the block
        if (threadIdx.x < kUfEdge) edge[threadIdx.x] = -1;
        if (threadIdx.x == 0) a.bempty[blk] = 1;
        return;
    }
    if (threadIdx.x == 0) a.bempty[blk] = 0;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) cnt[(w * kRowsPerThread + k) * kB + tx] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        if (roots[k] < 0) continue;
        const int r = r0 + w * kRowsPerThread + k, c = c0 + tx;
        if (count_area) atomicAdd(cnt + roots[k], 1);
        else if (r == 0 || c == 0 || r == a.H - 1 || c == a.W - 1) cnt[roots[k]] = 1;
    }
    __syncthreads();
    // every pixel's local root, so that the output pass need not label the block again
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int r = r0 + w * kRowsPerThread + k, c = c0 + tx;
        if (r < a.H && c < a.W) a.lroot[(int64_t)r * a.W + c] = roots[k] >= 0 ? (uint16_t)roots[k] : (uint16_t)0xFFFFu;
    }
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int lr = w * kRowsPerThread + k;
        const int i = lr * kB + tx;
        const int32_t g = roots[k] >= 0 ? global_index(a, roots[k]) : -1;
        if (lr == 0) edge[tx] = g;
        if (lr == kB - 1) edge[kB + tx] = g;
        if (tx == 0) edge[2 * kB + lr] = g;
        if (tx == kB - 1) edge[3 * kB + lr] = g;
        const bool is_root = roots[k] == i;
        if (is_root) {
            a.U[g] = g;
            a.A[g] = cnt[i];
        }
        const unsigned rm = __ballot_sync(0xffffffffu, is_root);
        if (rm) {
            uint32_t base = 0;
            const int leader = __ffs(rm) - 1;
            if (tx == leader) base = atomicAdd(a.nlist, (uint32_t)__popc(rm));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (is_root) a.list[base + __popc(rm & ((1u << tx) - 1))] = g;
        }
    }
}

// 2. merges across block edges, one CTA of 96 threads per block: threads
// 0..31 the top row (with the row above), 32..63 the left column (with the
// column to the left), 64..95 the right column (up-right neighbours, 8
// only). The nodes are the local roots recorded on the block edges. Pixels
// adjacent along one block row or column already share a local root, so
// along an edge only the first pixel pair of each pair of touching runs
// needs a union; the others are skipped.
template <int CONN>
__global__ void __launch_bounds__(96) uf_border_kernel(UfArgs a)
{
    const int bx = blockIdx.x, by = blockIdx.y, nbx = gridDim.x;
    const int pos = threadIdx.x;
    auto E = [&](int x, int y) -> const int32_t * { return a.edge + ((int64_t)y * nbx + x) * kUfEdge; };
    const int32_t *me = E(bx, by);
    if (pos < 32) {
        if (by == 0) return;
        const int k = pos;
        const int32_t p = me[k];
        if (p < 0) return;
        const int32_t *ab = E(bx, by - 1) + kB;          // bottom row of the block above
        const bool left_in = k > 0 && me[k - 1] >= 0;
        const bool right_in = k < kB - 1 && me[k + 1] >= 0;
        if (ab[k] >= 0 && !(left_in && ab[k - 1] >= 0)) union_g(a.U, p, ab[k]);
        if (CONN == 8) {
            const int32_t ul = k > 0 ? ab[k - 1] : (bx > 0 ? E(bx - 1, by - 1)[kB + kB - 1] : -1);
            const int32_t ur = k < kB - 1 ? ab[k + 1] : (bx + 1 < nbx ? E(bx + 1, by - 1)[kB] : -1);
            if (ul >= 0 && !left_in) union_g(a.U, p, ul);
            if (ur >= 0 && !right_in) union_g(a.U, p, ur);
        }
    } else if (pos < 64) {
        if (bx == 0) return;
        const int k = pos - 32;
        const int32_t p = me[2 * kB + k];
        if (p < 0) return;
        const int32_t *lr = E(bx - 1, by) + 3 * kB;      // right column of the block to the left
        const bool up_in = k > 0 && me[2 * kB + k - 1] >= 0;
        if (lr[k] >= 0 && !(up_in && lr[k - 1] >= 0)) union_g(a.U, p, lr[k]);
        if (CONN == 8 && k > 0 && lr[k - 1] >= 0 && !up_in) union_g(a.U, p, lr[k - 1]);
    } else {
        if (CONN != 8 || bx + 1 >= nbx) return;
        const int k = pos - 64;
        if (k == 0) return;                              // handled as a top-row pixel
        const int32_t p = me[3 * kB + k];
        if (p < 0) return;
        const int32_t q = E(bx + 1, by)[2 * kB + k - 1];  // left column of the block to the right, row above
        if (q >= 0 && me[3 * kB + k - 1] < 0) union_g(a.U, p, q);
    }
}

// 3. final roots of the local roots, with areas or border flags
__global__ void uf_roots_kernel(UfArgs a, bool count_area)
{
    const uint32_t n = *a.nlist;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t L = a.list[i];
        const int32_t root = find_g_halve(a.U, L);
        if (root == L) continue;
        a.U[L] = root;     // plain store: no concurrent value can be smaller
        if (count_area) atomicAdd(a.A + root, a.A[L]);
        else if (a.A[L]) a.A[root] = 1;
    }
}

cudaError_t uf_build(const UfArgs &a, int conn, int source, bool count_area, bool flag_border, cudaStream_t s)
{
    (void)flag_border;
    const dim3 grid_blk((unsigned)ceil_div(a.W, kB), (unsigned)ceil_div(a.H, kB));
    cudaError_t e = cudaMemsetAsync(a.nlist, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (conn == 8) uf_local_kernel<8><<<grid_blk, kThreads, 0, s>>>(a, source, count_area);
    else uf_local_kernel<4><<<grid_blk, kThreads, 0, s>>>(a, source, count_area);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (conn == 8) uf_border_kernel<8><<<grid_blk, 96, 0, s>>>(a);
    else uf_border_kernel<4><<<grid_blk, 96, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uf_roots_kernel<<<1024, 256, 0, s>>>(a, count_area);
    return cudaGetLastError();
}

// 4a. labels with the area filter, from every pixel's local root (recorded
// by pass 1); optionally the kept pixels as a bit plane (bit c % 32 of word
// r * ceil(W / 32) + c / 32), which is all the distance transform needs
__global__ void __launch_bounds__(kThreads) uf_labels_kernel(UfArgs a, int32_t *labels, int64_t ld_lab, int32_t amin,
                                                        int32_t amax, int32_t *n_kept, uint32_t *fgbits)
{
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = blockIdx.y * kB, c0 = blockIdx.x * kB, c = c0 + tx;
    const int64_t wpr = ceil_div(a.W, 32);
    const bool empty = a.bempty[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] != 0;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int r = r0 + w * kRowsPerThread + k;
        const bool in = r < a.H && c < a.W;
        const uint32_t lr = in && !empty ? a.lroot[(int64_t)r * a.W + c] : 0xFFFFu;
        int32_t out = -1;
        if (lr != 0xFFFFu) {
            const int32_t root = a.U[global_index(a, (int)lr)];
            const int32_t area = a.A[root];
            if (area >= amin && area <= amax) {
                out = root;
                if (n_kept && root == (int32_t)((int64_t)r * a.W + c)) atomicAdd(n_kept, 1);
            }
        }
        if (in) labels[(int64_t)r * ld_lab + c] = out;
        if (fgbits) {
            const uint32_t bits = __ballot_sync(0xffffffffu, out >= 0);
            if (tx == 0 && r < a.H) fgbits[(int64_t)r * wpr + blockIdx.x] = bits;
        }
    }
}

cudaError_t uf_labels_out(const UfArgs &a, int conn, int32_t *labels, int64_t ld_lab, int32_t min_area,
                          int32_t max_area, int32_t *n_kept, uint32_t *fgbits, cudaStream_t s)
{
    const dim3 grid_blk((unsigned)ceil_div(a.W, kB), (unsigned)ceil_div(a.H, kB));
    (void)conn;   // the components were built by uf_build with this connectivity
    uf_labels_kernel<<<grid_blk, kThreads, 0, s>>>(a, labels, ld_lab, min_area, max_area, n_kept, fgbits);
    return cudaGetLastError();
}

}  // namespace rtk
