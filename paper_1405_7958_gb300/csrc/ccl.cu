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
//      local root it records the local area and lists the root in the
//      block's own slots; for the pixels on the block's four edges it records
//      their local root;
//   2. local roots of pixels that touch across a block edge are merged in
//      global memory (only those roots are nodes of the global forest);
//   3. every listed local root is pointed at its final root, to which it adds
//      its area;
//   4. the output pass maps every pixel through its local root (recorded by
//      pass 1) to its final root and applies the area filter.
// Every stage is one launch over all the blocks of all the images of a batch
// (a table of images; each CTA finds its image by the block numbering).
#include "ccl.cuh"


namespace rtk {

constexpr int kB = kUfBlock;
constexpr int kRowsPerThread = 4;                     // warp w owns rows kRowsPerThread * w + 0, 1, ...
constexpr int kThreads = 32 * kB / kRowsPerThread;    // threads per block CTA

namespace {

size_t piece(size_t bytes) { return (size_t)round_up((int64_t)bytes, 256); }

}  // namespace

size_t uf_workspace_bytes(int H, int W)
{
    const size_t N = (size_t)H * W;
    const size_t nblk = (size_t)ceil_div(W, kB) * ceil_div(H, kB);
    return 2 * piece(N * sizeof(int32_t)) + piece(nblk * kUfEdge * sizeof(int32_t)) +
           piece(nblk * kUfMaxRoots * sizeof(int32_t)) + piece(nblk * sizeof(uint16_t)) +
           piece(N * sizeof(uint16_t)) + piece(nblk);
}

void uf_carve(UfImage &d, char *base, int H, int W)
{
    const size_t N = (size_t)H * W;
    d.H = H;
    d.W = W;
    d.nbx = (int)ceil_div(W, kB);
    d.nby = (int)ceil_div(H, kB);
    const size_t nblk = (size_t)d.nbx * d.nby;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base + off;
        off += piece(bytes);
        return p;
    };
    d.U = reinterpret_cast<int32_t *>(take(N * sizeof(int32_t)));
    d.A = reinterpret_cast<int32_t *>(take(N * sizeof(int32_t)));
    d.edge = reinterpret_cast<int32_t *>(take(nblk * kUfEdge * sizeof(int32_t)));
    d.list = reinterpret_cast<int32_t *>(take(nblk * kUfMaxRoots * sizeof(int32_t)));
    d.cnt = reinterpret_cast<uint16_t *>(take(nblk * sizeof(uint16_t)));
    d.lroot = reinterpret_cast<uint16_t *>(take(N * sizeof(uint16_t)));
    d.bempty = reinterpret_cast<uint8_t *>(take(nblk));
}

void uf_add(UfBatch &b, const UfImage &d)
{
    if (b.n == 0) b.nblk = 0;
    UfImage &e = b.img[b.n++];
    e = d;
    e.blk_base = b.nblk;
    b.nblk += (int64_t)d.nbx * d.nby;
}

// The image and block (bx, by) of CTA `g` of a launch over all blocks.
struct BlockRef {
    const UfImage *d;
    int bx, by;
    int64_t blk;   // block index inside the image
};

__device__ __forceinline__ BlockRef find_block(const UfBatch &b, int64_t g)
{
    int k = 0;
    while (k + 1 < b.n && g >= b.img[k + 1].blk_base) ++k;
    BlockRef r;
    r.d = &b.img[k];
    // an image has at most 1024 x 1024 blocks: 32-bit arithmetic (64-bit
    // division is a long software sequence)
    const int lb = (int)(g - r.d->blk_base);
    r.blk = lb;
    r.by = lb / r.d->nbx;
    r.bx = lb - r.by * r.d->nbx;
    return r;
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
// Labels block (bx, by) of image d in shared memory. Inside a row, a run of
// foreground pixels is one tree from the start: every pixel points at the
// run's first pixel (found from the row's ballot mask). Rows are then joined
// with one union per pair of touching runs: for 4-connectivity at the first
// column where the runs overlap; for 8-connectivity the first pixel of a run
// joins each run of the row above that starts within its three upper
// neighbours, and any other pixel joins only a run of the row above that
// starts at its upper-right neighbour. On return roots[k] holds the local
// index (lr * 32 + c) of the root of the thread's k-th pixel, or -1.
template <int CONN>
__device__ __forceinline__ bool local_labels(const UfImage &d, int bx, int by, int *P, uint32_t *M,
                                             int roots[kRowsPerThread])
{
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = by * kB, c0 = bx * kB;
    // the block's row masks: thread t reads 4 adjacent pixels of row t / 8
    // (one 32-bit load where aligned), eight threads combine a row's mask
    {
        const int rr = threadIdx.x >> 3, qq = threadIdx.x & 7;
        const int gr = r0 + rr, gc = c0 + 4 * qq;
        uint32_t nib = 0;
        if (gr < d.H && gc < d.W) {
            const uint8_t *px = d.in + (int64_t)gr * d.ld_in + gc;
            if (gc + 3 < d.W && (reinterpret_cast<uintptr_t>(px) & 3u) == 0) {
                const uint32_t v = *reinterpret_cast<const uint32_t *>(px);
                nib = (uint32_t)((v & 0xffu) != 0) | (uint32_t)((v & 0xff00u) != 0) << 1 |
                      (uint32_t)((v & 0xff0000u) != 0) << 2 | (uint32_t)((v & 0xff000000u) != 0) << 3;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (gc + k < d.W) nib |= (uint32_t)(px[k] != 0) << k;
            }
        }
        uint32_t m = nib << (4 * qq);
        m |= __shfl_xor_sync(0xffffffffu, m, 1);
        m |= __shfl_xor_sync(0xffffffffu, m, 2);
        m |= __shfl_xor_sync(0xffffffffu, m, 4);
        if (qq == 0) M[rr] = m;
        // a block without foreground (most of a sparse mask) has nothing to join
        if (!__syncthreads_or(m != 0)) {
#pragma unroll
            for (int k = 0; k < kRowsPerThread; ++k) roots[k] = -1;
            return false;
        }
    }
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int lr = w * kRowsPerThread + k;
        const uint32_t m = M[lr];
        const bool f = (m >> tx) & 1u;
        const uint32_t starts = m & ~(m << 1);
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
        const int i = (w * kRowsPerThread + k) * kB + tx;
        roots[k] = P[i] >= 0 ? find_s_halve(P, i) : -1;
    }
    return true;
}

__device__ __forceinline__ int32_t global_index(const UfImage &d, int bx, int by, int local)
{
    const int r = by * kB + local / kB, c = bx * kB + local % kB;
    return (int32_t)((int64_t)r * d.W + c);
}

// 1. block-local components, their roots, areas and edges. The first block
// of an image also clears its kept-component count (read by stage 4).
template <int CONN>
__global__ void __launch_bounds__(kThreads) uf_local_kernel(UfBatch b)
{
    __shared__ int P[kB * kB];
    __shared__ int cnt[kB * kB];
    __shared__ uint32_t M[kB];
    __shared__ int nroots;
    const BlockRef br = find_block(b, blockIdx.x);
    const UfImage &d = *br.d;
    const int bx = br.bx, by = br.by;
    const int64_t blk = br.blk;
    if (blk == 0 && threadIdx.x == 0 && d.n_kept) *d.n_kept = 0;
    const int tx = threadIdx.x & 31, w = threadIdx.x >> 5;
    int roots[kRowsPerThread];
    const bool nonempty = local_labels<CONN>(d, bx, by, P, M, roots);
    const int r0 = by * kB, c0 = bx * kB;
    int32_t *edge = d.edge + blk * kUfEdge;
    if (!nonempty) {   // no roots, no edge roots; the later stages skip the block
        if (threadIdx.x < kUfEdge) edge[threadIdx.x] = -1;
        if (threadIdx.x == 0) {
            d.bempty[blk] = 1;
            d.cnt[blk] = 0;
        }
        return;
    }
    if (threadIdx.x == 0) {
        d.bempty[blk] = 0;
        nroots = 0;
    }
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) cnt[(w * kRowsPerThread + k) * kB + tx] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k)
        if (roots[k] >= 0) atomicAdd(cnt + roots[k], 1);
    __syncthreads();
    // every pixel's local root, so that the output pass need not label the block again
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int r = r0 + w * kRowsPerThread + k, c = c0 + tx;
        if (r < d.H && c < d.W) d.lroot[(int64_t)r * d.W + c] = roots[k] >= 0 ? (uint16_t)roots[k] : (uint16_t)0xFFFFu;
    }
    int32_t *list = d.list + blk * kUfMaxRoots;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        const int lr = w * kRowsPerThread + k;
        const int i = lr * kB + tx;
        const int32_t g = roots[k] >= 0 ? global_index(d, bx, by, roots[k]) : -1;
        if (lr == 0) edge[tx] = g;
        if (lr == kB - 1) edge[kB + tx] = g;
        if (tx == 0) edge[2 * kB + lr] = g;
        if (tx == kB - 1) edge[3 * kB + lr] = g;
        const bool is_root = roots[k] == i;
        if (is_root) {
            d.U[g] = g;
            d.A[g] = cnt[i];
        }
        const unsigned rm = __ballot_sync(0xffffffffu, is_root);
        if (rm) {
            int base = 0;
            const int leader = __ffs(rm) - 1;
            if (tx == leader) base = atomicAdd(&nroots, __popc(rm));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (is_root) list[base + __popc(rm & ((1u << tx) - 1))] = g;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) d.cnt[blk] = (uint16_t)nroots;
}

// 2. merges across block edges, one CTA of 96 threads per block: threads
// 0..31 the top row (with the row above), 32..63 the left column (with the
// column to the left), 64..95 the right column (up-right neighbours, 8
// only). The nodes are the local roots recorded on the block edges. Pixels
// adjacent along one block row or column already share a local root, so
// along an edge only the first pixel pair of each pair of touching runs
// needs a union; the others are skipped.
template <int CONN>
__global__ void __launch_bounds__(96) uf_border_kernel(UfBatch b)
{
    const BlockRef br = find_block(b, blockIdx.x);
    const UfImage &d = *br.d;
    const int bx = br.bx, by = br.by, nbx = d.nbx;
    const int pos = threadIdx.x;
    auto E = [&](int x, int y) -> const int32_t * { return d.edge + ((int64_t)y * nbx + x) * kUfEdge; };
    const int32_t *me = E(bx, by);
    if (pos < 32) {
        if (by == 0) return;
        const int k = pos;
        const int32_t p = me[k];
        if (p < 0) return;
        const int32_t *ab = E(bx, by - 1) + kB;          // bottom row of the block above
        const bool left_in = k > 0 && me[k - 1] >= 0;
        const bool right_in = k < kB - 1 && me[k + 1] >= 0;
        if (ab[k] >= 0 && !(left_in && ab[k - 1] >= 0)) union_g(d.U, p, ab[k]);
        if (CONN == 8) {
            const int32_t ul = k > 0 ? ab[k - 1] : (bx > 0 ? E(bx - 1, by - 1)[kB + kB - 1] : -1);
            const int32_t ur = k < kB - 1 ? ab[k + 1] : (bx + 1 < nbx ? E(bx + 1, by - 1)[kB] : -1);
            if (ul >= 0 && !left_in) union_g(d.U, p, ul);
            if (ur >= 0 && !right_in) union_g(d.U, p, ur);
        }
    } else if (pos < 64) {
        if (bx == 0) return;
        const int k = pos - 32;
        const int32_t p = me[2 * kB + k];
        if (p < 0) return;
        const int32_t *lr = E(bx - 1, by) + 3 * kB;      // right column of the block to the left
        const bool up_in = k > 0 && me[2 * kB + k - 1] >= 0;
        if (lr[k] >= 0 && !(up_in && lr[k - 1] >= 0)) union_g(d.U, p, lr[k]);
        if (CONN == 8 && k > 0 && lr[k - 1] >= 0 && !up_in) union_g(d.U, p, lr[k - 1]);
    } else {
        if (CONN != 8 || bx + 1 >= nbx) return;
        const int k = pos - 64;
        if (k == 0) return;                              // handled as a top-row pixel
        const int32_t p = me[3 * kB + k];
        if (p < 0) return;
        const int32_t q = E(bx + 1, by)[2 * kB + k - 1];  // left column of the block to the right, row above
        if (q >= 0 && me[3 * kB + k - 1] < 0) union_g(d.U, p, q);
    }
}

// 3. final roots of the local roots, with areas: a warp per block, lanes
// over the block's listed roots (four blocks per CTA)
__global__ void __launch_bounds__(128) uf_roots_kernel(UfBatch b)
{
    const int64_t g = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (g >= b.nblk) return;
    const int lane = threadIdx.x & 31;
    const BlockRef br = find_block(b, g);
    const UfImage &d = *br.d;
    const int n = d.cnt[br.blk];
    const int32_t *list = d.list + br.blk * kUfMaxRoots;
    for (int k = lane; k < n; k += 32) {
        const int32_t L = list[k];
        const int32_t root = find_g_halve(d.U, L);
        if (root == L) continue;
        d.U[L] = root;     // plain store: no concurrent value can be smaller
        atomicAdd(d.A + root, d.A[L]);
    }
}

// 4. labels with the area filter, from every pixel's local root (recorded
// by stage 1); optionally the kept pixels as a bit plane (bit c % 32 of word
// r * ceil(W / 32) + c / 32), which is all the distance transform needs.
// A thread takes 4 adjacent pixels of one row (8 threads a block row), so
// the labels leave in 16-byte stores where the row allows them.
__global__ void __launch_bounds__(kThreads) uf_labels_kernel(UfBatch b)
{
    const BlockRef br = find_block(b, blockIdx.x);
    const UfImage &d = *br.d;
    const int q = threadIdx.x & 7, lr = threadIdx.x >> 3;
    const int r = br.by * kB + lr, c = br.bx * kB + 4 * q;
    const bool empty = d.bempty[br.blk] != 0;
    int32_t out[4] = {-1, -1, -1, -1};
    const bool row_in = r < d.H;
    if (row_in && !empty && c < d.W) {
        const int64_t pix = (int64_t)r * d.W + c;
        uint32_t lrs[4];
        if ((d.W & 3) == 0) {   // 8-byte aligned: W and c are multiples of 4
            const uint2 v = *reinterpret_cast<const uint2 *>(d.lroot + pix);
            lrs[0] = v.x & 0xFFFFu, lrs[1] = v.x >> 16, lrs[2] = v.y & 0xFFFFu, lrs[3] = v.y >> 16;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) lrs[k] = c + k < d.W ? d.lroot[pix + k] : 0xFFFFu;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (lrs[k] == 0xFFFFu) continue;
            const int32_t root = d.U[global_index(d, br.bx, br.by, (int)lrs[k])];
            const int32_t area = d.A[root];
            if (area >= b.amin && area <= b.amax) {
                out[k] = root;
                if (d.n_kept && root == (int32_t)(pix + k)) atomicAdd(d.n_kept, 1);
            }
        }
    }
    if (row_in && c < d.W) {
        int32_t *dst = d.labels + (int64_t)r * d.ld_lab + c;
        if (c + 3 < d.W && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
            *reinterpret_cast<int4 *>(dst) = make_int4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (c + k < d.W) dst[k] = out[k];
        }
    }
    if (d.fgbits) {
        uint32_t bits = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) bits |= (uint32_t)(out[k] >= 0) << (4 * q + k);
        bits |= __shfl_xor_sync(0xffffffffu, bits, 1);
        bits |= __shfl_xor_sync(0xffffffffu, bits, 2);
        bits |= __shfl_xor_sync(0xffffffffu, bits, 4);
        if (q == 0 && row_in) d.fgbits[(int64_t)r * ceil_div(d.W, 32) + br.bx] = bits;
    }
}

cudaError_t launch_label_batch(const UfBatch &b, int conn, cudaStream_t s)
{
    if (b.n < 1 || b.n > kUfMaxImgs || (conn != 4 && conn != 8)) return cudaErrorInvalidValue;
    const unsigned nb = (unsigned)b.nblk;
    if (conn == 8) uf_local_kernel<8><<<nb, kThreads, 0, s>>>(b);
    else uf_local_kernel<4><<<nb, kThreads, 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (conn == 8) uf_border_kernel<8><<<nb, 96, 0, s>>>(b);
    else uf_border_kernel<4><<<nb, 96, 0, s>>>(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uf_roots_kernel<<<(unsigned)ceil_div(b.nblk, 4), 128, 0, s>>>(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    uf_labels_kernel<<<nb, kThreads, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace rtk
