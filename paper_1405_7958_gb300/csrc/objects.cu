// The per-object steps that follow the labels in the paper's pipeline
// (Section 5.1, "Example Application"):
//   * the feature computation stage, restructured as the paper describes:
//     the objects are cut out by their minimum bounding boxes, one thread
//     block per box computes the intermediate results (histograms,
//     co-occurrence matrix, moments), then one thread per object turns them
//     into the features;
//   * the Watershed after the Pre-Watershed step, which splits touching
//     nuclei: marker-controlled flooding of the distance map inside every
//     object, one thread block per object (in shared memory when the box is
//     small enough).
// Both start from the same enumeration of the objects of a label image
// whose labels are the linear index of each object's first pixel (as
// rt_label_area writes them): those first pixels are found in raster order
// (count per chunk, prefix sum, emit), which orders the objects by label
// and gives every label its object index; a pass over the pixels then
// grows each object's bounding box (warp-aggregated atomics).
#include "objects.cuh"

namespace rtk {

namespace {

size_t piece(size_t bytes) { return (size_t)round_up((int64_t)bytes, 256); }

constexpr int kThreads = 256;
constexpr unsigned long long kUnl = ~0ull;   // watershed state of a pixel without a basin yet

}  // namespace

size_t obj_workspace_bytes(int H, int W, bool features, bool watershed, int cap)
{
    const size_t N = (size_t)H * W;
    const size_t nch = (size_t)ceil_div((int64_t)N, kObjChunk);
    size_t b = piece(nch * 4) + piece(64) + piece(N * 4) + piece(N * 4) + piece(N * 16);
    if (features) b += piece((size_t)(cap > 0 ? cap : 1) * sizeof(ObjInter));
    if (watershed) b += piece(N * 4) + piece(N * 8) + piece(N) + piece(N * 4);
    return b;
}

void obj_carve(ObjArgs &a, char *base, bool features, bool watershed)
{
    const size_t N = (size_t)a.H * a.W;
    const size_t nch = (size_t)ceil_div((int64_t)N, kObjChunk);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base + off;
        off += piece(bytes);
        return p;
    };
    a.chunk_cnt = reinterpret_cast<uint32_t *>(take(nch * 4));
    a.ctl = reinterpret_cast<uint32_t *>(take(64));
    a.idx_of = reinterpret_cast<int32_t *>(take(N * 4));
    a.olabel = reinterpret_cast<int32_t *>(take(N * 4));
    a.box = reinterpret_cast<int32_t *>(take(N * 16));
    a.max_obj = (int64_t)N;
    a.inter = features ? reinterpret_cast<ObjInter *>(take((size_t)(a.cap > 0 ? a.cap : 1) * sizeof(ObjInter)))
                       : nullptr;
    if (watershed) {
        a.R = reinterpret_cast<int32_t *>(take(N * 4));
        a.st = reinterpret_cast<unsigned long long *>(take(N * 8));
        a.nm = reinterpret_cast<uint8_t *>(take(N));
        a.order = reinterpret_cast<int32_t *>(take(N * 4));
    } else {
        a.R = nullptr;
        a.st = nullptr;
        a.nm = nullptr;
        a.order = nullptr;
    }
}

// ------------------------------------------------------------ enumeration
// Warp per chunk of kObjChunk pixels (raster order): the object first pixels
// (L(p) == p) it holds. EMIT = 0: count them; EMIT = 1: write them at their
// rank after the chunk's prefix, with their object index and initial box.
template <int EMIT>
__global__ void __launch_bounds__(kThreads) obj_scan_pixels_kernel(ObjArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t ch = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    const int64_t N = (int64_t)a.H * a.W;
    const int64_t p0 = ch * kObjChunk;
    if (p0 >= N) return;
    uint32_t base = EMIT ? a.chunk_cnt[ch] : 0u, cnt = 0;
    // H * W <= 2^30: 32-bit positions; the row and column follow the pixel
    // index incrementally (one division per lane, then at most a few wraps)
    const uint32_t W = (uint32_t)a.W;
    uint32_t pl = (uint32_t)p0 + lane;
    uint32_t r = pl / W, c = pl - r * W;
    for (int j = 0; j < kObjChunk / 32; ++j, pl += 32) {
        if (j) {
            c += 32;
            while (c >= W) {
                c -= W;
                ++r;
            }
        }
        const int64_t p = pl;
        bool root = false;
        if (p < N) root = a.L[(int64_t)r * a.ld_L + c] == (int32_t)p;
        const uint32_t m = __ballot_sync(0xffffffffu, root);
        if (EMIT && root) {
            const int64_t k = (int64_t)base + cnt + __popc(m & ((1u << lane) - 1u));
            if (k < a.max_obj) {
                a.olabel[k] = (int32_t)p;
                a.idx_of[p] = (int32_t)k;
                int4 b;
                b.x = (int)r;
                b.y = (int)c;
                b.z = (int)r;
                b.w = (int)c;
                reinterpret_cast<int4 *>(a.box)[k] = b;
            }
        }
        cnt += __popc(m);
    }
    if (!EMIT && lane == 0) a.chunk_cnt[ch] = cnt;
}

// One CTA: exclusive prefix sum of the chunk counts in place; the total is
// the number of objects. Also resets the per-object work counter and the
// caller's counts.
__global__ void __launch_bounds__(1024) obj_prefix_kernel(ObjArgs a, int64_t nch)
{
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    const int64_t per = ceil_div(nch, 1024);
    const int64_t b0 = t * per, b1 = min(nch, b0 + per);
    uint32_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += a.chunk_cnt[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {   // inclusive scan of the thread sums
        const uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (int64_t i = b0; i < b1; ++i) {
        const uint32_t v = a.chunk_cnt[i];
        a.chunk_cnt[i] = run;
        run += v;
    }
    if (t == 1023) {
        a.ctl[0] = part[1023];
        a.ctl[1] = 0u;
        a.ctl[2] = 0u;
        a.ctl[3] = 0u;
        a.ctl[4] = 0u;
        if (a.n_obj) *a.n_obj = (int32_t)part[1023];
        if (a.n_basins) *a.n_basins = 0;
    }
}

// Thread per pixel, a warp per 32 columns of one row: pixels of one label
// in the warp are combined, and their leader grows the object's box. A
// label that is not the linear index of an earlier-or-equal pixel carrying
// that same label is not canonical: RT_EINVAL in the status. With a basin
// image, background pixels get -1 there.
__global__ void __launch_bounds__(kThreads) obj_box_kernel(ObjArgs a)
{
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const int r = blockIdx.y * (kThreads / 32) + (threadIdx.x >> 5);
    if (r >= a.H) return;   // whole warp: one row
    const bool inside = c < a.W;
    const int32_t l = inside ? a.L[(int64_t)r * a.ld_L + c] : -1;
    if (inside && l < 0 && a.basins) a.basins[(int64_t)r * a.ld_B + c] = -1;
    const uint32_t peers = __match_any_sync(0xffffffffu, l);
    if (l < 0) return;
    const int cmin = __reduce_min_sync(peers, c), cmax = __reduce_max_sync(peers, c);
    if ((threadIdx.x & 31) != __ffs(peers) - 1) return;
    const int64_t p = (int64_t)r * a.W + cmin;
    const int64_t N = (int64_t)a.H * a.W;
    if ((int64_t)l > p || (int64_t)l >= N) {
        raise_status(a.err, RT_EINVAL);
        return;
    }
    const int rr = (int)(l / a.W), cr = (int)(l - (int64_t)rr * a.W);
    if (a.L[(int64_t)rr * a.ld_L + cr] != l) {
        raise_status(a.err, RT_EINVAL);
        return;
    }
    const int32_t k = a.idx_of[l];
    atomicMax(a.box + 4 * (int64_t)k + 2, r);
    atomicMin(a.box + 4 * (int64_t)k + 1, cmin);
    atomicMax(a.box + 4 * (int64_t)k + 3, cmax);
}

cudaError_t launch_enumeration(const ObjArgs &a, cudaStream_t s, int *launches)
{
    const int64_t N = (int64_t)a.H * a.W;
    const int64_t nch = ceil_div(N, kObjChunk);
    const unsigned g = (unsigned)ceil_div(nch, kThreads / 32);
    obj_scan_pixels_kernel<0><<<g, kThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    obj_prefix_kernel<<<1, 1024, 0, s>>>(a, nch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    obj_scan_pixels_kernel<1><<<g, kThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    obj_box_kernel<<<dim3((unsigned)ceil_div(a.W, 32), (unsigned)ceil_div(a.H, kThreads / 32)), kThreads, 0, s>>>(a);
    *launches += 4;
    return cudaGetLastError();
}

// Next object for this block (dynamic: boxes differ in size); -1 when done.
__device__ __forceinline__ int next_object(const ObjArgs &a, int limit, int *slot)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t k = atomicAdd(a.ctl + 1, 1u);
        *slot = (int64_t)k < limit ? (int)k : -1;
    }
    __syncthreads();
    return *slot;
}

// --------------------------------------------------------------- features
// Block per object: intermediate results over the object's bounding box.
__global__ void __launch_bounds__(kThreads) obj_inter_kernel(ObjArgs a)
{
    __shared__ uint32_t hist[256], glcm[64];
    __shared__ unsigned long long sums[9];
    __shared__ int slot;
    const int n_obj = (int)min((int64_t)a.ctl[0], a.max_obj);
    const int limit = min(n_obj, a.cap);
    for (;;) {
        const int k = next_object(a, limit, &slot);
        if (k < 0) return;
        for (int i = threadIdx.x; i < 256; i += kThreads) hist[i] = 0u;
        if (threadIdx.x < 64) glcm[threadIdx.x] = 0u;
        if (threadIdx.x < 9) sums[threadIdx.x] = 0ull;
        __syncthreads();
        const int4 b = reinterpret_cast<const int4 *>(a.box)[k];
        const int32_t l = a.olabel[k];
        const int bh = b.z - b.x + 1, bw = b.w - b.y + 1;
        const int m = bh * bw;   // H * W <= 2^30
        int64_t area = 0, per = 0, sr = 0, sc = 0, srr = 0, scc = 0, src = 0, si = 0, sii = 0;
        for (int i = threadIdx.x; i < m; i += kThreads) {
            const int y = i / bw, x = i - y * bw;
            const int r = b.x + y, c = b.y + x;
            const int32_t *Lr = a.L + (int64_t)r * a.ld_L;
            if (Lr[c] != l) continue;
            const int v = a.I[(int64_t)r * a.ld_I + c];
            ++area;
            per += (r == 0 || Lr[c - a.ld_L] != l) + (r + 1 == a.H || Lr[c + a.ld_L] != l) +
                   (c == 0 || Lr[c - 1] != l);
            const bool right_in = c + 1 < a.W && Lr[c + 1] == l;
            per += !right_in;
            sr += y;
            sc += x;
            srr += (int64_t)y * y;
            scc += (int64_t)x * x;
            src += (int64_t)y * x;
            si += v;
            sii += (int64_t)v * v;
            atomicAdd(hist + v, 1u);
            if (right_in) atomicAdd(glcm + (v >> 5) * 8 + (a.I[(int64_t)r * a.ld_I + c + 1] >> 5), 1u);
        }
        const int64_t vals[9] = {area, per, sr, sc, srr, scc, src, si, sii};
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            unsigned long long v = (unsigned long long)vals[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0 && v) atomicAdd(sums + q, v);
        }
        __syncthreads();
        ObjInter &o = a.inter[k];
        if (threadIdx.x < 9) {
            int64_t *dst = &o.area;
            dst[threadIdx.x] = (int64_t)sums[threadIdx.x];
        }
        for (int i = threadIdx.x; i < 256; i += kThreads) o.hist[i] = hist[i];
        if (threadIdx.x < 64) o.glcm[threadIdx.x] = glcm[threadIdx.x];
    }
}

// Step 2, the features from the intermediate results. The paper runs one
// thread per object; with a few thousand nuclei per tile that leaves the GPU
// nearly idle behind long serial double-precision chains, so here a warp
// takes an object: lanes own 8 histogram bins and 2 co-occurrence cells each,
// and lane 0 forms the moment features. Every floating-point step is an
// explicitly rounded operation (no contraction into fused multiply-adds),
// starting from exact integer moments; only the entropy and the
// homogeneity sum their terms in a tree order instead of bin order.
__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;   // lane 0
}

__global__ void __launch_bounds__(128) obj_feature_kernel(ObjArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_obj = min((int64_t)a.ctl[0], a.max_obj);
    if (k >= n_obj || k >= a.cap) return;   // whole warp
    const ObjInter &o = a.inter[k];
    const int64_t n = o.area;
    const double da = (double)n;
    // histogram: this lane's bins 8 lane .. 8 lane + 7
    uint32_t hb[8];
    uint32_t tot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        hb[q] = o.hist[8 * lane + q];
        tot += hb[q];
    }
    double ent = 0.0;
    int lo = -1, hi = -1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (!hb[q]) continue;
        if (lo < 0) lo = 8 * lane + q;
        hi = 8 * lane + q;
        const double p = __ddiv_rn((double)hb[q], da);
        ent = __dsub_rn(ent, __dmul_rn(p, log2(p)));
    }
    ent = warp_sum_d(ent);
    const uint32_t has = __ballot_sync(0xffffffffu, tot != 0);
    const int vmin = __shfl_sync(0xffffffffu, lo, __ffs(has) - 1);
    const int vmax = __shfl_sync(0xffffffffu, hi, 31 - __clz(has));
    // median: the smallest v with 2 cum(v) >= n (exclusive prefix over lanes)
    uint32_t pre = tot;
#pragma unroll
    for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, pre, o2);
        if (lane >= o2) pre += t;
    }
    int64_t cum = (int64_t)pre - tot;
    int med = -1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        cum += hb[q];
        if (med < 0 && hb[q] && 2 * cum >= n) med = 8 * lane + q;
    }
    const uint32_t mh = __ballot_sync(0xffffffffu, med >= 0);
    med = __shfl_sync(0xffffffffu, med, __ffs(mh) - 1);
    // co-occurrence: this lane's cells 2 lane, 2 lane + 1
    int64_t n2 = 0, con = 0, en = 0;
    double hom = 0.0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c = 2 * lane + q;
        const int64_t g = o.glcm[c], d = (c >> 3) - (c & 7);
        n2 += g;
        con += d * d * g;
        en += g * g;
        hom = __dadd_rn(hom, __ddiv_rn((double)g, (double)(1 + (d < 0 ? -d : d))));
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        n2 += __shfl_down_sync(0xffffffffu, n2, o2);
        con += __shfl_down_sync(0xffffffffu, con, o2);
        en += __shfl_down_sync(0xffffffffu, en, o2);
    }
    hom = warp_sum_d(hom);
    if (lane != 0) return;
    const int4 b = reinterpret_cast<const int4 *>(a.box)[k];
    double *f = a.feat + k * kObjFeat;
    a.out_labels[k] = a.olabel[k];
    f[0] = da;
    f[1] = (double)o.per;
    f[2] = (double)(b.z - b.x + 1);
    f[3] = (double)(b.w - b.y + 1);
    f[4] = __dadd_rn((double)b.x, __ddiv_rn((double)o.sr, da));
    f[5] = __dadd_rn((double)b.y, __ddiv_rn((double)o.sc, da));
    const __int128 mrr = (__int128)n * o.srr - (__int128)o.sr * o.sr;
    const __int128 mcc = (__int128)n * o.scc - (__int128)o.sc * o.sc;
    const __int128 mrc = (__int128)n * o.src - (__int128)o.sr * o.sc;
    const double a2 = __dmul_rn(da, da);
    const double vrr = __ddiv_rn((double)mrr, a2), vcc = __ddiv_rn((double)mcc, a2), vrc = __ddiv_rn((double)mrc, a2);
    const double half = __ddiv_rn(__dadd_rn(vrr, vcc), 2.0), dh = __ddiv_rn(__dsub_rn(vrr, vcc), 2.0);
    const double disc = __dsqrt_rn(__dadd_rn(__dmul_rn(dh, dh), __dmul_rn(vrc, vrc)));
    const double l1 = __dadd_rn(half, disc);
    double l2 = __dsub_rn(half, disc);
    if (l2 < 0.0) l2 = 0.0;
    f[6] = __dmul_rn(4.0, __dsqrt_rn(l1));
    f[7] = __dmul_rn(4.0, __dsqrt_rn(l2));
    f[8] = l1 > 0.0 ? __dsqrt_rn(__dsub_rn(1.0, __ddiv_rn(l2, l1))) : 0.0;
    const double P = (double)o.per;
    f[9] = __ddiv_rn(__dmul_rn(__dmul_rn(4.0, 3.14159265358979323846), da), __dmul_rn(P, P));
    f[10] = __ddiv_rn((double)o.si, da);
    f[11] = __dsqrt_rn(__ddiv_rn((double)((__int128)n * o.sii - (__int128)o.si * o.si), a2));
    f[12] = vmin;
    f[13] = vmax;
    f[14] = med;
    f[15] = ent;
    f[16] = (double)n2;
    if (n2 > 0) {
        f[17] = __ddiv_rn((double)con, (double)n2);
        f[18] = __ddiv_rn((double)en, __dmul_rn((double)n2, (double)n2));
        f[19] = __ddiv_rn(hom, (double)n2);
    } else {
        f[17] = f[18] = f[19] = 0.0;
    }
}

int persistent_grid(const void *fn, size_t smem, int num_sms, int threads = kThreads)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (per_sm > 0 ? per_sm : 1) * num_sms;
}

cudaError_t launch_object_features(const ObjArgs &a, int num_sms, cudaStream_t s, int *launches)
{
    *launches = 0;
    cudaError_t e = launch_enumeration(a, s, launches);
    if (e != cudaSuccess) return e;
    if (a.cap < 1) return cudaSuccess;
    obj_inter_kernel<<<(unsigned)persistent_grid((const void *)obj_inter_kernel, 0, num_sms), kThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    obj_feature_kernel<<<(unsigned)ceil_div((int64_t)a.cap * 32, 128), 128, 0, s>>>(a);
    *launches += 2;
    return cudaGetLastError();
}

// -------------------------------------------------------------- watershed
// Views of one object's box for the watershed block: i = y * bw + x indexes
// the box. The shared-memory view holds D, R, the state and the flags of
// the box; the global view reads L and D in place and keeps R, the state
// and the flags in image-sized arrays (only the object's pixels are
// touched, so objects never share a word).
struct SmemView {
    int32_t *d, *r;
    unsigned long long *st;
    uint8_t *fl;   // bit 0: in the object, bit 1: not a maximum
    __device__ __forceinline__ bool in(int i) const { return fl[i] & 1u; }
    __device__ __forceinline__ int32_t D(int i) const { return d[i]; }
    __device__ __forceinline__ int32_t &R(int i) const { return r[i]; }
    __device__ __forceinline__ unsigned long long &S(int i) const { return st[i]; }
    __device__ __forceinline__ bool nm(int i) const { return fl[i] & 2u; }
    __device__ __forceinline__ void set_nm(int i) const { fl[i] |= 2u; }
};

struct GlobalView {
    const ObjArgs *a;
    int32_t label;
    int r0, c0, bw;
    __device__ __forceinline__ int64_t pix(int i) const
    {
        const int y = i / bw, x = i - y * bw;
        return (int64_t)(r0 + y) * a->W + (c0 + x);
    }
    __device__ __forceinline__ bool in(int i) const
    {
        const int y = i / bw, x = i - y * bw;
        return a->L[(int64_t)(r0 + y) * a->ld_L + c0 + x] == label;
    }
    __device__ __forceinline__ int32_t D(int i) const
    {
        const int y = i / bw, x = i - y * bw;
        return a->D[(int64_t)(r0 + y) * a->ld_D + c0 + x];
    }
    __device__ __forceinline__ int32_t &R(int i) const { return a->R[pix(i)]; }
    __device__ __forceinline__ unsigned long long &S(int i) const { return a->st[pix(i)]; }
    __device__ __forceinline__ bool nm(int i) const { return *reinterpret_cast<volatile uint8_t *>(a->nm + pix(i)) != 0; }
    __device__ __forceinline__ void set_nm(int i) const { a->nm[pix(i)] = 1u; }
};

// The threads that work on one object: a whole block (large boxes) or one
// warp (small boxes, eight objects per block in flight).
template <int NT>
struct BlockGroup {
    static constexpr int size = NT;
    int *red;   // shared reduction word
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
    __device__ __forceinline__ int32_t max(int32_t v) const
    {
        v = __reduce_max_sync(0xffffffffu, v);
        __syncthreads();
        if (threadIdx.x == 0) *red = -1;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicMax(red, v);
        __syncthreads();
        return *red;
    }
};


// Largest D below `below` over the object's pixels that have no basin yet
// (-1: none). The levels strictly descend, so the flooding ends; a pixel
// left unlabelled at one level (not yet connected to a basin) is taken at a
// lower one, when its level set joins a basin.
template <class V, class G>
__device__ __forceinline__ int32_t max_unlabelled(const V &v, const G &g, int m, int32_t below)
{
    int32_t mx = -1;
    for (int i = g.rank(); i < m; i += G::size)
        if (v.in(i) && v.S(i) == kUnl && v.D(i) < below) mx = max(mx, v.D(i));
    return g.max(mx);
}

template <class V, class G>
__device__ void watershed_object(const V &v, const G &g, const ObjArgs &a, int r0, int c0, int bh, int bw)
{
    const int m = bh * bw;   // H * W <= 2^30
    auto for_nbrs = [&](int i, auto &&fn) {
        const int y = i / bw, x = i - y * bw;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if (dy == 0 && dx == 0) continue;
                const int yy = y + dy, xx = x + dx;
                if (yy < 0 || yy >= bh || xx < 0 || xx >= bw) continue;
                const int j = yy * bw + xx;
                if (v.in(j)) fn(j);
            }
    };
    // 1. h-maxima transform: R = reconstruction of max(D - h, 0) under D
    for (int i = g.rank(); i < m; i += G::size)
        if (v.in(i)) v.R(i) = max(v.D(i) - a.h, 0);
    g.sync();
    for (;;) {
        int ch = 0;
        for (int i = g.rank(); i < m; i += G::size) {
            if (!v.in(i)) continue;
            volatile int32_t &Ri = v.R(i);
            int32_t mx = Ri;
            for_nbrs(i, [&](int j) { mx = max(mx, *(volatile int32_t *)&v.R(j)); });
            mx = min(mx, v.D(i));
            if (mx > Ri) {
                Ri = mx;
                ch = 1;
            }
        }
        if (!g.any(ch)) break;
    }
    // 2. not a maximum: a higher neighbour, or an equal one that is not
    for (int i = g.rank(); i < m; i += G::size) {
        if (!v.in(i)) continue;
        bool hi = false;
        const int32_t ri = v.R(i);
        for_nbrs(i, [&](int j) { hi |= v.R(j) > ri; });
        if (hi) v.set_nm(i);
    }
    g.sync();
    for (;;) {
        int ch = 0;
        for (int i = g.rank(); i < m; i += G::size) {
            if (!v.in(i) || v.nm(i)) continue;
            bool f = false;
            const int32_t ri = v.R(i);
            for_nbrs(i, [&](int j) { f |= v.R(j) == ri && v.nm(j); });
            if (f) {
                v.set_nm(i);
                ch = 1;
            }
        }
        if (!g.any(ch)) break;
    }
    // 3. markers: each plateau of maxima takes its smallest linear index
    for (int i = g.rank(); i < m; i += G::size) {
        if (!v.in(i)) continue;
        const int y = i / bw, x = i - y * bw;
        v.S(i) = v.nm(i) ? kUnl : (unsigned long long)(uint32_t)((r0 + y) * a.W + (c0 + x));
    }
    g.sync();
    for (;;) {
        int ch = 0;
        for (int i = g.rank(); i < m; i += G::size) {
            if (!v.in(i) || v.nm(i)) continue;
            volatile unsigned long long &Si = v.S(i);
            unsigned long long mn = Si;
            for_nbrs(i, [&](int j) {
                if (!v.nm(j)) {
                    const unsigned long long sj = *(volatile unsigned long long *)&v.S(j);
                    mn = sj < mn ? sj : mn;
                }
            });
            if (mn < Si) {
                Si = mn;
                ch = 1;
            }
        }
        if (!g.any(ch)) break;
    }
    int nb = 0;
    for (int i = g.rank(); i < m; i += G::size) {
        if (!v.in(i) || v.nm(i)) continue;
        const int y = i / bw, x = i - y * bw;
        nb += v.S(i) == (unsigned long long)(uint32_t)((r0 + y) * a.W + (c0 + x));
    }
    nb = __reduce_add_sync(0xffffffffu, nb);
    if ((g.rank() & 31) == 0 && nb) {
        atomicAdd(a.ctl + 2, (uint32_t)nb);
        if (a.n_basins) atomicAdd(a.n_basins, nb);
    }
    // 4. flooding by levels of D, highest first, in breadth-first layers. A
    // level ends after the first layer whose new pixels have no unlabelled
    // neighbour with D >= t (the next layer could only take such pixels);
    // the next level, the largest D below t among unlabelled pixels, is
    // found during the level's first layer (those pixels do not change
    // within the level).
    uint32_t layer = 1;
    int32_t t = max_unlabelled(v, g, m, INT32_MAX);
    while (t >= 0) {
        int32_t next = -1;
        for (bool first = true;; first = false) {
            int more = 0;
            for (int i = g.rank(); i < m; i += G::size) {
                if (!v.in(i) || v.S(i) != kUnl) continue;
                const int32_t di = v.D(i);
                if (di < t) {
                    if (first) next = max(next, di);
                    continue;
                }
                uint32_t mn = 0xffffffffu;
                for_nbrs(i, [&](int j) {
                    const unsigned long long sj = *(volatile unsigned long long *)&v.S(j);
                    if (sj != kUnl && (uint32_t)(sj >> 32) < layer) mn = min(mn, (uint32_t)sj);
                });
                if (mn != 0xffffffffu) {
                    *(volatile unsigned long long *)&v.S(i) = ((unsigned long long)layer << 32) | mn;
                    for_nbrs(i, [&](int j) {
                        more |= *(volatile unsigned long long *)&v.S(j) == kUnl && v.D(j) >= t;
                    });
                }
            }
            ++layer;
            if (first) next = g.max(next);
            if (!g.any(more)) break;
        }
        t = next;
    }
    // 5. basins out
    for (int i = g.rank(); i < m; i += G::size) {
        if (!v.in(i)) continue;
        const int y = i / bw, x = i - y * bw;
        a.basins[(int64_t)(r0 + y) * a.ld_B + (c0 + x)] = (int32_t)(uint32_t)v.S(i);
    }
}

constexpr int kWsThreads = 256;
constexpr int kWsLargePx = 1024;   // boxes above this start first
constexpr size_t kWsSmemBytes = (size_t)kWsSmemPx * (4 + 4 + 8 + 1) + 64;

// Carves a shared-memory view of `px` pixels at base (8-byte aligned).
__device__ __forceinline__ SmemView smem_view(unsigned char *base, int px)
{
    SmemView sv;
    sv.st = reinterpret_cast<unsigned long long *>(base);
    sv.d = reinterpret_cast<int32_t *>(sv.st + px);
    sv.r = sv.d + px;
    sv.fl = reinterpret_cast<uint8_t *>(sv.r + px);
    return sv;
}

// Thread per object: objects with a box of more than kWsLargePx pixels go to
// the front of `order`, the others to the back, so the long ones start first.
__global__ void obj_classify_kernel(ObjArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_obj = (int)min((int64_t)a.ctl[0], a.max_obj);
    if (k >= n_obj) return;
    const int4 b = reinterpret_cast<const int4 *>(a.box)[k];
    const int m = (b.z - b.x + 1) * (b.w - b.y + 1);
    if (m > kWsLargePx) a.order[atomicAdd(a.ctl + 3, 1u)] = k;
    else a.order[a.max_obj - 1 - atomicAdd(a.ctl + 4, 1u)] = k;
}

// A block per object, in the order above: the box in shared memory up to
// kWsSmemPx pixels, else in the image-sized global arrays.
__global__ void __launch_bounds__(kWsThreads) obj_watershed_kernel(ObjArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int slot, red;
    const SmemView sv = smem_view(smem, kWsSmemPx);
    const BlockGroup<kWsThreads> g{&red};
    const int n_obj = (int)min((int64_t)a.ctl[0], a.max_obj);
    const int n_big = (int)a.ctl[3];
    for (;;) {
        const int q = next_object(a, n_obj, &slot);
        if (q < 0) return;
        const int k = q < n_big ? a.order[q] : a.order[a.max_obj - 1 - (q - n_big)];
        const int4 b = reinterpret_cast<const int4 *>(a.box)[k];
        const int32_t l = a.olabel[k];
        const int bh = b.z - b.x + 1, bw = b.w - b.y + 1;
        const int m = bh * bw;   // H * W <= 2^30
        if (m <= kWsSmemPx) {
            for (int i = threadIdx.x; i < m; i += kWsThreads) {
                const int y = i / bw, x = i - y * bw;
                const int r = b.x + y, c = b.y + x;
                const bool in = a.L[(int64_t)r * a.ld_L + c] == l;
                sv.fl[i] = in ? 1u : 0u;
                sv.d[i] = in ? a.D[(int64_t)r * a.ld_D + c] : 0;
            }
            __syncthreads();
            watershed_object(sv, g, a, b.x, b.y, bh, bw);
        } else {
            GlobalView gv{&a, l, b.x, b.y, bw};
            for (int i = threadIdx.x; i < m; i += kWsThreads)
                if (gv.in(i)) a.nm[gv.pix(i)] = 0u;
            __syncthreads();
            watershed_object(gv, g, a, b.x, b.y, bh, bw);
        }
    }
}

cudaError_t launch_watershed(const ObjArgs &a, int num_sms, cudaStream_t s, int *launches)
{
    *launches = 0;
    cudaError_t e = launch_enumeration(a, s, launches);
    if (e != cudaSuccess) return e;
    obj_classify_kernel<<<(unsigned)ceil_div(a.max_obj, 256), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(obj_watershed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemBytes);
    if (e != cudaSuccess) return e;
    obj_watershed_kernel<<<(unsigned)persistent_grid((const void *)obj_watershed_kernel, kWsSmemBytes, num_sms,
                                                     kWsThreads),
                           kWsThreads, kWsSmemBytes, s>>>(a);
    *launches += 2;
    return cudaGetLastError();
}

}  // namespace rtk
