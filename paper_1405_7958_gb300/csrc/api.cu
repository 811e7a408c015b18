// C-ABI entry points of the segmentation library (declared in rt.h):
// argument validation, the context and its device workspace, and the
// launch sequence of every operation and of the segmentation chain.
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ccl.cuh"
#include "common.cuh"
#include "edt.cuh"
#include "features.cuh"
#include "fill.cuh"
#include "mlp.cuh"
#include "objects.cuh"
#include "recon.cuh"
#include "synth.cuh"

using namespace rtk;

struct PhaseRec {
    int phase;
    cudaEvent_t a, b;
};

struct rt_ctx {
    int device = 0;
    int num_sms = 0;
    void *ws = nullptr;       // device workspace
    size_t ws_bytes = 0;
    uint32_t *visits_dev = nullptr;  // [visits, iterations] of the last reconstruction (workspace)
    int64_t launches = 0;     // kernels launched
    bool timing = false;
    const uint16_t *picker_wb = nullptr;   // attached picker (caller-owned device memory)
    const float *picker_norm = nullptr;
    int32_t *picks_host = nullptr;         // pinned, mapped: picker classes of the last learned chunk
    int32_t *picks_mapped = nullptr;       // the same memory as the device sees it
    cudaEvent_t picks_ev = nullptr;        // recorded after their copy (not under stream capture)
    bool picks_ev_valid = false;
    int n_last_picks = 0;
    PickTable classes{{0, 0, 0, 0}, {4, 12, 24, 12}};   // picker classes (rt_set_picker_classes); entry 3 per call
    int max_iters = 0;                     // limits of the single-operation entry points (rt_set_limits)
    uint64_t timeout_ns = 0;
    int64_t fq_cap = 0;                    // entries per global frontier queue (0: one per padded pixel)
    std::vector<PhaseRec> recs;
    std::vector<cudaEvent_t> pool;
};

namespace {

cudaEvent_t take_event(rt_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one phase with events on the stream when timing is enabled.
class Phase {
  public:
    Phase(rt_ctx *ctx, int phase, cudaStream_t s) : ctx_(ctx), s_(s)
    {
        if (!ctx->timing) return;
        rec_.phase = phase;
        rec_.a = take_event(ctx);
        rec_.b = take_event(ctx);
        cudaEventRecord(rec_.a, s);
    }
    ~Phase()
    {
        if (!ctx_->timing || !rec_.a) return;
        cudaEventRecord(rec_.b, s_);
        ctx_->recs.push_back(rec_);
    }

  private:
    rt_ctx *ctx_;
    cudaStream_t s_;
    PhaseRec rec_{0, nullptr, nullptr};
};

constexpr uint64_t kSweepTimeoutNs = 20000000000ull;   // default bound on one propagation (20 s)

// Bump allocator over the context workspace (256-byte aligned pieces).
struct Carve {
    size_t off = 0;
    char *base = nullptr;
    template <class T>
    T *take(size_t count)
    {
        off = (size_t)round_up((int64_t)off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
        dev_ = dev;
    }
    ~DeviceGuard()
    {
        if (prev_ != dev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0, dev_ = 0;
};

rt_status ensure_ws(rt_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return RT_OK;
    if (ctx->ws) {
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        ctx->visits_dev = nullptr;
    }
    size_t want = (size_t)round_up((int64_t)bytes, 1 << 20);
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return RT_ENOMEM;
    }
    ctx->ws_bytes = want;
    return RT_OK;
}

bool bad_dims(int H, int W) { return H < 1 || W < 1 || H > kMaxSide || W > kMaxSide; }

bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + nb && pb < pa + na;
}

size_t span(int H, int64_t ld, size_t elem, int W) { return ((size_t)(H - 1) * ld + W) * elem; }

rt_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return RT_OK;
    cudaGetLastError();
    return RT_ECUDA;
}

// Zeroes n words of device memory. The chain clears its control words with
// this kernel rather than cudaMemsetAsync, so that nothing in it can wait
// behind the caller's copies on a copy engine.
__global__ void zero_words_kernel(uint32_t *p, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0u;
}
cudaError_t zero_words(void *p, int n, cudaStream_t s)
{
    zero_words_kernel<<<(n + 255) / 256 < 16 ? (n + 255) / 256 : 16, 256, 0, s>>>(static_cast<uint32_t *>(p), n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- recon
struct ReconWs {
    uint32_t *flags;   // per tile
    uint32_t *ctl;     // kCtlWords control words (recon.cuh)
    int32_t *err;
    int32_t *map;      // kGroups x ntiles tile lists when the variant is chosen per image
    uint32_t *fq[2];   // RT_FRONTIER: global frontier queues (fq_cap entries each), or null
    uint32_t *fctl;    //              their kFqCtlWords control words
    uint32_t fq_cap;
};

// Whether a call runs RT_FRONTIER somewhere: as its variant, or as one of
// the picker's classes under the learned policy (ctx NULL: the default
// classes, all RT_RASTER).
bool uses_frontier(const rt_ctx *ctx, int variant, bool learned)
{
    if (variant == RT_FRONTIER) return true;
    if (!learned || !ctx) return false;
    for (int c = 0; c < kPickClasses; ++c)
        if (ctx->classes.group[c] == RT_FRONTIER - RT_RASTER) return true;
    return false;
}

// Entries of each global frontier queue for batch b: the context's setting,
// else one per padded pixel of the batch.
uint32_t frontier_capacity(const rt_ctx *ctx, const ReconBatch &b)
{
    int64_t px = 0;
    for (int i = 0; i < b.n; ++i) px += (int64_t)b.img[i].Hp * b.img[i].Wp;
    const int64_t cap = ctx && ctx->fq_cap > 0 ? ctx->fq_cap : px;
    return (uint32_t)(cap < 0xffffffffLL ? cap : 0xffffffffLL);
}

// Reserve the sweep control block and per-image padded buffers (and the
// global frontier queues when fq_cap > 0).
void carve_recon(Carve &cv, ReconBatch &b, ReconWs &w, bool grouped = false, uint32_t fq_cap = 0)
{
    w.flags = cv.take<uint32_t>((size_t)b.ntiles);
    w.ctl = cv.take<uint32_t>(kCtlWords);
    w.err = cv.take<int32_t>(1);
    w.map = grouped ? cv.take<int32_t>((size_t)kGroups * b.ntiles) : nullptr;
    w.fq_cap = fq_cap;
    w.fq[0] = fq_cap ? cv.take<uint32_t>(fq_cap) : nullptr;
    w.fq[1] = fq_cap ? cv.take<uint32_t>(fq_cap) : nullptr;
    w.fctl = fq_cap ? cv.take<uint32_t>(kFqCtlWords) : nullptr;
    for (int i = 0; i < b.n; ++i) {
        ReconImage &d = b.img[i];
        d.Rw = cv.take<uint8_t>((size_t)d.Hp * d.Wp);
        d.Iw = cv.take<uint8_t>((size_t)d.Hp * d.Wp);
        d.Cw = cv.take<uint8_t>((size_t)d.tiles_x * d.tiles_y * kEdgeBytes);
    }
}

// Enqueue init + propagation for a batch whose buffers are carved. `err`
// receives the device status. With `pick` (device, one picker class per
// image) every image propagates with its own variant: one launch per variant
// group over the group's tile list, with no host round trip.
// Bounds of a propagation: max_iters > 0 allows max_iters tile visits per
// 32 x 64 tile on average; timeout_ns bounds its device time.
struct Limits {
    int max_iters;
    uint64_t timeout_ns;
    int strip = 0;   // tiles per warp strip of the raster propagation (0: the library's choice)
};

Limits ctx_limits(const rt_ctx *ctx) { return {ctx->max_iters, ctx->timeout_ns ? ctx->timeout_ns : kSweepTimeoutNs}; }

int default_max_local(int variant) { return variant == RT_HYBRID || variant == RT_FRONTIER ? 64 : 12; }

// sweep budget of every raster tile in a launch shared by several tiles
int shared_raster_budget(int max_local) { return max_local > 0 ? max_local : default_max_local(RT_RASTER); }

// In a launch shared by several tiles every raster class runs at the plain
// budget, so when the plain schedule and every class of the picker are
// raster, no pick can change a tile's schedule and the picker is not run.
bool picks_matter(const rt_ctx *ctx, const rt_seg_params &P, int n_tiles)
{
    if (n_tiles == 1) return true;
    if (P.variant != RT_AUTO && P.variant != RT_RASTER) return true;
    for (int c = 0; c < kPickClasses; ++c)
        if (ctx->classes.group[c] != 0) return true;
    return false;
}

rt_status run_recon(rt_ctx *ctx, ReconBatch &b, ReconWs &w, int conn, int variant, int max_local, int32_t *err,
                    cudaStream_t s, Limits lim, const int32_t *pick = nullptr)
{
    if (variant == RT_AUTO) variant = RT_RASTER;
    // the learned policy's schedules: the picker's classes, then the call's
    // plain schedule as the fall-back entry
    PickTable table = ctx->classes;
    table.group[kPickClasses] = variant - RT_RASTER;
    table.max_local[kPickClasses] = max_local > 0 ? max_local : default_max_local(variant);
    // A frontier entry names its tile in 21 bits, and the queues need their
    // workspace: without either, frontier schedules run as RT_HYBRID (the
    // same dense first pass, then per-tile queues; same output).
    const bool fq_ok = w.fq_cap > 0 && b.ntiles < kFqMaxTiles;
    for (int e = 0; e < kPickEntries; ++e)
        if (table.group[e] == RT_FRONTIER - RT_RASTER && !fq_ok) table.group[e] = RT_HYBRID - RT_RASTER;
    if (variant == RT_FRONTIER && !fq_ok) variant = RT_HYBRID;
    // The picker learned its budgets on lone tiles, where a tile's latency
    // sets the time and short visits can win. Tiles that share a launch with
    // others are bound by its throughput instead: there a budget below the
    // plain one only adds visits, and one above it adds visits too once
    // revisits start at the moved side of the halo (measured on uneven and
    // 4K batches). Raster classes run at the plain budget in shared launches.
    if (pick && b.n > 1)
        for (int c = 0; c < kPickClasses; ++c)
            if (table.group[c] == 0) table.max_local[c] = shared_raster_budget(max_local);
    // RT_RASTER / RT_QUEUE: every tile starts flagged for a dense visit (the
    // queue visit then seeds every pixel); RT_HYBRID / RT_FRONTIER: nothing
    // flagged, the dense pass over all tiles flags what remains.
    const uint32_t flag0 = variant == RT_HYBRID || variant == RT_FRONTIER ? 0u : 2u;
    RT_CUDA_TRY(zero_words(w.ctl, kCtlWords, s));
    ctx->launches += 1;
    {
        Phase ph(ctx, RT_PHASE_RECON_INIT, s);
        RT_CUDA_TRY(launch_recon_init(b, w.flags, w.ctl, flag0, pick, table, w.map, err, s));
        ctx->launches += 1;
    }
    ctx->visits_dev = w.ctl + kCtlVisits;
    SweepParams p;
    p.b = b;
    p.ntiles = b.ntiles;
    p.flags = w.flags;
    p.pending = w.ctl + kCtlPending;
    p.err = err;
    p.visits = w.ctl + kCtlVisits;
    p.timeout_ns = lim.timeout_ns;
    p.seg_max = lim.strip;
    const int64_t bound = (int64_t)lim.max_iters * b.ntiles;
    p.max_visits = lim.max_iters > 0 ? (uint32_t)(bound < 0xffffffffLL ? bound : 0xffffffffLL) : 0u;
    p.spent = w.ctl + kCtlSpent;
    p.abort = w.ctl + kCtlAbort;
    p.map = nullptr;
    p.nvirt = nullptr;
    p.pick = pick;
    p.table = table;
    p.fq[0] = w.fq[0];
    p.fq[1] = w.fq[1];
    p.fq_cap = w.fq_cap;
    p.fctl = w.fctl;
    int grid = 0;
    Phase ph(ctx, RT_PHASE_RECON_SWEEP, s);
    bool used[kGroups] = {false, false, false, false};   // groups some schedule of the table propagates in
    for (int e = 0; e < kPickEntries; ++e)
        if (table.group[e] >= 0 && table.group[e] < kGroups) used[table.group[e]] = true;
    for (int g = 0; g < (pick ? kGroups : 1); ++g) {
        if (pick && !used[g]) continue;
        const int v = pick ? RT_RASTER + g : variant;
        if (pick) {
            p.map = w.map + (size_t)g * b.ntiles;
            p.nvirt = w.ctl + kCtlGroupCount + g;
            p.pending = w.ctl + kCtlGroupPending + g;
        }
        p.max_local = max_local > 0 ? max_local : default_max_local(v);
        if (v == RT_HYBRID || v == RT_FRONTIER) {
            RT_CUDA_TRY(launch_recon_dense(p, conn, s));
            ctx->launches += 1;
        }
        if (v == RT_FRONTIER) {
            // seed and drain the global frontier queues; the directional
            // sweeps that follow find nothing flagged unless a queue
            // overflowed
            RT_CUDA_TRY(zero_words(w.fctl, kFqCtlWords, s));
            ctx->launches += 1;
            RT_CUDA_TRY(launch_recon_seed(p, conn, s));
            RT_CUDA_TRY(launch_recon_frontier(p, conn, ctx->num_sms, s, &grid));
            ctx->launches += 2;
            p.max_local = max_local > 0 ? max_local : default_max_local(RT_RASTER);
        }
        ctx->launches += 1;
        RT_CUDA_TRY(launch_recon_persistent(p, conn, v == RT_RASTER || v == RT_FRONTIER ? 0 : 1, ctx->num_sms, s,
                                            &grid));
    }
    return RT_OK;
}

void add_image(ReconBatch &b, const uint8_t *marker, int64_t ld_marker, const uint8_t *mask, int64_t ld_mask,
               int H, int W, int h_offset)
{
    ReconImage &d = b.img[b.n];
    std::memset(&d, 0, sizeof(d));
    d.marker = marker;
    d.ld_marker = ld_marker;
    d.mask = mask;
    d.ld_mask = ld_mask;
    d.h_offset = h_offset;
    plan_recon_image(d, H, W);
    d.tile_base = b.ntiles;
    b.ntiles += d.tiles_x * d.tiles_y;
    const int64_t words = (int64_t)d.Hp * d.Wp / 4;
    if (words > b.max_words) b.max_words = words;
    b.n++;
}

// the tiles' status words: the device status of the chunk that carried them
struct StatusOut {
    int32_t *dst[kMaxImgs];
};
__global__ void copy_status_kernel(const int32_t *src, StatusOut o, int n)
{
    if ((int)threadIdx.x < n && o.dst[threadIdx.x]) *o.dst[threadIdx.x] = *src;
}

// the picker's classes of a chunk into the caller-visible pinned buffer
// src NULL: every tile ran the plain schedule (class kPickClasses)
__global__ void copy_picks_kernel(const int32_t *src, int32_t *dst, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src ? src[i] : kPickClasses;
    __threadfence_system();
}

bool bad_params(const rt_seg_params &P)
{
    if (P.conn_recon != 4 && P.conn_recon != 8) return true;
    if (P.conn_fill != 4 && P.conn_fill != 8) return true;
    if (P.h_offset < 0 || P.h_offset > 255 || P.threshold < 0 || P.threshold > 256) return true;
    if (P.variant < RT_AUTO || P.variant > RT_FRONTIER) return true;
    if (P.policy != RT_POLICY_PLAIN && P.policy != RT_POLICY_LEARNED) return true;
    if (P.max_local < 0 || P.max_iters < 0 || P.timeout_ms < 0) return true;
    if (P.strip_tiles < 0 || P.strip_tiles > 32) return true;
    if (P.pick_min_prob < 0 || P.pick_min_prob > 1000) return true;
    return false;
}

bool bad_tile(const rt_tile &t)
{
    if (!t.img || !t.labels || !t.d2 || bad_dims(t.H, t.W)) return true;
    if (t.ld_img < t.W || t.ld_labels < t.W || t.ld_d2 < t.W) return true;
    if (t.recon && t.ld_recon < t.W) return true;
    if (t.filled && t.ld_filled < t.W) return true;
    return false;
}

// Workspace of one chunk (up to kMaxImgs tiles) of rt_segment_batch. Every
// stage runs once for the whole chunk, so every tile has its own buffers:
// padded reconstruction copies, the binary image, the fill's bit planes, the
// union-find arrays, the kept-pixel bit plane and the distance transform's
// column masks.
struct Chunk {
    ReconBatch b;
    ReconWs w;
    FeatBatch fb;
    float *feat = nullptr;
    int32_t *picks = nullptr;
    FillBatch fill;
    uint32_t *fill_flags = nullptr, *fill_pending = nullptr;
    UfBatch uf;
    EdtBitsBatch eb;
};

// Lays chunk [c0, c0 + cn) out in cv. With cv.base == nullptr only the size
// is measured (cv.off); no pointer is formed.
void layout_chunk(Carve &cv, Chunk &c, const rt_tile *tiles, int c0, int cn, const rt_seg_params &P, bool learned,
                  const rt_ctx *ctx)
{
    const bool real = cv.base != nullptr;
    std::memset(&c.b, 0, sizeof(c.b));
    for (int i = 0; i < cn; ++i) {
        const rt_tile &t = tiles[c0 + i];
        add_image(c.b, nullptr, 0, t.img, t.ld_img, t.H, t.W, P.h_offset);
    }
    carve_recon(cv, c.b, c.w, learned,
                uses_frontier(ctx, P.variant, learned) ? frontier_capacity(ctx, c.b) : 0u);
    if (learned) {
        c.fb.n = cn;
        for (int i = 0; i < cn; ++i) {
            const rt_tile &t = tiles[c0 + i];
            const size_t nb = (size_t)((t.H + 7) / 8) * ((t.W + 7) / 8);
            FeatImage &d = c.fb.img[i];
            d.img = t.img;
            d.ld = t.ld_img;
            d.H = t.H;
            d.W = t.W;
            d.hist = cv.take<uint32_t>(256);
            d.acc = cv.take<unsigned long long>(4);
            d.dark = cv.take<uint8_t>(nb);
            d.bmax = cv.take<uint8_t>(nb);
        }
        c.feat = cv.take<float>((size_t)cn * kNumFeatures);
        c.picks = cv.take<int32_t>((size_t)cn);
    }
    c.fill.n = 0;
    c.uf.n = 0;
    c.eb.n = 0;
    int fill_tiles = 0;
    for (int i = 0; i < cn; ++i) {
        const rt_tile &t = tiles[c0 + i];
        const int H = t.H, W = t.W;
        ReconImage &d = c.b.img[i];
        // B = (R < threshold); F replaces it in place unless the caller wants F
        uint8_t *B = cv.take<uint8_t>((size_t)H * W);
        d.out = t.recon;
        d.ld_out = t.ld_recon;
        d.bin = B;
        d.ld_bin = W;
        uint8_t *F = t.filled ? t.filled : B;
        const int64_t ldF = t.filled ? t.ld_filled : W;
        char *fws = cv.take<char>(fill_image_bytes(H, W));
        if (real) fill_add(c.fill, B, W, F, ldF, H, W, fws);
        fill_tiles += (int)(ceil_div(H, kFillTH) * ceil_div(W, kFillTW));
        char *uws = cv.take<char>(uf_workspace_bytes(H, W));
        uint32_t *kept = cv.take<uint32_t>((size_t)H * ceil_div(W, 32));
        char *ews = cv.take<char>(edt_bits_workspace_bytes(H, W));
        if (real) {
            UfImage u;
            std::memset(&u, 0, sizeof(u));
            uf_carve(u, uws, H, W);
            u.in = F;
            u.ld_in = ldF;
            u.labels = t.labels;
            u.ld_lab = t.ld_labels;
            u.n_kept = t.n_kept;
            u.fgbits = kept;
            uf_add(c.uf, u);
            edt_bits_add(c.eb, kept, H, W, t.d2, t.ld_d2, ews);
        }
    }
    c.fill_flags = cv.take<uint32_t>((size_t)fill_tiles);
    c.fill_pending = cv.take<uint32_t>(1);
    c.uf.amin = P.min_area;
    c.uf.amax = P.max_area;
}

// Workspace bytes rt_segment_batch needs for these tiles (the largest chunk).
size_t segment_ws_bytes(const rt_tile *tiles, int n, const rt_seg_params &P, bool learned, const rt_ctx *ctx)
{
    size_t most = 0;
    for (int c0 = 0; c0 < n; c0 += kMaxImgs) {
        const int cn = n - c0 < kMaxImgs ? n - c0 : kMaxImgs;
        Carve cv;
        Chunk c;
        layout_chunk(cv, c, tiles, c0, cn, P, learned, ctx);
        most = cv.off > most ? cv.off : most;
    }
    return most;
}

}  // namespace

// ================================================================= C ABI
extern "C" {

int rt_version(void) { return 201; }

const char *rt_status_str(int status)
{
    switch (status) {
    case RT_OK: return "RT_OK";
    case RT_EINVAL: return "RT_EINVAL: invalid argument";
    case RT_ENOMEM: return "RT_ENOMEM: device workspace allocation failed";
    case RT_ECUDA: return "RT_ECUDA: CUDA runtime error";
    case RT_ETIMEOUT: return "RT_ETIMEOUT: device iteration or wait bound reached";
    case RT_EMARKER: return "RT_EMARKER: marker above mask (clamped)";
    case RT_EQUEUE: return "RT_EQUEUE: frontier queue overflow";
    case RT_EUNAVAIL: return "RT_EUNAVAIL: variant or feature unavailable";
    case RT_ESIZE: return "RT_ESIZE: image larger than the fixed scratch of the allocation-free entry point";
    default: return "unknown rt_status";
    }
}

rt_status rt_create(rt_ctx **ctx, int device, size_t workspace_bytes)
{
    if (!ctx) return RT_EINVAL;
    *ctx = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return RT_ECUDA;
    }
    rt_ctx *c = new (std::nothrow) rt_ctx;
    if (!c) return RT_ENOMEM;
    c->device = device;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaHostAlloc((void **)&c->picks_host, kMaxImgs * sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->picks_mapped, c->picks_host, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->picks_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->picks_host) cudaFreeHost(c->picks_host);
        delete c;
        return RT_ECUDA;
    }
    if (workspace_bytes > 0 && ensure_ws(c, workspace_bytes) != RT_OK) {
        cudaEventDestroy(c->picks_ev);
        cudaFreeHost(c->picks_host);
        delete c;
        return RT_ENOMEM;
    }
    *ctx = c;
    return RT_OK;
}

rt_status rt_set_limits(rt_ctx *ctx, int max_iters, int timeout_ms)
{
    if (!ctx || max_iters < 0 || timeout_ms < 0) return RT_EINVAL;
    ctx->max_iters = max_iters;
    ctx->timeout_ns = (uint64_t)timeout_ms * 1000000ull;
    return RT_OK;
}

size_t rt_segment_workspace_bytes(const rt_ctx *ctx, const rt_tile *tiles, int n, const rt_seg_params *params)
{
    if ((!tiles && n > 0) || n < 0 || !params || bad_params(*params)) return 0;
    for (int i = 0; i < n; ++i)
        if (bad_tile(tiles[i])) return 0;
    return segment_ws_bytes(tiles, n, *params, params->policy == RT_POLICY_LEARNED, ctx);
}

rt_status rt_set_queue_capacity(rt_ctx *ctx, int64_t entries)
{
    if (!ctx || entries < 0 || entries > 0xffffffffLL) return RT_EINVAL;
    ctx->fq_cap = entries;
    return RT_OK;
}

void rt_destroy(rt_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
    }
    for (const PhaseRec &r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    if (ctx->picks_ev) cudaEventDestroy(ctx->picks_ev);
    if (ctx->picks_host) cudaFreeHost(ctx->picks_host);
    delete ctx;
}

size_t rt_workspace_bytes(const rt_ctx *ctx) { return ctx ? ctx->ws_bytes : 0; }

rt_status rt_timing_enable(rt_ctx *ctx, int enable)
{
    if (!ctx) return RT_EINVAL;
    ctx->timing = enable != 0;
    return RT_OK;
}

rt_status rt_timing_read(rt_ctx *ctx, double *ms, int64_t *count, int reset)
{
    if (!ctx) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    for (const PhaseRec &r : ctx->recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            cudaGetLastError();
            return RT_ECUDA;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            return RT_ECUDA;
        }
        if (r.phase >= 0 && r.phase < RT_NPHASES) {
            if (ms) ms[r.phase] += t;
            if (count) count[r.phase] += 1;
        }
    }
    if (reset) {
        for (const PhaseRec &r : ctx->recs) {
            ctx->pool.push_back(r.a);
            ctx->pool.push_back(r.b);
        }
        ctx->recs.clear();
    }
    return RT_OK;
}

int64_t rt_kernel_launches(const rt_ctx *ctx) { return ctx ? ctx->launches : 0; }

rt_status rt_recon_stats(rt_ctx *ctx, int64_t *visits, int64_t *iterations, int64_t *pops)
{
    if (!ctx) return RT_EINVAL;
    uint32_t v[3] = {0, 0, 0};
    if (ctx->visits_dev) {
        DeviceGuard g(ctx->device);
        if (cudaMemcpy(v, ctx->visits_dev, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return RT_ECUDA;
        }
    }
    if (visits) *visits = v[0];
    if (iterations) *iterations = v[1];
    if (pops) *pops = v[2];
    return RT_OK;
}

rt_status rt_marker(rt_ctx *ctx, const uint8_t *mask, int64_t ld_mask, uint8_t *marker, int64_t ld_marker, int H,
                    int W, int h_offset, void *stream)
{
    if (!ctx || !mask || !marker || bad_dims(H, W) || ld_mask < W || ld_marker < W || h_offset < 0 ||
        h_offset > 255)
        return RT_EINVAL;
    if (overlaps(mask, span(H, ld_mask, 1, W), marker, span(H, ld_marker, 1, W))) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    Phase ph(ctx, RT_PHASE_RECON_INIT, (cudaStream_t)stream);
    ctx->launches += 1;
    return cuda_status(launch_marker(mask, ld_mask, marker, ld_marker, H, W, h_offset, (cudaStream_t)stream));
}

rt_status rt_reconstruct(rt_ctx *ctx, const uint8_t *marker, int64_t ld_marker, const uint8_t *mask,
                         int64_t ld_mask, uint8_t *out, int64_t ld_out, int H, int W, int conn, int variant,
                         int h_offset, int32_t *dev_status, void *stream)
{
    if (!ctx || !mask || !out || bad_dims(H, W) || ld_mask < W || ld_out < W) return RT_EINVAL;
    if (conn != 4 && conn != 8) return RT_EINVAL;
    if (variant < RT_AUTO || variant > RT_FRONTIER) return RT_EINVAL;
    if (marker && ld_marker < W) return RT_EINVAL;
    if (!marker && (h_offset < 0 || h_offset > 255)) return RT_EINVAL;
    if (overlaps(out, span(H, ld_out, 1, W), mask, span(H, ld_mask, 1, W))) return RT_EINVAL;
    if (marker && marker != out && overlaps(out, span(H, ld_out, 1, W), marker, span(H, ld_marker, 1, W)))
        return RT_EINVAL;
    if (marker && marker == out && ld_marker != ld_out) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;

    ReconBatch b;
    std::memset(&b, 0, sizeof(b));
    add_image(b, marker, ld_marker, mask, ld_mask, H, W, h_offset);
    const uint32_t fq_cap = variant == RT_FRONTIER ? frontier_capacity(ctx, b) : 0u;
    Carve cv;
    ReconWs w;
    carve_recon(cv, b, w, false, fq_cap);
    rt_status st = ensure_ws(ctx, cv.off);
    if (st != RT_OK) return st;
    cv = Carve();
    cv.base = (char *)ctx->ws;
    carve_recon(cv, b, w, false, fq_cap);

    int32_t *err = dev_status ? dev_status : w.err;
    RT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    st = run_recon(ctx, b, w, conn, variant, 0, err, s, ctx_limits(ctx));
    if (st != RT_OK) return st;
    b.img[0].out = out;
    b.img[0].ld_out = ld_out;
    Phase ph(ctx, RT_PHASE_RECON_OUT, s);
    ctx->launches += 1;
    return cuda_status(launch_recon_out(b, 0, s));
}

rt_status rt_fill_holes(rt_ctx *ctx, const uint8_t *in, int64_t ld_in, uint8_t *out, int64_t ld_out, int H, int W,
                        int conn, int32_t *dev_status, void *stream)
{
    if (!ctx || !in || !out || bad_dims(H, W) || ld_in < W || ld_out < W) return RT_EINVAL;
    if (conn != 4 && conn != 8) return RT_EINVAL;
    if ((const void *)in != (const void *)out && overlaps(in, span(H, ld_in, 1, W), out, span(H, ld_out, 1, W)))
        return RT_EINVAL;
    if ((const void *)in == (const void *)out && ld_in != ld_out) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Carve cv;
    auto layout = [&](Carve &c, char *&fws, uint32_t *&flags, uint32_t *&pend, int32_t *&err) {
        fws = c.take<char>(fill_image_bytes(H, W));
        flags = c.take<uint32_t>((size_t)(ceil_div(H, kFillTH) * ceil_div(W, kFillTW)));
        pend = c.take<uint32_t>(1);
        err = c.take<int32_t>(1);
    };
    char *fws;
    uint32_t *flags, *pend;
    int32_t *err;
    layout(cv, fws, flags, pend, err);
    rt_status st = ensure_ws(ctx, cv.off);
    if (st != RT_OK) return st;
    cv = Carve();
    cv.base = (char *)ctx->ws;
    layout(cv, fws, flags, pend, err);
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    FillBatch fb;
    fb.n = 0;
    fill_add(fb, in, ld_in, out, ld_out, H, W, fws);
    fb.conn = conn;
    fb.flags = flags;
    fb.pending = pend;
    fb.err = dev_status ? dev_status : err;
    fb.timeout_ns = ctx_limits(ctx).timeout_ns;
    Phase ph(ctx, RT_PHASE_FILL, s);
    ctx->launches += 3;
    return cuda_status(launch_fill(fb, ctx->num_sms, s));
}

rt_status rt_label_area(rt_ctx *ctx, const uint8_t *bin, int64_t ld_bin, int32_t *labels, int64_t ld_lab, int H,
                        int W, int conn, int32_t min_area, int32_t max_area, int32_t *dev_n_kept,
                        int32_t *dev_status, void *stream)
{
    if (!ctx || !bin || !labels || bad_dims(H, W) || ld_bin < W || ld_lab < W) return RT_EINVAL;
    if (conn != 4 && conn != 8) return RT_EINVAL;
    if (overlaps(bin, span(H, ld_bin, 1, W), labels, span(H, ld_lab, 4, W))) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    rt_status st = ensure_ws(ctx, uf_workspace_bytes(H, W));
    if (st != RT_OK) return st;
    UfImage u;
    std::memset(&u, 0, sizeof(u));
    uf_carve(u, (char *)ctx->ws, H, W);
    u.in = bin;
    u.ld_in = ld_bin;
    u.labels = labels;
    u.ld_lab = ld_lab;
    u.n_kept = dev_n_kept;
    UfBatch b;
    b.n = 0;
    uf_add(b, u);
    b.amin = min_area;
    b.amax = max_area;
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    Phase ph(ctx, RT_PHASE_LABEL, s);
    ctx->launches += 4;
    return cuda_status(launch_label_batch(b, conn, s));
}

rt_status rt_edt(rt_ctx *ctx, const uint8_t *fg, int64_t ld_fg, int32_t *d2, int64_t ld_d2, int H, int W,
                 int32_t *dev_status, void *stream)
{
    if (!ctx || !fg || !d2 || bad_dims(H, W) || ld_fg < W || ld_d2 < W) return RT_EINVAL;
    if (overlaps(fg, span(H, ld_fg, 1, W), d2, span(H, ld_d2, 4, W))) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    Carve cv;
    cv.take<char>(edt_workspace_bytes(H, W));
    rt_status st = ensure_ws(ctx, cv.off + 1024);
    if (st != RT_OK) return st;
    cv = Carve();
    cv.base = (char *)ctx->ws;
    EdtArgs a;
    a.fg8 = fg;
    a.lab32 = nullptr;
    a.ld_in = ld_fg;
    a.H = H;
    a.W = W;
    a.d2 = d2;
    a.ld_d2 = ld_d2;
    a.g = cv.take<uint16_t>((size_t)H * W);
    a.seg = cv.take<int32_t>((size_t)2 * ceil_div(H, 32) * W);
    a.any_bg = cv.take<uint32_t>(1);
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    Phase ph(ctx, RT_PHASE_EDT, s);
    ctx->launches += 3;
    return cuda_status(launch_edt(a, s));
}

rt_status rt_watershed(rt_ctx *ctx, const int32_t *labels, int64_t ld_lab, const int32_t *d2, int64_t ld_d2, int H,
                       int W, int h, int32_t *basins, int64_t ld_b, int32_t *dev_n_basins, int32_t *dev_status,
                       void *stream)
{
    if (!ctx || !labels || !d2 || !basins || bad_dims(H, W) || ld_lab < W || ld_d2 < W || ld_b < W || h < 0)
        return RT_EINVAL;
    const size_t nb = span(H, ld_b, 4, W);
    if (overlaps(basins, nb, labels, span(H, ld_lab, 4, W)) || overlaps(basins, nb, d2, span(H, ld_d2, 4, W)))
        return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    rt_status st = ensure_ws(ctx, obj_workspace_bytes(H, W, false, true, 0));
    if (st != RT_OK) return st;
    ObjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.L = labels;
    a.ld_L = ld_lab;
    a.D = d2;
    a.ld_D = ld_d2;
    a.H = H;
    a.W = W;
    a.h = h;
    a.basins = basins;
    a.ld_B = ld_b;
    a.n_basins = dev_n_basins;
    obj_carve(a, (char *)ctx->ws, false, true);
    a.err = dev_status;
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    Phase ph(ctx, RT_PHASE_WATERSHED, s);
    int n = 0;
    const cudaError_t e = launch_watershed(a, ctx->num_sms, s, &n);
    ctx->launches += n;
    return cuda_status(e);
}

rt_status rt_object_features(rt_ctx *ctx, const int32_t *labels, int64_t ld_lab, const uint8_t *img, int64_t ld_img,
                             int H, int W, int32_t *obj_labels, double *feat, int cap, int32_t *dev_n_obj,
                             int32_t *dev_status, void *stream)
{
    if (!ctx || !labels || !img || bad_dims(H, W) || ld_lab < W || ld_img < W || cap < 0) return RT_EINVAL;
    if (cap > 0 && (!obj_labels || !feat)) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    rt_status st = ensure_ws(ctx, obj_workspace_bytes(H, W, true, false, cap));
    if (st != RT_OK) return st;
    ObjArgs a;
    std::memset(&a, 0, sizeof(a));
    a.L = labels;
    a.ld_L = ld_lab;
    a.I = img;
    a.ld_I = ld_img;
    a.H = H;
    a.W = W;
    a.cap = cap;
    a.out_labels = obj_labels;
    a.feat = feat;
    a.n_obj = dev_n_obj;
    obj_carve(a, (char *)ctx->ws, true, false);
    a.err = dev_status;
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    Phase ph(ctx, RT_PHASE_OBJECTS, s);
    int n = 0;
    const cudaError_t e = launch_object_features(a, ctx->num_sms, s, &n);
    ctx->launches += n;
    return cuda_status(e);
}

rt_status rt_synth_tile(rt_ctx *ctx, uint8_t *out, int64_t ld, int H, int W, uint64_t seed, int n_shapes, int kind,
                        int vlo, int vhi, int rmin, int rmax, int amin, int amax, int flat, int noise, void *stream)
{
    if (!ctx || !out || bad_dims(H, W) || ld < W || n_shapes < 0 || (kind != 0 && kind != 1)) return RT_EINVAL;
    if (vlo < 0 || vhi > 255 || vlo > vhi || rmin < 0 || rmax < rmin || amin < 0 || amax < amin) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    rt_status st = ensure_ws(ctx, synth_workspace_bytes(H, W));
    if (st != RT_OK) return st;
    SynthArgs a;
    a.H = H;
    a.W = W;
    a.k0 = (uint32_t)(seed & 0xffffffffu);
    a.k1 = (uint32_t)(seed >> 32);
    a.n_shapes = n_shapes;
    a.kind = kind;
    a.vlo = vlo;
    a.vhi = vhi;
    a.rmin = rmin;
    a.rmax = rmax;
    a.amin = amin;
    a.amax = amax;
    a.flat = flat != 0;
    a.noise = noise != 0;
    ctx->launches += 3;
    return cuda_status(launch_synth(a, ctx->ws, out, ld, s));
}

rt_status rt_tile_features(rt_ctx *ctx, const uint8_t *const *imgs, const int64_t *lds, const int *Hs, const int *Ws,
                           int n, float *out, void *stream)
{
    if (!ctx || !imgs || !lds || !Hs || !Ws || !out || n < 1 || n > kMaxFeatImgs) return RT_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!imgs[i] || bad_dims(Hs[i], Ws[i]) || lds[i] < Ws[i]) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    auto layout = [&](Carve &cv, FeatBatch &fb) {
        fb.n = n;
        for (int i = 0; i < n; ++i) {
            const size_t nb = (size_t)((Hs[i] + 7) / 8) * ((Ws[i] + 7) / 8);
            FeatImage &d = fb.img[i];
            d.img = imgs[i];
            d.ld = lds[i];
            d.H = Hs[i];
            d.W = Ws[i];
            d.hist = cv.take<uint32_t>(256);
            d.acc = cv.take<unsigned long long>(4);
            d.dark = cv.take<uint8_t>(nb);
            d.bmax = cv.take<uint8_t>(nb);
        }
    };
    FeatBatch fb;
    Carve cv;
    layout(cv, fb);
    rt_status st = ensure_ws(ctx, cv.off);
    if (st != RT_OK) return st;
    cv = Carve();
    cv.base = (char *)ctx->ws;
    layout(cv, fb);
    ctx->launches += 4;
    return cuda_status(launch_features(fb, out, s));
}

rt_status rt_mlp_forward(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x, int B, float *logits,
                         float *act, int32_t *pick, float min_prob, int fallback, void *stream)
{
    if (!ctx || !wb || !norm || !x || B < 1 || !(min_prob <= 1.0f) || fallback < 0) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_status(launch_mlp_forward(wb, norm, x, B, logits, act, pick, min_prob, fallback, (cudaStream_t)stream));
}

rt_status rt_mlp_forward_tc(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x, int B, float *logits,
                            float *act, int32_t *pick, float min_prob, int fallback, int32_t *dev_status, void *stream)
{
    if (!ctx || !wb || !norm || !x || B < 1 || !(min_prob <= 1.0f) || fallback < 0) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_status(
        launch_mlp_forward_tc(wb, norm, x, B, logits, act, pick, min_prob, fallback, dev_status, (cudaStream_t)stream));
}

rt_status rt_set_picker_classes(rt_ctx *ctx, const int *variants, const int *max_locals)
{
    if (!ctx || !variants || !max_locals) return RT_EINVAL;
    PickTable t = ctx->classes;
    for (int c = 0; c < kPickClasses; ++c) {
        const int v = variants[c] == RT_AUTO ? RT_RASTER : variants[c];
        if (v < RT_RASTER || v > RT_FRONTIER || max_locals[c] < 0) return RT_EINVAL;
        t.group[c] = v - RT_RASTER;
        t.max_local[c] = max_locals[c] > 0 ? max_locals[c] : default_max_local(v);
    }
    ctx->classes = t;
    return RT_OK;
}

rt_status rt_mlp_backward(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x, const float *act,
                          const float *logits, const int32_t *label, int B, float *grad, float *loss, void *stream)
{
    if (!ctx || !wb || !norm || !x || !act || !logits || !label || !grad || B < 1) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    rt_status st = ensure_ws(ctx, mlp_backward_workspace_bytes(B));
    if (st != RT_OK) return st;
    ctx->launches += 2;
    return cuda_status(launch_mlp_backward(wb, norm, x, act, logits, label, B, grad, loss, (float *)ctx->ws,
                                           (cudaStream_t)stream));
}

rt_status rt_mlp_backward_tc(rt_ctx *ctx, const uint16_t *wb, const float *norm, const float *x, const float *act,
                             const float *logits, const int32_t *label, int B, float *grad, float *loss,
                             int32_t *dev_status, void *stream)
{
    if (!ctx || !wb || !norm || !x || !act || !logits || !label || !grad || B < 1) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    rt_status st = ensure_ws(ctx, mlp_backward_tc_workspace_bytes(B));
    if (st != RT_OK) return st;
    ctx->launches += 2;
    return cuda_status(launch_mlp_backward_tc(wb, norm, x, act, logits, label, B, grad, loss, (float *)ctx->ws,
                                              dev_status, (cudaStream_t)stream));
}

rt_status rt_feature_norm(rt_ctx *ctx, const float *x, int B, float *norm, void *stream)
{
    if (!ctx || !x || !norm || B < 1) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_status(launch_feature_norm(x, B, norm, (cudaStream_t)stream));
}

rt_status rt_mlp_adamw(rt_ctx *ctx, float *master, uint16_t *wb, const float *grad, float *m, float *v, int step,
                       float lr, float beta1, float beta2, float eps, float weight_decay, void *stream)
{
    if (!ctx || !master || !wb || !grad || !m || !v || step < 1) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_status(
        launch_mlp_adamw(master, wb, grad, m, v, step, lr, beta1, beta2, eps, weight_decay, (cudaStream_t)stream));
}

int rt_last_picks(const rt_ctx *ctx, int *classes, int cap)
{
    if (!ctx) return 0;
    if (ctx->picks_ev_valid) {
        DeviceGuard g(ctx->device);
        if (cudaEventSynchronize(ctx->picks_ev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    }
    const int n = ctx->n_last_picks < cap ? ctx->n_last_picks : cap;
    for (int i = 0; classes && i < n; ++i) {
        const int c = ctx->picks_host[i];
        classes[i] = (c >= 0 && c < kPickClasses) ? c : kPickClasses;
    }
    return ctx->n_last_picks;
}

rt_status rt_set_picker(rt_ctx *ctx, const uint16_t *wb, const float *norm)
{
    if (!ctx || (!wb) != (!norm)) return RT_EINVAL;
    ctx->picker_wb = wb;
    ctx->picker_norm = norm;
    return RT_OK;
}

void rt_seg_params_default(rt_seg_params *p)
{
    if (!p) return;
    p->h_offset = 30;
    p->threshold = 80;
    p->min_area = 20;
    p->max_area = 1000;
    p->conn_recon = 8;
    p->conn_fill = 4;
    p->variant = RT_AUTO;
    p->max_local = 0;
    p->policy = RT_POLICY_PLAIN;
    p->max_iters = 0;
    p->timeout_ms = 0;
    p->pick_min_prob = 0;
    p->strip_tiles = 0;
}

rt_status rt_segment_batch(rt_ctx *ctx, const rt_tile *tiles, int n, const rt_seg_params *params, void *stream)
{
    if (!ctx || (!tiles && n > 0) || n < 0 || !params) return RT_EINVAL;
    const rt_seg_params &P = *params;
    if (bad_params(P)) return RT_EINVAL;
    for (int i = 0; i < n; ++i)
        if (bad_tile(tiles[i])) return RT_EINVAL;
    if (n == 0) return RT_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool learned = P.policy == RT_POLICY_LEARNED && ctx->picker_wb && ctx->picker_norm;
    Limits lim = ctx_limits(ctx);
    if (P.max_iters > 0) lim.max_iters = P.max_iters;
    if (P.timeout_ms > 0) lim.timeout_ns = (uint64_t)P.timeout_ms * 1000000ull;
    lim.strip = P.strip_tiles;
    // one allocation for the largest chunk, before anything is enqueued
    rt_status st = ensure_ws(ctx, segment_ws_bytes(tiles, n, P, learned, ctx));
    if (st != RT_OK) return st;

    for (int c0 = 0; c0 < n; c0 += kMaxImgs) {
        const int cn = n - c0 < kMaxImgs ? n - c0 : kMaxImgs;
        Chunk c;
        Carve cv;
        cv.base = (char *)ctx->ws;
        layout_chunk(cv, c, tiles, c0, cn, P, learned, ctx);
        RT_CUDA_TRY(zero_words(c.w.err, 1, s));
        ctx->launches += 1;
        if (!learned) {
            st = run_recon(ctx, c.b, c.w, P.conn_recon, P.variant, P.max_local, c.w.err, s, lim);
            if (st != RT_OK) return st;
        } else {
            // the picker chooses a variant per tile on the device; the
            // propagation reads its choices directly (no host round trip)
            const bool pick = picks_matter(ctx, P, cn);
            if (pick) {
                Phase ph(ctx, RT_PHASE_PICK, s);
                RT_CUDA_TRY(launch_features_pick(c.fb, c.feat, ctx->picker_wb, ctx->picker_norm, c.picks,
                                                 (float)P.pick_min_prob / 1000.0f, kPickClasses, s));
                ctx->launches += 4;
            }
            st = run_recon(ctx, c.b, c.w, P.conn_recon, P.variant, P.max_local, c.w.err, s, lim,
                           pick ? c.picks : nullptr);
            if (st != RT_OK) return st;
            // written by a kernel into the mapped pinned buffer: a copy-engine
            // transfer here would queue behind the caller's read-backs on the
            // same engine and hold up the rest of the chain
            copy_picks_kernel<<<1, 32, 0, s>>>(pick ? c.picks : nullptr, ctx->picks_mapped, cn);
            RT_CUDA_TRY(cudaGetLastError());
            ctx->launches += 1;
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusActive;
            if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cudaGetLastError();
            ctx->picks_ev_valid = cap == cudaStreamCaptureStatusNone;
            if (ctx->picks_ev_valid) RT_CUDA_TRY(cudaEventRecord(ctx->picks_ev, s));
            ctx->n_last_picks = cn;
        }
        {
            Phase ph(ctx, RT_PHASE_RECON_OUT, s);
            ctx->launches += 1;
            RT_CUDA_TRY(launch_recon_out(c.b, P.threshold, s));
        }
        {
            c.fill.conn = P.conn_fill;
            c.fill.flags = c.fill_flags;
            c.fill.pending = c.fill_pending;
            c.fill.err = c.w.err;
            c.fill.timeout_ns = lim.timeout_ns;
            Phase ph(ctx, RT_PHASE_FILL, s);
            ctx->launches += 3;
            RT_CUDA_TRY(launch_fill(c.fill, ctx->num_sms, s));
        }
        {
            Phase ph(ctx, RT_PHASE_LABEL, s);
            ctx->launches += 4;
            RT_CUDA_TRY(launch_label_batch(c.uf, 8, s));
        }
        {
            Phase ph(ctx, RT_PHASE_EDT, s);
            ctx->launches += 3;
            RT_CUDA_TRY(launch_edt_bits_batch(c.eb, s));
        }
        StatusOut so;
        bool any_status = false;
        for (int i = 0; i < cn; ++i) {
            so.dst[i] = tiles[c0 + i].status;
            any_status |= so.dst[i] != nullptr;
        }
        if (any_status) {
            copy_status_kernel<<<1, 32, 0, s>>>(c.w.err, so, cn);
            ctx->launches += 1;
            RT_CUDA_TRY(cudaGetLastError());
        }
    }
    return RT_OK;
}

}  // extern "C"
