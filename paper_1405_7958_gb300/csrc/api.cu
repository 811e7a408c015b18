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
    int32_t *picks_host = nullptr;         // pinned: picker classes of the last learned chunk
    cudaEvent_t picks_ev = nullptr;        // recorded after their copy (not under stream capture)
    bool picks_ev_valid = false;
    int n_last_picks = 0;
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

constexpr uint64_t kSweepTimeoutNs = 20000000000ull;   // 20 s bound on one propagation

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

// ---------------------------------------------------------------- recon
struct ReconWs {
    uint32_t *flags;   // per tile
    uint32_t *ctl;     // kCtlWords control words (recon.cuh)
    int32_t *err;
    int32_t *map;      // kGroups x ntiles tile lists when the variant is chosen per image
};

// Reserve the sweep control block and per-image padded buffers.
void carve_recon(Carve &cv, ReconBatch &b, ReconWs &w, bool grouped = false)
{
    w.flags = cv.take<uint32_t>((size_t)b.ntiles);
    w.ctl = cv.take<uint32_t>(kCtlWords);
    w.err = cv.take<int32_t>(1);
    w.map = grouped ? cv.take<int32_t>((size_t)kGroups * b.ntiles) : nullptr;
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
rt_status run_recon(rt_ctx *ctx, ReconBatch &b, ReconWs &w, int conn, int variant, int max_local, int32_t *err,
                    cudaStream_t s, const int32_t *pick = nullptr)
{
    if (variant == RT_AUTO) variant = RT_RASTER;
    // RT_RASTER / RT_QUEUE: every tile starts flagged for a dense visit (the
    // queue visit then seeds every pixel); RT_HYBRID: nothing flagged, the
    // dense pass over all tiles flags what remains.
    const uint32_t flag0 = variant == RT_HYBRID ? 0u : 2u;
    RT_CUDA_TRY(cudaMemsetAsync(w.ctl, 0, kCtlWords * sizeof(uint32_t), s));
    {
        Phase ph(ctx, RT_PHASE_RECON_INIT, s);
        RT_CUDA_TRY(launch_recon_init(b, w.flags, w.ctl, flag0, pick, w.map, err, s));
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
    p.timeout_ns = kSweepTimeoutNs;
    p.map = nullptr;
    p.nvirt = nullptr;
    int grid = 0;
    Phase ph(ctx, RT_PHASE_RECON_SWEEP, s);
    for (int g = 0; g < (pick ? kGroups : 1); ++g) {
        const int v = pick ? RT_RASTER + g : variant;
        if (pick) {
            p.map = w.map + (size_t)g * b.ntiles;
            p.nvirt = w.ctl + kCtlGroupCount + g;
            p.pending = w.ctl + kCtlGroupPending + g;
        }
        p.max_local = max_local > 0 ? max_local : (v == RT_HYBRID ? 64 : 12);
        if (v == RT_HYBRID) {
            RT_CUDA_TRY(launch_recon_dense(p, conn, s));
            ctx->launches += 1;
        }
        ctx->launches += 1;
        RT_CUDA_TRY(launch_recon_persistent(p, conn, v == RT_RASTER ? 0 : 1, ctx->num_sms, s, &grid));
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

// Union-find workspace for an H x W image.
void carve_uf(Carve &cv, UfArgs &a, int H, int W)
{
    const size_t N = (size_t)H * W;
    const size_t nblk = (size_t)ceil_div(W, kUfBlock) * ceil_div(H, kUfBlock);
    a.U = cv.take<int32_t>(N);
    a.A = cv.take<int32_t>(N);
    a.edge = cv.take<int32_t>(nblk * kUfEdge);
    a.list = cv.take<int32_t>(N / 2 + 2);
    a.nlist = cv.take<uint32_t>(1);
    a.lroot = cv.take<uint16_t>(N);
    a.bempty = cv.take<uint8_t>(nblk);
}

// a tile's status word: the device status of the chunk that carried it
__global__ void copy_status_kernel(const int32_t *src, int32_t *dst)
{
    if (threadIdx.x == 0) *dst = *src;
}

}  // namespace

// ================================================================= C ABI
extern "C" {

int rt_version(void) { return 100; }

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

rt_status rt_create(rt_ctx **ctx, int device)
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
        cudaHostAlloc((void **)&c->picks_host, kMaxImgs * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->picks_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->picks_host) cudaFreeHost(c->picks_host);
        delete c;
        return RT_ECUDA;
    }
    *ctx = c;
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
    if (variant < RT_AUTO || variant > RT_HYBRID) return RT_EINVAL;
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
    Carve cv;
    ReconWs w;
    carve_recon(cv, b, w);
    rt_status st = ensure_ws(ctx, cv.off);
    if (st != RT_OK) return st;
    cv = Carve();
    cv.base = (char *)ctx->ws;
    carve_recon(cv, b, w);

    int32_t *err = dev_status ? dev_status : w.err;
    RT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    st = run_recon(ctx, b, w, conn, variant, 0, err, s);
    if (st != RT_OK) return st;
    Phase ph(ctx, RT_PHASE_RECON_OUT, s);
    ctx->launches += 1;
    return cuda_status(launch_recon_out(b.img[0].Rw, b.img[0].Wp, out, ld_out, H, W, nullptr, 0, 0, s));
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
    fb.timeout_ns = kSweepTimeoutNs;
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
    UfArgs a;
    Carve cv;
    carve_uf(cv, a, H, W);
    rt_status st = ensure_ws(ctx, cv.off);
    if (st != RT_OK) return st;
    cv = Carve();
    cv.base = (char *)ctx->ws;
    carve_uf(cv, a, H, W);
    a.in = bin;
    a.ld_in = ld_bin;
    a.H = H;
    a.W = W;
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    if (dev_n_kept) RT_CUDA_TRY(cudaMemsetAsync(dev_n_kept, 0, sizeof(int32_t), s));
    Phase ph(ctx, RT_PHASE_LABEL, s);
    ctx->launches += 4;
    RT_CUDA_TRY(uf_build(a, conn, kFgNonzero, true, false, s));
    return cuda_status(uf_labels_out(a, conn, labels, ld_lab, min_area, max_area, dev_n_kept, nullptr, s));
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
    a.bits = nullptr;
    a.ld_in = ld_fg;
    a.H = H;
    a.W = W;
    a.d2 = d2;
    a.ld_d2 = ld_d2;
    a.g = cv.take<uint16_t>((size_t)H * W);
    a.cmask = nullptr;
    a.seg = cv.take<int32_t>((size_t)2 * ceil_div(H, 32) * W);
    a.any_bg = cv.take<uint32_t>(1);
    if (dev_status) RT_CUDA_TRY(cudaMemsetAsync(dev_status, 0, sizeof(int32_t), s));
    Phase ph(ctx, RT_PHASE_EDT, s);
    ctx->launches += 3;
    return cuda_status(launch_edt(a, s));
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
                         float *act, int32_t *pick, void *stream)
{
    if (!ctx || !wb || !norm || !x || B < 1) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_status(launch_mlp_forward(wb, norm, x, B, logits, act, pick, (cudaStream_t)stream));
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

rt_status rt_mlp_adamw(rt_ctx *ctx, float *master, uint16_t *wb, const float *grad, float *m, float *v, int step,
                       float lr, float beta1, float beta2, float eps, float weight_decay, void *stream)
{
    if (!ctx || !master || !wb || !grad || !m || !v || step < 1) return RT_EINVAL;
    DeviceGuard g(ctx->device);
    ctx->launches += 1;
    return cuda_status(
        launch_mlp_adamw(master, wb, grad, m, v, step, lr, beta1, beta2, eps, weight_decay, (cudaStream_t)stream));
}

int rt_last_picks(const rt_ctx *ctx, int *variants, int cap)
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
    for (int i = 0; variants && i < n; ++i) {
        const int g = ctx->picks_host[i];
        variants[i] = (g >= 0 && g < kGroups) ? RT_RASTER + g : RT_RASTER;
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
}

rt_status rt_segment_batch(rt_ctx *ctx, const rt_tile *tiles, int n, const rt_seg_params *params, void *stream)
{
    if (!ctx || (!tiles && n > 0) || n < 0 || !params) return RT_EINVAL;
    const rt_seg_params &P = *params;
    if (P.conn_recon != 4 && P.conn_recon != 8) return RT_EINVAL;
    if (P.conn_fill != 4 && P.conn_fill != 8) return RT_EINVAL;
    if (P.h_offset < 0 || P.h_offset > 255 || P.threshold < 0 || P.threshold > 256) return RT_EINVAL;
    if (P.variant < RT_AUTO || P.variant > RT_HYBRID) return RT_EINVAL;
    if (P.policy != RT_POLICY_PLAIN && P.policy != RT_POLICY_LEARNED) return RT_EINVAL;
    int64_t maxN = 0;
    for (int i = 0; i < n; ++i) {
        const rt_tile &t = tiles[i];
        if (!t.img || !t.labels || !t.d2 || bad_dims(t.H, t.W)) return RT_EINVAL;
        if (t.ld_img < t.W || t.ld_labels < t.W || t.ld_d2 < t.W) return RT_EINVAL;
        if (t.recon && t.ld_recon < t.W) return RT_EINVAL;
        if (t.filled && t.ld_filled < t.W) return RT_EINVAL;
        if ((int64_t)t.H * t.W > maxN) maxN = (int64_t)t.H * t.W;
    }
    if (n == 0) return RT_OK;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;

    for (int c0 = 0; c0 < n; c0 += kMaxImgs) {
        const int cn = n - c0 < kMaxImgs ? n - c0 : kMaxImgs;
        ReconBatch b;
        std::memset(&b, 0, sizeof(b));
        for (int i = 0; i < cn; ++i) {
            const rt_tile &t = tiles[c0 + i];
            add_image(b, nullptr, 0, t.img, t.ld_img, t.H, t.W, P.h_offset);
        }
        // workspace: recon buffers for the chunk, binary B per tile, then one
        // shared set of union-find / EDT buffers (tiles run one after another)
        int maxH = 0, maxW = 0;
        for (int i = 0; i < cn; ++i) {
            maxH = b.img[i].H > maxH ? b.img[i].H : maxH;
            maxW = b.img[i].W > maxW ? b.img[i].W : maxW;
        }
        const bool learned = P.policy == RT_POLICY_LEARNED && ctx->picker_wb && ctx->picker_norm;
        FeatBatch fb;
        float *feat = nullptr;
        int32_t *picks_dev = nullptr;
        std::vector<char *> fill_ws;
        uint32_t *fill_flags = nullptr, *fill_pending = nullptr;
        uint32_t *kept_bits = nullptr;   // kept pixels of the tile being labeled, for its distance transform
        auto layout = [&](Carve &cv, ReconWs &w, std::vector<uint8_t *> &Bs, char *&uf_ws,
                          char *&edt_ws) {
            carve_recon(cv, b, w, learned);
            if (learned) {
                fb.n = cn;
                for (int i = 0; i < cn; ++i) {
                    const rt_tile &t = tiles[c0 + i];
                    const size_t nb = (size_t)((t.H + 7) / 8) * ((t.W + 7) / 8);
                    FeatImage &d = fb.img[i];
                    d.img = t.img;
                    d.ld = t.ld_img;
                    d.H = t.H;
                    d.W = t.W;
                    d.hist = cv.take<uint32_t>(256);
                    d.acc = cv.take<unsigned long long>(4);
                    d.dark = cv.take<uint8_t>(nb);
                    d.bmax = cv.take<uint8_t>(nb);
                }
                feat = cv.take<float>((size_t)cn * kNumFeatures);
                picks_dev = cv.take<int32_t>((size_t)cn);
            }
            Bs.resize(cn);
            for (int i = 0; i < cn; ++i) Bs[i] = cv.take<uint8_t>((size_t)b.img[i].H * b.img[i].W);
            // union-find pieces sized for (maxH, maxW), enough for every tile of the chunk
            uf_ws = cv.take<char>(uf_workspace_bytes(maxH, maxW));
            edt_ws = cv.take<char>(edt_workspace_bytes(maxH, maxW) + (size_t)maxN * 2);
            fill_ws.resize(cn);
            int fill_tiles = 0;
            for (int i = 0; i < cn; ++i) {
                fill_ws[i] = cv.take<char>(fill_image_bytes(b.img[i].H, b.img[i].W));
                fill_tiles += (int)(ceil_div(b.img[i].H, kFillTH) * ceil_div(b.img[i].W, kFillTW));
            }
            fill_flags = cv.take<uint32_t>((size_t)fill_tiles);
            kept_bits = cv.take<uint32_t>((size_t)maxH * ceil_div(maxW, 32));
            fill_pending = cv.take<uint32_t>(1);
        };
        Carve cv;
        ReconWs w;
        std::vector<uint8_t *> Bs;
        char *uf_ws, *edt_ws;
        layout(cv, w, Bs, uf_ws, edt_ws);
        rt_status st = ensure_ws(ctx, cv.off);
        if (st != RT_OK) return st;
        cv = Carve();
        cv.base = (char *)ctx->ws;
        layout(cv, w, Bs, uf_ws, edt_ws);

        RT_CUDA_TRY(cudaMemsetAsync(w.err, 0, sizeof(int32_t), s));
        if (!learned) {
            st = run_recon(ctx, b, w, P.conn_recon, P.variant, P.max_local, w.err, s);
            if (st != RT_OK) return st;
        } else {
            // the picker chooses a variant per tile on the device; the
            // propagation reads its choices directly (no host round trip)
            {
                Phase ph(ctx, RT_PHASE_PICK, s);
                RT_CUDA_TRY(launch_features(fb, feat, s));
                RT_CUDA_TRY(launch_mlp_forward(ctx->picker_wb, ctx->picker_norm, feat, cn, nullptr, nullptr,
                                               picks_dev, s));
                ctx->launches += 5;
            }
            st = run_recon(ctx, b, w, P.conn_recon, P.variant, P.max_local, w.err, s, picks_dev);
            if (st != RT_OK) return st;
            RT_CUDA_TRY(cudaMemcpyAsync(ctx->picks_host, picks_dev, sizeof(int32_t) * cn, cudaMemcpyDeviceToHost, s));
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusActive;
            if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cudaGetLastError();
            ctx->picks_ev_valid = cap == cudaStreamCaptureStatusNone;
            if (ctx->picks_ev_valid) RT_CUDA_TRY(cudaEventRecord(ctx->picks_ev, s));
            ctx->n_last_picks = cn;
        }
        for (int i = 0; i < cn; ++i) {
            const rt_tile &t = tiles[c0 + i];
            const ReconImage &d = b.img[i];
            Phase ph(ctx, RT_PHASE_RECON_OUT, s);
            ctx->launches += 1;
            RT_CUDA_TRY(launch_recon_out(d.Rw, d.Wp, t.recon, t.ld_recon, t.H, t.W, Bs[i], t.W, P.threshold, s));
        }
        // hole filling for the whole chunk at once; F replaces the binary
        // image unless the caller wants F in its own buffer
        {
            FillBatch fb_;
            fb_.n = 0;
            for (int i = 0; i < cn; ++i) {
                const rt_tile &t = tiles[c0 + i];
                uint8_t *F = t.filled ? t.filled : Bs[i];
                fill_add(fb_, Bs[i], t.W, F, t.filled ? t.ld_filled : t.W, t.H, t.W, fill_ws[i]);
            }
            fb_.conn = P.conn_fill;
            fb_.flags = fill_flags;
            fb_.pending = fill_pending;
            fb_.err = w.err;
            fb_.timeout_ns = kSweepTimeoutNs;
            Phase ph(ctx, RT_PHASE_FILL, s);
            ctx->launches += 3;
            RT_CUDA_TRY(launch_fill(fb_, ctx->num_sms, s));
        }
        for (int i = 0; i < cn; ++i) {
            const rt_tile &t = tiles[c0 + i];
            const int H = t.H, W = t.W;
            const uint8_t *F = t.filled ? t.filled : Bs[i];
            const int64_t ldF = t.filled ? t.ld_filled : W;
            UfArgs la;
            Carve uc;
            uc.base = uf_ws;
            carve_uf(uc, la, H, W);
            la.H = H;
            la.W = W;
            la.in = F;
            la.ld_in = ldF;
            if (t.n_kept) RT_CUDA_TRY(cudaMemsetAsync(t.n_kept, 0, sizeof(int32_t), s));
            {
                Phase ph(ctx, RT_PHASE_LABEL, s);
                ctx->launches += 4;
                RT_CUDA_TRY(uf_build(la, 8, kFgNonzero, true, false, s));
                RT_CUDA_TRY(uf_labels_out(la, 8, t.labels, t.ld_labels, P.min_area, P.max_area, t.n_kept, kept_bits, s));
            }
            EdtArgs ea;
            ea.fg8 = nullptr;
            ea.lab32 = nullptr;
            ea.bits = kept_bits;
            ea.ld_in = t.ld_labels;
            ea.H = H;
            ea.W = W;
            ea.d2 = t.d2;
            ea.ld_d2 = t.ld_d2;
            Carve ec;
            ec.base = edt_ws;
            ea.g = nullptr;   // the bit-plane path computes g while staging each row
            ea.cmask = ec.take<uint32_t>((size_t)ceil_div(H, 32) * W);
            ea.seg = ec.take<int32_t>((size_t)2 * ceil_div(H, 32) * W);
            ea.any_bg = ec.take<uint32_t>(1);
            {
                Phase ph(ctx, RT_PHASE_EDT, s);
                ctx->launches += 3;
                RT_CUDA_TRY(launch_edt(ea, s));
            }
            if (t.status) {
                copy_status_kernel<<<1, 32, 0, s>>>(w.err, t.status);
                ctx->launches += 1;
                RT_CUDA_TRY(cudaGetLastError());
            }
        }
    }
    return RT_OK;
}

}  // extern "C"
