"""GB300 (sm_103a) segmentation hot path of the Region Templates microscopy
pipeline: reconstruction by dilation (ReconToNuclei), hole filling
(FillHoles), connected-component labeling with an area filter (BWLabel +
AreaThreshold) and the exact squared Euclidean distance transform (the
Pre-Watershed input), behind the C ABI of include/rt.h.

This module marshals torch CUDA tensors into the C ABI; torch provides device
memory and streams only. All operations run in the library's own CUDA
kernels. There is no CPU fallback: without the built library or a GPU every
call raises.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import torch

from . import _native
from ._native import (RT_AUTO, RT_EINVAL, RT_EMARKER, RT_ETIMEOUT, RT_EUNAVAIL, RT_FRONTIER, RT_HYBRID,  # noqa: F401
                      RT_OK, RT_QUEUE, RT_RASTER)

__all__ = [
    "Context", "SegParams", "marker", "reconstruct", "fill_holes", "label_area", "edt",
    "segment_batch", "RT_AUTO", "RT_RASTER", "RT_QUEUE", "RT_HYBRID", "RT_FRONTIER",
]

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _native.load()
    return _lib


class RtError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {lib().rt_status_str(code).decode()} (code {code})")
        self.code = code


def _check(code: int, where: str):
    if code != RT_OK:
        raise RtError(code, where)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev_ptr(t: torch.Tensor, dtype: torch.dtype, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D {dtype} tensor")
    if t.stride(1) != 1:
        raise ValueError(f"{name} must have unit column stride")
    return t.data_ptr(), t.stride(0)


class Context:
    """Owns a library context (device workspace) on one CUDA device."""

    def __init__(self, device: int | None = None, workspace_bytes: int = 0):
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().rt_create(ctypes.byref(h), device, int(workspace_bytes)), "rt_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        return lib().rt_workspace_bytes(self._h)

    def set_limits(self, max_iters: int = 0, timeout_ms: int = 0):
        """Bounds of the propagations of the single-operation calls (and the
        defaults of segment_batch): tile visits per tile, device time."""
        _check(lib().rt_set_limits(self._h, int(max_iters), int(timeout_ms)), "rt_set_limits")

    def set_queue_capacity(self, entries: int = 0):
        """Entries of each global frontier queue of RT_FRONTIER (0: one per
        padded pixel of the call's images). A full queue hands over to the
        directional sweeps, with the same output."""
        _check(lib().rt_set_queue_capacity(self._h, int(entries)), "rt_set_queue_capacity")

    def timing(self, enable: bool = True):
        _check(lib().rt_timing_enable(self._h, int(enable)), "rt_timing_enable")

    def read_timing(self, reset: bool = True) -> dict:
        """Per-phase {name: (milliseconds, intervals)} since the last reset."""
        ms = (ctypes.c_double * _native.RT_NPHASES)()
        cnt = (ctypes.c_int64 * _native.RT_NPHASES)()
        _check(lib().rt_timing_read(self._h, ms, cnt, int(reset)), "rt_timing_read")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(_native.PHASES)}

    def kernel_launches(self) -> int:
        return lib().rt_kernel_launches(self._h)

    def recon_stats(self) -> tuple:
        """(tile visits, dense sweep iterations, queue pops) of the last reconstruction."""
        v, it, pops = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().rt_recon_stats(self._h, ctypes.byref(v), ctypes.byref(it), ctypes.byref(pops)),
               "rt_recon_stats")
        return v.value, it.value, pops.value

    def close(self):
        if self._h:
            lib().rt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default = {}


def default_context(device: int | None = None) -> Context:
    if device is None:
        device = torch.cuda.current_device()
    if device not in _default:
        _default[device] = Context(device)
    return _default[device]


def marker(mask: torch.Tensor, h_offset: int = 30, out=None, ctx=None, stream=None) -> torch.Tensor:
    ctx = ctx or default_context(mask.device.index)
    mp, mld = _dev_ptr(mask, torch.uint8, "mask")
    H, W = mask.shape
    out = torch.empty_like(mask, memory_format=torch.contiguous_format) if out is None else out
    op, old = _dev_ptr(out, torch.uint8, "out")
    _check(lib().rt_marker(ctx.handle, mp, mld, op, old, H, W, h_offset, _stream(stream)), "rt_marker")
    return out


def reconstruct(mask: torch.Tensor, marker: torch.Tensor | None = None, *, h_offset: int = 30, conn: int = 8,
                variant: int = RT_AUTO, out=None, status=None, ctx=None, stream=None) -> torch.Tensor:
    """Reconstruction by dilation of `marker` under `mask` (uint8 CUDA
    tensors). marker=None derives it from the mask with h_offset."""
    ctx = ctx or default_context(mask.device.index)
    ip, ild = _dev_ptr(mask, torch.uint8, "mask")
    H, W = mask.shape
    jp, jld = (None, 0) if marker is None else _dev_ptr(marker, torch.uint8, "marker")
    out = torch.empty((H, W), dtype=torch.uint8, device=mask.device) if out is None else out
    op, old = _dev_ptr(out, torch.uint8, "out")
    sp = None if status is None else status.data_ptr()
    _check(lib().rt_reconstruct(ctx.handle, jp, jld, ip, ild, op, old, H, W, conn, variant, h_offset, sp,
                                _stream(stream)), "rt_reconstruct")
    return out


def fill_holes(binary: torch.Tensor, *, conn: int = 4, out=None, status=None, ctx=None, stream=None):
    ctx = ctx or default_context(binary.device.index)
    bp, bld = _dev_ptr(binary, torch.uint8, "binary")
    H, W = binary.shape
    out = torch.empty((H, W), dtype=torch.uint8, device=binary.device) if out is None else out
    op, old = _dev_ptr(out, torch.uint8, "out")
    sp = None if status is None else status.data_ptr()
    _check(lib().rt_fill_holes(ctx.handle, bp, bld, op, old, H, W, conn, sp, _stream(stream)), "rt_fill_holes")
    return out


def label_area(binary: torch.Tensor, min_area: int = 20, max_area: int = 1000, *, conn: int = 8, out=None,
               n_kept=None, status=None, ctx=None, stream=None):
    ctx = ctx or default_context(binary.device.index)
    bp, bld = _dev_ptr(binary, torch.uint8, "binary")
    H, W = binary.shape
    out = torch.empty((H, W), dtype=torch.int32, device=binary.device) if out is None else out
    op, old = _dev_ptr(out, torch.int32, "out")
    kp = None if n_kept is None else n_kept.data_ptr()
    sp = None if status is None else status.data_ptr()
    _check(lib().rt_label_area(ctx.handle, bp, bld, op, old, H, W, conn, min_area, max_area, kp, sp,
                               _stream(stream)), "rt_label_area")
    return out


def edt(fg: torch.Tensor, *, out=None, status=None, ctx=None, stream=None):
    ctx = ctx or default_context(fg.device.index)
    fp, fld = _dev_ptr(fg, torch.uint8, "fg")
    H, W = fg.shape
    out = torch.empty((H, W), dtype=torch.int32, device=fg.device) if out is None else out
    op, old = _dev_ptr(out, torch.int32, "out")
    sp = None if status is None else status.data_ptr()
    _check(lib().rt_edt(ctx.handle, fp, fld, op, old, H, W, sp, _stream(stream)), "rt_edt")
    return out


def watershed(labels: torch.Tensor, d2: torch.Tensor, h: int = 2, *, out=None, n_basins=None, status=None, ctx=None,
              stream=None) -> torch.Tensor:
    """Marker-controlled watershed of the squared distance map inside every
    labelled object (int32 CUDA tensors); basin label per object pixel, -1
    elsewhere."""
    ctx = ctx or default_context(labels.device.index)
    lp, lld = _dev_ptr(labels, torch.int32, "labels")
    dp, dld = _dev_ptr(d2, torch.int32, "d2")
    H, W = labels.shape
    out = torch.empty((H, W), dtype=torch.int32, device=labels.device) if out is None else out
    op, old = _dev_ptr(out, torch.int32, "out")
    np_ = None if n_basins is None else n_basins.data_ptr()
    sp = None if status is None else status.data_ptr()
    _check(lib().rt_watershed(ctx.handle, lp, lld, dp, dld, H, W, int(h), op, old, np_, sp, _stream(stream)),
           "rt_watershed")
    return out


def object_features(labels: torch.Tensor, image: torch.Tensor, cap: int, *, n_obj=None, status=None, ctx=None,
                    stream=None):
    """Per-object features of the labelled objects over the uint8 image:
    (labels int32[cap], features float64[cap, 20]) for the first min(cap, n)
    objects in label order; n_obj (device int32[1]) receives n."""
    ctx = ctx or default_context(labels.device.index)
    lp, lld = _dev_ptr(labels, torch.int32, "labels")
    ip, ild = _dev_ptr(image, torch.uint8, "image")
    H, W = labels.shape
    dev = labels.device
    olab = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    feat = torch.empty((max(cap, 1), _native.RT_NOBJFEAT), dtype=torch.float64, device=dev)
    np_ = None if n_obj is None else n_obj.data_ptr()
    sp = None if status is None else status.data_ptr()
    _check(lib().rt_object_features(ctx.handle, lp, lld, ip, ild, H, W, olab.data_ptr(), feat.data_ptr(), int(cap),
                                    np_, sp, _stream(stream)), "rt_object_features")
    return olab[:cap], feat[:cap]


def synth_tile(H: int, W: int, seed: int, n_shapes: int, *, kind: str = "ellipse", vlo: int = 30, vhi: int = 100,
               rmin: int = 4, rmax: int = 12, amin: int = 4, amax: int = 14, background: str = "perlin",
               noise: bool = True, out=None, device=None, ctx=None, stream=None) -> torch.Tensor:
    """Seeded nuclei tile drawn on the GPU; same bytes as synth.tile() with
    the same arguments."""
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    ctx = ctx or default_context(torch.device(device).index)
    out = torch.empty((H, W), dtype=torch.uint8, device=device) if out is None else out
    op, old = _dev_ptr(out, torch.uint8, "out")
    _check(lib().rt_synth_tile(ctx.handle, op, old, H, W, int(seed), int(n_shapes), 1 if kind == "disk" else 0,
                               vlo, vhi, rmin, rmax, amin, amax, 1 if background == "flat" else 0, int(bool(noise)),
                               _stream(stream)), "rt_synth_tile")
    return out


def config2_tile(seed: int = 2000, H: int = 4096, W: int = 4096, n_shapes: int | None = None, **kw):
    """GPU twin of synth.config2_tile."""
    if n_shapes is None:
        n_shapes = int(round(3000 * H * W / (4096 * 4096)))
    return synth_tile(H, W, seed, n_shapes, kind="ellipse", vlo=30, vhi=100, **kw)


def tile_features(images, *, out=None, ctx=None, stream=None) -> torch.Tensor:
    """The picker's 24 features of each uint8 CUDA tile (n <= 32 per call
    chunk; longer lists are processed in chunks). Returns float32 n x 24."""
    if not images:
        return torch.empty((0, _native.RT_NFEATURES), dtype=torch.float32)
    ctx = ctx or default_context(images[0].device.index)
    n = len(images)
    out = torch.empty((n, _native.RT_NFEATURES), dtype=torch.float32, device=images[0].device) if out is None else out
    for c0 in range(0, n, 32):
        chunk = images[c0:c0 + 32]
        m = len(chunk)
        ptrs = (ctypes.c_void_p * m)()
        lds = (ctypes.c_int64 * m)()
        hs = (ctypes.c_int * m)()
        ws = (ctypes.c_int * m)()
        for i, img in enumerate(chunk):
            ptrs[i], lds[i] = _dev_ptr(img, torch.uint8, "image")
            hs[i], ws[i] = img.shape
        _check(lib().rt_tile_features(ctx.handle, ptrs, lds, hs, ws, m, out[c0:].data_ptr(), _stream(stream)),
               "rt_tile_features")
    return out


class Picker:
    """The learned variant picker: parameters on the GPU (bf16 working copy,
    fp32 master, AdamW moments) and the normalisation of the features. Every
    computation runs in the library's kernels."""

    NPARAM = _native.RT_MLP_NPARAM

    def __init__(self, device=None, seed: int = 0, norm=None, ctx=None):
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        self.ctx = ctx or default_context(self.device.index)
        g = torch.Generator().manual_seed(seed)
        # He-style initial weights (drawn on the host once), zero biases
        p = torch.zeros(self.NPARAM, dtype=torch.float32)
        p[0:1536] = torch.randn(1536, generator=g) * (2.0 / 24) ** 0.5
        p[1600:5696] = torch.randn(4096, generator=g) * (2.0 / 64) ** 0.5
        p[5760:5952] = torch.randn(192, generator=g) * (1.0 / 64) ** 0.5
        self.master = p.to(self.device)
        self.wb = self.master.to(torch.bfloat16).view(torch.int16).contiguous()
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.grad = torch.zeros_like(self.master)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.norm = torch.cat([torch.zeros(24), torch.ones(24)]).to(self.device) if norm is None else norm
        self.step_count = 0

    def set_norm(self, feats: torch.Tensor, stream=None):
        """Input normalisation from a training set (B x 24 float32 on the
        device), computed by the library (rt_feature_norm)."""
        x = feats.to(device=self.device, dtype=torch.float32).contiguous()
        norm = torch.empty(48, dtype=torch.float32, device=self.device)
        _check(lib().rt_feature_norm(self.ctx.handle, x.data_ptr(), x.shape[0], norm.data_ptr(), _stream(stream)),
               "rt_feature_norm")
        self.norm = norm

    def forward(self, x: torch.Tensor, with_act: bool = False, min_prob: float = 0.0, fallback: int = 3,
                stream=None, tensor_cores: bool = False, status=None):
        """Logits, saved activations (with_act) and picks; a pick whose
        softmax probability is below min_prob becomes `fallback`.
        tensor_cores: the tensor-core forward (bf16 operands, for training
        batches); status: its device status word (int32, nullable)."""
        B = x.shape[0]
        logits = torch.empty((B, 3), dtype=torch.float32, device=self.device)
        act = torch.empty((B, 128), dtype=torch.float32, device=self.device) if with_act else None
        pick = torch.empty(B, dtype=torch.int32, device=self.device)
        args = (self.ctx.handle, self.wb.data_ptr(), self.norm.data_ptr(), x.contiguous().data_ptr(), B,
                logits.data_ptr(), None if act is None else act.data_ptr(), pick.data_ptr(), float(min_prob),
                int(fallback))
        if tensor_cores:
            _check(lib().rt_mlp_forward_tc(*args, None if status is None else status.data_ptr(), _stream(stream)),
                   "rt_mlp_forward_tc")
        else:
            _check(lib().rt_mlp_forward(*args, _stream(stream)), "rt_mlp_forward")
        return logits, act, pick

    def backward(self, x, act, logits, label, stream=None, tensor_cores: bool = False, status=None):
        """Gradient (into self.grad) and loss of the batch; tensor_cores: the
        tensor-core backward (bf16 operands), from a tensor-core forward's
        act and logits."""
        args = (self.ctx.handle, self.wb.data_ptr(), self.norm.data_ptr(), x.contiguous().data_ptr(), act.data_ptr(),
                logits.data_ptr(), label.to(torch.int32).contiguous().data_ptr(), x.shape[0], self.grad.data_ptr(),
                self.loss.data_ptr())
        if tensor_cores:
            _check(lib().rt_mlp_backward_tc(*args, None if status is None else status.data_ptr(), _stream(stream)),
                   "rt_mlp_backward_tc")
        else:
            _check(lib().rt_mlp_backward(*args, _stream(stream)), "rt_mlp_backward")
        return self.grad, self.loss

    def step(self, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4, stream=None):
        self.step_count += 1
        _check(lib().rt_mlp_adamw(self.ctx.handle, self.master.data_ptr(), self.wb.data_ptr(), self.grad.data_ptr(),
                                  self.m.data_ptr(), self.v.data_ptr(), self.step_count, lr, beta1, beta2, eps,
                                  weight_decay, _stream(stream)), "rt_mlp_adamw")

    def attach(self, ctx=None):
        """Use this picker in rt_segment_batch(policy=learned) on ctx."""
        ctx = ctx or self.ctx
        _check(lib().rt_set_picker(ctx.handle, self.wb.data_ptr(), self.norm.data_ptr()), "rt_set_picker")

    def state_dict(self) -> dict:
        return {k: getattr(self, k).detach().cpu() for k in ("master", "wb", "m", "v", "norm")} | {
            "step_count": self.step_count}

    def load_state_dict(self, sd: dict):
        for k in ("master", "wb", "m", "v", "norm"):
            setattr(self, k, sd[k].to(self.device).contiguous())
        self.step_count = int(sd["step_count"])


PICKER_CLASSES = ((RT_RASTER, 4), (RT_RASTER, 12), (RT_RASTER, 24))   # the library's default table


def set_picker_classes(classes, ctx=None):
    """The picker's three schedules on ctx: ((variant, max_local), ...)."""
    ctx = ctx or default_context()
    v = (ctypes.c_int * 3)(*[int(c[0]) for c in classes])
    m = (ctypes.c_int * 3)(*[int(c[1]) for c in classes])
    _check(lib().rt_set_picker_classes(ctx.handle, v, m), "rt_set_picker_classes")


def last_picks(ctx=None) -> list:
    """Classes (0..2, or 3 = fell back to the plain schedule) the picker
    chose for the tiles of the last learned chunk."""
    ctx = ctx or default_context()
    buf = (ctypes.c_int * 32)()
    n = lib().rt_last_picks(ctx.handle, buf, 32)
    return [buf[i] for i in range(min(n, 32))]


@dataclass
class SegParams:
    h_offset: int = 30
    threshold: int = 80
    min_area: int = 20
    max_area: int = 1000
    conn_recon: int = 8
    conn_fill: int = 4
    variant: int = RT_AUTO
    max_local: int = 0
    policy: int = 0          # 0 plain (fixed variant), 1 learned (attached picker)
    max_iters: int = 0       # tile visits per tile allowed to the propagation (0: the context's bound)
    timeout_ms: int = 0      # device-time bound of each propagation (0: the context's)
    pick_min_prob: int = 0   # learned: a pick stands only at softmax probability >= this / 1000
    strip_tiles: int = 0     # tiles per warp strip of the raster propagation (0: the library's choice)

    def to_c(self) -> _native.RtSegParams:
        p = _native.RtSegParams()
        for k in self.__dataclass_fields__:
            setattr(p, k, int(getattr(self, k)))
        return p


def segment_workspace_bytes(shapes, params: SegParams | None = None, ctx: Context | None = None) -> int:
    """Device workspace bytes segment_batch needs for tiles of these (H, W)
    shapes on `ctx` (its picker classes and frontier-queue capacity; None:
    the defaults) -- the library's exact figure, rt_segment_workspace_bytes."""
    n = len(shapes)
    if n == 0:
        return 0
    tiles = (_native.RtTile * n)()
    for i, (H, W) in enumerate(shapes):
        t = tiles[i]
        t.H, t.W = int(H), int(W)
        t.img = t.labels = t.d2 = 1            # placeholders: the size query reads no pointer
        t.ld_img = t.ld_labels = t.ld_d2 = int(W)
    cp = (params or SegParams()).to_c()
    return int(lib().rt_segment_workspace_bytes(ctx._h if ctx is not None else None, tiles, n, ctypes.byref(cp)))


def segment_batch(images, params: SegParams | None = None, *, outputs=None, want_recon: bool = True,
                  want_filled: bool = True, ctx=None, stream=None):
    """Run the segmentation chain on a list of uint8 CUDA tiles. Returns a list
    of dicts with R, F (if requested), L, D, n_kept and status tensors. Pass
    `outputs` (a list from a previous call) to reuse the buffers."""
    if not images:
        return []
    ctx = ctx or default_context(images[0].device.index)
    params = params or SegParams()
    n = len(images)
    tiles = (_native.RtTile * n)()
    if outputs is None:
        outputs = []
        for img in images:
            H, W = img.shape
            dev = img.device
            o = {
                "L": torch.empty((H, W), dtype=torch.int32, device=dev),
                "D": torch.empty((H, W), dtype=torch.int32, device=dev),
                "n_kept": torch.zeros(1, dtype=torch.int32, device=dev),
                "status": torch.zeros(1, dtype=torch.int32, device=dev),
            }
            if want_recon:
                o["R"] = torch.empty((H, W), dtype=torch.uint8, device=dev)
            if want_filled:
                o["F"] = torch.empty((H, W), dtype=torch.uint8, device=dev)
            outputs.append(o)
    for i, (img, o) in enumerate(zip(images, outputs)):
        ip, ild = _dev_ptr(img, torch.uint8, "image")
        t = tiles[i]
        t.img, t.ld_img = ip, ild
        t.H, t.W = img.shape
        if "R" in o:
            t.recon, t.ld_recon = _dev_ptr(o["R"], torch.uint8, "R")
        if "F" in o:
            t.filled, t.ld_filled = _dev_ptr(o["F"], torch.uint8, "F")
        t.labels, t.ld_labels = _dev_ptr(o["L"], torch.int32, "L")
        t.d2, t.ld_d2 = _dev_ptr(o["D"], torch.int32, "D")
        t.n_kept = o["n_kept"].data_ptr()
        t.status = o["status"].data_ptr()
    cp = params.to_c()
    _check(lib().rt_segment_batch(ctx.handle, tiles, n, ctypes.byref(cp), _stream(stream)), "rt_segment_batch")
    return outputs
