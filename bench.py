#!/usr/bin/env python
"""Throughput of the segmentation chain on 4096 x 4096 nuclei tiles.

One step = the whole chain (marker, reconstruction by dilation, threshold,
hole filling, labeling with the area filter, squared EDT) over one batch of
synthetic 4096 x 4096 tiles already resident in HBM. The metric is 4K x 4K
tiles per second (outputs bit-exact with the CPU oracle, checked by the
tests). Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl native|reference]

--impl reference times the CPU oracle (the plain C implementation the tests
check against) on the host cores on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "4Kx4K tiles/s (bit-exact segmentation chain)"
UNIT = "tiles/s"
BYTES_CHAIN = 9          # compulsory bytes/px: input 1 + labels 4 + EDT 4
BYTES_RF = 2             # R and F outputs, 1 byte each
BYTES_RECON = 2          # reconstruction: read mask 1, write R 1
BYTES_PASS = 3           # one directional raster pass over a pixel: read R and I, write R
PASSES_PER_ITERATION = 3 # a dense tile iteration: down, up and row passes
TILE_PX = 32 * 64        # pixels of one warp tile
# ncu summary of the propagation kernel on the bench workload: its DRAM
# traffic per launch is reported while the kernel sources still hash to the
# value recorded there (else traffic is null: the counters are stale)
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "recon_persistent_8x4k.md")
KERNEL_SOURCES = ("paper_1405_7958_gb300/csrc/recon.cu", "paper_1405_7958_gb300/csrc/recon.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8, help="tiles per step per GPU")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="serving leg at 800 tiles/s (0: skip)")
    ap.add_argument("--streams", type=int, default=3, help="streams the timed steps alternate between")
    ap.add_argument("--no-configs", action="store_true", help="skip the configuration 1 and 3 legs")
    return ap.parse_args()


def _gen(args):
    seed, size = args
    import synth
    return synth.config2_tile(seed, H=size, W=size)


def make_tiles(n, rank, size):
    """Seeded 4K nuclei tiles, generated in a spawn pool before any CUDA call."""
    import multiprocessing as mp
    seeds = [(2000 + 100 * rank + i, size) for i in range(n)]
    workers = max(1, min(n, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen, seeds)


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the propagation kernel from its committed ncu
    summary, or None when the summary is missing or the kernel has changed."""
    try:
        with open(TRAFFIC_PROFILE) as fh:
            text = fh.read()
    except OSError:
        return None
    fields = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    try:
        if fields.get("kernel sources sha256/16") != kernel_hash():
            return None
        return int(fields["dram bytes per launch (read + write)"])
    except (KeyError, ValueError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def window(self, t0, t1):
        """Keep only samples that arrived during [t0, t1] (wall clock)."""
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        mhz, maxes, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        t0, t1 = getattr(self, "t0", 0.0), getattr(self, "t1", float("inf"))
        for ts, ln in self.lines:
            if ts < t0 or ts > t1 + 0.25:
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": max(maxes), "samples": len(mhz),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------- CPU oracle
def cpu_model() -> str:
    """The host CPU's model name (from lscpu or /proc/cpuinfo; Arm cores
    report their implementer / part numbers instead of a name)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:   # a missing tool or odd output only loses the name
        pass
    try:
        with open("/proc/cpuinfo", errors="replace") as fh:
            info = fh.read()
        for key in ("model name", "CPU part"):
            for line in info.splitlines():
                if line.lower().startswith(key.lower()):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine() or "unknown"


def host_cores() -> int:
    """Cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_tiles_per_s(tiles, threads):
    """Oracle chain over `tiles`, one tile per host thread (the C oracle
    releases the GIL). Returns (tiles/s, seconds)."""
    import concurrent.futures as cf

    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(oracle.chain, tiles))
    dt = time.perf_counter() - t0
    return len(tiles) / dt, dt


def oracle_per_op_ms(tile):
    """Single-thread milliseconds of each step of the oracle chain on one tile."""
    import oracle
    oracle.build()
    out = {}
    t = time.perf_counter()
    J = oracle.marker(tile, 30)
    R = oracle.recon(J, tile, 8)
    out["marker_recon"] = time.perf_counter() - t
    t = time.perf_counter()
    B = oracle.threshold_below(R, 80)
    out["threshold"] = time.perf_counter() - t
    t = time.perf_counter()
    F = oracle.fill_holes(B, 4)
    out["fill"] = time.perf_counter() - t
    t = time.perf_counter()
    L = oracle.label_area(F, 20, 1000, 8)
    out["label_area"] = time.perf_counter() - t
    t = time.perf_counter()
    oracle.edt((L >= 0).astype("uint8"))
    out["edt"] = time.perf_counter() - t
    t = time.perf_counter()
    oracle.chain(tile)
    out["chain"] = time.perf_counter() - t
    return {k: round(1000 * v, 1) for k, v in out.items()}


def cpu_baseline(tiles, batch, size):
    """The oracle on all host cores, one tile per core (the first tile per
    op single-threaded as well)."""
    cores = host_cores()
    v, dt = oracle_tiles_per_s(tiles, cores)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "nproc": cores, "per_op_single_thread_ms": oracle_per_op_ms(tiles[0]),
            "sample": f"{len(tiles)} distinct {size}x{size} tiles of the bench's generator, one per host thread "
                      f"on all {cores} cores, {dt:.1f} s wall; per-op times: one tile on one thread"}


def run_reference(a, rank, world):
    if rank != 0:
        return
    cores = host_cores()
    n = max(a.batch, cores)
    tiles = make_tiles(n, 0, a.size)
    for _ in range(a.warmup):
        oracle_tiles_per_s(tiles, cores)
    times = []
    for _ in range(a.steps):
        _, dt = oracle_tiles_per_s(tiles, cores)
        times.append(dt)
    total = sum(times)
    value = n * a.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32",
        "data": "synthetic",
        "config": {"workload": f"segmentation chain on {a.size}x{a.size} nuclei tiles",
                   "tiles_per_step": n, "side": a.size},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"{n} tiles of {a.size}x{a.size} per step, one tile per host thread on all "
                                   f"{cores} cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- native
class Pipeline:
    """Timed steps alternating between `nst` CUDA streams (one library
    context each), every step flushing L2 on its own stream first. The timed
    region is bracketed by events on the first stream, which the others
    join at both ends."""

    def __init__(self, rt, dev, nst, picker=None):
        import torch
        self.torch = torch
        self.ctxs = [rt.Context(dev.index) for _ in range(nst)]
        if picker is not None:
            for c in self.ctxs:
                picker.attach(c)
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(nst)]
        self.flush = [torch.empty(256 << 20, dtype=torch.uint8, device=dev) for _ in range(nst)]   # > 129 MB L2

    def run(self, fn, steps, warmup, barrier, timing=False):
        """fn(k, ctx, stream) enqueues step k. Returns (total ms, per-step ms,
        kernel launches in the timed steps, phase times if timing)."""
        torch = self.torch
        nst = len(self.streams)

        def step(k, ev=None):
            j = k % nst
            s = self.streams[j]
            with torch.cuda.stream(s):
                self.flush[j].fill_(k & 0xFF)
                if ev is not None:
                    ev[0].record(s)
                fn(k, self.ctxs[j], s)
                if ev is not None:
                    ev[1].record(s)

        for k in range(max(warmup, nst)):
            step(k)
        torch.cuda.synchronize()
        if timing:
            for c in self.ctxs:
                c.timing(True)
                c.read_timing(reset=True)
        l0 = sum(c.kernel_launches() for c in self.ctxs)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        t0.record(self.streams[0])
        for s in self.streams[1:]:
            s.wait_event(t0)
        for k in range(steps):
            step(k, evs[k])
        for s in self.streams[1:]:
            ej = torch.cuda.Event()
            ej.record(s)
            self.streams[0].wait_event(ej)
        t1.record(self.streams[0])
        barrier()
        launches = sum(c.kernel_launches() for c in self.ctxs) - l0
        phases = {}
        if timing:
            for c in self.ctxs:
                for name, (ms, n) in c.read_timing(reset=True).items():
                    m0, n0 = phases.get(name, (0.0, 0))
                    phases[name] = (m0 + ms, n0 + n)
                c.timing(False)
        return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in evs], launches, phases

    def close(self):
        for c in self.ctxs:
            c.close()


def copy_rates(dev, nbytes=1 << 30):
    """Plain pinned host <-> device copy rates (GB/s, best of 3) on this machine:
    each direction alone, and both directions at once (two streams), which
    share the host link."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name, (dst, src) in (("h2d_gbs", (d, h)), ("d2h_gbs", (h, d))):
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            e1.synchronize()
            best = max(best, nbytes / (e0.elapsed_time(e1) / 1000) / 1e9)
        out[name] = round(best, 1)
    sa, sb = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    both = {"h2d_concurrent_gbs": 0.0, "d2h_concurrent_gbs": 0.0}
    for _ in range(3):
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(sa):
            ev[0].record(sa)
            d.copy_(h, non_blocking=True)
            ev[1].record(sa)
        with torch.cuda.stream(sb):
            ev[2].record(sb)
            h2.copy_(d2, non_blocking=True)
            ev[3].record(sb)
        torch.cuda.synchronize()
        both["h2d_concurrent_gbs"] = max(both["h2d_concurrent_gbs"], nbytes / (ev[0].elapsed_time(ev[1]) / 1000) / 1e9)
        both["d2h_concurrent_gbs"] = max(both["d2h_concurrent_gbs"], nbytes / (ev[2].elapsed_time(ev[3]) / 1000) / 1e9)
    out.update({k: round(v, 1) for k, v in both.items()})
    del h, h2, d, d2
    return out


def config3_leg(rt, ctx, dev, stream_ctor):
    """Configuration 3: 64 uneven tiles (sides 1024..4096 step 256, 50..400
    nuclei per Mpx) in one call captured in a CUDA graph, parameters from
    the autotuner, replayed on the capture stream; outputs of tiles 0, 31,
    32 and 63 (both chunks, both sides of the chunk boundary) checked
    against the oracle after the timed replays; null if any differs."""
    import concurrent.futures as cf

    import torch

    import oracle
    import synth
    from paper_1405_7958_gb300 import autotune
    specs = synth.batch_sizes(64, 3000)
    b3 = [rt.synth_tile(H, W, sd, ns, ctx=ctx) for H, W, ns, sd in specs]
    px3 = sum(H * W for H, W, _, _ in specs)
    tuned = autotune.tune(b3, reps=2, ctx=ctx)["best"]
    p3 = rt.SegParams(variant=int(tuned["variant"]), max_local=int(tuned["max_local"]),
                      strip_tiles=int(tuned["strip_tiles"]))
    g3s = stream_ctor()
    with torch.cuda.stream(g3s):
        o3 = rt.segment_batch(b3, p3, ctx=ctx, stream=g3s, want_recon=False, want_filled=False)
    g3s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=g3s):
        rt.segment_batch(b3, p3, outputs=o3, ctx=ctx, stream=g3s, want_recon=False, want_filled=False)
    with torch.cuda.stream(g3s):
        for _ in range(2):
            graph.replay()
        for o in o3:
            o["L"].fill_(-5)
            o["D"].fill_(-5)
        t3 = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(g3s)
            graph.replay()
            e1.record(g3s)
            t3.append((e0, e1))
    g3s.synchronize()
    t3 = [a.elapsed_time(b) for a, b in t3]
    sample = (0, 31, 32, 63)
    hosts = [b3[i].cpu().numpy() for i in sample]
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        want = list(ex.map(oracle.chain, hosts))
    ok = all(np.array_equal(o3[i]["L"].cpu().numpy(), w["L"]) and np.array_equal(o3[i]["D"].cpu().numpy(), w["D"])
             for i, w in zip(sample, want))
    ms3 = statistics.median(t3)
    res = {"tiles": 64, "megapixels": px3 / 1e6, "tuned": tuned, "graph_replay_ms": ms3, "replays": 5,
           "oracle_checked_tiles": list(sample), "outputs_match_oracle": ok,
           "chain_bytes_per_replay": BYTES_CHAIN * px3,
           "chain_gbs": BYTES_CHAIN * px3 / (ms3 / 1000.0) / 1e9,
           "tile4k_equiv_s": px3 / 2 ** 24 / (ms3 / 1000.0) if ok else None,
           "tiles_s": 64 / (ms3 / 1000.0) if ok else None}
    del o3, b3, graph
    return res



def timed_ms(fn, reps):
    """Median milliseconds of fn() on the current stream (CUDA events)."""
    import torch
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def objects_leg(rt, ctx, outs, imgs):
    """The steps after the chain on the bench's tiles: per-nucleus features
    (rt_object_features) and the watershed of the distance map (rt_watershed,
    h = 2), one tile per call; median of 5 after a warm-up call."""
    import torch
    cap = 20000
    n_obj = torch.zeros(1, dtype=torch.int32, device=imgs[0].device)
    n_bas = torch.zeros(1, dtype=torch.int32, device=imgs[0].device)
    basins = [torch.empty_like(o["L"]) for o in outs]

    def feats():
        for o, im in zip(outs, imgs):
            rt.object_features(o["L"], im, cap, n_obj=n_obj, ctx=ctx)

    def sheds():
        for o, b in zip(outs, basins):
            rt.watershed(o["L"], o["D"], 2, out=b, n_basins=n_bas, ctx=ctx)

    feats()
    sheds()
    f_ms, w_ms = timed_ms(feats, 5), timed_ms(sheds, 5)
    nobj, nbas = int(n_obj.item()), int(n_bas.item())
    n = len(imgs)
    return {"tiles": n, "features_ms_per_tile": f_ms / n, "watershed_ms_per_tile": w_ms / n,
            "nuclei_last_tile": nobj, "basins_last_tile": nbas,
            "nuclei_features_per_s": nobj * n / (f_ms / 1000.0) if nobj else None,
            "features_per_nucleus": 20, "watershed_h": 2}


def picker_train_leg(rt, dev, B=256):
    """One training step of the picker network (forward with saved
    activations, backward, AdamW) on a batch of B samples, on the tensor
    cores and on the fp32 kernels; median of 50 after 5 warm-up steps."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(3)
    x = (torch.randn(B, 24, generator=g) * 3 + 1).to(dev)
    y = torch.randint(0, 3, (B,), generator=g, dtype=torch.int32).to(dev)
    res = {"batch": B}
    for name, tc in (("tensor_cores_us", True), ("fp32_us", False)):
        pk = rt.Picker(device=dev, seed=1)
        pk.set_norm(x)

        def step():
            logits, act, _ = pk.forward(x, with_act=True, tensor_cores=tc)
            pk.backward(x, act, logits, y, tensor_cores=tc)
            pk.step()

        for _ in range(5):
            step()
        res[name] = timed_ms(step, 50) * 1000.0
    return res


def slide_leg(rt, ctx, side=16384):
    """Whole-slide segmentation: one side x side slide (16 tiles of 4096^2,
    nuclei across every seam) as one image; median of 3 after a warm-up."""
    import torch
    slide = rt.config2_tile(515151, H=side, W=side, ctx=ctx)
    out = rt.segment_batch([slide], ctx=ctx, want_recon=False, want_filled=False)
    ms = timed_ms(lambda: rt.segment_batch([slide], outputs=out, ctx=ctx, want_recon=False, want_filled=False), 3)
    ok = int(out[0]["status"].item()) == 0
    res = {"side": side, "ms": ms, "status_ok": ok, "megapixels_s": side * side / 1e6 / (ms / 1000.0),
           "tile4k_equiv_s": side * side / 2 ** 24 / (ms / 1000.0), "nuclei_kept": int(out[0]["n_kept"].item())}
    del out, slide
    torch.cuda.empty_cache()
    return res


def run_native(a, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1405_7958_gb300 as rt

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = rt.Context(local_rank)
    # the bench's tiles, drawn on the GPU by the generator's bit-exact twin
    imgs = [rt.config2_tile(2000 + 100 * rank + i, H=a.size, W=a.size, ctx=ctx) for i in range(a.batch)]
    torch.cuda.synchronize()
    # the metric's configuration: batched, with the trained variant picker
    from paper_1405_7958_gb300 import picker as pkmod
    picker = pkmod.load(os.path.join(ROOT, "paper_1405_7958_gb300", "data", "picker_config4.npz"), device=dev)
    picker.attach(ctx)
    learned = rt.SegParams(policy=1, pick_min_prob=600)    # the trained picker with its confidence fall-back
    plain = rt.SegParams()
    nst = max(1, a.streams)
    pipe = Pipeline(rt, dev, nst, picker)
    outs_l = [None] * nst
    outs_p = [None] * nst
    outs_1 = [[None] * a.batch for _ in range(nst)]

    def step_learned(k, c, s):
        j = k % nst
        outs_l[j] = rt.segment_batch(imgs, learned, outputs=outs_l[j], ctx=c, stream=s)

    def step_plain(k, c, s):
        j = k % nst
        outs_p[j] = rt.segment_batch(imgs, plain, outputs=outs_p[j], ctx=c, stream=s)

    def step_per_tile(k, c, s):
        j = k % nst
        for i, im in enumerate(imgs):
            o = outs_1[j][i]
            outs_1[j][i] = rt.segment_batch([im], plain, outputs=None if o is None else [o], ctx=c, stream=s)[0]

    sampler = ClockSampler(local_rank)
    sampler.start()
    wall0 = time.time()
    total_ms, step_ms, launches, phases = pipe.run(step_learned, a.steps, a.warmup, barrier, timing=True)
    sampler.window(wall0, time.time())
    clocks = sampler.stop()
    visits = pipe.ctxs[0].recon_stats()
    picks = rt.last_picks(pipe.ctxs[0])
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    px = a.size * a.size
    value = world * a.batch * a.steps / (total_ms / 1000.0)

    # the propagation launch alone: the same steps on one stream (no other
    # step's kernels beside it), for the kernel's own duration
    pipe1 = Pipeline(rt, dev, 1, picker)
    outs_a = [None]

    def step_alone(k, c, s):
        outs_a[0] = rt.segment_batch(imgs, learned, outputs=outs_a[0], ctx=c, stream=s)

    _, _, _, phases_alone = pipe1.run(step_alone, max(5, a.steps // 4), a.warmup, barrier, timing=True)
    pipe1.close()

    # the plain legs on the same harness (same streams, contexts, flushes)
    k2 = max(5, a.steps // 4)
    plain_ms, _, plain_launches, _ = pipe.run(step_plain, k2, a.warmup, barrier)
    per_tile_ms, _, per_tile_launches, _ = pipe.run(step_per_tile, k2, a.warmup, barrier)
    batched_plain = a.batch * k2 / (plain_ms / 1000)
    per_tile_plain = a.batch * k2 / (per_tile_ms / 1000)
    torch.cuda.synchronize()
    # batched, plain and one-at-a-time produce the same bytes
    for o_l, o_p, o_1 in zip(outs_l[0], outs_p[0], outs_1[0]):
        assert torch.equal(o_l["L"], o_p["L"]) and torch.equal(o_l["D"], o_1["D"])

    # configuration 1: reconstruction only, one 512^2 image, median of 200
    # timed runs after 20 warm-up runs, with the bytes the passes moved
    config1 = None
    config3 = None
    objects = None
    slide = None
    train_step = None
    stream = torch.cuda.current_stream()
    if not a.no_configs and world == 1:
        import synth
        c1 = torch.from_numpy(synth.config1_image(1000)).to(dev)
        r1 = torch.empty_like(c1)
        for _ in range(20):
            rt.reconstruct(c1, None, h_offset=30, out=r1, ctx=ctx, stream=stream)
        t1 = []
        for _ in range(200):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rt.reconstruct(c1, None, h_offset=30, out=r1, ctx=ctx, stream=stream)
            e1.record(stream)
            e1.synchronize()
            t1.append(e0.elapsed_time(e1))
        v1, it1, _ = ctx.recon_stats()
        config1 = {"image": "512x512, 60 disks, flat background", "median_ms": statistics.median(t1), "reps": 200,
                   "warmup": 20, "tile_visits": v1, "tile_iterations": it1,
                   "pass_bytes": it1 * PASSES_PER_ITERATION * TILE_PX * BYTES_PASS,
                   "compulsory_bytes": BYTES_RECON * 512 * 512}
        config3 = config3_leg(rt, ctx, dev, lambda: torch.cuda.Stream(device=dev))
        objects = objects_leg(rt, ctx, outs_l[0], imgs)
        slide = slide_leg(rt, ctx)
        train_step = picker_train_leg(rt, dev)

    serving = None
    if a.serve_seconds > 0 and world == 1:
        from paper_1405_7958_gb300 import serve
        spool = serve.make_pool(32, 5000, ctx=ctx)
        hp = serve.host_pool(spool)
        serve.run_batched(serve.arrivals(800.0, 1.0, len(spool), 9, spool), spool, policy=1, picker=picker, hp=hp)
        reqs = serve.arrivals(800.0, a.serve_seconds, len(spool), 801, spool)
        serve.run_batched(reqs, spool, policy=1, picker=picker, hp=hp)
        serving = {"rate_tiles_s": 800, "seconds": a.serve_seconds, "tiles": "512..4096 px sides",
                   **serve.summarize(reqs, a.serve_seconds)}

    # dominant kernel: the propagation sweeps (one launch per step)
    sweep_ms, sweep_n = phases["recon_sweep"]
    peak, peak_kind = load_peaks()
    roof = None
    if sweep_n:
        per_launch_s = sweep_ms / sweep_n / 1000.0
        algo_bytes = BYTES_RECON * px * a.batch
        ach = algo_bytes / per_launch_s / 1e9
        its = visits[1]       # dense tile iterations of one step (the last one)
        pass_bytes = its * PASSES_PER_ITERATION * TILE_PX * BYTES_PASS
        ms_alone, n_alone = phases_alone["recon_sweep"]
        alone_s = ms_alone / max(n_alone, 1) / 1000.0
        roof = {"kernel": "recon_persistent_kernel<8,0>", "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "launch_ms_alone": alone_s * 1000, "achieved_alone": algo_bytes / alone_s / 1e9,
                "frac_alone": algo_bytes / alone_s / 1e9 / peak,
                "frac": ach / peak, "peak_source": peak_kind, "traffic": profiled_traffic(),
                "algorithmic_bytes_per_launch": algo_bytes, "launch_ms": per_launch_s * 1000,
                "pass_bytes_per_launch": pass_bytes, "pass_equivalent_gbs": pass_bytes / per_launch_s / 1e9,
                "pass_equivalent_frac": pass_bytes / per_launch_s / 1e9 / peak}

    # end to end through the public API with host buffers: every step copies
    # its inputs from pinned host memory, runs the chain and copies labels and
    # distances back. Steps alternate between the compute streams (one context
    # each). The input copies run on a stream of their own two steps ahead,
    # the read-backs on another, into and from input and output sets rotated
    # over twice as many steps as there are compute streams, so no compute
    # stream waits behind a copy queue
    e2e = None
    if not a.no_e2e:
        nset = 2 * nst
        ahead = 2
        h_in = [im.cpu().pin_memory() for im in imgs]
        h_L = [[torch.empty((a.size, a.size), dtype=torch.int32).pin_memory() for _ in imgs] for _ in range(nset)]
        h_D = [[torch.empty((a.size, a.size), dtype=torch.int32).pin_memory() for _ in imgs] for _ in range(nset)]
        d_in = [[torch.empty_like(x, device=dev) for x in imgs] for _ in range(nset)]
        read_s = torch.cuda.Stream(device=dev)
        in_s = torch.cuda.Stream(device=dev)
        outs_e = [None] * nset
        read_done = [None] * nset
        used = [None] * nset     # the set's last compute, after which its inputs may be overwritten
        in_ready = [None] * nset
        n_steps = [0]            # steps to run: no inputs are loaded past the last one

        def e2e_load(k):
            b = k % nset
            with torch.cuda.stream(in_s):
                if used[b] is not None:
                    in_s.wait_event(used[b])
                for h, d in zip(h_in, d_in[b]):
                    d.copy_(h, non_blocking=True)
                in_ready[b] = torch.cuda.Event()
                in_ready[b].record(in_s)

        def e2e_step(k):
            j, b = k % nst, k % nset
            s = pipe.streams[j]
            with torch.cuda.stream(s):
                s.wait_event(in_ready[b])
                if read_done[b] is not None:
                    s.wait_event(read_done[b])      # the set's previous read-back has finished
                outs_e[b] = rt.segment_batch(d_in[b], learned, outputs=outs_e[b], ctx=pipe.ctxs[j], stream=s,
                                             want_recon=False, want_filled=False)
                computed = torch.cuda.Event()
                computed.record(s)
                used[b] = computed
            read_s.wait_event(computed)
            with torch.cuda.stream(read_s):
                for o, hl, hd in zip(outs_e[b], h_L[b], h_D[b]):
                    hl.copy_(o["L"], non_blocking=True)
                    hd.copy_(o["D"], non_blocking=True)
                read_done[b] = torch.cuda.Event()
                read_done[b].record(read_s)
            if k + ahead < n_steps[0]:
                e2e_load(k + ahead)

        nwarm = max(nset, a.warmup)
        n_steps[0] = nwarm              # warm-up: inputs of warm-up steps only
        for k in range(ahead):
            e2e_load(k)
        for k in range(nwarm):
            e2e_step(k)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(pipe.streams[0])
        for s in pipe.streams[1:] + [read_s, in_s]:
            s.wait_event(e0)
        # timed: every step's input copy is inside the region. The region
        # starts with an empty pipeline (the first inputs' copies) and ends
        # draining it (the last read-backs), so it runs at least 60 steps
        # for a steady-state rate
        ke = max(a.steps, 60)
        n_steps[0] = nwarm + ke
        for k in range(nwarm, nwarm + ahead):
            e2e_load(k)
        for k in range(nwarm, nwarm + ke):
            e2e_step(k)
        for s in pipe.streams[1:] + [read_s, in_s]:
            ev = torch.cuda.Event()
            ev.record(s)
            pipe.streams[0].wait_event(ev)
        e1.record(pipe.streams[0])
        barrier()
        tt = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        # the read-back matches the device result
        torch.cuda.synchronize()
        assert np.array_equal(h_L[0][0].numpy(), outs_e[0][0]["L"].cpu().numpy())
        rates = copy_rates(dev)
        h2d, d2h = a.batch * px, a.batch * px * 8
        e2e = {"value": world * a.batch * ke / (float(tt.item()) / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke,
               "streams": nst, "output_sets": nset, "input_lookahead_steps": ahead, "copy_gbs": rates,
               "copy_bound_tiles_s": a.batch / max(h2d / (rates["h2d_gbs"] * 1e9), d2h / (rates["d2h_gbs"] * 1e9)),
               "copy_bound_concurrent_tiles_s": a.batch / max(h2d / (rates["h2d_concurrent_gbs"] * 1e9),
                                                              d2h / (rates["d2h_concurrent_gbs"] * 1e9))}
        del h_in, h_L, h_D, d_in

    cpu = None
    if rank == 0 and not a.no_cpu:
        n_cpu = max(a.batch, host_cores())
        cpu_tiles = [im.cpu().numpy() for im in imgs]
        cpu_tiles += [rt.config2_tile(3000 + i, H=a.size, W=a.size, ctx=ctx).cpu().numpy()
                      for i in range(n_cpu - len(cpu_tiles))]
        cpu = cpu_baseline(cpu_tiles, a.batch, a.size)
    pipe.close()

    if world > 1:
        dist.barrier()
    if rank == 0:
        chain_bytes = (BYTES_CHAIN + BYTES_RF) * px * a.batch * a.steps * world
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/i32", "data": "synthetic",
            "config": {"workload": f"segmentation chain, {a.batch} x {a.size}x{a.size} nuclei tiles per step per GPU",
                       "tiles_per_step": a.batch, "side": a.size, "parallelism": f"replicas x{world}",
                       "l2": "flushed before every step (256 MB write on the step's stream)",
                       "streams": nst,
                       "pipelining": "consecutive steps alternate between the streams (one context each); "
                                     "the plain legs run on the same harness"},
            "chain_hbm_gbs": chain_bytes / (total_ms / 1000.0) / 1e9,
            "roofline": roof,
            "phases_ms_per_step": {k: v[0] / a.steps for k, v in phases.items()},
            "phases_note": "sum of per-phase event times over the steps / steps; phases of overlapping steps overlap",
            "recon_visits_iterations_per_step": visits,
            "batched_learned_tiles_s": value,
            "batched_plain_tiles_s": world * batched_plain,
            "plain_per_tile_tiles_s": world * per_tile_plain,
            "launches_per_step": {"batched_learned": launches / a.steps, "batched_plain": plain_launches / k2,
                                  "per_tile_plain": per_tile_launches / k2},
            "picker_choices": picks,
            "serving_batched_learned": serving,
            "config1_recon_512": config1,
            "config3_uneven_64_graph": config3,
            "objects_per_tile": objects,
            "slide": slide,
            "picker_train_step": train_step,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "step_ms": [round(x, 4) for x in step_ms],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_native(a, rank, world, local_rank)


if __name__ == "__main__":
    main()
