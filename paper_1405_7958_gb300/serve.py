"""Serving loop with continuous batching for the segmentation chain.

Requests (single tiles, sides 512..4096) arrive as a Poisson process. The
batched server reserves, at start-up, one library context per stream with
the workspace of the largest batch it will launch (the library's exact
figure, rt_segment_workspace_bytes), so nothing is allocated inside the
loop; the rest of the device-memory budget holds the requests' own buffers
(input, labels, distances: 9 bytes per pixel). It admits arrived requests,
in arrival order, while their buffers fit the budget beside those in use
and the batch's workspace fits the context's reservation, launches every
admitted group as one batch on a free stream, and keeps admitting and
launching while earlier batches are still on the GPU, so host-to-device
copies, compute and device-to-host copies of different batches overlap.
The plain server runs one tile at a time on one stream with the fixed
variant. Latency is the time from a request's arrival to its labels and
distance map being in host memory.

    python -m paper_1405_7958_gb300.serve --rates 50 200 800 --duration 10
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np
import torch

import paper_1405_7958_gb300 as rt

BYTES_PER_PX = 9            # a request's device buffers: input 1 + labels 4 + distances 4
BATCH_TILES_4K = 8          # the largest batch a context reserves workspace for, in 4096^2 tiles


@dataclass
class Request:
    rid: int
    arrival: float          # seconds since the start
    H: int
    W: int
    pool: int               # index of its host tile
    done: float = -1.0
    out_L: torch.Tensor | None = None
    out_D: torch.Tensor | None = None


@dataclass
class Batch:
    reqs: list
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    slot: int
    dev: list = field(default_factory=list)


class PinnedPool:
    """Reusable pinned host buffers by shape (allocating pinned memory per
    request would stall the loop); reserve() allocates them before the
    timed run."""

    def __init__(self):
        self.free = {}

    def reserve(self, shapes, per_shape: int, dtype=torch.int32):
        for shape in set(tuple(x) for x in shapes):
            lst = self.free.setdefault((shape, dtype), [])
            while len(lst) < per_shape:
                lst.append(torch.empty(shape, dtype=dtype).pin_memory())

    def get(self, shape, dtype=torch.int32):
        lst = self.free.get((shape, dtype))
        if lst:
            return lst.pop()
        return torch.empty(shape, dtype=dtype).pin_memory()

    def put(self, t):
        self.free.setdefault((tuple(t.shape), t.dtype), []).append(t)


def make_pool(n: int, seed: int, lo: int = 512, hi: int = 4096, step: int = 256, ctx=None):
    """n distinct tiles drawn on the GPU and kept in pinned host memory."""
    import synth
    specs = synth.batch_sizes(n, seed, lo, hi, step)
    pool = []
    for H, W, ns, s in specs:
        t = rt.synth_tile(H, W, s, ns, ctx=ctx)
        pool.append(t.cpu().pin_memory())
    return pool


def arrivals(rate: float, duration: float, n_pool: int, seed: int, pool):
    rng = np.random.default_rng(seed)
    t, out, k = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        p = int(rng.integers(0, n_pool))
        H, W = pool[p].shape
        out.append(Request(k, t, H, W, p))
        k += 1


def _wait_until(t0: float, t: float):
    while True:
        d = t - (time.perf_counter() - t0)
        if d <= 0:
            return
        time.sleep(min(d, 2e-4))


def _fetch(o, r, hp: PinnedPool):
    r.out_L = hp.get((r.H, r.W))
    r.out_D = hp.get((r.H, r.W))
    r.out_L.copy_(o["L"], non_blocking=True)
    r.out_D.copy_(o["D"], non_blocking=True)


def _release(r, hp: PinnedPool, keep: bool):
    if not keep:
        hp.put(r.out_L)
        hp.put(r.out_D)
        r.out_L = r.out_D = None


def request_bytes(r) -> int:
    return r.H * r.W * BYTES_PER_PX


def admit(pending: list, in_use: int, budget_bytes: int, max_batch: int, ws_fits=None):
    """Takes requests from the front of `pending` (arrival order) while their
    device bytes fit the budget beside the bytes in use, at most max_batch,
    and (with ws_fits) while the batch's workspace fits the context's
    reservation; a request larger than the whole budget is taken alone once
    nothing else is in use. Returns (taken requests, bytes in use)."""
    take = []
    while pending and len(take) < max_batch:
        need = request_bytes(pending[0])
        if in_use + need > budget_bytes and (take or in_use > 0):
            break
        if take and ws_fits is not None and not ws_fits([(r.H, r.W) for r in take] + [(pending[0].H, pending[0].W)]):
            break
        in_use += need
        take.append(pending.pop(0))
    return take, in_use


def host_pool(pool, per_shape: int = 8) -> PinnedPool:
    """Pinned read-back buffers for every tile shape of the pool (two per
    request: labels and distances), allocated before the timed run."""
    hp = PinnedPool()
    hp.reserve([t.shape for t in pool], 2 * per_shape)
    return hp


def run_plain(reqs, pool, variant=rt.RT_RASTER, ctx=None, keep: bool = False, hp: PinnedPool | None = None):
    """One tile at a time, fixed variant, one stream."""
    ctx = ctx or rt.Context()
    s = torch.cuda.Stream()
    hp = hp or PinnedPool()
    params = rt.SegParams(variant=variant)
    t0 = time.perf_counter()
    for r in reqs:
        _wait_until(t0, r.arrival)
        with torch.cuda.stream(s):
            d_in = pool[r.pool].to("cuda", non_blocking=True)
            o = rt.segment_batch([d_in], params, ctx=ctx, stream=s, want_recon=False, want_filled=False)[0]
            _fetch(o, r, hp)
        s.synchronize()
        r.done = time.perf_counter() - t0
        _release(r, hp, keep)
    return reqs


def run_batched(reqs, pool, budget_bytes: int = 40 << 30, max_batch: int = 32, n_streams: int = 3,
                policy: int = 0, picker=None, keep: bool = False, hp: PinnedPool | None = None):
    """Continuous batching under a device-memory budget (policy 1: the
    attached picker chooses each tile's variant)."""
    hp = hp or PinnedPool()
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    params = rt.SegParams(policy=policy, pick_min_prob=600 if policy else 0)   # learned: with the fall-back
    reserve = rt.segment_workspace_bytes([(4096, 4096)] * BATCH_TILES_4K, params)
    ctxs = [rt.Context(workspace_bytes=reserve) for _ in range(n_streams)]
    held = [c.workspace_bytes() for c in ctxs]
    budget_bytes -= sum(held)
    # The requests' device buffers come from torch's caching allocator. One
    # block of the whole remaining budget, allocated and freed here, stays in
    # its cache, so no allocation inside the loop reaches cudaMalloc, which
    # would wait for every stream's work to finish.
    if budget_bytes > 0:
        torch.empty(budget_bytes, dtype=torch.uint8, device="cuda")
    if picker is not None:
        for c in ctxs:
            picker.attach(c)

    def ws_fits(shapes):
        return rt.segment_workspace_bytes(shapes, params) <= reserve

    busy = [None] * n_streams
    pending, nxt, done_n = [], 0, 0
    in_use = 0
    t0 = time.perf_counter()
    while done_n < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            pending.append(reqs[nxt])
            nxt += 1
        # retire finished batches
        for k, b in enumerate(busy):
            if b is not None and b.event.query():
                tnow = time.perf_counter() - t0
                for r in b.reqs:
                    r.done = tnow
                    in_use -= request_bytes(r)
                    _release(r, hp, keep)
                done_n += len(b.reqs)
                busy[k] = None
        # admit and launch on a free stream
        free = [k for k, b in enumerate(busy) if b is None]
        if pending and free:
            take, in_use = admit(pending, in_use, budget_bytes, max_batch, ws_fits)
            if take:
                k = free[0]
                s = streams[k]
                with torch.cuda.stream(s):
                    d_in = [pool[r.pool].to("cuda", non_blocking=True) for r in take]
                    outs = rt.segment_batch(d_in, params, ctx=ctxs[k], stream=s, want_recon=False,
                                            want_filled=False)
                    for r, o in zip(take, outs):
                        _fetch(o, r, hp)
                    ev = torch.cuda.Event()
                    ev.record(s)
                busy[k] = Batch(take, s, ev, k, d_in)
                continue
        if nxt < len(reqs) and not pending:
            _wait_until(t0, min(reqs[nxt].arrival, (time.perf_counter() - t0) + 1e-4))
        else:
            time.sleep(2e-5)
    grown = [c.workspace_bytes() != h for c, h in zip(ctxs, held)]
    for c in ctxs:
        c.close()
    if any(grown):
        raise RuntimeError("a serving context grew its workspace inside the loop")
    return reqs


def summarize(reqs, duration: float) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs]) * 1000.0
    end = max(r.done for r in reqs) if reqs else duration
    px = sum(r.H * r.W for r in reqs)
    return {"requests": len(reqs), "throughput_tiles_s": len(reqs) / max(end, 1e-9),
            "throughput_4k_equiv_s": px / 2 ** 24 / max(end, 1e-9),
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_ms": float(lat.mean()) if len(lat) else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", type=float, nargs="+", default=[50, 200, 800])
    ap.add_argument("--duration", type=float, default=30.0)
    ap.add_argument("--warmup", type=float, default=2.0, help="seconds of arrivals at the same rate first")
    ap.add_argument("--pool", type=int, default=48)
    ap.add_argument("--picker", default=None, help="trained picker weights (.npz) for the batched server")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    ctx = rt.Context()
    pool = make_pool(a.pool, 5000, ctx=ctx)
    hp = host_pool(pool)
    picker = None
    if a.picker:
        from paper_1405_7958_gb300 import picker as pk
        picker = pk.load(a.picker)
    res = {}
    for lam in a.rates:
        res[str(lam)] = {}
        for mode in ("plain", "batched"):
            reqs = arrivals(lam, a.duration, len(pool), int(lam) * 7 + 1, pool)
            # warm-up at the same rate (first launches, torch's caching allocator)
            warm = arrivals(lam, a.warmup, len(pool), 99, pool)
            if mode == "plain":
                run_plain(warm, pool, ctx=ctx, hp=hp)
                torch.cuda.synchronize()
                run_plain(reqs, pool, ctx=ctx, hp=hp)
            else:
                pol = 1 if picker is not None else 0
                run_batched(warm, pool, policy=pol, picker=picker, hp=hp)
                torch.cuda.synchronize()
                run_batched(reqs, pool, policy=pol, picker=picker, hp=hp)
            res[str(lam)][mode] = summarize(reqs, a.duration)
            print(json.dumps({"rate": lam, "mode": mode, **res[str(lam)][mode]}), flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
