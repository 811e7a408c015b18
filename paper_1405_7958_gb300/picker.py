"""Training and evaluation of the learned variant picker.

The picker chooses, per tile, how its reconstruction propagates (RT_RASTER,
RT_QUEUE or RT_HYBRID; all three give identical bytes). Its training data
are timings the method itself produces: every tile is drawn on the GPU,
reconstructed with each variant (CUDA events on the launch stream, median of
`reps` runs), and checked to give the same output under all three; the
label is the fastest variant. Training runs the library's own forward,
backward and AdamW kernels; torch only holds the buffers.

    python -m paper_1405_7958_gb300.picker --train 4000 --eval 512 \
        --out picker.npz --report picker_report.json
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

import paper_1405_7958_gb300 as rt

VARIANTS = (rt.RT_RASTER, rt.RT_QUEUE, rt.RT_HYBRID)
NAMES = ("raster", "queue", "hybrid")


def tile_specs(n: int, seed: int, lo: int = 1024, hi: int = 4096, step: int = 256):
    """(H, W, n_shapes, tile_seed) of n tiles: sides uniform over
    {lo, lo+step, ..., hi}, nuclei density uniform in [50, 400] per Mpx."""
    import synth
    return synth.batch_sizes(n, seed, lo, hi, step)


def variant_times(ctx, img: torch.Tensor, reps: int = 3, stream=None):
    """Median reconstruction time (ms) of each variant on one tile, and
    whether all variants produced the same bytes."""
    stream = stream or torch.cuda.current_stream()
    outs, times = [], []
    for v in VARIANTS:
        out = torch.empty_like(img)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rt.reconstruct(img, None, h_offset=30, conn=8, variant=v, out=out, ctx=ctx, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        times.append(float(np.median(ts)))
        outs.append(out)
    same = all(torch.equal(outs[0], o) for o in outs[1:])
    return times, same


def build_dataset(n: int, seed: int, reps: int = 3, ctx=None, log_every: int = 500, cache: str | None = None):
    """Features (n x 24) and variant times (n x 3, ms) of n GPU-drawn tiles.
    With `cache`, finished rows are saved and a rerun resumes from them."""
    ctx = ctx or rt.Context()
    specs = tile_specs(n, seed)
    feats = np.zeros((n, 24), np.float32)
    times = np.zeros((n, 3), np.float64)
    start = 0
    if cache and os.path.exists(cache):
        z = np.load(cache)
        k = int(z["done"])
        if z["feats"].shape[0] == n:
            feats[:k], times[:k], start = z["feats"][:k], z["times"][:k], k
    # one warm-up of every variant
    warm = rt.synth_tile(1024, 1024, 1, 40, ctx=ctx)
    variant_times(ctx, warm, 1)
    t0 = time.time()
    for i in range(start, n):
        H, W, ns, s = specs[i]
        img = rt.synth_tile(H, W, s, ns, ctx=ctx)
        feats[i] = rt.tile_features([img], ctx=ctx).cpu().numpy()[0]
        tv, same = variant_times(ctx, img, reps)
        if not same:
            raise RuntimeError(f"variants disagree on tile {i} (seed {s})")
        times[i] = tv
        if log_every and (i + 1) % log_every == 0:
            print(f"  dataset {i + 1}/{n}  {time.time() - t0:.0f} s", flush=True)
            if cache:
                np.savez(cache, feats=feats, times=times, done=i + 1)
    if cache:
        np.savez(cache, feats=feats, times=times, done=n)
    return feats, times


def train(feats: np.ndarray, times: np.ndarray, epochs: int = 60, batch: int = 256, lr: float = 3e-3,
          seed: int = 0, device=None) -> rt.Picker:
    """Cross-entropy on the fastest variant, mini-batch AdamW, all on the GPU."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(np.ascontiguousarray(feats)).to(device)
    y = torch.from_numpy(times.argmin(axis=1).astype(np.int32)).to(device)
    pk = rt.Picker(device=device, seed=seed)
    pk.set_norm(x)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(device)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = x[idx].contiguous(), y[idx].contiguous()
            logits, act, _ = pk.forward(xb, with_act=True)
            pk.backward(xb, act, logits, yb)
            pk.step(lr=lr)
    return pk


def evaluate(pk: rt.Picker, feats: np.ndarray, times: np.ndarray) -> dict:
    """Selection accuracy, regret, and the summed reconstruction time of the
    picks against the plain schedule (RT_RASTER for every tile) and against
    the best variant per tile."""
    x = torch.from_numpy(np.ascontiguousarray(feats)).to(pk.device)
    _, _, pick = pk.forward(x)
    pick = pick.cpu().numpy()
    best = times.argmin(axis=1)
    chosen = times[np.arange(len(times)), pick]
    return {
        "tiles": int(len(times)),
        "accuracy": float((pick == best).mean()),
        "pick_counts": {NAMES[k]: int((pick == k).sum()) for k in range(3)},
        "best_counts": {NAMES[k]: int((best == k).sum()) for k in range(3)},
        "regret_mean_ms": float((chosen - times.min(axis=1)).mean()),
        "time_learned_ms": float(chosen.sum()),
        "time_plain_ms": float(times[:, 0].sum()),
        "time_best_ms": float(times.min(axis=1).sum()),
        "gain_vs_plain": float(times[:, 0].sum() / chosen.sum()),
    }


def save(pk: rt.Picker, path: str):
    sd = pk.state_dict()
    np.savez(path, **{k: (v.numpy() if hasattr(v, "numpy") else np.asarray(v)) for k, v in sd.items()})


def load(path: str, device=None) -> rt.Picker:
    z = np.load(path)
    pk = rt.Picker(device=device)
    pk.load_state_dict({k: torch.from_numpy(np.asarray(z[k])) for k in ("master", "wb", "m", "v", "norm")}
                       | {"step_count": int(z["step_count"])})
    return pk


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4000)
    ap.add_argument("--eval", type=int, default=512)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--out", default="picker.npz")
    ap.add_argument("--report", default="picker_report.json")
    ap.add_argument("--cache", default=None, help="dataset cache prefix (resumable)")
    a = ap.parse_args()
    ctx = rt.Context()
    t0 = time.time()
    ftr, ttr = build_dataset(a.train, 4000 + a.seed, a.reps, ctx,
                             cache=(a.cache + "_train.npz") if a.cache else None)
    fev, tev = build_dataset(a.eval, 4500 + a.seed, a.reps, ctx,
                             cache=(a.cache + "_eval.npz") if a.cache else None)
    t1 = time.time()
    pk = train(ftr, ttr, epochs=a.epochs, seed=a.seed)
    t2 = time.time()
    rep = {"train": evaluate(pk, ftr, ttr), "eval": evaluate(pk, fev, tev),
           "dataset_s": t1 - t0, "train_s": t2 - t1, "epochs": a.epochs, "reps": a.reps}
    save(pk, a.out)
    with open(a.report, "w") as fh:
        json.dump(rep, fh, indent=1)
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
