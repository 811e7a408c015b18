"""Training and evaluation of the learned schedule picker.

The picker chooses, per tile, how its reconstruction propagates: one of three
schedules (a variant and its sweep iterations per dense tile visit; by
default the raster sweeps with 4, 12 and 24 iterations), all giving
identical bytes; a pick it is not confident of falls back to the plain
schedule (the raster sweeps with 12 iterations, the library's default). Its training data
are timings the method itself produces: every tile is drawn on the GPU,
segmented with each schedule and with the plain one (CUDA events on the
launch stream, median of `reps` runs), and checked to give the same labels
and distances under all four; the label is the fastest of the three.
Training runs the library's own kernels: the tensor-core forward and
backward (tcgen05, bf16 operands, fp32 accumulation), AdamW and the input
normalisation; torch only holds the buffers. The picks (evaluation and the
segmentation chain) come from the fp32 forward.

The robustness study (the paper's PATS evaluation perturbs the speedup
estimates its scheduler relies on, Section 5.5) adds Gaussian noise of
sigma feature standard deviations to the held-out features and reports,
with and without the confidence fall-back to the plain schedule, what the
picks cost against the plain schedule.

    python -m paper_1405_7958_gb300.picker --train 20000 --eval 512 \
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

SCHEDULES = rt.PICKER_CLASSES            # class c runs SCHEDULES[c] = (variant, max_local)
PLAIN_SCHEDULE = (rt.RT_RASTER, 12)      # the fixed schedule without the picker
TIMED = SCHEDULES + (PLAIN_SCHEDULE,)    # times[:, c]: class c, then the plain schedule
NAMES = tuple(f"raster/{m}" if v == rt.RT_RASTER else f"{v}/{m}" for v, m in SCHEDULES)
PLAIN = len(SCHEDULES)                   # the fall-back class: the plain schedule's column


def tile_specs(n: int, seed: int, lo: int = 1024, hi: int = 4096, step: int = 256):
    """(H, W, n_shapes, tile_seed) of n tiles: sides uniform over
    {lo, lo+step, ..., hi}, nuclei density uniform in [50, 400] per Mpx."""
    import synth
    return synth.batch_sizes(n, seed, lo, hi, step)


def schedule_times(ctx, img: torch.Tensor, reps: int = 3, stream=None):
    """Median chain time (ms) of each class's schedule and of the plain
    schedule on one tile, and whether all of them produced the same labels
    and distances."""
    stream = stream or torch.cuda.current_stream()
    outs, times = [], []
    for v, m in TIMED:
        if (v, m) in TIMED[:len(times)]:           # the plain schedule is also a class: timed once
            k = TIMED.index((v, m))
            times.append(times[k])
            outs.append(outs[k])
            continue
        p = rt.SegParams(variant=v, max_local=m)
        o = rt.segment_batch([img], p, ctx=ctx, stream=stream, want_recon=False, want_filled=False)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rt.segment_batch([img], p, outputs=o, ctx=ctx, stream=stream, want_recon=False, want_filled=False)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        times.append(float(np.median(ts)))
        outs.append(o[0])
    same = all(torch.equal(outs[0]["L"], o["L"]) and torch.equal(outs[0]["D"], o["D"]) for o in outs[1:])
    return times, same


def build_dataset(n: int, seed: int, reps: int = 3, ctx=None, log_every: int = 500, cache: str | None = None):
    """Features (n x 24) and schedule times (n x 4, ms: the three classes,
    then the plain schedule) of n GPU-drawn tiles.
    With `cache`, finished rows are saved and a rerun resumes from them."""
    ctx = ctx or rt.Context()
    specs = tile_specs(n, seed)
    feats = np.zeros((n, 24), np.float32)
    times = np.zeros((n, len(TIMED)), np.float64)
    start = 0
    if cache and os.path.exists(cache):
        z = np.load(cache)
        k = int(z["done"])
        if z["feats"].shape[0] == n and z["times"].shape[1] == len(TIMED):
            feats[:k], times[:k], start = z["feats"][:k], z["times"][:k], k
    # one warm-up of every schedule
    warm = rt.synth_tile(1024, 1024, 1, 40, ctx=ctx)
    schedule_times(ctx, warm, 1)
    t0 = time.time()
    for i in range(start, n):
        H, W, ns, s = specs[i]
        img = rt.synth_tile(H, W, s, ns, ctx=ctx)
        feats[i] = rt.tile_features([img], ctx=ctx).cpu().numpy()[0]
        tv, same = schedule_times(ctx, img, reps)
        if not same:
            raise RuntimeError(f"schedules disagree on tile {i} (seed {s})")
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
    """Cross-entropy on the fastest of the three classes, mini-batch AdamW,
    all on the GPU (forward and backward on the tensor cores)."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(np.ascontiguousarray(feats)).to(device)
    y = torch.from_numpy(times[:, :PLAIN].argmin(axis=1).astype(np.int32)).to(device)
    pk = rt.Picker(device=device, seed=seed)
    pk.set_norm(x)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = x.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(device)
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = x[idx].contiguous(), y[idx].contiguous()
            logits, act, _ = pk.forward(xb, with_act=True, tensor_cores=True)
            pk.backward(xb, act, logits, yb, tensor_cores=True)
            pk.step(lr=lr)
    return pk


def choose(pk: rt.Picker, feats: np.ndarray, min_prob: float = 0.0) -> np.ndarray:
    """The picker's classes for these features (class 3: fell back to the
    plain schedule), from the library's forward kernel."""
    x = torch.from_numpy(np.ascontiguousarray(feats, dtype=np.float32)).to(pk.device)
    _, _, pick = pk.forward(x, min_prob=min_prob, fallback=3)
    return pick.cpu().numpy()


def cost(times: np.ndarray, pick: np.ndarray) -> np.ndarray:
    """Per-tile time of the picks (a fall-back runs the plain schedule)."""
    cls = np.where(pick < PLAIN, pick, PLAIN)
    return times[np.arange(len(times)), cls]


def evaluate(pk: rt.Picker, feats: np.ndarray, times: np.ndarray, min_prob: float = 0.0) -> dict:
    """Selection accuracy, regret, and the summed time of the picks against
    the plain schedule for every tile and against the best class per tile
    (and the slowest of all four schedules per tile)."""
    pick = choose(pk, feats, min_prob)
    cls = times[:, :PLAIN]
    best = cls.argmin(axis=1)
    chosen = cost(times, pick)
    return {
        "tiles": int(len(times)),
        "accuracy": float((pick == best).mean()),
        "pick_counts": {NAMES[k]: int((pick == k).sum()) for k in range(len(SCHEDULES))} | {
            "fell_back": int((pick >= len(SCHEDULES)).sum())},
        "best_counts": {NAMES[k]: int((best == k).sum()) for k in range(len(SCHEDULES))},
        "regret_mean_ms": float((chosen - cls.min(axis=1)).mean()),
        "time_learned_ms": float(chosen.sum()),
        "time_plain_ms": float(times[:, PLAIN].sum()),
        "time_best_ms": float(cls.min(axis=1).sum()),
        "time_best_single_class_ms": float(cls.sum(axis=0).min()),
        "time_worst_ms": float(times.max(axis=1).sum()),
        "gain_vs_plain": float(times[:, PLAIN].sum() / chosen.sum()),
    }


def robustness(pk: rt.Picker, feats: np.ndarray, times: np.ndarray, sigmas=(0.0, 0.5, 1.0, 2.0, 4.0),
               min_probs=(0.0, 0.6, 0.8, 0.95), seed: int = 7, repeats: int = 5) -> list:
    """Estimate-error study: Gaussian noise of sigma feature standard
    deviations on the inputs (`repeats` draws), picks with and without the
    confidence fall-back; what they cost against the plain schedule (> 1:
    slower than plain) and how often the picker fell back."""
    rng = np.random.default_rng(seed)
    sd = pk.norm[24:].cpu().numpy().astype(np.float64)
    plain = times[:, PLAIN].sum()
    rows = []
    for sg in sigmas:
        draws = [feats + sg * sd * rng.standard_normal(feats.shape) for _ in range(repeats if sg > 0 else 1)]
        for mp in min_probs:
            ratios, fb = [], []
            for x in draws:
                pick = choose(pk, x.astype(np.float32), mp)
                ratios.append(float(cost(times, pick).sum() / plain))
                fb.append(float((pick >= len(SCHEDULES)).mean()))
            rows.append({"sigma": sg, "min_prob": mp, "time_vs_plain": float(np.mean(ratios)),
                         "time_vs_plain_max": float(np.max(ratios)), "fell_back": float(np.mean(fb))})
    rows.append({"bounds": {"best_vs_plain": float(times[:, :PLAIN].min(axis=1).sum() / plain),
                            "worst_vs_plain": float(times.max(axis=1).sum() / plain)}})
    return rows


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
    ap.add_argument("--train", type=int, default=20000)
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
    rep = {"schedules": [{"class": k, "variant": v, "max_local": m} for k, (v, m) in enumerate(SCHEDULES)],
           "plain_schedule": {"variant": PLAIN_SCHEDULE[0], "max_local": PLAIN_SCHEDULE[1]},
           "plain_class": PLAIN, "train": evaluate(pk, ftr, ttr), "eval": evaluate(pk, fev, tev),
           "robustness_eval": robustness(pk, fev, tev),
           "dataset_s": t1 - t0, "train_s": t2 - t1, "epochs": a.epochs, "reps": a.reps}
    np.savez(os.path.splitext(a.report)[0] + "_eval_set.npz", feats=fev, times=tev)
    save(pk, a.out)
    with open(a.report, "w") as fh:
        json.dump(rep, fh, indent=1)
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
