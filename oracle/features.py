"""Per-tile features for the learned variant picker -- TEST INFRASTRUCTURE ONLY.

Plain numpy (fp64) definition of the 24 cheap statistics the picker reads
(the paper's PATS scheduler orders tasks by estimated speedup, Section 3.2.1;
here the estimate comes from a small network fed with these features). Only
tests/ and the benchmark's CPU legs use this module.

Features of a uint8 tile I (H x W), in order:
  0 H, 1 W, 2 ln(H*W)
  3 mean, 4 variance, 5 skewness, 6 kurtosis (not excess) of the 256-bin
    histogram (skewness and kurtosis are 0 when the variance is 0)
  7..15 lower percentiles 1, 5, 10, 25, 50, 75, 90, 95, 99: the smallest
    value v with #{I <= v} >= p/100 * H*W
  16 fraction of pixels < 80, 17 fraction < 110
  18 histogram entropy in bits
  19, 20 mean and (population) standard deviation over the 8 x 8 blocks
    (partial blocks at the right / bottom edge included) of the block's
    fraction of dark pixels (I < 80); 21 fraction of blocks whose dark
    fraction exceeds 0.1
  22 frontier estimate: on D = the 8 x 8 block maximum of I, with marker
    Jd = max(D - 30, 0) inside and Jd = D on D's border, the fraction of
    pixels p of D with max over q in {up-left, up, up-right, left} of
    min(Jd(q), D(p)) > Jd(p); 23 ln(1 + the same count)
"""
from __future__ import annotations

import numpy as np

PCTS = (1, 5, 10, 25, 50, 75, 90, 95, 99)
NFEAT = 24


def features(I: np.ndarray) -> np.ndarray:
    I = np.ascontiguousarray(I)
    if I.dtype != np.uint8 or I.ndim != 2:
        raise TypeError("expected a 2-D uint8 array")
    H, W = I.shape
    N = H * W
    f = np.zeros(NFEAT, dtype=np.float64)
    f[0], f[1], f[2] = H, W, np.log(float(N))
    hist = np.bincount(I.ravel(), minlength=256).astype(np.float64)
    v = np.arange(256, dtype=np.float64)
    p = hist / N
    mean = float((p * v).sum())
    var = float((p * (v - mean) ** 2).sum())
    f[3], f[4] = mean, var
    if var > 0:
        sd = np.sqrt(var)
        f[5] = float((p * (v - mean) ** 3).sum()) / sd ** 3
        f[6] = float((p * (v - mean) ** 4).sum()) / sd ** 4
    cdf = np.cumsum(hist)
    for k, q in enumerate(PCTS):
        f[7 + k] = float(np.argmax(cdf >= q / 100.0 * N))
    f[16] = hist[:80].sum() / N
    f[17] = hist[:110].sum() / N
    nz = p[p > 0]
    f[18] = float(-(nz * np.log2(nz)).sum())
    # 8 x 8 blocks
    bh, bw = -(-H // 8), -(-W // 8)
    pad = np.zeros((bh * 8, bw * 8), dtype=np.int64)
    pad[:H, :W] = I < 80
    cnt = np.zeros((bh * 8, bw * 8), dtype=np.int64)
    cnt[:H, :W] = 1
    dark = pad.reshape(bh, 8, bw, 8).sum(axis=(1, 3))
    npx = cnt.reshape(bh, 8, bw, 8).sum(axis=(1, 3))
    frac = dark / npx
    f[19] = float(frac.mean())
    f[20] = float(frac.std())
    f[21] = float((frac > 0.1).mean())
    # frontier on the block maximum
    mx = np.zeros((bh * 8, bw * 8), dtype=np.int64)
    mx[:H, :W] = I
    D = mx.reshape(bh, 8, bw, 8).max(axis=(1, 3))
    Jd = np.maximum(D - 30, 0)
    Jd[0, :], Jd[-1, :], Jd[:, 0], Jd[:, -1] = D[0, :], D[-1, :], D[:, 0], D[:, -1]
    count = 0
    for r in range(bh):
        for c in range(bw):
            best = -1
            for dr, dc in ((-1, -1), (-1, 0), (-1, 1), (0, -1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < bh and 0 <= cc < bw:
                    best = max(best, min(int(Jd[rr, cc]), int(D[r, c])))
            if best > Jd[r, c]:
                count += 1
    f[22] = count / float(bh * bw)
    f[23] = np.log1p(count)
    return f
