"""Seeded synthetic microscopy tiles: the inputs shared by the oracle and the GPU path.

This module only draws inputs. It holds none of the segmentation arithmetic
(no marker, reconstruction, threshold, fill, labeling or distance transform),
so the oracle and the CUDA path can both consume its images without sharing
any of the method's code.

The paper evaluates on 4K x 4K tiles cut from brain-tumour whole-slide images
(Section 5, "Experimental Results"). That dataset is not available, so these
tiles stand in for it: dark, roughly elliptical nuclei on a bright, slowly
varying background with additive noise, at the paper's 4K x 4K tile size.

Every random draw comes from the counter-based generator Philox4x32-10
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC 2011), and all geometry is integer arithmetic. The image is therefore a
pure function of (H, W, seed, parameters), reproducible bit for bit on any
machine and by any implementation of the same definition.

Definition of one tile (all integer):

* key = (seed mod 2^32, seed div 2^32); stream s in counter word 3.
* Background, stream 1 ("Perlin-like" lattice noise): three octaves with cell
  sizes 512, 256, 128 px and weights 4, 2, 1. Octave lattice node (i, j)
  takes value ``(x0 >> 21) - 1024`` in [-1024, 1023], from counter
  (i, j, octave, 1). Bilinear interpolation on integer weights; the three
  octaves are combined at a common scale of 1/512^2 and mapped to
  ``200 + round(15 * t / (7 * 1024))`` where t is the weighted sum, so the
  background spans 200 +- 15. ``background="flat"`` gives a constant 200.
* Shapes, stream 0: shape k draws counter (k, 0, 0, 0) and (k, 1, 0, 0).
  Centres are in 1/16 px, uniform over the tile. Ellipses have semi-axes
  a, b uniform in [4, 14] px (1/16 px steps) and an orientation given by an
  integer direction (u, v) uniform in [-64, 64]^2; pixel centre (r, c) is
  inside iff ``(u dx + v dy)^2 b^2 + (-v dx + u dy)^2 a^2 <= a^2 b^2 (u^2+v^2)``
  with dx, dy the offsets in 1/16 px. Disks have radius in [rmin, rmax] px.
  Intensities are uniform integers in [vlo, vhi]. Overlaps keep the darker
  value (minimum), so the drawing order does not matter.
* Noise, stream 2: pixel p = r*W + c reads counter (p >> 1, 0, 0, 2) and uses
  words (x0, x1) if p is even, (x2, x3) if odd. The noise is a sum of twelve
  3-bit fields minus 42 (Irwin-Hall, standard deviation 7.94 ~ sigma 8):
  ten fields from the first word, two from the low 6 bits of the second.
* Pixel value = clip(min(background, shapes) + noise, 0, 255) as uint8.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x32_10", "tile", "config1_image", "config2_tile", "batch_sizes",
    "batch_tiles", "serpentine", "spiral", "checkerboard", "random_binary",
]

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, key0: int, key1: int):
    """Philox4x32 with 10 rounds, vectorised over counter arrays.

    Returns four uint32 arrays. Each round multiplies words 0 and 2 by the
    two Philox constants (64-bit products split into hi/lo), mixes the highs
    with words 1, 3 and the key, and the key is bumped by the Weyl constants
    between rounds.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(key0) & 0xFFFFFFFF
    k1 = int(key1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def _key(seed: int):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def _umul(x: np.ndarray, n: int) -> np.ndarray:
    """Uniform integer in [0, n) from a uint32 by a 32x32 -> high-word multiply."""
    return ((x.astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def _background(H: int, W: int, key, flat: bool) -> np.ndarray:
    if flat:
        return np.full((H, W), 200, dtype=np.int64)
    total = np.zeros((H, W), dtype=np.int64)
    for octave, (cell, weight) in enumerate(((512, 4), (256, 2), (128, 1))):
        ny = H // cell + 2
        nx = W // cell + 2
        ii, jj = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        x0, _, _, _ = philox4x32_10(ii, jj, octave, 1, *key)
        lat = (x0.astype(np.int64) >> 21) - 1024           # [-1024, 1023]
        r = np.arange(H)
        c = np.arange(W)
        i0, ty = r // cell, r % cell
        j0, tx = c // cell, c % cell
        # interpolate along x on every lattice row, then along y (exact ints,
        # scaled by cell per axis)
        rows = lat[:, j0] * (cell - tx)[None, :] + lat[:, j0 + 1] * tx[None, :]
        val = rows[i0, :] * (cell - ty)[:, None] + rows[i0 + 1, :] * ty[:, None]
        scale = (512 // cell) ** 2                            # to units of 1/512^2
        total += weight * scale * val
    den = 7 * 1024 * 512 * 512
    num = 15 * total
    # round half away from zero, integer only
    q = np.where(num >= 0, (num + den // 2) // den, -((-num + den // 2) // den))
    return 200 + q


def _shapes(H: int, W: int, n: int, key, kind: str, vlo: int, vhi: int,
            rmin: int, rmax: int, amin: int, amax: int):
    """Draw n shapes; returns a list of (cy16, cx16, params..., value)."""
    if n == 0:
        return []
    k = np.arange(n)
    a0, a1, a2, a3 = philox4x32_10(k, 0, 0, 0, *key)
    b0, b1, b2, b3 = philox4x32_10(k, 1, 0, 0, *key)
    cy = _umul(a0, H * 16)
    cx = _umul(a1, W * 16)
    val = vlo + _umul(a2, vhi - vlo + 1)
    out = []
    if kind == "disk":
        rad = rmin * 16 + _umul(a3, (rmax - rmin) * 16 + 1)
        for i in range(n):
            out.append((int(cy[i]), int(cx[i]), int(rad[i]), int(val[i])))
    else:
        sa = amin * 16 + _umul(a3, (amax - amin) * 16 + 1)
        sb = amin * 16 + _umul(b0, (amax - amin) * 16 + 1)
        u = _umul(b1, 129) - 64
        v = _umul(b2, 129) - 64
        for i in range(n):
            uu, vv = int(u[i]), int(v[i])
            if uu == 0 and vv == 0:
                uu = 1
            out.append((int(cy[i]), int(cx[i]), int(sa[i]), int(sb[i]), uu, vv, int(val[i])))
    return out


def _render(H: int, W: int, shapes, kind: str) -> np.ndarray:
    """Minimum over covering shapes; 255 where none covers."""
    layer = np.full((H, W), 255, dtype=np.int64)
    for s in shapes:
        cy, cx = s[0], s[1]
        reach = (s[2] if kind == "disk" else max(s[2], s[3])) // 16 + 2
        r0 = max(0, cy // 16 - reach)
        r1 = min(H, cy // 16 + reach + 1)
        c0 = max(0, cx // 16 - reach)
        c1 = min(W, cx // 16 + reach + 1)
        if r0 >= r1 or c0 >= c1:
            continue
        dy = (np.arange(r0, r1, dtype=np.int64) * 16 - cy)[:, None]
        dx = (np.arange(c0, c1, dtype=np.int64) * 16 - cx)[None, :]
        if kind == "disk":
            inside = dx * dx + dy * dy <= s[2] * s[2]
        else:
            a, b, u, v = s[2], s[3], s[4], s[5]
            p = u * dx + v * dy
            q = -v * dx + u * dy
            inside = p * p * (b * b) + q * q * (a * a) <= (a * a) * (b * b) * (u * u + v * v)
        sub = layer[r0:r1, c0:c1]
        np.minimum(sub, np.where(inside, s[-1], 255), out=sub)
    return layer


def _noise(H: int, W: int, key) -> np.ndarray:
    out = np.empty(H * W, dtype=np.int64)
    n_blk = (H * W + 1) // 2
    # chunk to bound temporary memory on large tiles
    step = 1 << 21
    for s0 in range(0, n_blk, step):
        blk = np.arange(s0, min(n_blk, s0 + step), dtype=np.uint64)
        x0, x1, x2, x3 = philox4x32_10(blk, 0, 0, 2, *key)
        pair = []
        for lo, hi in ((x0, x1), (x2, x3)):
            acc = np.zeros(blk.shape, dtype=np.int64)
            lo = lo.astype(np.int64)
            hi = hi.astype(np.int64)
            for f in range(10):
                acc += (lo >> (3 * f)) & 7
            acc += hi & 7
            acc += (hi >> 3) & 7
            pair.append(acc - 42)
        even = 2 * s0
        n_here = min(H * W, 2 * (s0 + blk.size)) - even
        inter = np.empty(2 * blk.size, dtype=np.int64)
        inter[0::2] = pair[0]
        inter[1::2] = pair[1]
        out[even:even + n_here] = inter[:n_here]
    return out.reshape(H, W)


def tile(H: int, W: int, seed: int, n_shapes: int, *, kind: str = "ellipse",
         vlo: int = 30, vhi: int = 100, rmin: int = 4, rmax: int = 12,
         amin: int = 4, amax: int = 14, background: str = "perlin",
         noise: bool = True) -> np.ndarray:
    """One synthetic tile as a C-contiguous uint8 array of shape (H, W)."""
    if H < 1 or W < 1:
        raise ValueError("H and W must be >= 1")
    key = _key(seed)
    img = _background(H, W, key, background == "flat")
    shapes = _shapes(H, W, n_shapes, key, kind, vlo, vhi, rmin, rmax, amin, amax)
    np.minimum(img, _render(H, W, shapes, kind), out=img)
    if noise:
        img += _noise(H, W, key)
    return np.ascontiguousarray(np.clip(img, 0, 255).astype(np.uint8))


def config1_image(seed: int = 1000) -> np.ndarray:
    """512 x 512 mask image: flat 200 background, 60 dark disks (values 40..90,
    radii 4..12 px), noise sigma ~8."""
    return tile(512, 512, seed, 60, kind="disk", vlo=40, vhi=90, rmin=4, rmax=12,
                background="flat")


def config2_tile(seed: int = 2000, H: int = 4096, W: int = 4096, n_shapes: int | None = None) -> np.ndarray:
    """4K x 4K nuclei tile: ~3000 ellipses (semi-axes 4..14 px, values
    30..100) on a 200 +- 15 lattice-noise background, noise sigma ~8. Smaller
    H, W keep the nuclei density (3000 per 4096^2)."""
    if n_shapes is None:
        n_shapes = int(round(3000 * H * W / (4096 * 4096)))
    return tile(H, W, seed, n_shapes, kind="ellipse", vlo=30, vhi=100)


def batch_sizes(n: int, seed: int, lo: int = 1024, hi: int = 4096, step: int = 256,
                square: bool = False):
    """Side lengths for a batch of uneven tiles: H, W uniform over
    {lo, lo+step, ..., hi} (independently unless square) and a nuclei
    density uniform in [50, 400] per megapixel; returns a list of
    (H, W, n_shapes, tile_seed)."""
    key = _key(seed)
    k = np.arange(n)
    x0, x1, x2, _ = philox4x32_10(k, 0, 0, 7, *key)
    n_sides = (hi - lo) // step + 1
    hs = lo + step * _umul(x0, n_sides)
    ws = hs if square else lo + step * _umul(x1, n_sides)
    dens = 50 + _umul(x2, 351)
    out = []
    for i in range(n):
        H, W = int(hs[i]), int(ws[i])
        out.append((H, W, int(round(int(dens[i]) * H * W / 1e6)), seed * 1000 + i))
    return out


def batch_tiles(n: int, seed: int, **kw):
    """Tiles for batch_sizes(n, seed, **kw)."""
    return [tile(H, W, s, ns) for (H, W, ns, s) in batch_sizes(n, seed, **kw)]


# ----------------------------------------------------------------- adversarial
def serpentine(H: int, W: int, wall: int = 1, gap: int = 1, low: int = 10, high: int = 250) -> np.ndarray:
    """A maze of horizontal corridors joined at alternating ends: the longest
    possible geodesic path for a given size (value `high` on the corridor,
    `low` on the walls)."""
    img = np.full((H, W), low, dtype=np.uint8)
    period = wall + gap
    flip = False
    r = 0
    while r < H:
        img[r:r + gap, :] = high
        wr = r + gap
        if wr < H:
            if flip:
                img[wr:wr + wall, 0] = high
            else:
                img[wr:wr + wall, W - 1] = high
        flip = not flip
        r += period
    return img


def spiral(n: int, low: int = 10, high: int = 250) -> np.ndarray:
    """A square spiral corridor, 1 px wide with 1 px walls, inside an n x n
    image: information entering at (0, 0) must travel its whole length."""
    img = np.full((n, n), low, dtype=np.uint8)
    r = c = 0
    img[0, 0] = high
    steps = ((0, 1), (1, 0), (0, -1), (-1, 0))
    d = 0
    turns = 0

    def free(y, x):
        return 0 <= y < n and 0 <= x < n and img[y, x] == low

    while turns < 2:
        dr, dc = steps[d]
        ny, nx = r + dr, c + dc
        fy, fx = r + 2 * dr, c + 2 * dc
        far_ok = not (0 <= fy < n and 0 <= fx < n) or img[fy, fx] == low
        if free(ny, nx) and far_ok:
            r, c = ny, nx
            img[r, c] = high
            turns = 0
        else:
            d = (d + 1) % 4
            turns += 1
    return img


def checkerboard(H: int, W: int, lo: int = 0, hi: int = 1) -> np.ndarray:
    r, c = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.where((r + c) % 2 == 0, hi, lo).astype(np.uint8)


def random_binary(H: int, W: int, seed: int, p_permille: int = 500) -> np.ndarray:
    """Binary image with P(pixel = 1) = p_permille / 1000."""
    key = _key(seed)
    idx = np.arange(H * W, dtype=np.uint64)
    x0, _, _, _ = philox4x32_10(idx, 0, 0, 3, *key)
    return (_umul(x0, 1000) < p_permille).astype(np.uint8).reshape(H, W)
