"""Pins of the per-object oracles (the feature computation stage and the
watershed after Pre-Watershed, Section 5.1) against values fixed outside
them: hand-worked fixtures, scipy.ndimage and numpy statistics of each
object, closed forms (rectangles, a lone pixel, one basin per object when h
exceeds every distance), and properties every watershed has (each basin is
connected and holds exactly one marker)."""
import numpy as np
import pytest
from scipy import ndimage, stats

import oracle
import synth
from golden.load import load

F = {n: i for i, n in enumerate(oracle.FEATURE_NAMES)}


def test_object_features_golden():
    g = load("objects_small.txt")
    L = g["L"].astype(np.int32)
    r, c = np.mgrid[0:5, 0:7]
    I = (7 * (7 * r + c)).astype(np.uint8)
    labels, f = oracle.object_features(L, I)
    assert labels.tolist() == [int(x) for x in g["objects"][:, 0]]
    for row, (lab, area, per, bh, bw, cr2, cc2, vrr36, vcc36, vrc36, s, vmin, vmax, med, nd, n2, con, en, hom2) in \
            zip(f, g["objects"]):
        assert row[F["area"]] == area and row[F["perimeter"]] == per
        assert row[F["bbox_h"]] == bh and row[F["bbox_w"]] == bw
        assert row[F["centroid_r"]] == cr2 / 2 and row[F["centroid_c"]] == cc2 / 2
        lam = np.linalg.eigvalsh(np.array([[vrr36, vrc36], [vrc36, vcc36]], float) / 36)
        assert np.isclose(row[F["major_axis"]], 4 * np.sqrt(lam[1]))
        assert np.isclose(row[F["minor_axis"]], 4 * np.sqrt(max(lam[0], 0)))
        ecc = np.sqrt(1 - max(lam[0], 0) / lam[1]) if lam[1] > 0 else 0.0
        assert np.isclose(row[F["eccentricity"]], ecc)
        assert np.isclose(row[F["compactness"]], 4 * np.pi * area / per ** 2)
        assert np.isclose(row[F["mean"]], s / area)
        assert row[F["min"]] == vmin and row[F["max"]] == vmax and row[F["median"]] == med
        assert np.isclose(row[F["entropy"]], np.log2(nd))      # every value once: uniform histogram
        assert row[F["glcm_pairs"]] == n2
        if n2:
            assert np.isclose(row[F["glcm_contrast"]], con / n2)
            assert np.isclose(row[F["glcm_energy"]], en / n2 ** 2)
            assert np.isclose(row[F["glcm_homogeneity"]], hom2 / 2 / n2)
        else:
            assert row[F["glcm_contrast"]] == row[F["glcm_energy"]] == row[F["glcm_homogeneity"]] == 0


def _chain_labels(seed, H, W):
    I = synth.config2_tile(seed, H=H, W=W)
    return oracle.chain(I), I


def test_object_features_match_scipy_and_numpy():
    """On the chain's kept nuclei of a 700 x 900 tile: bounding boxes, areas,
    centroids, intensity moments and extrema from scipy.ndimage; perimeter,
    covariance axes, median, entropy and co-occurrences recounted with numpy
    on each object's own mask."""
    out, I = _chain_labels(5, 700, 900)
    L = out["L"]
    labels, f = oracle.object_features(L, I)
    assert len(labels) == out["n_kept"] and np.array_equal(labels, np.unique(L[L >= 0]))
    assert f[:, F["area"]].sum() == (L >= 0).sum()
    idx = labels.tolist()
    Ii = I.astype(np.float64)
    assert np.array_equal(f[:, F["area"]], ndimage.sum(np.ones_like(Ii), L, idx))
    com = np.array(ndimage.center_of_mass(np.ones_like(Ii), L, idx))
    assert np.allclose(f[:, [F["centroid_r"], F["centroid_c"]]], com, rtol=1e-12)
    assert np.allclose(f[:, F["mean"]], ndimage.mean(Ii, L, idx), rtol=1e-12)
    assert np.allclose(f[:, F["std"]], np.sqrt(ndimage.variance(Ii, L, idx)), rtol=1e-9, atol=1e-9)
    assert np.array_equal(f[:, F["min"]], ndimage.minimum(Ii, L, idx))
    assert np.array_equal(f[:, F["max"]], ndimage.maximum(Ii, L, idx))
    lab_img, _ = ndimage.label(L >= 0, structure=np.ones((3, 3)))
    for k, lab in enumerate(idx[:60]):
        rr, cc = np.nonzero(L == lab)
        sl = (slice(rr.min(), rr.max() + 1), slice(cc.min(), cc.max() + 1))
        assert f[k, F["bbox_h"]] == rr.max() - rr.min() + 1 and f[k, F["bbox_w"]] == cc.max() - cc.min() + 1
        m = np.pad(L == lab, 1)
        per = sum(int((m & ~np.roll(m, s, axis=a)).sum()) for a in (0, 1) for s in (1, -1))
        assert f[k, F["perimeter"]] == per
        lam = np.linalg.eigvalsh(np.cov(np.stack([rr, cc]).astype(float), bias=True))
        assert np.isclose(f[k, F["major_axis"]], 4 * np.sqrt(lam[1]), rtol=1e-9)
        assert np.isclose(f[k, F["minor_axis"]], 4 * np.sqrt(max(lam[0], 0)), rtol=1e-9, atol=1e-7)
        v = np.sort(I[rr, cc])
        assert f[k, F["median"]] == v[(len(v) + 1) // 2 - 1]           # lower median
        _, counts = np.unique(v, return_counts=True)
        assert np.isclose(f[k, F["entropy"]], stats.entropy(counts, base=2))
        inn = (L[sl] == lab)
        q = (I[sl] >> 5).astype(int)
        pair = inn[:, :-1] & inn[:, 1:]
        a, b = q[:, :-1][pair], q[:, 1:][pair]
        assert f[k, F["glcm_pairs"]] == pair.sum()
        if pair.sum():
            G = np.zeros((8, 8))
            np.add.at(G, (a, b), 1)
            P = G / G.sum()
            ii, jj = np.mgrid[0:8, 0:8]
            assert np.isclose(f[k, F["glcm_contrast"]], ((ii - jj) ** 2 * P).sum())
            assert np.isclose(f[k, F["glcm_energy"]], (P ** 2).sum())
            assert np.isclose(f[k, F["glcm_homogeneity"]], (P / (1 + np.abs(ii - jj))).sum())
        assert lab_img[rr[0], cc[0]] > 0


def test_object_features_closed_forms():
    L = np.full((20, 30), -1, np.int32)
    L[2:9, 3:14] = 5          # a 7 x 11 rectangle
    L[15, 20] = 200           # a lone pixel
    I = np.full((20, 30), 40, np.uint8)
    labels, f = oracle.object_features(L, I)
    assert labels.tolist() == [5, 200]
    assert f[0, F["perimeter"]] == 2 * (7 + 11) and f[0, F["area"]] == 77
    # a rectangle's coordinate variances are (n^2 - 1) / 12 per side
    assert np.isclose(f[0, F["major_axis"]], 4 * np.sqrt((11 ** 2 - 1) / 12))
    assert np.isclose(f[0, F["minor_axis"]], 4 * np.sqrt((7 ** 2 - 1) / 12))
    assert f[0, F["std"]] == 0 and f[0, F["entropy"]] == 0 and f[0, F["glcm_contrast"]] == 0
    assert f[0, F["glcm_energy"]] == 1 and f[0, F["glcm_homogeneity"]] == 1 and f[0, F["glcm_pairs"]] == 7 * 10
    assert np.isclose(f[1, F["compactness"]], np.pi / 4) and f[1, F["eccentricity"]] == 0


def test_watershed_golden():
    g = load("watershed_dumbbell.txt")
    L, D = g["L"].astype(np.int32), g["D"].astype(np.int32)
    for h in (0, 1):
        B, n = oracle.watershed(L, D, h, return_count=True)
        assert np.array_equal(B, g[f"B_h{h}"]) and n == g[f"basins_h{h}"]


def _two_disks(H=60, W=90, r=14, sep=22):
    rr, cc = np.mgrid[0:H, 0:W]
    cy, cx = H // 2, W // 2
    m = ((rr - cy) ** 2 + (cc - (cx - sep // 2)) ** 2 <= r * r) | ((rr - cy) ** 2 + (cc - (cx + sep // 2)) ** 2 <= r * r)
    return m


def test_watershed_splits_two_touching_disks():
    m = _two_disks()
    L = np.where(m, np.argmax(m.ravel()), -1).astype(np.int32)
    D = oracle.edt(m.astype(np.uint8))
    B, n = oracle.watershed(L, D, 2, return_count=True)
    assert n == 2
    left, right = np.unique(B[m])
    H, W = m.shape
    cy, cx = H // 2, W // 2
    # the outer side of each disk (beyond its centre) is its own basin
    assert (B[:, :cx - 11][m[:, :cx - 11]] == left).all() and (B[:, cx + 12:][m[:, cx + 12:]] == right).all()
    # on the centre row the two markers are equally far from the neck's
    # centre column (a tie: the smaller label); every other pixel of the row
    # is nearer its own side
    row = B[cy][m[cy]]
    cols = np.nonzero(m[cy])[0]
    assert (row[cols <= cx] == left).all() and (row[cols > cx] == right).all()
    assert (B[m] == left).sum() > 0.4 * m.sum() and (B[m] == right).sum() > 0.4 * m.sum()


def test_watershed_properties_on_chain_objects():
    """On the chain's kept nuclei of a 700 x 900 tile, for several h: every
    object pixel gets a basin; a basin's label is the index of one of its own
    pixels, inside the same object; every basin is 8-connected; with h above
    every distance each object is one basin labelled by its own label."""
    out, I = _chain_labels(7, 700, 900)
    L, D = out["L"], out["D"]
    obj = L >= 0
    for h in (0, 2, 8):
        B, n = oracle.watershed(L, D, h, return_count=True)
        assert ((B >= 0) == obj).all()
        ids = np.unique(B[obj])
        assert len(ids) == n >= len(np.unique(L[obj]))
        flat, lf = B.ravel(), L.ravel()
        assert (flat[ids] == ids).all()                     # a basin's label is the index of one of its pixels
        for bid in ids[:200]:
            inside = B == bid
            assert (L[inside] == lf[bid]).all()             # ... and the basin lies inside that pixel's object
            assert ndimage.label(inside, structure=np.ones((3, 3)))[1] == 1   # 8-connected
    B, n = oracle.watershed(L, D, int(D.max()) + 1, return_count=True)
    assert np.array_equal(B, L) and n == len(np.unique(L[obj]))


@pytest.mark.parametrize("h", [0, 3])
def test_watershed_single_peak_is_one_basin(h):
    rr, cc = np.mgrid[0:41, 0:41]
    m = (rr - 20) ** 2 + (cc - 20) ** 2 <= 15 ** 2
    L = np.where(m, np.argmax(m.ravel()), -1).astype(np.int32)
    D = ((rr - 20) ** 2 + (cc - 20) ** 2).max() - ((rr - 20) ** 2 + (cc - 20) ** 2)   # one peak at the centre
    D = np.where(m, D, 0).astype(np.int32)
    B, n = oracle.watershed(L, D, h, return_count=True)
    # the marker is the plateau D >= max - h of the h-maxima transform; its
    # label is the plateau's first pixel in raster order
    first = int(np.argmax((m & (D >= D[m].max() - h)).ravel()))
    assert n == 1 and (B[m] == first).all()
