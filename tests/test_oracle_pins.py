"""Pins for the CPU oracle: checks against what the mathematics fixes.

The paper prints no worked example and no per-op values, so every pin here is
independent of the oracle's own code: hand-worked fixtures (tests/golden),
brute force on tiny inputs by a different characterisation (maximin paths,
nearest-background search), library routines that compute the same
definition (scipy.ndimage), closed forms and invariants. A plausible mistake
in the oracle (a dropped neighbour, a wrong border rule, an off-by-one in the
envelope) fails at least one of them.
"""
import heapq

import numpy as np
import pytest
from scipy import ndimage as ndi

import oracle
import synth
from golden.load import load

CROSS = ndi.generate_binary_structure(2, 1)
SQUARE = ndi.generate_binary_structure(2, 2)


def rand_img(rng, H, W, lo=0, hi=256):
    return rng.integers(lo, hi, size=(H, W)).astype(np.uint8)


# ------------------------------------------------------------------- Philox
def test_philox_known_answers():
    # Random123 known-answer vectors for philox4x32-10 (Salmon et al. 2011).
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = tuple(int(x) for x in synth.philox4x32_10(*ctr, *key))
        assert got == want


def test_generator_deterministic_and_shaped():
    a = synth.config2_tile(7, H=256, W=320)
    b = synth.config2_tile(7, H=256, W=320)
    assert a.shape == (256, 320) and a.dtype == np.uint8
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.config2_tile(8, H=256, W=320))
    # dark nuclei on a bright background
    assert 170 < np.median(a) < 230
    assert (a < 110).mean() > 0.01


# ------------------------------------------------------------ reconstruction
def maximin_recon(J, I, conn):
    """Brute force by a second characterisation: R(p) = max over q and over
    conn-paths q -> p of min(J(q), min of I along the path), computed as a
    widest-path search with a max-heap from every pixel at once."""
    H, W = I.shape
    best = np.minimum(J, I).astype(np.int64)
    heap = [(-int(best[r, c]), r, c) for r in range(H) for c in range(W)]
    heapq.heapify(heap)
    nb = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    if conn == 8:
        nb += [(-1, -1), (-1, 1), (1, -1), (1, 1)]
    done = np.zeros((H, W), bool)
    while heap:
        v, r, c = heapq.heappop(heap)
        v = -v
        if done[r, c] or v != best[r, c]:
            continue
        done[r, c] = True
        for dr, dc in nb:
            rr, cc = r + dr, c + dc
            if 0 <= rr < H and 0 <= cc < W:
                cand = min(v, int(I[rr, cc]))
                if cand > best[rr, cc]:
                    best[rr, cc] = cand
                    heapq.heappush(heap, (-cand, rr, cc))
    return best.astype(np.uint8)


def scipy_recon(J, I, conn):
    """Iterated 3x3 grey dilation clipped by the mask, to a fixed point."""
    fp = SQUARE if conn == 8 else CROSS
    R = np.minimum(J, I)
    while True:
        nxt = np.minimum(ndi.grey_dilation(R, footprint=fp, mode="constant", cval=0), I)
        if np.array_equal(nxt, R):
            return R
        R = nxt


@pytest.mark.parametrize("conn", [4, 8])
def test_recon_fixpoint_vs_maximin_bruteforce(conn):
    rng = np.random.default_rng(11)
    for _ in range(60):
        H, W = rng.integers(1, 9, size=2)
        I = rand_img(rng, H, W)
        J = rand_img(rng, H, W)   # marker may exceed mask: clamped by min(J, I)
        want = maximin_recon(J, I, conn)
        assert np.array_equal(oracle.recon_fixpoint(J, I, conn), want)
        assert np.array_equal(oracle.recon(J, I, conn), want)


@pytest.mark.parametrize("conn", [4, 8])
def test_recon_vs_scipy_grey_dilation(conn):
    rng = np.random.default_rng(3)
    for H, W in [(64, 64), (37, 91), (1, 50), (50, 1)]:
        I = rand_img(rng, H, W)
        J = (I.astype(np.int32) - rng.integers(0, 60, size=(H, W))).clip(0, 255).astype(np.uint8)
        want = scipy_recon(J, I, conn)
        assert np.array_equal(oracle.recon_fixpoint(J, I, conn), want)
        assert np.array_equal(oracle.recon(J, I, conn), want)


def test_recon_config1_three_ways():
    I = synth.config1_image()
    J = oracle.marker(I)
    Rv = oracle.recon(J, I)
    assert np.array_equal(Rv, oracle.recon_fixpoint(J, I))
    assert np.array_equal(Rv, scipy_recon(J, I, 8))


def test_recon_golden():
    g = load("recon_1d.txt")
    for conn in (4, 8):
        assert np.array_equal(oracle.recon(g["J"].astype(np.uint8), g["I"].astype(np.uint8), conn), g["R"])
        assert np.array_equal(oracle.recon_fixpoint(g["J"].astype(np.uint8), g["I"].astype(np.uint8), conn),
                              g["R"])
    g = load("recon_diag.txt")
    for conn, key in ((8, "R8"), (4, "R4")):
        for f in (oracle.recon, oracle.recon_fixpoint):
            assert np.array_equal(f(g["J"].astype(np.uint8), g["I"].astype(np.uint8), conn), g[key])


@pytest.mark.parametrize("conn", [4, 8])
def test_recon_binary_equals_binary_propagation(conn):
    """On {0,1} images reconstruction is binary propagation of the marker
    inside the mask (scipy.ndimage.binary_propagation)."""
    rng = np.random.default_rng(5)
    for seed in range(5):
        mask = synth.random_binary(48, 40, seed, 600)
        mark = (synth.random_binary(48, 40, seed + 100, 30) & mask)
        want = ndi.binary_propagation(mark.astype(bool), structure=SQUARE if conn == 8 else CROSS,
                                      mask=mask.astype(bool)).astype(np.uint8)
        assert np.array_equal(oracle.recon(mark, mask, conn), want)
        assert np.array_equal(oracle.recon_fixpoint(mark, mask, conn), want)


def test_recon_invariants_and_adversarial():
    rng = np.random.default_rng(9)
    imgs = [synth.spiral(31), synth.serpentine(24, 33), synth.checkerboard(17, 19, 0, 200),
            synth.config2_tile(4, H=96, W=128), np.zeros((5, 7), np.uint8), np.full((6, 4), 255, np.uint8)]
    for I in imgs:
        J = np.zeros_like(I)
        J[0, 0] = I[0, 0]
        R = oracle.recon(J, I)
        assert np.array_equal(R, oracle.recon_fixpoint(J, I))
        assert (R <= I).all() and (R >= np.minimum(J, I)).all()
        assert np.array_equal(oracle.recon(R, I), R)                       # idempotent
        assert np.array_equal(oracle.recon(I, I), I)
        assert not oracle.recon(np.zeros_like(I), I).any()
        Jh = oracle.marker(I)
        Rh = oracle.recon(Jh, I)
        assert (Rh.astype(int) >= I.astype(int) - 30).all() and (Rh <= I).all()
    # the spiral forces propagation along its whole corridor
    S = synth.spiral(31, low=0)
    J = np.zeros_like(S)
    J[0, 0] = 250
    assert np.array_equal(oracle.recon(J, S), S)
    J[0, 0] = 100
    assert np.array_equal(oracle.recon(J, S), np.where(S == 250, 100, 0).astype(np.uint8))
    _, iters = oracle.recon_fixpoint(J, S, 8, return_iters=True)
    assert iters > 200    # the corridor is long: the definition needs many steps


def test_marker_definition():
    I = np.arange(35, dtype=np.uint8).reshape(5, 7) * 7
    J = oracle.marker(I, 30)
    inner = I[1:-1, 1:-1].astype(int) - 30
    assert np.array_equal(J[1:-1, 1:-1], np.maximum(inner, 0))
    assert np.array_equal(J[0], I[0]) and np.array_equal(J[-1], I[-1])
    assert np.array_equal(J[:, 0], I[:, 0]) and np.array_equal(J[:, -1], I[:, -1])


# ---------------------------------------------------------------- fill holes
def test_fill_golden():
    g = load("fill_ring_gap.txt")
    B = g["B"].astype(np.uint8)
    assert np.array_equal(oracle.fill_holes(B, 4), g["F4"])
    assert np.array_equal(oracle.fill_holes(B, 8), g["F8"])


@pytest.mark.parametrize("conn", [4, 8])
def test_fill_vs_scipy(conn):
    for seed in range(8):
        B = synth.random_binary(41 + seed, 57, seed, 450 + 20 * seed)
        want = ndi.binary_fill_holes(B.astype(bool), structure=CROSS if conn == 4 else SQUARE)
        F = oracle.fill_holes(B, conn)
        assert np.array_equal(F, want.astype(np.uint8))
        assert (F >= B).all()
        assert np.array_equal(oracle.fill_holes(F, conn), F)


def test_fill_on_chain_tile_vs_scipy():
    I = synth.config2_tile(21, H=256, W=256)
    B = oracle.threshold_below(oracle.recon(oracle.marker(I), I), 80)
    want = ndi.binary_fill_holes(B.astype(bool), structure=CROSS)
    assert np.array_equal(oracle.fill_holes(B, 4), want.astype(np.uint8))


# ------------------------------------------------------------------ labeling
def scipy_labels(F, conn, amin, amax):
    lab, n = ndi.label(F != 0, structure=SQUARE if conn == 8 else CROSS)
    out = np.full(F.shape, -1, np.int64)
    if n == 0:
        return out
    idx = np.arange(F.size).reshape(F.shape)
    first = np.full(n + 1, np.iinfo(np.int64).max)
    np.minimum.at(first, lab.ravel(), idx.ravel())
    area = np.bincount(lab.ravel(), minlength=n + 1)
    keep = (area >= amin) & (area <= amax)
    keep[0] = False
    m = keep[lab]
    out[m] = first[lab[m]]
    return out


def test_label_golden():
    g = load("label_area.txt")
    F = g["F"].astype(np.uint8)
    L, n = oracle.label_area(F, g["min_area"], g["max_area"], return_count=True)
    assert np.array_equal(L, g["L"]) and n == 1
    assert np.array_equal(oracle.label_area(F, 0, 10 ** 9), g["Lall"])


@pytest.mark.parametrize("conn", [4, 8])
def test_label_vs_scipy(conn):
    for seed in range(8):
        F = synth.random_binary(33 + 3 * seed, 45, seed, 300 + 40 * seed)
        for amin, amax in ((0, 10 ** 9), (3, 12), (20, 1000)):
            L = oracle.label_area(F, amin, amax, conn)
            assert np.array_equal(L, scipy_labels(F, conn, amin, amax))


def test_label_invariants():
    F = synth.checkerboard(9, 11)
    L = oracle.label_area(F, 0, 10 ** 9)
    assert set(np.unique(L)) == {-1, 0}           # one 8-connected component
    L4 = oracle.label_area(F, 0, 10 ** 9, conn=4)
    assert (L4[F == 1] == np.flatnonzero(F.ravel() == 1)).all()   # all singletons
    F = synth.random_binary(64, 64, 3, 550)
    L = oracle.label_area(F, 0, 10 ** 9)
    fl = L.ravel()
    idx = np.arange(fl.size)
    fgm = fl >= 0
    assert (fl[fgm] <= idx[fgm]).all()
    assert (fl[fl[fgm]] == fl[fgm]).all()
    assert fgm.sum() == (F != 0).sum()


# ----------------------------------------------------------------------- EDT
def test_edt_golden():
    g = load("edt_small.txt")
    fg = g["fg"].astype(np.uint8)
    assert np.array_equal(oracle.edt(fg), g["D"])
    assert np.array_equal(oracle.edt_brute(fg), g["D"])


def test_edt_vs_bruteforce_tiny():
    rng = np.random.default_rng(17)
    for _ in range(80):
        H, W = rng.integers(1, 12, size=2)
        fg = (rng.random((H, W)) < rng.random()).astype(np.uint8)
        want = oracle.edt_brute(fg)
        assert np.array_equal(oracle.edt(fg), want)
        for _ in range(3):
            r, c = rng.integers(0, H), rng.integers(0, W)
            assert oracle.edt_at(fg, r, c) == want[r, c]


def scipy_edt_sq(fg):
    d, ind = ndi.distance_transform_edt(fg != 0, return_indices=True)
    r, c = np.indices(fg.shape)
    return (ind[0] - r) ** 2 + (ind[1] - c) ** 2


def test_edt_vs_scipy():
    for seed in range(6):
        fg = synth.random_binary(70 + seed, 90, seed, 900 + 15 * seed)
        assert np.array_equal(oracle.edt(fg), scipy_edt_sq(fg))
    I = synth.config2_tile(5, H=300, W=260)
    out = oracle.chain(I)
    fg = (out["L"] >= 0).astype(np.uint8)
    assert np.array_equal(out["D"], scipy_edt_sq(fg))


def test_edt_closed_forms():
    H, W = 23, 31
    for r0, c0 in ((0, 0), (11, 17), (22, 30)):
        fg = np.ones((H, W), np.uint8)
        fg[r0, c0] = 0
        r, c = np.indices((H, W))
        assert np.array_equal(oracle.edt(fg), (r - r0) ** 2 + (c - c0) ** 2)
    assert (oracle.edt(np.ones((4, 5), np.uint8)) == -1).all()      # no background
    assert (oracle.edt(np.zeros((4, 5), np.uint8)) == 0).all()
    fg = synth.random_binary(40, 40, 1, 950)
    D = oracle.edt(fg)
    squares = {a * a + b * b for a in range(41) for b in range(41)}
    assert set(np.unique(D)) <= squares
    assert (D[fg == 0] == 0).all() and (D[fg != 0] > 0).all()


# --------------------------------------------------------------------- chain
def test_chain_is_composition():
    I = synth.config2_tile(2, H=200, W=240)
    out = oracle.chain(I)
    R = oracle.recon(oracle.marker(I, 30), I, 8)
    F = oracle.fill_holes(oracle.threshold_below(R, 80), 4)
    L = oracle.label_area(F, 20, 1000)
    D = oracle.edt((L >= 0).astype(np.uint8))
    assert np.array_equal(out["R"], R) and np.array_equal(out["F"], F)
    assert np.array_equal(out["L"], L) and np.array_equal(out["D"], D)
    assert out["n_kept"] == len(np.unique(L[L >= 0]))


def test_chain_vs_scipy_pipeline():
    I = synth.config2_tile(12, H=256, W=256)
    J = oracle.marker(I, 30)
    R = scipy_recon(J, I, 8)
    B = (R < 80)
    F = ndi.binary_fill_holes(B, structure=CROSS).astype(np.uint8)
    L = scipy_labels(F, 8, 20, 1000)
    D = scipy_edt_sq((L >= 0).astype(np.uint8))
    out = oracle.chain(I)
    assert np.array_equal(out["R"], R)
    assert np.array_equal(out["F"], F)
    assert np.array_equal(out["L"], L)
    assert np.array_equal(out["D"], D)
