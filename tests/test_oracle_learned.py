"""Pins for the learned-picker parts of the oracle (features and network):
closed forms, hand-computable cases, finite differences, and library
cross-checks (numpy.percentile / scipy.stats)."""
import numpy as np
import pytest
from scipy import stats

from golden.load import load
from oracle import features as F
from oracle import mlp as M


def test_features_constant_image():
    I = np.full((17, 23), 90, np.uint8)
    f = F.features(I)
    assert f[0] == 17 and f[1] == 23 and np.isclose(f[2], np.log(17 * 23))
    assert f[3] == 90 and f[4] == 0 and f[5] == 0 and f[6] == 0
    assert (f[7:16] == 90).all()
    assert f[16] == 0 and f[17] == 1 and f[18] == 0
    assert f[19] == 0 and f[20] == 0 and f[21] == 0
    # block max 90, marker 60 inside: every non-border block pixel is raised
    bh, bw = 3, 3
    assert np.isclose(f[22], 1 / 9) and np.isclose(f[23], np.log1p(1))


def test_features_match_library_statistics():
    rng = np.random.default_rng(1)
    I = rng.integers(0, 256, size=(61, 77)).astype(np.uint8)
    f = F.features(I)
    x = I.ravel().astype(np.float64)
    assert np.isclose(f[3], x.mean()) and np.isclose(f[4], x.var())
    assert np.isclose(f[5], stats.skew(x)) and np.isclose(f[6], stats.kurtosis(x, fisher=False))
    for k, q in enumerate(F.PCTS):
        assert f[7 + k] == np.percentile(x, q, method="inverted_cdf")
    assert np.isclose(f[16], (x < 80).mean()) and np.isclose(f[17], (x < 110).mean())
    _, counts = np.unique(I, return_counts=True)
    assert np.isclose(f[18], stats.entropy(counts, base=2))


def test_features_blocks_by_hand():
    I = np.full((16, 9), 200, np.uint8)      # blocks: 2 x 2 (the right ones 8 x 1)
    I[0:8, 0:8] = 10                          # top-left block all dark
    I[8, 8] = 10                              # one dark pixel in the 8x1 bottom-right block
    f = F.features(I)
    fr = np.array([1.0, 0.0, 0.0, 1 / 8])
    assert np.isclose(f[19], fr.mean()) and np.isclose(f[20], fr.std()) and np.isclose(f[21], 0.5)


def test_mlp_zero_network_closed_form():
    p = np.zeros(M.NPARAM)
    norm = np.concatenate([np.zeros(24), np.ones(24)])
    x = np.random.default_rng(0).normal(size=(5, 24))
    assert np.isclose(M.loss(p, norm, x, np.array([0, 1, 2, 0, 1])), np.log(3))
    g = M.backward(p, norm, x, np.array([0, 1, 2, 0, 1]))
    w = M.unflatten(g)
    # only b3 receives gradient: mean of softmax(0) - onehot
    assert np.allclose(w["b3"], (1 / 3) - np.array([2, 2, 1]) / 5)
    assert not np.any(w["W1"]) and not np.any(w["W2"]) and not np.any(w["W3"])


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(scale=0.3, size=M.NPARAM)
    norm = np.concatenate([rng.normal(size=24), rng.uniform(0.5, 2, size=24)])
    x = rng.normal(size=(7, 24))
    y = rng.integers(0, 3, size=7)
    g = M.backward(p, norm, x, y)
    idx = rng.choice(M.NPARAM, size=60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(M.NPARAM)
        e[i] = h
        num = (M.loss(p + e, norm, x, y) - M.loss(p - e, norm, x, y)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num)


def test_bf16_decode():
    bits = np.array([0x3F80, 0xC000, 0x0000, 0x3E80], np.uint16)
    assert np.array_equal(M.bf16_bits_to_f64(bits), [1.0, -2.0, 0.0, 0.25])


def test_adamw_first_step_closed_form():
    master = np.array([1.0, -1.0])
    grad = np.array([0.5, -2.0])
    new, m, v = M.adamw(master, grad, np.zeros(2), np.zeros(2), 1, lr=0.1, wd=0.0, eps=0.0)
    # first bias-corrected step moves every parameter by lr * sign(grad)
    assert np.allclose(new, master - 0.1 * np.sign(grad))


def _frontier_image(D):
    """48 x 48 image whose 8 x 8 block maxima are D: the block's maximum sits
    at a position that varies from block to block, the rest holds D // 2."""
    bh, bw = D.shape
    I = np.zeros((8 * bh, 8 * bw), np.uint8)
    for r in range(bh):
        for c in range(bw):
            I[8 * r:8 * r + 8, 8 * c:8 * c + 8] = D[r, c] // 2
            I[8 * r + (r + c) % 8, 8 * c + (2 * r + c) % 8] = D[r, c]
    return I


def _count_with(D, offsets):
    """The frontier count of the fixture's rule with another neighbour set
    (written out here, not taken from the oracle)."""
    Jd = np.maximum(D - 30, 0)
    Jd[0, :], Jd[-1, :], Jd[:, 0], Jd[:, -1] = D[0, :], D[-1, :], D[:, 0], D[:, -1]
    n = 0
    for r in range(D.shape[0]):
        for c in range(D.shape[1]):
            vals = [min(Jd[r + dr, c + dc], D[r, c]) for dr, dc in offsets
                    if 0 <= r + dr < D.shape[0] and 0 <= c + dc < D.shape[1]]
            n += bool(vals) and max(vals) > Jd[r, c]
    return n


def test_features_frontier_golden():
    g = load("features_frontier.txt")
    D = g["D"]
    f = F.features(_frontier_image(D))
    n = g["count_causal"]
    assert np.isclose(f[22], n / D.size) and np.isclose(f[23], np.log1p(n))
    # the fixture tells the causal set from the plausible wrong ones
    anti = ((1, 1), (1, 0), (1, -1), (0, 1))
    all8 = tuple((dr, dc) for dr in (-1, 0, 1) for dc in (-1, 0, 1) if (dr, dc) != (0, 0))
    assert _count_with(D, anti) == g["count_anticausal"] != n
    assert _count_with(D, all8) == g["count_all8"] != n
