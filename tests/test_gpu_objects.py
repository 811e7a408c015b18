"""GPU parity of the per-object steps after the labels (the watershed after
Pre-Watershed and the feature computation stage, Section 5.1) against the
CPU oracle: hand-worked fixtures, the chain's own labels and distances on
ragged tiles and a full 4096 x 4096 tile, objects whose bounding box is too
large for shared memory (the global-memory path), degenerate inputs.
Labels, basins and integer-valued features are compared exactly; the other
features within 1e-12 relative (the same double-precision steps on both
sides; only the logarithm of the entropy may round differently)."""
import numpy as np
import pytest

import oracle
import synth
from golden.load import load

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL = 1e-12


@pytest.fixture(scope="module")
def rt():
    import paper_1405_7958_gb300 as rt
    return rt


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def check_features(rt, L, I, cap=None):
    want_lab, want = oracle.object_features(L, I)
    n = len(want_lab)
    cap = n if cap is None else cap
    n_obj = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    lab, f = rt.object_features(dev(L), dev(I), cap, n_obj=n_obj, status=st)
    assert int(host(st)[0]) == 0 and int(host(n_obj)[0]) == n
    k = min(cap, n)
    got_lab, got = host(lab)[:k], host(f)[:k]
    assert np.array_equal(got_lab, want_lab[:k])
    ints = list(oracle.INTEGER_FEATURES)
    assert np.array_equal(got[:, ints], want[:k, ints])
    assert np.allclose(got, want[:k], rtol=RTOL, atol=RTOL)
    return got


def check_watershed(rt, L, D, h):
    want, nb = oracle.watershed(L, D, h, return_count=True)
    n_b = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    out = torch.full(L.shape, -7, dtype=torch.int32, device="cuda")
    rt.watershed(dev(L), dev(D), h, out=out, n_basins=n_b, status=st)
    assert int(host(st)[0]) == 0
    assert np.array_equal(host(out), want)
    assert int(host(n_b)[0]) == nb
    return want


def test_features_golden(rt):
    g = load("objects_small.txt")
    r, c = np.mgrid[0:5, 0:7]
    check_features(rt, g["L"].astype(np.int32), (7 * (7 * r + c)).astype(np.uint8))


def test_watershed_golden(rt):
    g = load("watershed_dumbbell.txt")
    for h in (0, 1):
        assert np.array_equal(check_watershed(rt, g["L"].astype(np.int32), g["D"].astype(np.int32), h), g[f"B_h{h}"])


@pytest.mark.parametrize("shape", [(700, 900), (333, 1031), (64, 64), (1, 500)])
def test_objects_on_chain_outputs(rt, shape):
    H, W = shape
    I = synth.config2_tile(40 + H, H=H, W=W)
    c = oracle.chain(I)
    check_features(rt, c["L"], I)
    for h in (0, 2, 8):
        check_watershed(rt, c["L"], c["D"], h)


def test_objects_full_4k_tile(rt):
    I = synth.config2_tile(2000)
    c = oracle.chain(I)
    got = check_features(rt, c["L"], I)
    assert len(got) == c["n_kept"]
    check_watershed(rt, c["L"], c["D"], 2)


def test_large_boxes_take_the_global_path(rt):
    """Objects whose bounding box exceeds the shared-memory box (4096
    pixels): a 150 x 120 ellipse pair, a diagonal line across 900 x 900 and a
    ring, next to small disks; both paths in one launch."""
    H, W = 1000, 1400
    rr, cc = np.mgrid[0:H, 0:W]
    m = np.zeros((H, W), bool)
    m |= ((rr - 150) / 70.0) ** 2 + ((cc - 200) / 55.0) ** 2 <= 1
    m |= ((rr - 150) / 70.0) ** 2 + ((cc - 290) / 55.0) ** 2 <= 1
    d = np.arange(50, 950)
    m[d, d + 380] = True
    m[d[:-1], d[:-1] + 381] = True
    m |= np.abs(np.hypot(rr - 700, cc - 300) - 120) <= 3
    for k in range(12):
        m |= (rr - 400 - 40 * (k % 3)) ** 2 + (cc - 1100 - 40 * (k // 3)) ** 2 <= 64
    L = oracle.label_area(m.astype(np.uint8), 1, 10 ** 9)
    D = oracle.edt((L >= 0).astype(np.uint8))
    I = synth.config2_tile(77, H=H, W=W)
    f = check_features(rt, L, I)
    assert (f[:, 2] * f[:, 3]).max() > 4096
    for h in (0, 3):
        check_watershed(rt, L, D, h)


def test_objects_degenerate_inputs(rt):
    empty = np.full((40, 50), -1, np.int32)
    assert len(check_features(rt, empty, np.zeros((40, 50), np.uint8))) == 0
    check_watershed(rt, empty, np.zeros((40, 50), np.int32), 2)
    # one object covering the image; single pixels at the corners
    full = np.zeros((33, 65), np.int32)
    check_features(rt, full, synth.config2_tile(3, H=33, W=65))
    check_watershed(rt, full, oracle.edt(np.pad(np.ones((31, 63), np.uint8), 1)), 1)
    dots = np.full((9, 10), -1, np.int32)
    for r, c in ((0, 0), (0, 9), (8, 0), (8, 9), (4, 5)):
        dots[r, c] = r * 10 + c
    check_features(rt, dots, synth.config2_tile(4, H=9, W=10))
    check_watershed(rt, dots, np.where(dots >= 0, 1, 0).astype(np.int32), 0)


def test_features_cap_and_strides(rt):
    I = synth.config2_tile(12, H=500, W=600)
    c = oracle.chain(I)
    n = c["n_kept"]
    assert n > 10
    check_features(rt, c["L"], I, cap=7)
    # strided label and image views
    Lb = torch.full((500, 613), 123, dtype=torch.int32, device="cuda")
    Lb[:, :600] = dev(c["L"])
    Ib = torch.zeros((500, 640), dtype=torch.uint8, device="cuda")
    Ib[:, :600] = dev(I)
    lab, f = rt.object_features(Lb[:, :600], Ib[:, :600], n)
    want_lab, want = oracle.object_features(c["L"], I)
    assert np.array_equal(host(lab), want_lab) and np.allclose(host(f), want, rtol=RTOL, atol=RTOL)


def test_non_canonical_labels_are_reported(rt):
    L = np.full((20, 20), -1, np.int32)
    L[5:8, 5:8] = 3            # 3 is not the index of a pixel of this object
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rt.object_features(dev(L), dev(np.zeros((20, 20), np.uint8)), 4, status=st)
    assert int(host(st)[0]) == rt.RT_EINVAL
