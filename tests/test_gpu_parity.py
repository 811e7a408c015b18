"""GPU parity: every CUDA op against the CPU oracle, bit-exact (all outputs
are integers with a unique correct value). Inputs come from the seeded
generator in synth/; expected values only from oracle/."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rt():
    import paper_1405_7958_gb300 as rt
    return rt


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def strided(a, pad=13):
    """A CUDA view of `a` whose row stride exceeds its width."""
    H, W = a.shape
    big = torch.full((H, W + pad), 77, dtype=torch.from_numpy(a[:0]).dtype, device="cuda")
    big[:, :W] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return big[:, :W]


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


SIZES = [(1, 1), (1, 300), (300, 1), (7, 5), (64, 128), (65, 129), (200, 333), (513, 257)]


# ------------------------------------------------------------ reconstruction
def test_marker_matches_oracle(rt):
    for H, W in SIZES:
        I = synth.config2_tile(3, H=H, W=W)
        assert np.array_equal(host(rt.marker(dev(I), 30)), oracle.marker(I, 30))


def test_recon_config1(rt):
    I = synth.config1_image(1000)
    want = oracle.recon(oracle.marker(I, 30), I, 8)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = host(rt.reconstruct(dev(I), None, h_offset=30, conn=8, status=st))
    assert np.array_equal(got, want)
    assert int(st.item()) == rt.RT_OK
    J = rt.marker(dev(I), 30)
    assert np.array_equal(host(rt.reconstruct(dev(I), J, conn=8)), want)


VARIANTS = ["RT_RASTER", "RT_QUEUE", "RT_HYBRID", "RT_FRONTIER"]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("conn", [4, 8])
def test_recon_random_sizes(rt, conn, variant):
    rng = np.random.default_rng(7)
    for H, W in SIZES:
        I = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
        J = np.minimum(I, rng.integers(0, 256, size=(H, W))).astype(np.uint8)
        J[rng.random((H, W)) < 0.98] = 0
        want = oracle.recon(J, I, conn)
        got = host(rt.reconstruct(dev(I), dev(J), conn=conn, variant=getattr(rt, variant)))
        assert np.array_equal(got, want), (H, W)


def test_recon_strided_and_alias(rt):
    I = synth.config2_tile(5, H=257, W=383)
    J = oracle.marker(I, 30)
    want = oracle.recon(J, I, 8)
    out = strided(np.zeros_like(I), pad=29)
    rt.reconstruct(strided(I), strided(J, pad=7), conn=8, out=out)
    assert np.array_equal(host(out), want)
    Jd = dev(J)                         # out aliases the marker
    rt.reconstruct(dev(I), Jd, conn=8, out=Jd)
    assert np.array_equal(host(Jd), want)


def test_recon_marker_above_mask_reports_and_clamps(rt):
    rng = np.random.default_rng(2)
    I = rng.integers(0, 200, size=(90, 140)).astype(np.uint8)
    J = rng.integers(0, 256, size=(90, 140)).astype(np.uint8)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = host(rt.reconstruct(dev(I), dev(J), conn=8, status=st))
    assert np.array_equal(got, oracle.recon(J, I, 8))
    assert int(st.item()) == rt.RT_EMARKER


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("conn", [4, 8])
def test_recon_adversarial(rt, conn, variant):
    cases = [synth.spiral(129, low=0), synth.serpentine(131, 200), synth.checkerboard(97, 161, 0, 200),
             np.zeros((70, 90), np.uint8), np.full((70, 90), 255, np.uint8)]
    for I in cases:
        J = np.zeros_like(I)
        J[0, 0] = I[0, 0]
        got = host(rt.reconstruct(dev(I), dev(J), conn=conn, variant=getattr(rt, variant)))
        assert np.array_equal(got, oracle.recon(J, I, conn))


@pytest.mark.parametrize("variant", VARIANTS)
def test_recon_full_4k_tile(rt, variant):
    I = synth.config2_tile(2000)
    want = oracle.recon(oracle.marker(I, 30), I, 8)
    got = host(rt.reconstruct(dev(I), None, h_offset=30, conn=8, variant=getattr(rt, variant)))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("conn", [4, 8])
def test_frontier_queue_overflow_hands_over_to_the_sweeps(rt, conn):
    """RT_FRONTIER with global queues too small for the seeds or for the
    drain's spills: the directional sweeps finish the propagation from the
    drained state, and the bytes are the oracle's. Capacity 0 restores the
    default (one entry per padded pixel)."""
    ctx = rt.Context()
    cases = [synth.config2_tile(11, H=700, W=900), synth.spiral(129, low=0),
             synth.tile(640, 832, 5, 60, background="flat")]
    for I in cases:
        J = oracle.marker(I, 30)
        want = oracle.recon(J, I, conn)
        for cap in (1, 64, 3000, 0):
            ctx.set_queue_capacity(cap)
            st = torch.zeros(1, dtype=torch.int32, device="cuda")
            got = host(rt.reconstruct(dev(I), dev(J), conn=conn, variant=rt.RT_FRONTIER, status=st, ctx=ctx))
            assert np.array_equal(got, want), (I.shape, cap)
            assert int(st.item()) == rt.RT_OK
    ctx.close()


def test_frontier_pops_follow_the_front(rt):
    """On a flat-background tile the dense first pass leaves a thin front:
    the frontier drain pops pixels (counted in the statistics), and the
    output is the oracle's."""
    ctx = rt.Context()
    I = synth.tile(1024, 1024, 3, 200, background="flat")
    want = oracle.recon(oracle.marker(I, 30), I, 8)
    got = host(rt.reconstruct(dev(I), None, h_offset=30, conn=8, variant=rt.RT_FRONTIER, ctx=ctx))
    assert np.array_equal(got, want)
    visits, iters, pops = ctx.recon_stats()
    assert pops > 0 and visits >= (1024 // 32) * (1024 // 64)
    ctx.close()


# ---------------------------------------------------------------- fill holes
@pytest.mark.parametrize("conn", [4, 8])
def test_fill_holes(rt, conn):
    for k, (H, W) in enumerate(SIZES + [(1000, 1100)]):
        B = synth.random_binary(H, W, 40 + k, 420 + 10 * k)
        assert np.array_equal(host(rt.fill_holes(dev(B), conn=conn)), oracle.fill_holes(B, conn)), (H, W)


def test_fill_holes_chain_mask_and_strides(rt):
    I = synth.config2_tile(9, H=777, W=901)
    B = oracle.threshold_below(oracle.recon(oracle.marker(I), I), 80)
    want = oracle.fill_holes(B, 4)
    out = strided(np.zeros_like(B), pad=5)
    rt.fill_holes(strided(B, pad=3), conn=4, out=out)
    assert np.array_equal(host(out), want)
    Bd = dev(B)
    rt.fill_holes(Bd, conn=4, out=Bd)   # in place
    assert np.array_equal(host(Bd), want)


# ------------------------------------------------------------------ labeling
@pytest.mark.parametrize("conn", [4, 8])
def test_label_area(rt, conn):
    for k, (H, W) in enumerate(SIZES + [(1000, 1100)]):
        F = synth.random_binary(H, W, 70 + k, 300 + 40 * (k % 8))
        for amin, amax in ((0, 2 ** 31 - 1), (3, 40), (20, 1000)):
            n = torch.zeros(1, dtype=torch.int32, device="cuda")
            got = host(rt.label_area(dev(F), amin, amax, conn=conn, n_kept=n))
            want, kept = oracle.label_area(F, amin, amax, conn, return_count=True)
            assert np.array_equal(got, want), (H, W, amin, amax)
            assert int(n.item()) == kept


def test_label_checkerboard_and_strided(rt):
    F = synth.checkerboard(100, 130)
    assert np.array_equal(host(rt.label_area(dev(F), 0, 10 ** 9)), oracle.label_area(F, 0, 10 ** 9))
    F = synth.random_binary(300, 410, 5, 550)
    out = torch.full((300, 450), 99, dtype=torch.int32, device="cuda")[:, :410]
    rt.label_area(strided(F), 20, 1000, out=out)
    assert np.array_equal(host(out), oracle.label_area(F, 20, 1000))


# ----------------------------------------------------------------------- EDT
def test_edt(rt):
    rng = np.random.default_rng(4)
    for k, (H, W) in enumerate(SIZES + [(700, 1000)]):
        for dens in (50, 500, 950, 999):
            fg = (rng.integers(0, 1000, size=(H, W)) < dens).astype(np.uint8)
            assert np.array_equal(host(rt.edt(dev(fg))), oracle.edt(fg)), (H, W, dens)


def test_edt_special_cases(rt):
    assert (host(rt.edt(dev(np.ones((37, 53), np.uint8)))) == -1).all()
    assert (host(rt.edt(dev(np.zeros((37, 53), np.uint8)))) == 0).all()
    fg = np.ones((123, 77), np.uint8)
    fg[100, 3] = 0
    r, c = np.indices(fg.shape)
    assert np.array_equal(host(rt.edt(dev(fg))), (r - 100) ** 2 + (c - 3) ** 2)
    fg = synth.random_binary(200, 250, 8, 900)
    out = torch.zeros((200, 300), dtype=torch.int32, device="cuda")[:, :250]
    rt.edt(strided(fg), out=out)
    assert np.array_equal(host(out), oracle.edt(fg))


# --------------------------------------------------------------------- chain
def check_chain(out, I):
    want = oracle.chain(I)
    if "R" in out:
        assert np.array_equal(host(out["R"]), want["R"])
    if "F" in out:
        assert np.array_equal(host(out["F"]), want["F"])
    assert np.array_equal(host(out["L"]), want["L"])
    assert np.array_equal(host(out["D"]), want["D"])
    assert int(out["n_kept"].item()) == want["n_kept"]
    assert int(out["status"].item()) == 0


def test_chain_small(rt):
    I = synth.config2_tile(11, H=512, W=512)
    check_chain(rt.segment_batch([dev(I)])[0], I)


def test_chain_edt_bit_plane_edge_cases(rt):
    """The chain's distance transform runs on the kept-pixel bit plane. Its
    degenerate inputs: every pixel kept (no background anywhere: -1), a kept
    band across the whole width (for rows inside it the nearest background
    lies several 32-row segments away, above and below), a tall kept bar,
    and nothing kept (0 everywhere); ragged sizes throughout."""
    band = np.full((300, 120), 200, np.uint8)
    band[40:251, :] = 40
    bar = np.full((300, 200), 200, np.uint8)
    bar[10:291, 50:61] = 40
    cases = [np.full((77, 101), 40, np.uint8), band, bar, np.full((45, 70), 200, np.uint8)]
    p = rt.SegParams(max_area=10 ** 9)
    got = []
    for I in cases:
        out = rt.segment_batch([dev(I)], p)[0]
        want = oracle.chain(I, max_area=10 ** 9)
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(out[k]), want[k]), (I.shape, k)
        assert int(out["n_kept"].item()) == want["n_kept"]
        assert int(out["status"].item()) == 0
        got.append(host(out["D"]))
    # closed forms
    assert (got[0] == -1).all()
    r = np.arange(300)[:, None]
    inside = (r >= 40) & (r <= 250)
    assert np.array_equal(got[1], np.broadcast_to(np.where(inside, np.minimum(r - 39, 251 - r) ** 2, 0), (300, 120)))
    assert (got[3] == 0).all()


def test_chain_batch_uneven(rt):
    shapes = [(300, 700), (1024, 256), (129, 131)]
    imgs = [synth.config2_tile(100 + i, H=H, W=W) for i, (H, W) in enumerate(shapes)]
    outs = rt.segment_batch([dev(x) for x in imgs])
    for o, I in zip(outs, imgs):
        check_chain(o, I)
    # the same tiles alone give the same bytes
    alone = rt.segment_batch([dev(imgs[1])])[0]
    assert np.array_equal(host(alone["L"]), host(outs[1]["L"]))


def test_chain_full_4k(rt):
    I = synth.config2_tile(2000)
    out = rt.segment_batch([dev(I)], want_recon=True, want_filled=True)[0]
    check_chain(out, I)


def test_chain_independent_of_schedule(rt):
    """Bytes do not depend on the variant or on how the propagation is scheduled."""
    I = synth.config2_tile(31, H=700, W=900)
    runs = [rt.segment_batch([dev(I)], rt.SegParams(variant=getattr(rt, v), max_local=m))[0]
            for v in VARIANTS for m in (1, 32)]
    for other in runs[1:]:
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(runs[0][k]), host(other[k]))
    check_chain(runs[0], I)


def test_chain_bench_configuration(rt):
    """The benchmark's workload exactly as it runs there: 8 distinct 4096^2
    tiles in one batched call with the trained picker attached, on two
    streams with one context each (consecutive calls overlap), every output of
    every tile against the oracle."""
    import concurrent.futures as cf
    import os
    from paper_1405_7958_gb300 import picker as pkmod
    seeds = [2000 + i for i in range(8)]
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        imgs = list(ex.map(synth.config2_tile, seeds))
        want = list(ex.map(oracle.chain, imgs))
    d = [dev(x) for x in imgs]
    pk = pkmod.load(os.path.join(os.path.dirname(rt.__file__), "data", "picker_config4.npz"))
    ctxs = [rt.Context(), rt.Context()]
    for c in ctxs:
        pk.attach(c)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [None, None]
    for k in range(4):
        j = k % 2
        with torch.cuda.stream(streams[j]):
            outs[j] = rt.segment_batch(d, rt.SegParams(policy=1), outputs=outs[j], ctx=ctxs[j], stream=streams[j])
    torch.cuda.synchronize()
    for o_s in outs:
        for o, w in zip(o_s, want):
            assert int(host(o["status"])[0]) == 0
            for k in ("R", "F", "L", "D"):
                assert np.array_equal(host(o[k]), w[k])
            assert int(host(o["n_kept"])[0]) == w["n_kept"]
    for c in ctxs:
        c.close()
