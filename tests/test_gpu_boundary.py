"""GPU tests of the boundary's bounds and sizing: an iteration bound or a
time bound that runs out stops the propagation with RT_ETIMEOUT and leaves
the context usable (the next call gives the oracle's bytes); a batch of more
than 32 uneven tiles (two chunks) eager and replayed from a CUDA graph,
every tile against the oracle; a context reserved with the library's
workspace figure never grows; the feature normalisation against numpy; the
raster propagation's strip length changes no byte."""
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("variant", ["RT_RASTER", "RT_QUEUE", "RT_HYBRID", "RT_FRONTIER"])
def test_visit_bound_runs_out_and_context_recovers(rt, variant):
    """A spiral corridor needs many visits of each of its 15 tiles; with one
    visit per tile allowed the propagation stops with RT_ETIMEOUT, below the
    reconstruction (it only ever raises pixels towards it). RT_FRONTIER's
    dense first pass spends the one visit per tile, and the drain's pops count
    against the same bound (2048 pops per visit)."""
    I = synth.spiral(129, low=0)
    J = np.zeros_like(I)
    J[0, 0] = I[0, 0]
    want = oracle.recon(J, I, 8)
    ctx = rt.Context()
    v = getattr(rt, variant)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.set_limits(max_iters=1)
    got = host(rt.reconstruct(dev(I), dev(J), conn=8, variant=v, status=st, ctx=ctx))
    assert int(st.item()) == rt.RT_ETIMEOUT
    assert (got <= want).all() and not np.array_equal(got, want)
    ctx.set_limits(0, 0)
    got = host(rt.reconstruct(dev(I), dev(J), conn=8, variant=v, status=st, ctx=ctx))
    assert int(st.item()) == rt.RT_OK
    assert np.array_equal(got, want)
    ctx.close()


@pytest.mark.parametrize("variant", ["RT_RASTER", "RT_FRONTIER"])
def test_time_bound_runs_out_and_context_recovers(rt, variant):
    """A 768 x 768 spiral's front crosses thousands of tile edges one after
    another (each ring of the corridor crosses every tile on its way), and a
    pixel frontier follows its 300,000-pixel corridor one step at a time; 2 ms
    of device time is not enough for either."""
    I = synth.spiral(768, low=0)
    J = np.zeros_like(I)
    J[0, 0] = I[0, 0]
    ctx = rt.Context()
    v = getattr(rt, variant)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.set_limits(timeout_ms=2)
    rt.reconstruct(dev(I), dev(J), conn=8, variant=v, status=st, ctx=ctx)
    assert int(host(st)[0]) == rt.RT_ETIMEOUT
    ctx.set_limits(0, 0)
    got = host(rt.reconstruct(dev(I), dev(J), conn=8, variant=v, status=st, ctx=ctx))
    assert int(st.item()) == rt.RT_OK
    assert np.array_equal(got, oracle.recon(J, I, 8))
    ctx.close()


def test_chain_visit_bound_in_params(rt):
    """rt_seg_params.max_iters bounds the chain's propagation the same way:
    the tile's status says RT_ETIMEOUT; the same call without the bound on
    the same context gives the oracle's outputs."""
    I = synth.spiral(300, low=0, high=60)      # dark corridor: R < 80 along it
    ctx = rt.Context()
    out = rt.segment_batch([dev(I)], rt.SegParams(max_iters=1), ctx=ctx)[0]
    assert int(host(out["status"])[0]) == rt.RT_ETIMEOUT
    out = rt.segment_batch([dev(I)], rt.SegParams(), outputs=[out], ctx=ctx)[0]
    assert int(host(out["status"])[0]) == rt.RT_OK
    want = oracle.chain(I)
    for k in ("R", "F", "L", "D"):
        assert np.array_equal(host(out[k]), want[k])
    ctx.close()


def test_batch_of_40_uneven_tiles_eager_and_graph(rt):
    """40 tiles of ragged uneven sizes run as a chunk of 32 and a chunk of 8
    in one call, eager and replayed from a CUDA graph: every output of every
    tile equals the oracle's."""
    specs = synth.batch_sizes(40, 77, lo=33, hi=33 + 29 * 14, step=29)
    imgs = [synth.tile(H, W, s, ns) for H, W, ns, s in specs]
    want = [oracle.chain(x) for x in imgs]
    d = [dev(x) for x in imgs]
    ctx = rt.Context()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = rt.segment_batch(d, ctx=ctx, stream=s)
    s.synchronize()
    for o, w in zip(outs, want):
        assert int(host(o["status"])[0]) == 0
        assert int(host(o["n_kept"])[0]) == w["n_kept"]
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(o[k]), w[k])
    for o in outs:
        for k in ("R", "F", "L", "D", "n_kept"):
            o[k].fill_(-7 if o[k].dtype == torch.int32 else 7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rt.segment_batch(d, outputs=outs, ctx=ctx, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for o, w in zip(outs, want):
        assert int(host(o["n_kept"])[0]) == w["n_kept"]
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(o[k]), w[k])
    ctx.close()


@pytest.mark.parametrize("cap", [0, 500])
def test_batch_frontier_variant(rt, cap):
    """rt_segment_batch with RT_FRONTIER for every tile (one seeding and one
    drain over the whole chunk, entries naming tiles of several images), with
    the default queues and with queues small enough to overflow: every
    output is the oracle's, and the size query counts the queues."""
    shapes = [(300, 500), (640, 256), (1024, 1024), (77, 1300), (513, 700)]
    imgs = [synth.tile(H, W, 60 + i, 1 + H * W // 4000, background="flat" if i % 2 else "perlin")
            for i, (H, W) in enumerate(shapes)]
    want = [oracle.chain(x) for x in imgs]
    ctx = rt.Context()
    ctx.set_queue_capacity(cap)
    p = rt.SegParams(variant=rt.RT_FRONTIER)
    need = rt.segment_workspace_bytes(shapes, p, ctx=ctx)
    assert need > rt.segment_workspace_bytes(shapes, rt.SegParams())
    outs = rt.segment_batch([dev(x) for x in imgs], p, ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.workspace_bytes() >= need
    for o, w in zip(outs, want):
        assert int(host(o["status"])[0]) == 0
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(o[k]), w[k])
    ctx.close()


def test_reserved_workspace_is_enough(rt):
    shapes = [(700, 1031), (64, 4000), (1024, 1024)]
    imgs = [synth.config2_tile(40 + i, H=H, W=W) for i, (H, W) in enumerate(shapes)]
    need = rt.segment_workspace_bytes(shapes)
    assert need > 0
    ctx = rt.Context(workspace_bytes=need)
    have = ctx.workspace_bytes()
    assert have >= need
    outs = rt.segment_batch([dev(x) for x in imgs], ctx=ctx)
    torch.cuda.synchronize()
    assert ctx.workspace_bytes() == have
    for o, x in zip(outs, imgs):
        w = oracle.chain(x)
        assert np.array_equal(host(o["L"]), w["L"]) and np.array_equal(host(o["D"]), w["D"])
    ctx.close()


def test_feature_norm_matches_numpy(rt):
    rng = np.random.default_rng(5)
    x = (rng.normal(size=(1000, 24)) * rng.uniform(0.1, 50, size=24) + rng.normal(size=24) * 100).astype(np.float32)
    x[:, 7] = 3.0                                           # a constant column: sd clamped to 1e-6
    pk = rt.Picker(seed=0)
    pk.set_norm(dev(x))
    norm = host(pk.norm)
    xd = x.astype(np.float64)
    assert np.allclose(norm[:24], xd.mean(axis=0), rtol=1e-6, atol=1e-6)
    sd = np.maximum(xd.std(axis=0, ddof=1), 1e-6)
    assert np.allclose(norm[24:], sd, rtol=1e-6)
    assert norm[24 + 7] == np.float32(1e-6)


@pytest.mark.parametrize("strip", [1, 3, 8, 16, 32])
def test_strip_lengths_give_the_oracle_bytes(rt, strip):
    """The raster propagation's strip of tiles per warp (rt_seg_params
    strip_tiles, an autotuner knob) changes only which warp visits a tile
    first: every length gives the oracle's bytes, on ragged tiles in one call
    (a strip may cross from one image into the next) and on a spiral whose
    front crosses many strips."""
    shapes = [(700, 1031), (257, 300), (1100, 640)]
    imgs = [synth.config2_tile(300 + i, H=H, W=W) for i, (H, W) in enumerate(shapes)]
    outs = rt.segment_batch([dev(x) for x in imgs], rt.SegParams(strip_tiles=strip))
    for o, x in zip(outs, imgs):
        want = oracle.chain(x)
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(o[k]), want[k]), k
    I = synth.spiral(257, low=0)
    (o,) = rt.segment_batch([dev(I)], rt.SegParams(strip_tiles=strip, h_offset=255))
    J = np.zeros_like(I)
    J[0, :], J[-1, :], J[:, 0], J[:, -1] = I[0, :], I[-1, :], I[:, 0], I[:, -1]
    assert np.array_equal(host(o["R"]), oracle.recon(J, I, 8))


def test_strip_length_out_of_range_is_rejected(rt):
    x = dev(synth.config2_tile(5, H=64, W=64))
    for bad in (-1, 33):
        with pytest.raises(RuntimeError):
            rt.segment_batch([x], rt.SegParams(strip_tiles=bad))
