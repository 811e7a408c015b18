"""GPU tests of the learned picker path and the GPU tile generator: the
generator against the Python generator (bit-exact), the features and the
network (forward, backward, AdamW) against the fp64 oracle, and the chain
under the learned policy against the plain one (identical bytes)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import features as OF
from oracle import mlp as OM

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rt():
    import paper_1405_7958_gb300 as rt
    return rt


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


GEN_CASES = [
    dict(H=512, W=512, seed=1000, n_shapes=60, kind="disk", vlo=40, vhi=90, rmin=4, rmax=12, background="flat"),
    dict(H=700, W=1031, seed=7, n_shapes=150, kind="ellipse"),
    dict(H=1, W=300, seed=3, n_shapes=2, kind="ellipse"),
    dict(H=600, W=520, seed=2**40 + 5, n_shapes=0, kind="ellipse"),
    dict(H=300, W=300, seed=11, n_shapes=40, kind="ellipse", noise=False),
]


@pytest.mark.parametrize("case", GEN_CASES)
def test_gpu_generator_matches_python(rt, case):
    want = synth.tile(**case)
    got = host(rt.synth_tile(**case))
    assert np.array_equal(got, want)


def test_gpu_generator_4k_tile(rt):
    assert np.array_equal(host(rt.config2_tile(2003)), synth.config2_tile(2003))


def test_features_match_oracle(rt):
    from test_oracle_learned import _frontier_image
    from golden.load import load
    imgs = [synth.config2_tile(5, H=333, W=517), synth.config1_image(1000), synth.random_binary(64, 40, 2, 500) * 200,
            np.full((9, 13), 77, np.uint8), synth.config2_tile(9, H=1024, W=2048),
            _frontier_image(load("features_frontier.txt")["D"])]
    got = host(rt.tile_features([torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in imgs]))
    for g, x in zip(got, imgs):
        want = OF.features(x)
        assert np.array_equal(g[7:16], want[7:16])                       # percentiles are integers
        assert np.allclose(g, want, rtol=2e-6, atol=2e-6), (g - want)


def _picker_inputs(rng, B):
    x = rng.normal(size=(B, 24)).astype(np.float32) * 3 + 1
    y = rng.integers(0, 3, size=B).astype(np.int32)
    return x, y


def test_mlp_forward_and_backward_match_oracle(rt):
    rng = np.random.default_rng(0)
    pk = rt.Picker(seed=1)
    norm = np.concatenate([rng.normal(size=24), rng.uniform(0.5, 2.0, size=24)]).astype(np.float32)
    pk.norm = torch.from_numpy(norm).cuda()
    x, y = _picker_inputs(rng, 777)
    xd = torch.from_numpy(x).cuda()
    logits, act, pick = pk.forward(xd, with_act=True)
    grad, loss = pk.backward(xd, act, logits, torch.from_numpy(y).cuda())
    p = OM.bf16_bits_to_f64(host(pk.wb))
    _, h1, h2, z = OM.forward(p, norm, x)
    assert np.allclose(host(logits), z, rtol=1e-4, atol=1e-4)
    assert np.array_equal(host(pick), z.argmax(axis=1))
    assert np.allclose(host(act)[:, :64], h1, rtol=1e-4, atol=1e-4)
    g_want = OM.backward(p, norm, x, y)
    g_got = host(grad).astype(np.float64)
    for name, shape in OM.SHAPES:
        a, b = OM.unflatten(g_got)[name].ravel(), OM.unflatten(g_want)[name].ravel()
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-7, name
        if np.linalg.norm(b) > 0:
            assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.999, name
    assert np.isclose(float(host(loss)[0]), OM.loss(p, norm, x, y), rtol=1e-5)


def test_mlp_forward_small_and_large_batches_agree(rt):
    """Chunks of up to 64 samples run one warp per sample, larger batches one
    thread per sample: the same sums in the same order, the same bits."""
    rng = np.random.default_rng(2)
    pk = rt.Picker(seed=3)
    x, _ = _picker_inputs(rng, 300)
    xd = torch.from_numpy(x).cuda()
    big_logits, big_act, big_pick = pk.forward(xd, with_act=True, min_prob=0.5)
    for n in (1, 7, 64):
        logits, act, pick = pk.forward(xd[:n].contiguous(), with_act=True, min_prob=0.5)
        assert torch.equal(logits, big_logits[:n]) and torch.equal(act, big_act[:n])
        assert torch.equal(pick, big_pick[:n])


def _bf16_round(a):
    """Round float32 values to bf16 (nearest even), as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("B", [1, 128, 300, 2000])
def test_mlp_forward_tensor_cores_match_oracle(rt, B):
    """The tensor-core forward against the fp64 oracle network evaluated on
    the same bf16 operands: the normalised input (computed in fp32, as the
    kernel does) rounded to bf16, and each hidden layer rounded to bf16
    before it enters the next product. Accumulation order and fp32 sums may
    flip a hidden value across a bf16 rounding boundary, so the hidden
    layers compare within 1e-2 of their scale; the first hidden layer, whose
    inputs are rounded identically on both sides, within 1e-5. Batches of 1,
    128 and ragged 300 and 2000 samples (several thread blocks, partial
    last block)."""
    rng = np.random.default_rng(5)
    pk = rt.Picker(seed=7)
    norm = np.concatenate([rng.normal(size=24), rng.uniform(0.5, 2.0, size=24)]).astype(np.float32)
    pk.norm = torch.from_numpy(norm).cuda()
    x, _ = _picker_inputs(rng, B)
    xd = torch.from_numpy(x).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    logits, act, pick = pk.forward(xd, with_act=True, tensor_cores=True, status=st)
    assert int(host(st)[0]) == 0
    w = OM.unflatten(OM.bf16_bits_to_f64(host(pk.wb)))
    xn = _bf16_round((x - norm[:24]) / norm[24:])
    h1 = np.maximum(xn @ w["W1"].T + w["b1"], 0.0)
    got = host(act)
    scale1 = np.abs(h1).max() + 1e-30
    assert np.abs(got[:, :64] - h1).max() <= 1e-5 * scale1
    h2 = np.maximum(_bf16_round(got[:, :64]) @ w["W2"].T + w["b2"], 0.0)
    assert np.abs(got[:, 64:] - h2).max() <= 1e-5 * (np.abs(h2).max() + 1e-30)
    z = _bf16_round(got[:, 64:]) @ w["W3"].T + w["b3"]
    zl = host(logits)
    assert np.abs(zl - z).max() <= 1e-5 * (np.abs(z).max() + 1e-30)
    assert np.array_equal(host(pick), zl.argmax(axis=1))
    # against the fp32 forward: the same network up to the bf16 operand rounding
    l32, a32, p32 = pk.forward(xd, with_act=True)
    a32 = host(a32)
    assert np.abs(got - a32).max() <= 1e-2 * (np.abs(a32).max() + 1e-30)
    assert np.abs(zl - host(l32)).max() <= 2e-2 * (np.abs(host(l32)).max() + 1e-30)


@pytest.mark.parametrize("B", [1, 256, 777])
def test_mlp_backward_tensor_cores_match_oracle(rt, B):
    """The tensor-core backward against the fp64 oracle gradient (relative
    2e-2 per parameter tensor, cosine above 0.999, as for the fp32 backward:
    the deltas and activations enter its products as bf16), and against the
    fp32 backward on the same forward outputs (relative 1e-2); W3 and b3,
    computed in fp32 on both paths, agree to 1e-5. Deterministic: a second
    call gives the same bits. One, two and seven blocks of 128 samples."""
    rng = np.random.default_rng(11)
    pk = rt.Picker(seed=2)
    norm = np.concatenate([rng.normal(size=24), rng.uniform(0.5, 2.0, size=24)]).astype(np.float32)
    pk.norm = torch.from_numpy(norm).cuda()
    x, y = _picker_inputs(rng, B)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    logits, act, _ = pk.forward(xd, with_act=True, tensor_cores=True, status=st)
    grad, loss = pk.backward(xd, act, logits, yd, tensor_cores=True, status=st)
    g_tc, l_tc = host(grad).astype(np.float64).copy(), float(host(loss)[0])
    pk.backward(xd, act, logits, yd, tensor_cores=True, status=st)
    assert np.array_equal(host(grad), g_tc.astype(np.float32)) and int(host(st)[0]) == 0
    grad32, loss32 = pk.backward(xd, act, logits, yd)
    g_32 = host(grad32).astype(np.float64)
    assert np.isclose(l_tc, float(host(loss32)[0]), rtol=1e-6)
    p = OM.bf16_bits_to_f64(host(pk.wb))
    g_want = OM.backward(p, norm, x, y)
    for name, _ in OM.SHAPES:
        a, w, c = (OM.unflatten(v)[name].ravel() for v in (g_tc, g_want, g_32))
        assert np.linalg.norm(a - w) <= 2e-2 * np.linalg.norm(w) + 1e-7, name
        if np.linalg.norm(w) > 0:
            assert a @ w / (np.linalg.norm(a) * np.linalg.norm(w)) > 0.999, name
        tol = 1e-5 if name in ("W3", "b3") else 1e-2
        assert np.linalg.norm(a - c) <= tol * np.linalg.norm(c) + 1e-7, name
    assert np.isclose(l_tc, OM.loss(p, norm, x, y), rtol=1e-2)


def test_adamw_step_matches_oracle(rt):
    rng = np.random.default_rng(2)
    pk = rt.Picker(seed=3)
    g = rng.normal(size=pk.NPARAM).astype(np.float32)
    pk.grad.copy_(torch.from_numpy(g))
    master0 = host(pk.master).astype(np.float64)
    pk.step(lr=1e-2, weight_decay=1e-3)
    pk.step(lr=1e-2, weight_decay=1e-3)
    m1, mm, vv = OM.adamw(master0, g.astype(np.float64), 0.0, 0.0, 1, 1e-2, wd=1e-3)
    m2, _, _ = OM.adamw(m1, g.astype(np.float64), mm, vv, 2, 1e-2, wd=1e-3)
    got = host(pk.master)
    assert np.allclose(got, m2, rtol=1e-5, atol=1e-6)
    # the bf16 copy is the master rounded to nearest even
    want_bits = torch.from_numpy(got).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(host(pk.wb), want_bits)


def test_training_reduces_loss(rt):
    """Training with the tensor-core forward and backward and AdamW fits a
    separable labelling."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(512, 24)).astype(np.float32)
    y = (x[:, 0] > 0.3).astype(np.int32) + (x[:, 1] > 0.8).astype(np.int32)
    pk = rt.Picker(seed=5)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    pk.set_norm(xd)
    losses = []
    for _ in range(150):
        logits, act, _ = pk.forward(xd, with_act=True, tensor_cores=True)
        _, loss = pk.backward(xd, act, logits, yd, tensor_cores=True)
        losses.append(float(loss.item()))
        pk.step(lr=1e-2)
    assert losses[-1] < 0.5 * losses[0]
    _, _, pick = pk.forward(xd)
    assert (host(pick) == y).mean() > 0.9


VARIANT_CLASSES = ((1, 12), (2, 0), (3, 0))    # RT_RASTER, RT_QUEUE, RT_HYBRID as the three classes
FRONTIER_CLASSES = ((1, 12), (4, 0), (3, 0))   # RT_RASTER, RT_FRONTIER, RT_HYBRID


@pytest.mark.parametrize("classes", [None, VARIANT_CLASSES, FRONTIER_CLASSES], ids=["budgets", "variants", "frontier"])
def test_learned_policy_same_bytes_as_plain(rt, classes):
    """Every class of the picker, forced (the default visit budgets, and a
    table of the three variants): the oracle's bytes; a confidence threshold
    no pick reaches sends every tile to the plain schedule (class 3). With
    the default budgets, tiles sharing a launch all run the plain budget, so
    the picker is skipped there and every tile reports class 3; the picks
    are checked on each tile alone."""
    imgs = [synth.config2_tile(40 + i, H=H, W=W) for i, (H, W) in enumerate([(300, 500), (640, 256), (1024, 1024)])]
    want = [oracle.chain(x) for x in imgs]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    pk = rt.Picker(seed=9)
    # steer the untrained network to every class: bias b3 one-hot per run
    for cls in range(3):
        b3 = torch.full((3,), -1.0)
        b3[cls] = 1.0
        pk.master[5760:5952] = 0.0                 # W3 = 0: the logits are b3 (softmax max 0.78)
        pk.master[5952:5955] = b3.cuda()
        pk.wb = pk.master.to(torch.bfloat16).view(torch.int16).contiguous()
        ctx = rt.Context()
        if classes:
            rt.set_picker_classes(classes, ctx)
        pk.attach(ctx)
        for min_prob, picks in ((0, [cls] * 3), (700, [cls] * 3), (800, [3] * 3)):
            params = rt.SegParams(policy=1, pick_min_prob=min_prob)
            outs = rt.segment_batch(d, params, ctx=ctx)
            assert rt.last_picks(ctx) == (picks if classes else [3] * 3)
            for o, w in zip(outs, want):
                for k in ("R", "F", "L", "D"):
                    assert np.array_equal(host(o[k]), w[k])
            if not classes:
                for x, w, p in zip(d, want, picks):
                    (o,) = rt.segment_batch([x], params, ctx=ctx)
                    assert rt.last_picks(ctx) == [p]
                    for k in ("R", "F", "L", "D"):
                        assert np.array_equal(host(o[k]), w[k])
        ctx.close()


def test_chain_picks_equal_the_network_forward(rt):
    """The chain computes its picks in the features' last launch; they equal
    the network's forward on rt_tile_features of the same tiles (the same
    bits), alone and in a chunk whose classes make the picks matter, with and
    without the confidence fall-back."""
    import os
    from paper_1405_7958_gb300 import picker as pkmod
    pk = pkmod.load(os.path.join(os.path.dirname(rt.__file__), "data", "picker_config4.npz"))
    shapes = [(1024, 1280), (2048, 1536), (300, 500), (1536, 3072)]
    imgs = [rt.synth_tile(H, W, 500 + i, 60 + 40 * i) for i, (H, W) in enumerate(shapes)]
    feats = rt.tile_features(imgs)
    for min_prob in (0, 600, 990):
        want = host(pk.forward(feats, min_prob=min_prob / 1000.0, fallback=3)[2]).tolist()
        ctx = rt.Context()
        pk.attach(ctx)
        params = rt.SegParams(policy=1, pick_min_prob=min_prob)
        got = []
        for im in imgs:
            rt.segment_batch([im], params, ctx=ctx)
            got += rt.last_picks(ctx)
        assert got == want
        rt.set_picker_classes(VARIANT_CLASSES, ctx)
        rt.segment_batch(imgs, params, ctx=ctx)
        assert rt.last_picks(ctx) == want
        ctx.close()


def _height_picker(rt):
    """A hand-set network whose class depends on the tile height alone:
    h = H / 1024, logits (0.5, h, 2h - 0.75) -> raster below H = 512, queue
    below 768, hybrid above (all weights exact in bf16)."""
    pk = rt.Picker(seed=0)
    w = torch.zeros(pk.NPARAM, dtype=torch.float32)
    w[0] = 2.0 ** -10                # W1[0][0]
    w[1600] = 1.0                    # W2[0][0]
    w[5760 + 64] = 1.0               # W3[1][0]
    w[5760 + 128] = 2.0              # W3[2][0]
    w[5952:5955] = torch.tensor([0.5, 0.0, -0.75])
    pk.master.copy_(w)
    pk.wb = pk.master.to(torch.bfloat16).view(torch.int16).contiguous()
    pk.norm = torch.cat([torch.zeros(24), torch.ones(24)]).cuda()
    return pk


def test_learned_policy_mixed_variants_in_one_batch(rt):
    """Tiles of one call take different variants (chosen on the device);
    every tile still gives the oracle's bytes."""
    shapes = [(1024, 700), (300, 500), (640, 256), (300, 300), (1100, 640), (700, 900)]
    imgs = [synth.config2_tile(60 + i, H=H, W=W) for i, (H, W) in enumerate(shapes)]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    pk = _height_picker(rt)
    ctx = rt.Context()
    rt.set_picker_classes(VARIANT_CLASSES, ctx)
    pk.attach(ctx)
    outs = rt.segment_batch(d, rt.SegParams(policy=1), ctx=ctx)
    want_picks = [0 if H < 512 else 1 if H < 768 else 2 for H, _ in shapes]
    assert rt.last_picks(ctx) == want_picks
    for o, x in zip(outs, imgs):
        want = oracle.chain(x)
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(host(o[k]), want[k])
    ctx.close()


@pytest.mark.parametrize("classes", [VARIANT_CLASSES, FRONTIER_CLASSES], ids=["variants", "frontier"])
def test_learned_policy_in_cuda_graph(rt, classes):
    """The learned path has no host round trip, so it captures into a CUDA
    graph (the frontier class included: its queue counters are reset by a
    memset node); replays give the oracle's bytes and the same picks."""
    shapes = [(300, 500), (700, 640), (1100, 333)]
    imgs = [synth.config2_tile(80 + i, H=H, W=W) for i, (H, W) in enumerate(shapes)]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    pk = _height_picker(rt)
    ctx = rt.Context()
    rt.set_picker_classes(classes, ctx)
    pk.attach(ctx)
    s = torch.cuda.Stream()
    p = rt.SegParams(policy=1)
    with torch.cuda.stream(s):
        outs = rt.segment_batch(d, p, ctx=ctx, stream=s)          # eager: allocates the workspace
    s.synchronize()
    for o in outs:
        for k in ("R", "F", "L", "D"):
            o[k].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rt.segment_batch(d, p, outputs=outs, ctx=ctx, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert rt.last_picks(ctx) == [0, 1, 2]
        for o, x in zip(outs, imgs):
            want = oracle.chain(x)
            for k in ("R", "F", "L", "D"):
                assert np.array_equal(host(o[k]), want[k])
    ctx.close()


def _trained(rt):
    import os
    from paper_1405_7958_gb300 import picker as pkmod
    data = os.path.join(os.path.dirname(rt.__file__), "data")
    pk = pkmod.load(os.path.join(data, "picker_config4.npz"))
    with open(os.path.join(data, "picker_config4_report.json")) as fh:
        import json
        rep = json.load(fh)
    ev = np.load(os.path.join(data, "picker_config4_report_eval_set.npz"))
    return pkmod, pk, rep, ev["feats"], ev["times"]


def test_trained_picker_report_replays_on_the_gpu(rt):
    """The library's forward kernel on the committed held-out features gives
    the report's picks, its gain over the plain schedule (above 1), and the
    robustness study's figures (same seeded noise, same kernels)."""
    pkmod, pk, rep, feats, times = _trained(rt)
    ev = pkmod.evaluate(pk, feats, times)
    assert ev["pick_counts"] == rep["eval"]["pick_counts"]
    assert ev["gain_vs_plain"] == pytest.approx(rep["eval"]["gain_vs_plain"], rel=1e-12) and ev["gain_vs_plain"] > 1
    rows = pkmod.robustness(pk, feats, times)
    for got, want in zip(rows, rep["robustness_eval"]):
        if "sigma" in want:
            assert got["sigma"] == want["sigma"] and got["min_prob"] == want["min_prob"]
            assert got["time_vs_plain"] == pytest.approx(want["time_vs_plain"], rel=1e-9)
            assert got["fell_back"] == pytest.approx(want["fell_back"], abs=1e-12)


def test_trained_picker_on_new_held_out_tiles(rt):
    """16 new held-out uneven tiles (seeds outside the training and
    evaluation sets), each alone (the regime the picker was trained in) and
    all in one call, with the trained picker (confidence fall-back at 0.6)
    and with the plain schedule: identical outputs; the measured times
    (median of 7, CUDA events, learned and plain runs alternating) are
    printed. In the shared launch every tile runs the plain budget, so the
    picker is skipped and every tile reports class 3. The gain over the plain schedule
    net of the picker's own cost (features and network) is bounded below; the
    picker's gain before its cost is asserted on the committed held-out set
    (test_trained_picker_report_replays_on_the_gpu)."""
    import statistics
    _, pk, _, _, _ = _trained(rt)
    specs = synth.batch_sizes(16, 9100)
    imgs = [rt.synth_tile(H, W, s, ns) for H, W, ns, s in specs]
    ctx_l, ctx_p = rt.Context(), rt.Context()
    pk.attach(ctx_l)
    learned, plain = rt.SegParams(policy=1, pick_min_prob=600), rt.SegParams()

    def timed(batch, ol, op):
        # learned and plain runs alternate, so drifting clocks or a busy
        # neighbour on the machine weigh on both medians alike
        tl, tp = [], []
        for _ in range(7):
            for params, ctx, outs, ts in ((learned, ctx_l, ol, tl), (plain, ctx_p, op, tp)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                rt.segment_batch(batch, params, outputs=outs, ctx=ctx)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        return statistics.median(tl), statistics.median(tp)

    gains = {}
    for mode, groups in (("alone", [[im] for im in imgs]), ("batched", [imgs])):
        t_l = t_p = 0.0
        picks = []
        for g in groups:
            ol = rt.segment_batch(g, learned, ctx=ctx_l)
            picks += rt.last_picks(ctx_l)
            op = rt.segment_batch(g, plain, ctx=ctx_p)
            torch.cuda.synchronize()
            for a, b in zip(ol, op):
                for k in ("R", "F", "L", "D"):
                    assert torch.equal(a[k], b[k])
            a, b = timed(g, ol, op)
            t_l += a
            t_p += b
        assert len(picks) == 16 and all(0 <= c <= 3 for c in picks)
        if mode == "batched":
            assert picks == [3] * 16
        gains[mode] = t_p / t_l
        print(f"{mode}: trained picker {t_l:.2f} ms, plain {t_p:.2f} ms, gain {gains[mode]:.3f}, picks {picks}")
    assert min(gains.values()) > 0.95
    ctx_l.close()
    ctx_p.close()
