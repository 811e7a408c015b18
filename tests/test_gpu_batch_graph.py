"""The uneven-batch chain (tiles of different sizes in one call) captured in
a CUDA graph: replays give the same bytes as the eager call and as the
oracle; the autotuner's choice gives the same bytes too."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_graph_replay_equals_eager_and_oracle(tmp_path):
    import paper_1405_7958_gb300 as rt
    from paper_1405_7958_gb300 import autotune
    specs = synth.batch_sizes(6, 31, lo=256, hi=1024, step=128)
    imgs = [synth.tile(H, W, s, ns) for H, W, ns, s in specs]
    d = [torch.from_numpy(x).cuda() for x in imgs]
    ctx = rt.Context()
    table = autotune.Table(str(tmp_path / "tune.json"))
    params = table.params(d, reps=1, ctx=ctx)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        outs = rt.segment_batch(d, params, ctx=ctx, stream=s)      # eager (allocates the workspace)
    s.synchronize()
    eager = [{k: o[k].clone() for k in ("R", "F", "L", "D")} for o in outs]
    for o in outs:
        for k in ("R", "F", "L", "D"):
            o[k].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rt.segment_batch(d, params, outputs=outs, ctx=ctx, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for o, e, x in zip(outs, eager, imgs):
            for k in ("R", "F", "L", "D"):
                assert torch.equal(o[k], e[k])
    for o, x in zip(outs, imgs):
        want = oracle.chain(x)
        for k in ("R", "F", "L", "D"):
            assert np.array_equal(o[k].cpu().numpy(), want[k])
