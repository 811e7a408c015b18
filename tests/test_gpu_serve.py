"""Serving loop: every result of the continuously batched server is the
same, byte for byte, as the tile run alone; the plain server likewise."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_served_results_equal_standalone_runs():
    import paper_1405_7958_gb300 as rt
    from paper_1405_7958_gb300 import serve
    pool = serve.make_pool(6, 77, lo=512, hi=1280)
    alone = []
    for t in pool:
        o = rt.segment_batch([t.cuda()], want_recon=False, want_filled=False)[0]
        alone.append((o["L"].cpu().numpy(), o["D"].cpu().numpy()))
    for runner in (serve.run_batched, serve.run_plain):
        reqs = serve.arrivals(300.0, 0.4, len(pool), 5, pool)
        assert len(reqs) > 20
        runner(reqs, pool, keep=True)
        torch.cuda.synchronize()
        for r in reqs:
            assert r.done >= r.arrival
            L, D = alone[r.pool]
            assert np.array_equal(r.out_L.numpy(), L) and np.array_equal(r.out_D.numpy(), D)
        s = serve.summarize(reqs, 0.4)
        assert s["p99_ms"] >= s["p50_ms"] > 0
