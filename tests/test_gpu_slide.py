"""Whole-slide segmentation across tile seams. An 8192 x 8192 slide (2 x 2
tiles of 4096 x 4096, nuclei everywhere, also across both seams) runs as
one image through rt_segment_batch: the reconstruction propagates across
every seam of its 32 x 64 warp tiles (each visit reads its neighbours'
edge rows and columns as halo, and a changed edge flags the neighbour for
another visit), and the union-find joins components across every 32 x 32
block edge. Every output equals the CPU oracle's chain on the whole slide.
Cutting the slide into four independent 4096 x 4096 tiles instead gives
different labels: nuclei on a seam are cut in two."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_slide_2x2_tiles_equals_whole_slide_oracle():
    import paper_1405_7958_gb300 as rt
    S = 8192
    slide = rt.config2_tile(424242, H=S, W=S)          # ~12,000 nuclei, GPU twin of the generator
    torch.cuda.synchronize()
    I = slide.cpu().numpy()
    want = oracle.chain(I)
    out = rt.segment_batch([slide])[0]
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0
    for k in ("R", "F", "L", "D"):
        assert np.array_equal(out[k].cpu().numpy(), want[k]), k
    assert int(out["n_kept"].item()) == want["n_kept"]
    L = want["L"]
    h = 4096
    crossing = np.intersect1d(L[h - 1, :][L[h - 1, :] >= 0], L[h, :][L[h, :] >= 0]).size + \
        np.intersect1d(L[:, h - 1][L[:, h - 1] >= 0], L[:, h][L[:, h] >= 0]).size
    assert crossing > 0                                 # some kept nuclei do cross a seam
    # the same slide cut into four independent tiles does not give the slide's labels
    quads = [slide[r:r + h, c:c + h].contiguous() for r in (0, h) for c in (0, h)]
    outs = rt.segment_batch(quads)
    torch.cuda.synchronize()
    tiled = np.zeros_like(L)
    for (r, c), o in zip(((0, 0), (0, h), (h, 0), (h, h)), outs):
        q = o["L"].cpu().numpy()
        tiled[r:r + h, c:c + h] = np.where(q >= 0, (q // h + r) * S + (q % h + c), -1)
    assert not np.array_equal(tiled, L)
