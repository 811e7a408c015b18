"""The C-ABI library builds for sm_103a, loads on the host and exports every
symbol include/rt.h declares (no GPU needed: nothing is computed here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1405_7958_gb300 import build
    return build.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rt.h")).read()
    return sorted(set(re.findall(r"RT_API\s+[\w\s\*]*?\b(rt_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("rt_reconstruct", "rt_fill_holes", "rt_label_area", "rt_edt", "rt_segment_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_lists_every_export(built):
    from paper_1405_7958_gb300 import _native
    assert sorted(_native.EXPORTS) == declared_symbols()
    lib = _native.load(built)
    assert lib.rt_version() == 201
    assert lib.rt_status_str(4).decode().startswith("RT_ETIMEOUT")


def test_argument_validation_without_gpu(built):
    """Synchronous validation happens before any CUDA call."""
    from paper_1405_7958_gb300 import _native
    lib = _native.load(built)
    bogus = ctypes.c_void_p(1)
    # NULL context
    assert lib.rt_reconstruct(None, None, 0, bogus, 8, bogus, 8, 4, 4, 8, 0, 30, None, None) == _native.RT_EINVAL
    assert lib.rt_edt(None, bogus, 8, bogus, 8, 4, 4, None, None) == _native.RT_EINVAL
    assert lib.rt_create(None, 0, 0) == _native.RT_EINVAL
    assert lib.rt_set_limits(None, 1, 1) == _native.RT_EINVAL
    assert lib.rt_set_queue_capacity(None, 1) == _native.RT_EINVAL
    assert lib.rt_feature_norm(None, bogus, 4, bogus, None) == _native.RT_EINVAL


def _tiles(shapes):
    from paper_1405_7958_gb300 import _native
    tiles = (_native.RtTile * len(shapes))()
    for t, (H, W) in zip(tiles, shapes):
        t.H, t.W = H, W
        t.img = t.labels = t.d2 = 1
        t.ld_img = t.ld_labels = t.ld_d2 = W
    return tiles


def test_segment_workspace_query_without_gpu(built):
    """The batch workspace figure is computed on the host: positive, at
    least the compulsory per-tile buffers, the largest chunk of 32 tiles, and
    0 for invalid arguments."""
    from paper_1405_7958_gb300 import _native
    lib = _native.load(built)
    p = _native.RtSegParams()
    lib.rt_seg_params_default(ctypes.byref(p))
    one = lib.rt_segment_workspace_bytes(None, _tiles([(4096, 4096)]), 1, ctypes.byref(p))
    # padded R and mask copies (2 B/px), the binary image (1), union-find arrays (>= 10)
    assert one >= 13 * 4096 * 4096
    two = lib.rt_segment_workspace_bytes(None, _tiles([(4096, 4096)] * 2), 2, ctypes.byref(p))
    assert two >= 2 * one - 4096
    # 33 tiles run as a chunk of 32 and a chunk of 1: the figure is the larger chunk
    small = [(512, 600)] * 33
    w33 = lib.rt_segment_workspace_bytes(None, _tiles(small), 33, ctypes.byref(p))
    w32 = lib.rt_segment_workspace_bytes(None, _tiles(small), 32, ctypes.byref(p))
    assert w33 == w32
    bad = _tiles([(0, 5)])
    assert lib.rt_segment_workspace_bytes(None, bad, 1, ctypes.byref(p)) == 0
    p.conn_recon = 5
    assert lib.rt_segment_workspace_bytes(None, _tiles([(64, 64)]), 1, ctypes.byref(p)) == 0


def test_frontier_workspace_without_gpu(built):
    """RT_FRONTIER adds its two global queues (one 4-byte entry per padded
    pixel each) and their control words to the batch workspace; variants past
    RT_FRONTIER are invalid."""
    from paper_1405_7958_gb300 import _native
    lib = _native.load(built)
    p = _native.RtSegParams()
    lib.rt_seg_params_default(ctypes.byref(p))
    shapes = [(1000, 1100)]
    plain = lib.rt_segment_workspace_bytes(None, _tiles(shapes), 1, ctypes.byref(p))
    p.variant = _native.RT_FRONTIER
    front = lib.rt_segment_workspace_bytes(None, _tiles(shapes), 1, ctypes.byref(p))
    padded = 1024 * 1152                       # 1000 x 1100 in 32 x 64 tiles
    extra = front - plain
    assert 8 * padded <= extra <= 8 * padded + 4 * 2052 + 3 * 256
    p.variant = _native.RT_FRONTIER + 1
    assert lib.rt_segment_workspace_bytes(None, _tiles(shapes), 1, ctypes.byref(p)) == 0
