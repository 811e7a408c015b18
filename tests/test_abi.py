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
    assert lib.rt_version() == 100
    assert lib.rt_status_str(4).decode().startswith("RT_ETIMEOUT")


def test_argument_validation_without_gpu(built):
    """Synchronous validation happens before any CUDA call."""
    from paper_1405_7958_gb300 import _native
    lib = _native.load(built)
    bogus = ctypes.c_void_p(1)
    # NULL context
    assert lib.rt_reconstruct(None, None, 0, bogus, 8, bogus, 8, 4, 4, 8, 0, 30, None, None) == _native.RT_EINVAL
    assert lib.rt_edt(None, bogus, 8, bogus, 8, 4, 4, None, None) == _native.RT_EINVAL
    assert lib.rt_create(None, 0) == _native.RT_EINVAL
