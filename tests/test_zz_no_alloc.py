"""The allocation-free EDT entry point (rt_edt_noalloc), called through the C
ABI, against the regular rt_edt on two calls in a row.

rt_edt_noalloc exists for callers that cannot allocate device memory while
they run (a serving loop that reserved its budget at start-up, a plug-in
whose host owns all device allocations); its scratch is a fixed array built
into the library. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call_noalloc(lib, fg, out, status, stream):
    H, W = fg.shape
    return lib.rt_edt_noalloc(fg.data_ptr(), fg.stride(0), out.data_ptr(), out.stride(0), H, W,
                              status.data_ptr(), stream)


def test_noalloc_edt_matches_rt_edt_on_two_calls():
    import paper_1405_7958_gb300 as rt
    lib = rt.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # two different images in a row: the shared scratch must not carry the
    # first call's contents into the second one
    for seed, (H, W), dens in ((1, (700, 900), 900), (2, (1024, 1024), 600)):
        fg = torch.from_numpy(synth.random_binary(H, W, seed, dens)).cuda()
        got = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
        st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        assert _call_noalloc(lib, fg, got, st, stream) == rt.RT_OK
        want = rt.edt(fg)
        torch.cuda.synchronize()
        assert int(st.item()) == rt.RT_OK
        assert torch.equal(got, want)


def test_noalloc_edt_rejects_images_beyond_its_scratch():
    import paper_1405_7958_gb300 as rt
    from paper_1405_7958_gb300 import _native
    lib = rt.lib()
    stream = torch.cuda.current_stream().cuda_stream
    fg = torch.zeros((1025, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty((1025, 1024), dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call_noalloc(lib, fg, out, st, stream) == _native.RT_ESIZE
    assert lib.rt_status_str(_native.RT_ESIZE).decode().startswith("RT_ESIZE")
