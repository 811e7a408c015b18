"""The allocation-free EDT entry point (rt_edt_noalloc), called through the C
ABI, against the regular rt_edt and the CPU oracle on two calls in a row,
and at the edges of its fixed scratch.

rt_edt_noalloc exists for callers that cannot allocate device memory while
they run (a serving loop that reserved its budget at start-up, a plug-in
whose host owns all device allocations); its scratch is a fixed array built
into the library. The file sorts last so that, in a run that stops at the
first failure, every other test has run before it; its tests do not depend
on that order: each output buffer starts as a sentinel, and the scratch's
contents from any earlier call never matter (two different images back to
back check exactly that)."""
import ctypes

import numpy as np
import pytest

import oracle
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
        assert np.array_equal(got.cpu().numpy(), oracle.edt(fg.cpu().numpy()))


def test_noalloc_edt_at_the_edges_of_its_scratch():
    """The widest rows it takes (32 x 32768: exactly its pixel limit, and rows
    wider than 24576 pixels need the opt-in shared memory of the row pass),
    one 32768-pixel row with a closed form, and an image without background
    (every distance -1)."""
    import paper_1405_7958_gb300 as rt
    lib = rt.lib()
    stream = torch.cuda.current_stream().cuda_stream
    row = np.ones((1, 32768), np.uint8)
    row[0, [0, 20000]] = 0
    c = np.arange(32768)
    cases = [(synth.random_binary(32, 32768, 3, 990), None),
             (row, np.minimum(c, np.abs(c - 20000)).astype(np.int64) ** 2),
             (np.ones((300, 500), np.uint8), np.full((300, 500), -1))]
    for img, closed in cases:
        H, W = img.shape
        fg = torch.from_numpy(img).cuda()
        got = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
        st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        assert _call_noalloc(lib, fg, got, st, stream) == rt.RT_OK
        torch.cuda.synchronize()
        assert int(st.item()) == rt.RT_OK
        g = got.cpu().numpy()
        assert np.array_equal(g, oracle.edt(img))
        if closed is not None:
            assert np.array_equal(g, closed.reshape(H, W))


def test_noalloc_edt_rejects_images_beyond_its_scratch():
    import paper_1405_7958_gb300 as rt
    from paper_1405_7958_gb300 import _native
    lib = rt.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for H, W in ((1025, 1024), (33, 32768), (2, 32768 + 1)):
        fg = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
        out = torch.empty((H, W), dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = _call_noalloc(lib, fg, out, st, stream)
        assert rc == (_native.RT_EINVAL if W > 32768 else _native.RT_ESIZE), (H, W, rc)
    assert lib.rt_status_str(_native.RT_ESIZE).decode().startswith("RT_ESIZE")
