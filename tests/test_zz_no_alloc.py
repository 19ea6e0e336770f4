"""iwpp_reconstruct_noalloc: the entry point for callers that cannot allocate device
memory (it uses the library's own static scratch array). Called through the C ABI, its
results must equal iwpp_reconstruct's, bit for bit, on two calls in a row that share the
array. This file is collected last so that a failure here stops a -x run only after every
other test has run; it passes alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest

from paper_1605_00930_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def iw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_00930_gb300 import build
    build.build()
    from paper_1605_00930_gb300 import iwpp
    iwpp.lib()
    return iwpp


def _with_workspace(iw, marker, mask, conn, op, dtype_code):
    m = torch.from_numpy(marker).cuda()
    I = torch.from_numpy(mask).cuda()
    need = iw.iwpp_workspace_bytes(marker.shape[0], marker.shape[1], dtype_code)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    assert iw.iwpp_reconstruct(P(m.data_ptr()), P(I.data_ptr()), marker.shape[0], marker.shape[1], conn,
                               iw.OPS[op], dtype_code, P(ws.data_ptr()), need, s) == 0
    assert iw.iwpp_sync_status(P(ws.data_ptr()), s) == 0
    return m.cpu().numpy()


def _noalloc(iw, marker, mask, conn, op, dtype_code):
    m = torch.from_numpy(marker).cuda()
    I = torch.from_numpy(mask).cuda()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = ctypes.c_int(-1)
    rc = iw.iwpp_reconstruct_noalloc(ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(I.data_ptr()),
                                     marker.shape[0], marker.shape[1], conn, iw.OPS[op], dtype_code, s, st)
    assert rc == 0, iw.STATUS.get(rc)
    assert st.value == 0, iw.STATUS.get(st.value)
    return m.cpu().numpy()


def _cases():
    a = synth.tissue_case(700, 1033, nblobs=50)                       # u8, dilation
    field = synth.blob_field_u8(513, 301, 20, synth.rng_for(91))
    mask16 = synth.to_u16(field)
    b = synth.Case(synth.fillholes_marker(mask16), mask16, 4, "erode")  # u16, fill-holes
    return a, b


def test_noalloc_matches_workspace_entry_point_twice(iw):
    import oracle
    oracle.build()
    a, b = _cases()
    for case, code in ((a, 0), (b, 1)):                                 # two calls in a row
        ref = _with_workspace(iw, case.marker, case.mask, case.conn, case.op, code)
        got = _noalloc(iw, case.marker, case.mask, case.conn, case.op, code)
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_array_equal(got, oracle.reconstruct(case.marker, case.mask, case.conn, case.op))
    # and the first one again, after the array was used for a different image
    np.testing.assert_array_equal(_noalloc(iw, a.marker, a.mask, a.conn, a.op, 0),
                                  _with_workspace(iw, a.marker, a.mask, a.conn, a.op, 0))


def test_noalloc_allocates_nothing(iw):
    """After a first call on the device (which loads the library's device code and its
    scratch array), further calls leave the device's free memory and torch's allocator
    unchanged."""
    a, b = _cases()
    m = torch.from_numpy(a.marker).cuda()
    I = torch.from_numpy(a.mask).cuda()
    m0 = m.clone()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    st = ctypes.c_int(-1)
    assert iw.iwpp_reconstruct_noalloc(P(m.data_ptr()), P(I.data_ptr()), m.shape[0], m.shape[1], a.conn,
                                       iw.OPS[a.op], 0, s, st) == 0 and st.value == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        m.copy_(m0)
        assert iw.iwpp_reconstruct_noalloc(P(m.data_ptr()), P(I.data_ptr()), m.shape[0], m.shape[1], a.conn,
                                           iw.OPS[a.op], 0, s, None) == 0
    assert iw.iwpp_reconstruct_noalloc(P(m.data_ptr()), P(I.data_ptr()), m.shape[0], m.shape[1], a.conn,
                                       iw.OPS[a.op], 0, s, st) == 0 and st.value == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_status_refused_during_capture(iw):
    """Waiting for the status would end a stream capture: the call refuses it."""
    a, _ = _cases()
    m = torch.from_numpy(a.marker).cuda()
    I = torch.from_numpy(a.mask).cuda()
    P = ctypes.c_void_p
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    st = ctypes.c_int(-1)
    with torch.cuda.graph(g, stream=side):
        s = ctypes.c_void_p(side.cuda_stream)
        rc = iw.iwpp_reconstruct_noalloc(P(m.data_ptr()), P(I.data_ptr()), m.shape[0], m.shape[1], a.conn,
                                         iw.OPS[a.op], 0, s, st)
        m.add_(0)   # keep the captured graph non-empty
    assert rc == 1   # IWPP_ERR_ARG, nothing enqueued
    assert st.value == -1


def test_noalloc_rejects_images_beyond_its_scratch(iw):
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    P = ctypes.c_void_p(buf.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert iw.iwpp_workspace_bytes(65535, 65535, 0) > 8 << 20
    assert iw.iwpp_reconstruct_noalloc(P, P, 65535, 65535, 8, 0, 0, s, None) == 3   # IWPP_ERR_WORKSPACE
