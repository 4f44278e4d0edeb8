"""ccl_label_static: the allocation-free entry point.

It exists for callers that cannot allocate device memory (a host framework
that owns every device allocation, a plug-in handed only input/output
pointers, a latency-critical loop that cannot take cudaMalloc's device
synchronisation).  Its scratch is a fixed device array inside libccl.so, so
these tests check, through the C ABI, that two calls in a row on the shared
array give exactly the labels of the allocating entry point (ccl_label), and
that images too large for the array are refused before anything is enqueued.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synthetic
from paper_1708_08180_gb300 import _lib

LIMIT = _lib.CCL_STATIC_SCRATCH_BYTES


def test_static_limit_covers_4096_square_and_refuses_larger():
    lib = _lib.load()
    for h, w in ((4096, 4096), (4096, 1), (1, 4096), (4096, 257), (3000, 4096), (33, 4096)):
        for conn in (4, 8):
            assert 0 < lib.ccl_workspace_bytes(h, w, conn) <= LIMIT, (h, w, conn)
    P = ctypes.c_void_p
    # too large for the array: refused on the host, nothing enqueued
    assert lib.ccl_workspace_bytes(8192, 8192, 8) > LIMIT
    assert lib.ccl_label_static(P(256), P(512), 8192, 8192, 8, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_static(None, P(512), 64, 64, 8, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_static(P(256), P(512), 64, 64, 5, None) == _lib.CCL_ERR_INVALID_ARG


@pytest.mark.gpu
def test_two_calls_in_a_row_match_ccl_label():
    torch = pytest.importorskip("torch")
    lib = _lib.load()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    cases = [(synthetic.bernoulli(1500, 2100, 0.5, 1, cfg_id=50), 8),
             (synthetic.bernoulli(777, 513, 0.6, 2, cfg_id=50), 4),
             (synthetic.bernoulli(4096, 4096, 0.45, 3, cfg_id=50), 8)]
    for img, conn in cases:
        h, w = img.shape
        dimg = torch.from_numpy(img).to(dev)
        # reference: the allocating entry point with its own workspace
        ref = torch.empty((h, w), dtype=torch.int32, device=dev)
        ws = torch.empty(lib.ccl_workspace_bytes(h, w, conn), dtype=torch.uint8, device=dev)
        assert lib.ccl_label(dimg.data_ptr(), ref.data_ptr(), h, w, conn, ws.data_ptr(),
                             ws.numel(), stream.cuda_stream) == _lib.CCL_OK
        # two calls in a row on the shared static scratch
        outs = []
        for _ in range(2):
            out = torch.full((h, w), -3, dtype=torch.int32, device=dev)
            assert lib.ccl_label_static(dimg.data_ptr(), out.data_ptr(), h, w, conn,
                                        stream.cuda_stream) == _lib.CCL_OK
            outs.append(out)
        assert lib.ccl_sync(stream.cuda_stream) == _lib.CCL_OK
        want = ref.cpu().numpy()
        for out in outs:
            np.testing.assert_array_equal(out.cpu().numpy(), want)
