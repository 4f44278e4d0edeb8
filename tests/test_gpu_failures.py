"""Failure detection on the GPU, without faulting it: a union-find walk made to
run out of hops (a lowered hop budget) must end its kernel and be reported by
ccl_sync as CCL_ERR_TIMEOUT, after which the context is still usable; an
injected allocation failure must return CCL_ERR_OOM with nothing enqueued; and
the binding must reject caller tensors it cannot pass to the library."""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402
from paper_1708_08180_gb300 import _lib  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("which", ["global", "both"])
def test_exhausted_hop_budget_is_reported_and_recoverable(conn, which):
    """The serpentine's single component crosses every tile seam: every tile
    but the first holds a border root whose global root is elsewhere, and the
    link kernel walks it up the global forest, so a budget of one hop runs out
    for certain.  (Walks in a tile's shared-memory forest run only for unions
    that lose a race or overflow the union queue, so the shared-memory budget
    is lowered together with the global one, not alone.)"""
    img = synthetic.serpentine(4096, 4096)
    dimg = torch.from_numpy(img).to(DEV)
    out = torch.zeros((4096, 4096), dtype=torch.int32, device=DEV)
    ws = torch.empty(ccl.ccl_workspace_bytes(4096, 4096, conn), dtype=torch.uint8, device=DEV)
    ccl.ccl_sync()
    try:
        ccl.ccl_set_hop_budget(1 if which == "both" else 0, 1)
        ccl.ccl_label(dimg, conn, out=out, ws=ws)
        with pytest.raises(ccl.CclError) as e:
            ccl.ccl_sync()
        assert e.value.status == _lib.CCL_ERR_TIMEOUT
    finally:
        ccl.ccl_set_hop_budget(0, 0)
    # the error word was cleared by the report; the next call is exact
    ccl.ccl_label(dimg, conn, out=out, ws=ws)
    ccl.ccl_sync()
    assert np.array_equal(out.cpu().numpy(), oracle.label(img, conn))


def test_injected_allocation_failure_enqueues_nothing():
    img = synthetic.bernoulli(300, 400, 0.5, 1, cfg_id=29)
    dimg = torch.from_numpy(img).to(DEV)
    out = torch.full((300, 400), -9, dtype=torch.int32, device=DEV)
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    ccl.ccl_shutdown()            # no library workspace cached: the call must allocate
    ccl.ccl_inject_alloc_failures(1)
    try:
        st = lib.ccl_label(dimg.data_ptr(), out.data_ptr(), 300, 400, 8, None, 0, stream)
        assert st == _lib.CCL_ERR_OOM
        ccl.ccl_sync()
        assert bool((out == -9).all()), "a failed call wrote its output"
    finally:
        ccl.ccl_inject_alloc_failures(0)
    st = lib.ccl_label(dimg.data_ptr(), out.data_ptr(), 300, 400, 8, None, 0, stream)
    assert st == _lib.CCL_OK
    ccl.ccl_sync()
    assert np.array_equal(out.cpu().numpy(), oracle.label(img, 8))


def test_binding_rejects_bad_outputs_and_workspaces():
    img = torch.zeros((16, 24), dtype=torch.uint8, device=DEV)
    good = torch.empty((16, 24), dtype=torch.int32, device=DEV)
    bad_outs = [torch.empty((16, 24), dtype=torch.int32),             # host memory
                torch.empty((16, 24), dtype=torch.int64, device=DEV),  # dtype
                torch.empty((24, 16), dtype=torch.int32, device=DEV),  # shape
                torch.empty((24, 16), dtype=torch.int32, device=DEV).t()]   # not contiguous
    for o in bad_outs:
        for call in (lambda: ccl.ccl_label(img, 8, out=o), lambda: ccl.ccl_label_tiled(img, 8, 32, out=o),
                     lambda: ccl.ccl_label_static(img, 8, out=o),
                     lambda: ccl.ccl_label_regions(img, (0, 1), 8, out=o),
                     lambda: ccl.ccl_label_batched([img], 8, outs=[o])):
            with pytest.raises(TypeError):
                call()
    need = ccl.ccl_workspace_bytes(16, 24, 8)
    for ws in (torch.empty(need, dtype=torch.uint8), torch.empty(need // 4 + 1, dtype=torch.int32, device=DEV)):
        with pytest.raises(TypeError):
            ccl.ccl_label(img, 8, out=good, ws=ws)
    ccl.ccl_sync()
