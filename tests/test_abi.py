"""The C-ABI library loads, exports every declared entry point and validates
arguments on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import oracle
import paper_1708_08180_gb300 as ccl
from paper_1708_08180_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for path in HEADERS:
        src = open(path).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(ccl_[a-z0-9_]+)\s*\(", src):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("ccl_label", "ccl_label_batched", "ccl_server_create", "ccl_server_submit",
                     "ccl_server_wait", "ccl_server_destroy", "ccl_workspace_bytes",
                     "ccl_status_string", "ccl_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ccl_[a-z0-9_]+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing


def test_status_strings(lib):
    assert ccl.ccl_status_string(0) == "CCL_OK"
    assert ccl.ccl_status_string(1) == "CCL_ERR_INVALID_ARG"
    assert ccl.ccl_status_string(8) == "CCL_ERR_PENDING"
    assert ccl.ccl_status_string(99) == "CCL_ERR_UNKNOWN"


def test_tile_table_and_workspace_sizes(lib):
    assert ccl.ccl_default_tile_width(8192, 8192, 8) == 256
    assert ccl.ccl_default_tile_width(64, 40, 8) == 64
    assert ccl.ccl_default_tile_width(64, 7, 4) == 32
    assert ccl.ccl_default_tile_width(0, 7, 4) == 0
    assert ccl.ccl_default_tile_width(5, 7, 6) == 0
    # bits (H * ceil(W/32) words) + per-tile records; grows with the image
    a = ccl.ccl_workspace_bytes(1024, 1024, 8)
    b = ccl.ccl_workspace_bytes(2048, 2048, 8)
    assert 0 < a < b
    assert a % 256 == 0
    assert ccl.ccl_workspace_bytes(0, 5, 8) == 0
    assert ccl.ccl_workspace_bytes(5, 5, 5) == 0
    assert ccl.ccl_workspace_bytes_tiled(5, 5, 8, 48) == 0
    assert ccl.ccl_workspace_bytes(46341, 46341, 8) == 0      # > 2^31 - 2 pixels
    assert ccl.ccl_workspace_bytes(1, 2147483646, 4) > 0
    assert ccl.ccl_batched_workspace_bytes([(64, 64), (100, 3000)], 8) > 0
    # volumes: bits + per-brick records + per-brick forest slots; 0 when invalid
    v1 = ccl.ccl_workspace_bytes3d(16, 16, 32, 6)
    assert v1 > 0 and v1 % 256 == 0
    assert ccl.ccl_workspace_bytes3d(17, 16, 32, 6) > v1          # a second brick layer
    assert ccl.ccl_workspace_bytes3d(16, 16, 32, 4) == 0
    assert ccl.ccl_workspace_bytes3d(1291, 1291, 1291, 26) == 0   # > 2^31 - 2 voxels
    assert ccl.ccl_workspace_bytes3d(1 << 27, 1, 1, 6) == 0       # > 2^22 bricks
    assert ccl.ccl_workspace_bytes3d(1 << 26, 1, 1, 6) > 0


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw,tile", [((8, 8), (4, 2)), ((7, 9), (4, 2)), ((12, 10), (3, 5)),
                                     ((16, 32), (32, 4)), ((40, 70), (32, 16)), ((1, 9), (2, 2))])
def test_seam_pair_count_matches_enumeration(hw, tile, conn, lib):
    h, w = hw
    tw, th = tile
    assert ccl.ccl_seam_pair_count(h, w, conn, tw, th) == len(oracle.seam_pairs(h, w, conn, tw, th))


def test_host_validation_rejects_before_enqueueing(lib):
    P = ctypes.c_void_p
    # null pointers, bad sizes and bad connectivity fail before any CUDA call
    assert lib.ccl_label(None, None, 4, 4, 8, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label(P(256), P(512), 0, 4, 8, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label(P(256), P(512), 4, 4, 6, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label(P(256), P(512), 46341, 46341, 8, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_tiled(P(256), P(512), 4, 4, 8, 48, 0, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_tiled(P(256), P(512), 4, 4, 8, 32, 6, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    # a caller workspace that is too small or misaligned
    need = ccl.ccl_workspace_bytes(64, 64, 8)
    assert lib.ccl_label(P(256), P(512), 64, 64, 8, P(4096), need - 1, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label(P(256), P(512), 64, 64, 8, P(4096 + 16), need, None) == _lib.CCL_ERR_INVALID_ARG
    # every-region labelling: the level list is checked first, then the image
    lv = (ctypes.c_uint8 * 3)(0, 1, 1)
    addr = ctypes.addressof(lv)
    assert lib.ccl_label_regions(P(256), P(512), 4, 4, 8, None, 1, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_regions(P(256), P(512), 4, 4, 8, addr, 0, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_regions(P(256), P(512), 4, 4, 8, addr, 257, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_regions(P(256), P(512), 4, 4, 8, addr, 3, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG                                  # level 1 repeated
    assert lib.ccl_label_regions(None, P(512), 4, 4, 8, addr, 2, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_regions(P(256), P(512), 4, 4, 6, addr, 2, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG
    # volumes: connectivity 6, 18, 26 only; at most 2^31 - 2 voxels and 2^22 bricks
    assert lib.ccl_label3d(None, P(512), 2, 2, 2, 6, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label3d(P(256), P(512), 2, 2, 2, 8, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label3d(P(256), P(512), 0, 2, 2, 6, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label3d(P(256), P(512), 2048, 1024, 1024, 26, None, 0, None) == \
        _lib.CCL_ERR_INVALID_ARG
    need3 = ccl.ccl_workspace_bytes3d(20, 20, 40, 26)
    assert lib.ccl_label3d(P(256), P(512), 20, 20, 40, 26, P(4096), need3 - 1, None) == \
        _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label3d(P(256), P(512), 20, 20, 40, 26, P(4096 + 64), need3, None) == \
        _lib.CCL_ERR_INVALID_ARG
    arr = (_lib.ccl_image * 1)()
    assert lib.ccl_label_batched(arr, 1, 8, None, 0, None) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_label_batched(arr, 0, 8, None, 0, None) == _lib.CCL_ERR_INVALID_ARG


def test_server_argument_errors(lib):
    h = ctypes.c_void_p()
    assert lib.ccl_server_create(None, ctypes.byref(h)) == _lib.CCL_ERR_INVALID_ARG
    cfg = _lib.ccl_server_config(0, 0, 0, 6, 0)
    assert lib.ccl_server_create(ctypes.byref(cfg), ctypes.byref(h)) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_server_wait(None, 1, 0) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_server_destroy(None) == _lib.CCL_ERR_INVALID_ARG


def test_server_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    cfg = _lib.ccl_server_config(1 << 20, 4, 2, 8, 0)
    st = lib.ccl_server_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st in (_lib.CCL_ERR_CUDA, _lib.CCL_ERR_INVALID_ARG)
    assert not h.value


def test_tile_table_get_set_roundtrip(lib):
    n = _lib.CCL_TILE_CLASSES
    before = ccl.ccl_get_tile_table(8)
    assert len(before) == n and all(len(r) == n for r in before)
    # effective widths never exceed the class's need (<= 64 wide -> <= 64)
    assert all(w <= 64 for w in [row[0] for row in before])
    try:
        table = [[32] * n for _ in range(n)]
        ccl.ccl_set_tile_table(8, table)
        assert ccl.ccl_default_tile_width(4096, 4096, 8) == 32
        assert ccl.ccl_default_tile_width(4096, 4096, 4) == before_4096(lib)
        with pytest.raises(ccl.CclError):
            ccl.ccl_set_tile_table(8, [[48] * n for _ in range(n)])
        assert ccl.ccl_default_tile_width(4096, 4096, 8) == 32   # nothing installed on error
    finally:
        ccl.ccl_set_tile_table(8, [[256] * n for _ in range(n)])
    # workspace sizing covers every tile width
    for tw in (32, 64, 128, 256):
        assert ccl.ccl_workspace_bytes_tiled(1000, 3000, 8, tw) <= ccl.ccl_workspace_bytes(1000, 3000, 8)


def before_4096(lib):
    return lib.ccl_default_tile_width(4096, 4096, 4)


def test_binding_rejects_host_tensors_and_bad_shapes(lib):
    """The Python binding checks tensors before any library call: host tensors
    and wrong dtypes or ranks raise TypeError."""
    import torch

    img = torch.zeros((8, 8), dtype=torch.uint8)
    vol = torch.zeros((4, 4, 4), dtype=torch.uint8)
    for call in (lambda: ccl.ccl_label(img, 8), lambda: ccl.ccl_label_regions(img, (0, 1), 8),
                 lambda: ccl.ccl_label3d(vol, 26), lambda: ccl.ccl_label3d(img, 6),
                 lambda: ccl.ccl_label(img.float(), 8)):
        with pytest.raises(TypeError):
            call()


def test_failure_injection_hooks_validate_and_fail_allocation_on_host(lib):
    """An injected allocation failure makes a call that needs a library-owned
    workspace return CCL_ERR_OOM before any CUDA call (so this runs without a
    GPU); negative counts and budgets are refused."""
    P = ctypes.c_void_p
    assert lib.ccl_inject_alloc_failures(-1) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_set_hop_budget(-1, 0) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_set_hop_budget(0, -5) == _lib.CCL_ERR_INVALID_ARG
    assert lib.ccl_set_hop_budget(0, 0) == _lib.CCL_OK
    assert lib.ccl_inject_alloc_failures(2) == _lib.CCL_OK
    try:
        assert lib.ccl_label(P(256), P(512), 64, 64, 8, None, 0, None) == _lib.CCL_ERR_OOM
        assert lib.ccl_label_tiled(P(256), P(512), 64, 64, 4, 32, 0, None, 0, None) == \
            _lib.CCL_ERR_OOM
    finally:
        assert lib.ccl_inject_alloc_failures(0) == _lib.CCL_OK


def test_binding_rejects_bad_workspace_and_outputs_without_gpu(lib):
    """Host-memory images are refused before any output or workspace check."""
    import torch

    img = torch.zeros((8, 8), dtype=torch.uint8)
    with pytest.raises(TypeError):
        ccl.ccl_label_static(img, 8)
    with pytest.raises(TypeError):
        ccl.ccl_label_batched([img], 8)
    with pytest.raises(TypeError):
        ccl.ccl_component_stats(torch.zeros((8, 8), dtype=torch.int32), 4)
