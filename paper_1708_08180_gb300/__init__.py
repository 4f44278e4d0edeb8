"""GB300-native union-find connected-components labelling (CCL).

Python binding over the C ABI of ``libccl.so`` (``include/ccl.h``): argument
marshalling only -- every step of the labelling runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.

    >>> import torch, paper_1708_08180_gb300 as ccl
    >>> img = (torch.rand(1024, 1024, device="cuda") < 0.5).to(torch.uint8)
    >>> labels = ccl.label(img, conn=8)   # int32, 0 = background,
    ...                                   # 1 + smallest raster index of the component

Functions named ``ccl_*`` mirror the C entry points one to one.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, List, Optional, Sequence

from ._lib import (CCL_ERR_PENDING, CCL_ERR_TIMEOUT, CCL_FLAG_LOCAL_ONLY, CCL_OK, CclError,
                   ccl_image, ccl_server_config, check, load, status_string)

__all__ = [
    "CclError", "CCL_FLAG_LOCAL_ONLY", "label", "label_batched", "ccl_label", "ccl_label_tiled",
    "ccl_label_batched", "ccl_workspace_bytes", "ccl_workspace_bytes_tiled",
    "ccl_batched_workspace_bytes", "ccl_default_tile_width", "ccl_seam_pair_count", "ccl_sync",
    "ccl_shutdown", "ccl_status_string", "ccl_set_phase_events", "ccl_label_static", "Server",
    "ccl_get_tile_table", "ccl_set_tile_table", "ccl_autotune", "load",
    "ccl_stats_workspace_bytes", "ccl_component_stats", "component_stats", "COMPONENT_FIELDS",
    "ccl_label_regions", "label_regions", "ccl_label3d", "ccl_workspace_bytes3d", "label3d",
    "ccl_set_hop_budget", "ccl_inject_alloc_failures", "ccl_label_with_stats",
    "ccl_workspace_bytes_with_stats", "label_with_stats",
]

# ccl_component as int32 words: label, count, xmin, ymin, xmax, ymax, then the
# int64 sums of x and y (two words each)
COMPONENT_WORDS = 10
COMPONENT_FIELDS = ("label", "count", "xmin", "ymin", "xmax", "ymax", "sum_x", "sum_y")


def _torch():
    import torch

    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check_img(img):
    torch = _torch()
    if not isinstance(img, torch.Tensor) or not img.is_cuda:
        raise TypeError("image must be a CUDA tensor")
    if img.dtype != torch.uint8 or img.dim() != 2 or not img.is_contiguous():
        raise TypeError("image must be a contiguous 2-D uint8 tensor")


def _check_out(out, shape, device, what: str = "out"):
    """A caller-given output must be a contiguous int32 CUDA tensor of the given
    shape on the input's device: the library writes through its pointer."""
    torch = _torch()
    if not isinstance(out, torch.Tensor) or not out.is_cuda or out.device != device:
        raise TypeError(f"{what} must be a CUDA tensor on {device}")
    if out.dtype != torch.int32 or tuple(out.shape) != tuple(shape) or not out.is_contiguous():
        raise TypeError(f"{what} must be a contiguous int32 tensor of shape {tuple(shape)}")


def _check_ws(ws, device):
    """A caller-given workspace must be a contiguous uint8 CUDA tensor on the
    input's device; its byte size is passed to the library, which checks it."""
    torch = _torch()
    if not isinstance(ws, torch.Tensor) or not ws.is_cuda or ws.device != device:
        raise TypeError(f"ws must be a CUDA tensor on {device}")
    if ws.dtype != torch.uint8 or not ws.is_contiguous():
        raise TypeError("ws must be a contiguous uint8 tensor")


def ccl_status_string(status: int) -> str:
    return status_string(status)


def ccl_default_tile_width(height: int, width: int, conn: int) -> int:
    return int(load().ccl_default_tile_width(height, width, conn))


def ccl_workspace_bytes(height: int, width: int, conn: int) -> int:
    return int(load().ccl_workspace_bytes(height, width, conn))


def ccl_workspace_bytes_tiled(height: int, width: int, conn: int, tile_w: int) -> int:
    return int(load().ccl_workspace_bytes_tiled(height, width, conn, tile_w))


def ccl_seam_pair_count(height: int, width: int, conn: int, tile_w: int, tile_h: int) -> int:
    return int(load().ccl_seam_pair_count(height, width, conn, tile_w, tile_h))


def _workspace(nbytes: int, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def ccl_label_tiled(img, conn: int = 8, tile_w: int = 0, flags: int = 0, out=None, ws=None,
                    stream=None):
    """Label ``img`` (CUDA uint8, H x W) into ``out`` (CUDA int32, H x W).

    ``ws``: a CUDA uint8 tensor of at least ``ccl_workspace_bytes_tiled`` bytes
    (allocated here when None).  Enqueued on ``stream`` (default: current)."""
    torch = _torch()
    _check_img(img)
    h, w = img.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.int32, device=img.device)
    else:
        _check_out(out, (h, w), img.device)
    need = ccl_workspace_bytes_tiled(h, w, conn, tile_w)
    if need == 0:
        raise CclError(1, "ccl_workspace_bytes_tiled")
    if ws is None:
        ws = _workspace(need, img.device)
    else:
        _check_ws(ws, img.device)
    with torch.cuda.device(img.device):
        st = load().ccl_label_tiled(img.data_ptr(), out.data_ptr(), h, w, conn, tile_w, flags,
                                    ws.data_ptr(), ws.numel(), _stream_handle(stream))
    check(st, "ccl_label_tiled")
    return out


def ccl_label(img, conn: int = 8, out=None, ws=None, stream=None):
    """Label one image with the default tile shape (see ``ccl_label_tiled``)."""
    torch = _torch()
    _check_img(img)
    h, w = img.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.int32, device=img.device)
    else:
        _check_out(out, (h, w), img.device)
    need = ccl_workspace_bytes(h, w, conn)
    if need == 0:
        raise CclError(1, "ccl_workspace_bytes")
    if ws is None:
        ws = _workspace(need, img.device)
    else:
        _check_ws(ws, img.device)
    with torch.cuda.device(img.device):
        st = load().ccl_label(img.data_ptr(), out.data_ptr(), h, w, conn, ws.data_ptr(),
                              ws.numel(), _stream_handle(stream))
    check(st, "ccl_label")
    return out


def ccl_label_regions(img, levels: Sequence[int], conn: int = 8, out=None, ws=None,
                      stream=None):
    """Label every equal-value region of ``img`` whose byte value is in
    ``levels`` (distinct values 0..255): 1 + the smallest raster index of the
    region, 0 for pixels of other values.  One three-phase pass per level on
    ``stream``; ``ws`` as for ``ccl_label``."""
    torch = _torch()
    _check_img(img)
    h, w = img.shape
    lv = [int(v) for v in levels]
    if not lv or any(v < 0 or v > 255 for v in lv):
        raise ValueError("levels must be 1..256 byte values")
    if out is None:
        out = torch.empty((h, w), dtype=torch.int32, device=img.device)
    else:
        _check_out(out, (h, w), img.device)
    need = ccl_workspace_bytes(h, w, conn)
    if need == 0:
        raise CclError(1, "ccl_workspace_bytes")
    if ws is None:
        ws = _workspace(need, img.device)
    else:
        _check_ws(ws, img.device)
    host_levels = (ctypes.c_uint8 * len(lv))(*lv)
    with torch.cuda.device(img.device):
        st = load().ccl_label_regions(img.data_ptr(), out.data_ptr(), h, w, conn,
                                      ctypes.addressof(host_levels), len(lv), ws.data_ptr(),
                                      ws.numel(), _stream_handle(stream))
    check(st, "ccl_label_regions")
    return out


def label_regions(img, levels: Sequence[int] = (0, 1), conn: int = 8):
    """Every region of ``img`` whose value is in ``levels``, background
    included when 0 is listed (see ``ccl_label_regions``)."""
    return ccl_label_regions(img, levels, conn)


def ccl_workspace_bytes3d(depth: int, height: int, width: int, conn: int) -> int:
    return int(load().ccl_workspace_bytes3d(depth, height, width, conn))


def ccl_label3d(vol, conn: int = 26, out=None, ws=None, stream=None):
    """Label a 3-D volume ``vol`` (CUDA uint8, D x H x W, index [z, y, x]) into
    ``out`` (CUDA int32, same shape): 0 for background, 1 + the smallest voxel
    index ``(z*H + y)*W + x`` of the component.  ``conn``: 6, 18 or 26.  ``ws``:
    a CUDA uint8 tensor of at least ``ccl_workspace_bytes3d`` bytes (allocated
    here when None).  Enqueued on ``stream`` (default: current)."""
    torch = _torch()
    if not isinstance(vol, torch.Tensor) or not vol.is_cuda:
        raise TypeError("volume must be a CUDA tensor")
    if vol.dtype != torch.uint8 or vol.dim() != 3 or not vol.is_contiguous():
        raise TypeError("volume must be a contiguous 3-D uint8 tensor")
    d, h, w = vol.shape
    if out is None:
        out = torch.empty((d, h, w), dtype=torch.int32, device=vol.device)
    else:
        _check_out(out, (d, h, w), vol.device)
    need = ccl_workspace_bytes3d(d, h, w, conn)
    if need == 0:
        raise CclError(1, "ccl_workspace_bytes3d")
    if ws is None:
        ws = _workspace(need, vol.device)
    else:
        _check_ws(ws, vol.device)
    with torch.cuda.device(vol.device):
        st = load().ccl_label3d(vol.data_ptr(), out.data_ptr(), d, h, w, conn, ws.data_ptr(),
                                ws.numel(), _stream_handle(stream))
    check(st, "ccl_label3d")
    return out


def label3d(vol, conn: int = 26):
    """Canonical labels of a 3-D volume (see ``ccl_label3d``)."""
    return ccl_label3d(vol, conn)


def ccl_label_static(img, conn: int = 8, out=None, stream=None):
    """Label one image without allocating device memory in the library: the
    scratch is the library's fixed device array (see ``include/ccl.h``).  Only
    ``out`` is allocated here when None; images whose workspace exceeds
    ``CCL_STATIC_SCRATCH_BYTES`` raise.  Calls that overlap on the GPU race on
    the shared scratch, so keep them on one stream."""
    torch = _torch()
    _check_img(img)
    h, w = img.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.int32, device=img.device)
    else:
        _check_out(out, (h, w), img.device)
    with torch.cuda.device(img.device):
        st = load().ccl_label_static(img.data_ptr(), out.data_ptr(), h, w, conn,
                                     _stream_handle(stream))
    check(st, "ccl_label_static")
    return out


def _image_array(imgs, outs):
    arr = (ccl_image * len(imgs))()
    for k, (im, o) in enumerate(zip(imgs, outs)):
        arr[k].d_img = im.data_ptr()
        arr[k].d_labels = o.data_ptr()
        arr[k].height = im.shape[0]
        arr[k].width = im.shape[1]
    return arr


def ccl_batched_workspace_bytes(shapes: Sequence, conn: int = 8) -> int:
    """Workspace bytes for a batch given ``[(h, w), ...]`` or tensors."""
    arr = (ccl_image * len(shapes))()
    for k, s in enumerate(shapes):
        h, w = (s.shape if hasattr(s, "shape") else s)
        arr[k].d_img = 256
        arr[k].d_labels = 256
        arr[k].height, arr[k].width = int(h), int(w)
    return int(load().ccl_batched_workspace_bytes(arr, len(shapes), conn))


def ccl_label_batched(imgs: Sequence, conn: int = 8, outs: Optional[Sequence] = None, ws=None,
                      stream=None) -> List:
    """Label a list of CUDA uint8 images of any sizes in one batched launch."""
    torch = _torch()
    if len(imgs) == 0:
        return []
    for im in imgs:
        _check_img(im)
    dev = imgs[0].device
    for im in imgs:
        if im.device != dev:
            raise TypeError("every image of a batch must be on the same device")
    if outs is None:
        outs = [torch.empty(tuple(im.shape), dtype=torch.int32, device=im.device) for im in imgs]
    if len(outs) != len(imgs):
        raise ValueError("outs must hold one tensor per image")
    for im, o in zip(imgs, outs):
        _check_out(o, tuple(im.shape), dev, "each of outs")
    arr = _image_array(imgs, outs)
    need = int(load().ccl_batched_workspace_bytes(arr, len(imgs), conn))
    if need == 0:
        raise CclError(1, "ccl_batched_workspace_bytes")
    if ws is None:
        ws = _workspace(need, dev)
    else:
        _check_ws(ws, dev)
    with torch.cuda.device(dev):
        st = load().ccl_label_batched(arr, len(imgs), conn, ws.data_ptr(), ws.numel(),
                                      _stream_handle(stream))
    check(st, "ccl_label_batched")
    return list(outs)


def ccl_sync(stream=None) -> None:
    """Wait for ``stream`` and raise if a device-side bounded loop ran out."""
    check(load().ccl_sync(_stream_handle(stream)), "ccl_sync")


def ccl_set_phase_events(events) -> None:
    """Arm the per-kernel timing hook for this thread's next ccl_label call:
    ``events`` is 4 ``torch.cuda.Event(enable_timing=True)`` (or None)."""
    if events is None:
        load().ccl_set_phase_events(None)
        return
    for e in events:
        if not int(e.cuda_event):      # torch creates the CUDA event on first record
            e.record()
    arr = (ctypes.c_void_p * 4)(*[int(e.cuda_event) for e in events])
    load().ccl_set_phase_events(arr)


def ccl_get_tile_table(conn: int = 8) -> List[List[int]]:
    """The size-class table as rows (height class) of tile widths (width class)."""
    from ._lib import CCL_TILE_CLASSES as n

    arr = (ctypes.c_int * (n * n))()
    check(load().ccl_get_tile_table(conn, arr), "ccl_get_tile_table")
    return [list(arr[r * n:(r + 1) * n]) for r in range(n)]


def ccl_set_tile_table(conn: int, table: Sequence[Sequence[int]]) -> None:
    from ._lib import CCL_TILE_CLASSES as n

    flat = [int(v) for row in table for v in row]
    if len(flat) != n * n:
        raise ValueError(f"table must be {n}x{n}")
    arr = (ctypes.c_int * (n * n))(*flat)
    check(load().ccl_set_tile_table(conn, arr), "ccl_set_tile_table")


def ccl_autotune(conn: int = 8, reps: int = 3, stream=None) -> List[List[int]]:
    """Measure and install the fastest tile width per size class; returns the table."""
    check(load().ccl_autotune(conn, reps, _stream_handle(stream)), "ccl_autotune")
    return ccl_get_tile_table(conn)


def ccl_shutdown() -> None:
    check(load().ccl_shutdown(), "ccl_shutdown")


def ccl_set_hop_budget(smem_hops: int = 0, global_hops: int = 0) -> None:
    """Failure injection for tests: the union-find hop budgets of the 2-D
    kernels (0 = default); a walk that runs out makes ccl_sync raise
    CCL_ERR_TIMEOUT."""
    check(load().ccl_set_hop_budget(smem_hops, global_hops), "ccl_set_hop_budget")


def ccl_inject_alloc_failures(count: int) -> None:
    """Failure injection for tests: the next ``count`` library-owned workspace
    allocations fail with CCL_ERR_OOM (0 clears them)."""
    check(load().ccl_inject_alloc_failures(count), "ccl_inject_alloc_failures")


def ccl_stats_workspace_bytes(height: int, width: int, max_comps: int) -> int:
    return int(load().ccl_stats_workspace_bytes(height, width, max_comps))


def ccl_component_stats(labels, max_comps: int, comps=None, ncomps=None, ws=None, stream=None):
    """Enqueue the statistics of every component of a canonical CUDA int32
    label image.  ``comps``: CUDA int32 tensor (max_comps, 10) receiving the
    records (COMPONENT_FIELDS, the sums as int64 word pairs), in label order;
    ``ncomps``: CUDA int32 tensor (1,) receiving the component count.  Both
    are allocated here when None.  Returns (comps, ncomps)."""
    torch = _torch()
    if not isinstance(labels, torch.Tensor) or not labels.is_cuda or labels.dtype != torch.int32 \
            or labels.dim() != 2 or not labels.is_contiguous():
        raise TypeError("labels must be a contiguous 2-D int32 CUDA tensor")
    h, w = labels.shape
    if comps is None:
        comps = torch.empty((max(max_comps, 1), COMPONENT_WORDS), dtype=torch.int32,
                            device=labels.device)
    elif (not isinstance(comps, torch.Tensor) or not comps.is_cuda or comps.device != labels.device
          or comps.dtype != torch.int32 or comps.dim() != 2 or comps.shape[1] != COMPONENT_WORDS
          or comps.shape[0] < max_comps or not comps.is_contiguous()):
        raise TypeError(f"comps must be a contiguous int32 CUDA tensor (>= max_comps, "
                        f"{COMPONENT_WORDS}) on {labels.device}")
    if ncomps is None:
        ncomps = torch.empty(1, dtype=torch.int32, device=labels.device)
    else:
        _check_out(ncomps, (1,), labels.device, "ncomps")
    if ws is None:
        ws = _workspace(ccl_stats_workspace_bytes(h, w, max_comps), labels.device)
    else:
        _check_ws(ws, labels.device)
    check(load().ccl_component_stats(labels.data_ptr(), h, w, comps.data_ptr(), max_comps,
                                     ncomps.data_ptr(), ws.data_ptr(), ws.numel(),
                                     _stream_handle(stream)), "ccl_component_stats")
    return comps, ncomps


def component_stats(labels) -> dict:
    """Statistics of every component of a canonical CUDA label image (blocking):
    a dict of CPU numpy arrays keyed by COMPONENT_FIELDS, in label order."""
    import numpy as np

    _, ncomps = ccl_component_stats(labels, 0)         # the count first
    n = int(ncomps.item())
    comps, ncomps = ccl_component_stats(labels, n)     # then the records
    ccl_sync()
    return _records_to_dict(comps.cpu().numpy(), n)


def ccl_workspace_bytes_with_stats(height: int, width: int, conn: int) -> int:
    return int(load().ccl_workspace_bytes_with_stats(height, width, conn))


def ccl_label_with_stats(img, conn: int = 8, max_comps: int = 0, out=None, comps=None, ncomps=None,
                         ws=None, stream=None):
    """Label ``img`` and gather every component's statistics in the same pass.
    ``comps``: CUDA int32 tensor (>= max_comps, 10) receiving records
    (COMPONENT_FIELDS, sums as int64 word pairs) in unspecified order;
    ``ncomps``: CUDA int32 tensor (1,) receiving the component count.  Returns
    (out, comps, ncomps); tensors not given are allocated here."""
    torch = _torch()
    _check_img(img)
    h, w = img.shape
    if out is None:
        out = torch.empty((h, w), dtype=torch.int32, device=img.device)
    else:
        _check_out(out, (h, w), img.device)
    if comps is None:
        comps = torch.empty((max(max_comps, 1), COMPONENT_WORDS), dtype=torch.int32,
                            device=img.device)
    elif (not isinstance(comps, torch.Tensor) or not comps.is_cuda or comps.device != img.device
          or comps.dtype != torch.int32 or comps.dim() != 2 or comps.shape[1] != COMPONENT_WORDS
          or comps.shape[0] < max_comps or not comps.is_contiguous()):
        raise TypeError(f"comps must be a contiguous int32 CUDA tensor (>= max_comps, "
                        f"{COMPONENT_WORDS}) on {img.device}")
    if ncomps is None:
        ncomps = torch.empty(1, dtype=torch.int32, device=img.device)
    else:
        _check_out(ncomps, (1,), img.device, "ncomps")
    need = ccl_workspace_bytes_with_stats(h, w, conn)
    if need == 0:
        raise CclError(1, "ccl_workspace_bytes_with_stats")
    if ws is None:
        ws = _workspace(need, img.device)
    else:
        _check_ws(ws, img.device)
    with torch.cuda.device(img.device):
        st = load().ccl_label_with_stats(img.data_ptr(), out.data_ptr(), h, w, conn,
                                         comps.data_ptr(), max_comps, ncomps.data_ptr(),
                                         ws.data_ptr(), ws.numel(), _stream_handle(stream))
    check(st, "ccl_label_with_stats")
    return out, comps, ncomps


def _records_to_dict(raw, n: int) -> dict:
    import numpy as np

    raw = raw[:n]
    out = {f: raw[:, k].astype(np.int64) for k, f in enumerate(COMPONENT_FIELDS[:6])}
    wide = raw[:, 6:10].copy().view(np.int64)
    out["sum_x"] = wide[:, 0]
    out["sum_y"] = wide[:, 1]
    return out


def label_with_stats(img, conn: int = 8):
    """Labels and the statistics of every component, in one pass (blocking):
    (labels, dict of CPU numpy arrays keyed by COMPONENT_FIELDS, in label
    order).  The record capacity starts at one per 64 pixels and is raised to
    the exact count if that is exceeded."""
    import numpy as np

    h, w = img.shape
    cap = min(h * w // 2 + 2, h * w // 64 + 1024)
    out, comps, ncomps = ccl_label_with_stats(img, conn, cap)
    ccl_sync()
    n = int(ncomps.item())
    if n > cap:
        out, comps, ncomps = ccl_label_with_stats(img, conn, n, out=out)
        ccl_sync()
    st = _records_to_dict(comps.cpu().numpy(), n)
    order = np.argsort(st["label"], kind="stable")
    return out, {k: v[order] for k, v in st.items()}


def label(img, conn: int = 8, tile_w: int = 0):
    """Canonical labels of a CUDA uint8 image (blocking convenience wrapper)."""
    out = ccl_label_tiled(img, conn, tile_w)
    ccl_sync()
    return out


def label_batched(imgs: Iterable, conn: int = 8):
    outs = ccl_label_batched(list(imgs), conn)
    ccl_sync()
    return outs


class Server:
    """Continuous-batching server over host buffers (``ccl_server_*``).

    ``submit`` takes a contiguous host uint8 array/tensor and a host int32
    output of the same shape (pinned memory recommended); both must stay alive
    until ``wait``/``poll`` reports completion."""

    def __init__(self, conn: int = 8, hbm_budget_bytes: int = 0, max_batch: int = 0,
                 max_inflight: int = 0, device: int = 0):
        cfg = ccl_server_config(hbm_budget_bytes, max_batch, max_inflight, conn, device)
        h = ctypes.c_void_p()
        check(load().ccl_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ccl_server_create")
        self._h = h
        self._keep = {}

    @staticmethod
    def _ptr(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data

    def submit(self, img, out) -> int:
        h, w = img.shape
        rid = ctypes.c_uint64()
        st = load().ccl_server_submit(self._h, self._ptr(img), h, w, self._ptr(out),
                                      ctypes.byref(rid))
        check(st, "ccl_server_submit")
        self._keep[rid.value] = (img, out)
        return rid.value

    def wait(self, rid: int, timeout_ms: int = -1) -> None:
        st = load().ccl_server_wait(self._h, rid, timeout_ms)
        if st != CCL_ERR_TIMEOUT:
            self._keep.pop(rid, None)
        check(st, "ccl_server_wait")

    def poll(self, rid: int) -> bool:
        st = load().ccl_server_poll(self._h, rid)
        if st == CCL_ERR_PENDING:
            return False
        self._keep.pop(rid, None)
        check(st, "ccl_server_poll")
        return True

    def stats(self) -> dict:
        p50, p99, gp = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        done, rej = ctypes.c_uint64(), ctypes.c_uint64()
        check(load().ccl_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99),
                                      ctypes.byref(gp), ctypes.byref(done), ctypes.byref(rej)),
              "ccl_server_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "gpix_per_s": gp.value,
                "completed": done.value, "rejected": rej.value}

    def timing(self) -> dict:
        """Mean per-batch host-to-device copy, labelling and device-to-host copy
        times (ms, CUDA events) over the batches completed so far."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_uint64()
        check(load().ccl_server_timing(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                       ctypes.byref(n)), "ccl_server_timing")
        return {"h2d_ms": a.value, "label_ms": b.value, "d2h_ms": c.value, "batches": n.value}

    def close(self) -> None:
        if self._h:
            check(load().ccl_server_destroy(self._h), "ccl_server_destroy")
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
