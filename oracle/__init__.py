"""CPU oracle for canonical connected-components labelling.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The GPU library never
imports it, and it imports nothing from the GPU library.

Result definition (the paper's union-find reaches it exactly):
  * the paper gives each connected region one unique ID (§I);
  * its union-find links the larger root under the smaller with atomicMin
    (§II-A-3), so each component's root is its smallest index;
  * IDs are global raster indices ``x + y*imgWidth`` (Kernel 1, ID conversion;
    the Link step of §II-C).
With ``i = y*W + x``: ``out[i] = 0`` for background, else ``1 + min C(i)``.

Functions
  * ``label(img, conn)`` -- the C breadth-first flood fill (``ccl_oracle.c``).
  * ``label_many(imgs, conn)`` -- the same over a stack of equal-size images.
  * ``label_py(img, conn)`` -- a pure-Python twin for tiny inputs.
  * ``label_tiles(img, conn, tile_w, tile_h)`` -- each tile labelled as its own
    image, local indices mapped to global raster indices: the paper's "global
    label map after local merge" (§II-A-3 ID conversion, Fig. 4(a)).
  * ``seam_pairs(h, w, conn, tile_w, tile_h)`` -- the cross-tile adjacent pixel
    pairs the boundary analysis must union (§II-B, Eq. 1-2), enumerated one by
    one.
  * ``label_regions(img, levels, conn)`` -- every equal-value region whose
    value is in ``levels`` (the equality predicate the paper's kernels test,
    §II-A and §II-B), background included when 0 is listed: the sum over the
    levels of ``label`` applied to the level's indicator image.
  * ``label_regions_py(img, levels, conn)`` -- a pure-Python equal-value flood
    fill for tiny inputs.
  * ``label3d(vol, conn)`` / ``label3d_py`` -- the same definition for 3-D
    volumes (the "2D/3D grid" of §I), 6-, 18- or 26-connectivity: the C flood
    fill and a pure-Python twin.
  * ``component_stats(labels)`` -- per component of a canonical label image:
    pixel count, inclusive bounding box and coordinate sums (the size and
    location of each region, §I), by definition, in label order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from collections import deque

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccl_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libccl_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``ccl_oracle.c`` into a shared library with gcc (-O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-shared",
                           "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            for name in ("ccl_oracle_bfs",):
                fn = getattr(lib, name)
                fn.restype = ctypes.c_int
                fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.c_int64, ctypes.c_int]
            fn = lib.ccl_oracle_bfs3d
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_int]
            fn = lib.ccl_oracle_bfs_many
            fn.restype = ctypes.c_int
            fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
            _lib = lib
    return _lib


def _check_conn(conn: int) -> None:
    if conn not in (4, 8):
        raise ValueError(f"connectivity must be 4 or 8, got {conn}")


def label(img: np.ndarray, conn: int = 8) -> np.ndarray:
    """Canonical labels of a 2-D uint8 image (nonzero = foreground)."""
    _check_conn(conn)
    img = np.ascontiguousarray(img, dtype=np.uint8)
    if img.ndim != 2 or img.shape[0] < 1 or img.shape[1] < 1:
        raise ValueError("img must be a non-empty 2-D array")
    out = np.empty(img.shape, dtype=np.int32)
    rc = _load().ccl_oracle_bfs(img.ctypes.data, out.ctypes.data, img.shape[0],
                                img.shape[1], conn)
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    return out


def label_many(imgs: np.ndarray, conn: int = 8) -> np.ndarray:
    """Canonical labels of a stack ``imgs[k]`` of equal-size 2-D images."""
    _check_conn(conn)
    imgs = np.ascontiguousarray(imgs, dtype=np.uint8)
    if imgs.ndim != 3:
        raise ValueError("imgs must be (count, h, w)")
    out = np.empty(imgs.shape, dtype=np.int32)
    rc = _load().ccl_oracle_bfs_many(imgs.ctypes.data, out.ctypes.data, imgs.shape[0],
                                     imgs.shape[1], imgs.shape[2], conn)
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    return out


def _offsets(conn: int):
    if conn == 4:
        return ((1, 0), (-1, 0), (0, 1), (0, -1))
    return ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1))


def label_py(img, conn: int = 8) -> np.ndarray:
    """Pure-Python twin of ``label`` (raster scan + breadth-first flood fill)."""
    _check_conn(conn)
    img = np.asarray(img)
    h, w = img.shape
    out = np.zeros((h, w), dtype=np.int32)
    for y0 in range(h):
        for x0 in range(w):
            if img[y0, x0] == 0 or out[y0, x0] != 0:
                continue
            lab = 1 + y0 * w + x0
            out[y0, x0] = lab
            queue = deque([(x0, y0)])
            while queue:
                x, y = queue.popleft()
                for dx, dy in _offsets(conn):
                    qx, qy = x + dx, y + dy
                    if 0 <= qx < w and 0 <= qy < h and img[qy, qx] != 0 and out[qy, qx] == 0:
                        out[qy, qx] = lab
                        queue.append((qx, qy))
    return out


def _check_levels(levels) -> list:
    lv = [int(v) for v in levels]
    if not lv or len(set(lv)) != len(lv) or any(v < 0 or v > 255 for v in lv):
        raise ValueError("levels must be distinct byte values")
    return lv


def label_regions(img: np.ndarray, levels, conn: int = 8) -> np.ndarray:
    """Canonical labels of every equal-value region of ``img`` whose value is in
    ``levels``; 0 for pixels of other values.

    The paper's kernels join neighbours whose image values are equal (Kernel 1's
    row and column scans, §II-A; Kernel 2's boundary tests, §II-B).  Regions of
    different values are disjoint, so the result is the sum over the levels of
    the canonical labelling of the indicator image ``img == v``."""
    lv = _check_levels(levels)
    img = np.ascontiguousarray(img, dtype=np.uint8)
    out = np.zeros(img.shape, dtype=np.int32)
    for v in lv:
        out += label((img == v).astype(np.uint8), conn)
    return out


def label_regions_py(img, levels, conn: int = 8) -> np.ndarray:
    """Pure-Python twin of ``label_regions``: raster scan, and a breadth-first
    flood fill over neighbours holding the same value as the seed."""
    _check_conn(conn)
    lv = set(_check_levels(levels))
    img = np.asarray(img)
    h, w = img.shape
    out = np.zeros((h, w), dtype=np.int32)
    for y0 in range(h):
        for x0 in range(w):
            v = int(img[y0, x0])
            if v not in lv or out[y0, x0] != 0:
                continue
            lab = 1 + y0 * w + x0
            out[y0, x0] = lab
            queue = deque([(x0, y0)])
            while queue:
                x, y = queue.popleft()
                for dx, dy in _offsets(conn):
                    qx, qy = x + dx, y + dy
                    if 0 <= qx < w and 0 <= qy < h and int(img[qy, qx]) == v \
                            and out[qy, qx] == 0:
                        out[qy, qx] = lab
                        queue.append((qx, qy))
    return out


def _offsets3(conn: int):
    if conn not in (6, 18, 26):
        raise ValueError(f"3-D connectivity must be 6, 18 or 26, got {conn}")
    lim = {6: 1, 18: 2, 26: 3}[conn]
    return tuple((dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                 if 0 < abs(dx) + abs(dy) + abs(dz) <= lim)


def label3d(vol: np.ndarray, conn: int = 26) -> np.ndarray:
    """Canonical labels of a 3-D uint8 volume (nonzero = foreground), indexed
    ``vol[z, y, x]``, voxel index ``(z*H + y)*W + x``: 0 for background, 1 +
    the smallest index of the voxel's component.  ``conn``: 6 (faces), 18
    (faces and edges) or 26 (faces, edges and corners)."""
    _offsets3(conn)
    vol = np.ascontiguousarray(vol, dtype=np.uint8)
    if vol.ndim != 3 or min(vol.shape) < 1:
        raise ValueError("vol must be a non-empty 3-D array")
    out = np.empty(vol.shape, dtype=np.int32)
    rc = _load().ccl_oracle_bfs3d(vol.ctypes.data, out.ctypes.data, vol.shape[0], vol.shape[1],
                                  vol.shape[2], conn)
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    return out


def label3d_py(vol, conn: int = 26) -> np.ndarray:
    """Pure-Python twin of ``label3d`` for tiny volumes."""
    offs = _offsets3(conn)
    vol = np.asarray(vol)
    d, h, w = vol.shape
    out = np.zeros((d, h, w), dtype=np.int32)
    for z0 in range(d):
        for y0 in range(h):
            for x0 in range(w):
                if vol[z0, y0, x0] == 0 or out[z0, y0, x0] != 0:
                    continue
                lab = 1 + (z0 * h + y0) * w + x0
                out[z0, y0, x0] = lab
                queue = deque([(x0, y0, z0)])
                while queue:
                    x, y, z = queue.popleft()
                    for dx, dy, dz in offs:
                        qx, qy, qz = x + dx, y + dy, z + dz
                        if 0 <= qx < w and 0 <= qy < h and 0 <= qz < d \
                                and vol[qz, qy, qx] != 0 and out[qz, qy, qx] == 0:
                            out[qz, qy, qx] = lab
                            queue.append((qx, qy, qz))
    return out


def label_tiles(img: np.ndarray, conn: int, tile_w: int, tile_h: int) -> np.ndarray:
    """Label every tile_w x tile_h tile as if it were a separate image.

    A tile's local raster index ``l = ly*tile_w + lx`` of its component root is
    converted to the global raster index ``(tx*tile_w + lx) + (ty*tile_h + ly)*W``
    (Kernel 1's local-to-global ID conversion, read with ``lx = l % tile_w``,
    ``ly = l / tile_w``).  Partial tiles at the right/bottom edge are labelled
    over their in-image part only.
    """
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w = img.shape
    out = np.zeros((h, w), dtype=np.int32)
    for y0 in range(0, h, tile_h):
        for x0 in range(0, w, tile_w):
            sub = img[y0:y0 + tile_h, x0:x0 + tile_w]
            loc = label(sub, conn).astype(np.int64)
            sw = sub.shape[1]
            fg = loc > 0
            li = loc[fg] - 1
            ly, lx = li // sw, li % sw
            glob = np.zeros(sub.shape, dtype=np.int64)
            glob[fg] = 1 + (y0 + ly) * w + (x0 + lx)
            out[y0:y0 + tile_h, x0:x0 + tile_w] = glob.astype(np.int32)
    return out


def seam_pairs(h: int, w: int, conn: int, tile_w: int, tile_h: int):
    """All unordered pairs of in-bounds neighbouring pixels that lie in different
    tiles, as raster-index tuples ``(p, q)`` with ``p < q`` (pure enumeration).

    These are the cells the boundary analysis (§II-B) works on; Eq. 1-2 count
    the horizontal/vertical seam cells of a whole-tile grid.
    """
    _check_conn(conn)
    pairs = set()
    for y in range(h):
        for x in range(w):
            for dx, dy in _offsets(conn):
                qx, qy = x + dx, y + dy
                if not (0 <= qx < w and 0 <= qy < h):
                    continue
                if (x // tile_w, y // tile_h) == (qx // tile_w, qy // tile_h):
                    continue
                p, q = y * w + x, qy * w + qx
                pairs.add((min(p, q), max(p, q)))
    return pairs


def component_stats(labels: np.ndarray) -> dict:
    """Statistics of every component of a canonical label image, in increasing
    label order: ``label``, ``count`` (pixels), ``xmin ymin xmax ymax``
    (inclusive bounding box), ``sum_x sum_y`` (sums of the pixels' coordinates;
    the centroid is sum / count).  Plain definition: group the foreground
    pixels by label and reduce each group."""
    lab = np.asarray(labels)
    h, w = lab.shape
    ys, xs = np.nonzero(lab)
    vals = lab[ys, xs].astype(np.int64)
    if vals.size == 0:
        z = np.zeros(0, dtype=np.int64)
        return {k: z for k in ("label", "count", "xmin", "ymin", "xmax", "ymax", "sum_x", "sum_y")}
    uniq, inv = np.unique(vals, return_inverse=True)
    n = uniq.size
    count = np.bincount(inv, minlength=n).astype(np.int64)
    xmin = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    ymin = xmin.copy()
    xmax = np.full(n, -1, dtype=np.int64)
    ymax = xmax.copy()
    np.minimum.at(xmin, inv, xs)
    np.minimum.at(ymin, inv, ys)
    np.maximum.at(xmax, inv, xs)
    np.maximum.at(ymax, inv, ys)
    sum_x = np.bincount(inv, weights=xs.astype(np.float64), minlength=n)
    sum_y = np.bincount(inv, weights=ys.astype(np.float64), minlength=n)
    return {"label": uniq, "count": count, "xmin": xmin, "ymin": ymin, "xmax": xmax,
            "ymax": ymax, "sum_x": np.rint(sum_x).astype(np.int64),
            "sum_y": np.rint(sum_y).astype(np.int64)}

