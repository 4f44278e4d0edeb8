"""Test helpers: golden-file parsing and oracle-independent checks.

Nothing here is shared with the GPU library; the independent checks below
(transitive closure, two-pass Rosenfeld-Pfaltz count, canonicalised scipy
labels) exist to pin the oracle to something other than itself.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name: str) -> dict:
    """Parse a hand-worked fixture: {"image": arr, "conn4": arr, "conn8": arr,
    "tiles": (tw, th, arr) or None}."""
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.endswith(":"):
                cur = line[:-1]
                blocks[cur] = []
                continue
            blocks[cur].append([int(v) for v in line.split()])
    out = {k: np.array(v, dtype=np.int64) for k, v in blocks.items()}
    res = {"image": out["image"].astype(np.uint8), "conn4": out["conn4"],
           "conn8": out["conn8"], "tiles": None}
    for k, v in out.items():
        if k.startswith("tiles "):
            tw, th = (int(s) for s in k.split()[1].split("x"))
            res["tiles"] = (tw, th, v)
    return res


def golden_names():
    return sorted(n for n in os.listdir(GOLDEN) if n.endswith(".txt") and n != "README.txt"
                  and not n.startswith("regions_"))


def regions_golden_names():
    return sorted(n for n in os.listdir(GOLDEN) if n.startswith("regions_"))


def load_regions_golden(name: str) -> dict:
    """Parse a hand-worked multi-level fixture: blocks "image:", "levels:",
    "conn4:", "conn8:"."""
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.endswith(":"):
                cur = line[:-1]
                blocks[cur] = []
                continue
            blocks[cur].append([int(v) for v in line.split()])
    return {"image": np.array(blocks["image"], dtype=np.uint8),
            "levels": [v for row in blocks["levels"] for v in row],
            "conn4": np.array(blocks["conn4"], dtype=np.int64),
            "conn8": np.array(blocks["conn8"], dtype=np.int64)}


def all_images(h: int, w: int) -> np.ndarray:
    """Every binary h x w image, image k has pixel i = bit i of k."""
    n = h * w
    k = np.arange(1 << n, dtype=np.int64)
    bits = (k[:, None] >> np.arange(n)[None, :]) & 1
    return bits.reshape(-1, h, w).astype(np.uint8)


def closure_labels(imgs: np.ndarray, conn: int) -> np.ndarray:
    """Canonical labels by transitive closure of the adjacency relation.

    R starts as (adjacent or equal) restricted to foreground pairs and is
    squared until it stops changing; pixel i's label is 1 + the first j with
    R[i, j] (reachable), 0 for background.  Independent of any flood fill.
    """
    cnt, h, w = imgs.shape
    n = h * w
    ys, xs = np.divmod(np.arange(n), w)
    dy = np.abs(ys[:, None] - ys[None, :])
    dx = np.abs(xs[:, None] - xs[None, :])
    if conn == 4:
        adj = (dx + dy) <= 1
    else:
        adj = np.maximum(dx, dy) <= 1
    fg = imgs.reshape(cnt, n).astype(bool)
    r = (adj[None, :, :] & fg[:, :, None] & fg[:, None, :]).astype(np.float32)
    for _ in range(max(1, int(np.ceil(np.log2(max(n, 2)))) + 1)):
        r2 = (np.matmul(r, r) > 0).astype(np.float32)
        if np.array_equal(r2, r):
            break
        r = r2
    first = np.argmax(r > 0, axis=2)
    lab = np.where(fg, first + 1, 0)
    return lab.reshape(cnt, h, w).astype(np.int32)


def closure_labels_valued(imgs: np.ndarray, conn: int, levels) -> np.ndarray:
    """Canonical region labels by transitive closure, for multi-level images:
    R starts as (adjacent or equal) and (equal value) and (value in levels),
    and is squared until it stops changing; pixel i's label is 1 + the first j
    reachable from it, 0 for a value not in levels."""
    cnt, h, w = imgs.shape
    n = h * w
    ys, xs = np.divmod(np.arange(n), w)
    dy = np.abs(ys[:, None] - ys[None, :])
    dx = np.abs(xs[:, None] - xs[None, :])
    adj = ((dx + dy) <= 1) if conn == 4 else (np.maximum(dx, dy) <= 1)
    v = imgs.reshape(cnt, n).astype(np.int64)
    keep = np.isin(v, np.asarray(list(levels), dtype=np.int64))
    r = (adj[None] & (v[:, :, None] == v[:, None, :]) & keep[:, :, None]).astype(np.float32)
    for _ in range(max(1, int(np.ceil(np.log2(max(n, 2)))) + 1)):
        r2 = (np.matmul(r, r) > 0).astype(np.float32)
        if np.array_equal(r2, r):
            break
        r = r2
    first = np.argmax(r > 0, axis=2)
    lab = np.where(keep, first + 1, 0)
    return lab.reshape(cnt, h, w).astype(np.int32)


def all_images_valued(h: int, w: int, nval: int) -> np.ndarray:
    """Every h x w image over the values 0..nval-1 (image k: pixel i = digit i
    of k in base nval)."""
    n = h * w
    k = np.arange(nval ** n, dtype=np.int64)
    digits = (k[:, None] // (nval ** np.arange(n))[None, :]) % nval
    return digits.reshape(-1, h, w).astype(np.uint8)


def two_pass_count(img: np.ndarray, conn: int) -> int:
    """Number of components by the classical two-pass (Rosenfeld-Pfaltz)
    scheme: provisional labels from the already-visited neighbours (left, up,
    and up-left / up-right for 8-connectivity) plus an equivalence table."""
    img = np.asarray(img) != 0
    h, w = img.shape
    prov = np.zeros((h, w), dtype=np.int64)
    parent = [0]

    def root(a):
        while parent[a] != a:
            a = parent[a]
        return a

    nxt = 1
    if conn == 4:
        back = [(-1, 0), (0, -1)]
    else:
        back = [(-1, 0), (0, -1), (-1, -1), (1, -1)]
    for y in range(h):
        for x in range(w):
            if not img[y, x]:
                continue
            seen = []
            for ddx, ddy in back:
                qx, qy = x + ddx, y + ddy
                if 0 <= qx < w and 0 <= qy < h and prov[qy, qx]:
                    seen.append(prov[qy, qx])
            if not seen:
                parent.append(nxt)
                prov[y, x] = nxt
                nxt += 1
                continue
            roots = sorted({root(s) for s in seen})
            prov[y, x] = roots[0]
            for r in roots[1:]:
                parent[r] = roots[0]
    return len({root(v) for v in prov[img]}) if img.any() else 0


def canonical_from_arbitrary(lab: np.ndarray) -> np.ndarray:
    """Map an arbitrary component labelling (0 = background) to canonical form:
    each label replaced by 1 + the smallest raster index carrying it."""
    flat = lab.ravel().astype(np.int64)
    nlab = int(flat.max()) if flat.size else 0
    mins = np.full(nlab + 1, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(mins, flat, np.arange(flat.size, dtype=np.int64))
    out = np.where(flat > 0, mins[flat] + 1, 0)
    return out.reshape(lab.shape).astype(np.int32)


def scipy_canonical(img: np.ndarray, conn: int) -> np.ndarray:
    from scipy import ndimage

    structure = np.ones((3, 3), dtype=int) if conn == 8 else None
    lab, _ = ndimage.label(np.asarray(img) != 0, structure=structure)
    return canonical_from_arbitrary(lab)


def check_invariants(img: np.ndarray, lab: np.ndarray, conn: int) -> None:
    """Assert the properties every canonical labelling has."""
    img = np.asarray(img) != 0
    lab = np.asarray(lab).astype(np.int64)
    h, w = img.shape
    assert lab.shape == img.shape
    assert np.all((lab == 0) == ~img), "background iff label 0"
    idx = np.arange(h * w, dtype=np.int64).reshape(h, w)
    # label - 1 is a raster index not larger than the pixel's own index
    assert np.all(lab[img] - 1 <= idx[img])
    # adjacent foreground pixels carry equal labels
    offs = [(0, 1), (1, 0)] + ([(1, 1), (1, -1)] if conn == 8 else [])
    for dy, dx in offs:
        y0, y1 = 0, h - dy
        x0, x1 = max(0, -dx), w - max(0, dx)
        a = (slice(y0, y1), slice(x0, x1))
        b = (slice(y0 + dy, y1 + dy), slice(x0 + dx, x1 + dx))
        both = img[a] & img[b]
        assert np.array_equal(lab[a][both], lab[b][both]), f"neighbour mismatch {dy},{dx}"
    # a label value L marks its own pixel L-1, which is foreground and labelled L
    vals = np.unique(lab[img])
    flat = lab.ravel()
    assert np.all(flat[vals - 1] == vals), "root pixel carries its own label"
