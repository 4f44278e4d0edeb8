"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws pixels; it holds none of the labelling arithmetic and
imports neither the oracle nor the GPU library.  Every image is uint8 row-major
with foreground byte 1 (or ``fg`` when given) and background 0.

The paper measures on binarised natural images (lena, peppers; §III, Fig. 5)
that are not available here; blobby block noise and smoothed "video" frames
stand in for them, Bernoulli noise spans the percolation regimes, and the
serpentine/ring/full/empty images are the structural extremes.

Seeds: ``np.random.default_rng(SeedSequence([cfg_id, seed, h, w, round(100*p)]))``.
"""
from __future__ import annotations

import math

import numpy as np

# config ids used in the seed sequence
CFG_SMALL = 0       # 512x512 plain path
CFG_SWEEP = 1       # 1024^2..8192^2 density sweep
CFG_STRUCT = 2      # structured 4096^2 images
CFG_BATCH = 3       # batched composition
CFG_SERVE = 4       # serving trace


def rng_for(cfg_id: int, seed: int, h: int, w: int, p: float) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(
        [int(cfg_id), int(seed), int(h), int(w), int(round(100 * p))]))


def bernoulli(h: int, w: int, p: float, seed: int, cfg_id: int = CFG_SWEEP,
              fg: int = 1) -> np.ndarray:
    """i.i.d. Bernoulli(p) foreground."""
    rng = rng_for(cfg_id, seed, h, w, p)
    out = np.empty((h, w), dtype=np.uint8)
    rows = max(1, (1 << 24) // max(w, 1))          # bounded float32 scratch
    for y0 in range(0, h, rows):
        y1 = min(h, y0 + rows)
        out[y0:y1] = (rng.random((y1 - y0, w), dtype=np.float32) < p)
    if fg != 1:
        out *= np.uint8(fg)
    return out


def block_noise(h: int, w: int, g: int, seed: int, p: float = 0.5) -> np.ndarray:
    """Bernoulli(p) drawn per g x g cell; cell (i, j) covers rows [i*g, (i+1)*g)
    and columns [j*g, (j+1)*g)."""
    rng = rng_for(CFG_STRUCT, seed * 100 + g, h, w, p)
    ch, cw = -(-h // g), -(-w // g)
    cells = (rng.random((ch, cw), dtype=np.float32) < p).astype(np.uint8)
    return np.ascontiguousarray(np.repeat(np.repeat(cells, g, axis=0), g, axis=1)[:h, :w])


CFG_LEVELS = 5      # multi-level images


def multilevel(h: int, w: int, values, seed: int, g: int = 1) -> np.ndarray:
    """Each g x g cell takes one of ``values`` (bytes) uniformly at random;
    g = 1 is i.i.d. per pixel, larger g gives blobby regions of equal value."""
    vals = np.asarray(list(values), dtype=np.uint8)
    rng = rng_for(CFG_LEVELS, seed * 1000 + g * 7 + vals.size, h, w, 0.0)
    ch, cw = -(-h // g), -(-w // g)
    cells = vals[rng.integers(0, vals.size, size=(ch, cw))]
    if g == 1:
        return np.ascontiguousarray(cells)
    return np.ascontiguousarray(np.repeat(np.repeat(cells, g, axis=0), g, axis=1)[:h, :w])


CFG_VOLUME = 6      # 3-D volumes


def bernoulli3d(d: int, h: int, w: int, p: float, seed: int, g: int = 1) -> np.ndarray:
    """A d x h x w volume (index [z, y, x]) of i.i.d. Bernoulli(p) voxels, or of
    Bernoulli(p) g x g x g cells when g > 1 (blobby regions)."""
    rng = rng_for(CFG_VOLUME, seed * 100 + g, d * h, w, p)
    cd, ch, cw = -(-d // g), -(-h // g), -(-w // g)
    out = np.empty((cd, ch, cw), dtype=np.uint8)
    plane = max(1, (1 << 24) // max(ch * cw, 1))   # bounded float32 scratch
    for z0 in range(0, cd, plane):
        z1 = min(cd, z0 + plane)
        out[z0:z1] = rng.random((z1 - z0, ch, cw), dtype=np.float32) < p
    if g == 1:
        return out
    return np.ascontiguousarray(
        np.repeat(np.repeat(np.repeat(out, g, axis=0), g, axis=1), g, axis=2)[:d, :h, :w])


def serpentine(h: int, w: int, transpose: bool = False) -> np.ndarray:
    """One 1-pixel-wide path: rows y = 0 (mod 2) fully set, row y = 1 (mod 4)
    only at x = W-1, row y = 3 (mod 4) only at x = 0."""
    if transpose:
        return np.ascontiguousarray(serpentine(w, h).T)
    img = np.zeros((h, w), dtype=np.uint8)
    img[0::2, :] = 1
    img[1::4, w - 1] = 1
    img[3::4, 0] = 1
    return img


def rings(h: int, w: int, count: int = 64, spacing: int = 32, inset0: int = 16) -> np.ndarray:
    """Concentric 1-pixel square rings: ring k is the perimeter of the square
    with inset d_k = inset0 + spacing*k (rings that do not fit are skipped)."""
    img = np.zeros((h, w), dtype=np.uint8)
    for k in range(count):
        d = inset0 + spacing * k
        y1, x1 = h - 1 - d, w - 1 - d
        if y1 < d or x1 < d:
            break
        img[d, d:x1 + 1] = 1
        img[y1, d:x1 + 1] = 1
        img[d:y1 + 1, d] = 1
        img[d:y1 + 1, x1] = 1
    return img


def ring_insets(h: int, w: int, count: int = 64, spacing: int = 32, inset0: int = 16):
    out = []
    for k in range(count):
        d = inset0 + spacing * k
        if h - 1 - d < d or w - 1 - d < d:
            break
        out.append(d)
    return out


def full(h: int, w: int) -> np.ndarray:
    return np.ones((h, w), dtype=np.uint8)


def empty(h: int, w: int) -> np.ndarray:
    return np.zeros((h, w), dtype=np.uint8)


def checkerboard(h: int, w: int) -> np.ndarray:
    yy, xx = np.indices((h, w))
    return ((xx + yy) % 2 == 0).astype(np.uint8)


def structured_set(h: int = 4096, w: int = 4096, seed: int = 0):
    """The structured plain-path inputs as (name, image) pairs."""
    items = [(f"block_g{g}", block_noise(h, w, g, seed)) for g in (1, 2, 4, 8, 16)]
    items += [("serpentine", serpentine(h, w)), ("serpentine_T", serpentine(h, w, True)),
              ("rings", rings(h, w)), ("full", full(h, w)), ("empty", empty(h, w))]
    return items


def video_frames(count: int, seed: int, h: int = 1080, w: int = 1920, sigma: float = 4.0,
                 drift: int = 2) -> list:
    """Video-like frames: an N(0,1) noise field smoothed with a Gaussian
    (sigma px, periodic), frame t = crop shifted by drift*t px along x,
    foreground = value above the frame's median (about 50 % density)."""
    from scipy.ndimage import gaussian_filter

    rng = rng_for(CFG_SERVE, seed, h, w, 0.5)
    span = w + drift * max(count - 1, 0)
    field = gaussian_filter(rng.standard_normal((h, span)).astype(np.float32), sigma,
                            mode="wrap")
    frames = []
    for t in range(count):
        crop = field[:, drift * t: drift * t + w]
        frames.append(np.ascontiguousarray((crop > np.median(crop)).astype(np.uint8)))
    return frames


def batch_composition(seed: int, n: int = 256, lo: int = 64, hi: int = 2048):
    """(h, w, p) for a batch: h, w i.i.d. round(exp(U(ln lo, ln hi))), p ~ U(0.3, 0.7)."""
    rng = rng_for(CFG_BATCH, seed, n, hi, 0.5)
    hs = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(int)
    ws = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(int)
    ps = rng.uniform(0.3, 0.7, n)
    return [(int(a), int(b), float(c)) for a, b, c in zip(hs, ws, ps)]


def batch_images(seed: int, n: int = 256, lo: int = 64, hi: int = 2048):
    comp = batch_composition(seed, n, lo, hi)
    return [bernoulli(h, w, p, seed * 1000 + k, cfg_id=CFG_BATCH) for k, (h, w, p) in
            enumerate(comp)]


def serving_trace(rate_hz: float, count: int, seed: int, frame_frac: float = 0.5,
                  lo: int = 128, hi: int = 4096):
    """Poisson arrivals at ``rate_hz``: a list of (arrival_s, kind, h, w) where
    kind is "frame" (1920x1080 video frame) or "square" (side log-uniform in
    [lo, hi], Bernoulli 0.5)."""
    rng = rng_for(CFG_SERVE, seed, count, int(rate_hz), frame_frac)
    gaps = rng.exponential(1.0 / rate_hz, count)
    t = np.cumsum(gaps) - gaps[0]
    kinds = rng.random(count) < frame_frac
    sides = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(int)
    out = []
    for k in range(count):
        if kinds[k]:
            out.append((float(t[k]), "frame", 1080, 1920))
        else:
            out.append((float(t[k]), "square", int(sides[k]), int(sides[k])))
    return out
