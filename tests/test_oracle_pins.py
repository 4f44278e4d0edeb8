"""Pins for the CPU oracle (no GPU).

The oracle is the definition of the result; these tests tie it to things other
than itself: exhaustive transitive closure on every image up to 4x4,
hand-worked examples, closed forms, a library routine (scipy.ndimage.label,
canonicalised), invariants, and an independent two-pass component count.
"""
import numpy as np
import pytest

import oracle
import synthetic
from helpers import (all_images, all_images_valued, canonical_from_arbitrary,
                     check_invariants, closure_labels, closure_labels_valued, golden_names,
                     load_golden, load_regions_golden, regions_golden_names, scipy_canonical,
                     two_pass_count)

SIZES_4x4 = [(h, w) for h in range(1, 5) for w in range(1, 5)]


def test_exhaustive_count():
    assert sum(1 << (h * w) for h, w in SIZES_4x4) == 74954


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", SIZES_4x4, ids=lambda s: f"{s[0]}x{s[1]}")
def test_bruteforce_closure_all_images(hw, conn):
    h, w = hw
    imgs = all_images(h, w)
    got = oracle.label_many(imgs, conn)
    want = closure_labels(imgs, conn)
    bad = np.nonzero(np.any(got != want, axis=(1, 2)))[0]
    assert bad.size == 0, f"first mismatch image {bad[:5]}"


@pytest.mark.parametrize("conn", [4, 8])
def test_python_twin_matches_c(conn):
    imgs = all_images(3, 3)
    c = oracle.label_many(imgs, conn)
    for k in range(imgs.shape[0]):
        np.testing.assert_array_equal(oracle.label_py(imgs[k], conn), c[k])
    rng = np.random.default_rng(7)
    for _ in range(20):
        h, w = rng.integers(1, 24, size=2)
        img = (rng.random((h, w)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        np.testing.assert_array_equal(oracle.label_py(img, conn), oracle.label(img, conn))


@pytest.mark.parametrize("name", golden_names())
@pytest.mark.parametrize("conn", [4, 8])
def test_hand_worked(name, conn):
    g = load_golden(name)
    np.testing.assert_array_equal(oracle.label(g["image"], conn), g[f"conn{conn}"])
    np.testing.assert_array_equal(oracle.label_py(g["image"], conn), g[f"conn{conn}"])


def test_hand_worked_tiles():
    g = load_golden("tiles4.txt")
    tw, th, want = g["tiles"]
    for conn in (4, 8):
        np.testing.assert_array_equal(oracle.label_tiles(g["image"], conn, tw, th), want)


@pytest.mark.parametrize("conn", [4, 8])
def test_label_tiles_whole_image_tile(conn):
    img = synthetic.bernoulli(37, 53, 0.5, 3)
    np.testing.assert_array_equal(oracle.label_tiles(img, conn, 64, 64), oracle.label(img, conn))
    # 1x1 tiles: every foreground pixel is its own root
    idx = np.arange(img.size).reshape(img.shape) + 1
    np.testing.assert_array_equal(oracle.label_tiles(img, conn, 1, 1), np.where(img > 0, idx, 0))


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(1, 1), (1, 7), (7, 1), (5, 9), (64, 64), (33, 17)])
def test_closed_forms(hw, conn):
    h, w = hw
    assert not oracle.label(synthetic.empty(h, w), conn).any()
    assert np.all(oracle.label(synthetic.full(h, w), conn) == 1)
    cb = synthetic.checkerboard(h, w)
    lab = oracle.label(cb, conn)
    idx = np.arange(h * w).reshape(h, w)
    if conn == 4 or h == 1 or w == 1:
        np.testing.assert_array_equal(lab, np.where(cb > 0, idx + 1, 0))
    else:
        np.testing.assert_array_equal(lab, cb.astype(np.int32))
    stripes = np.zeros((h, w), np.uint8)
    stripes[0::2] = 1
    ys = np.arange(h)[:, None]
    want = np.where(stripes > 0, 1 + ys * w, 0)
    np.testing.assert_array_equal(oracle.label(stripes, conn), want)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(8, 8), (9, 13), (64, 40), (257, 131)])
def test_serpentine_closed_form(hw, conn):
    h, w = hw
    for tr in (False, True):
        img = synthetic.serpentine(h, w, transpose=tr)
        lab = oracle.label(img, conn)
        # the path starts at raster index 0 and visits every foreground pixel
        np.testing.assert_array_equal(lab, img.astype(np.int32))


@pytest.mark.parametrize("conn", [4, 8])
def test_rings_closed_form(conn):
    h, w = 700, 640
    img = synthetic.rings(h, w, count=64, spacing=32, inset0=16)
    lab = oracle.label(img, conn)
    want = np.zeros((h, w), np.int64)
    for d in synthetic.ring_insets(h, w):
        ring = np.zeros((h, w), bool)
        ring[d, d:w - d] = ring[h - 1 - d, d:w - d] = True
        ring[d:h - d, d] = ring[d:h - d, w - 1 - d] = True
        want[ring] = 1 + d * w + d
    np.testing.assert_array_equal(lab, want)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw,count", [((16, 16), 100), ((33, 17), 100), ((64, 64), 100),
                                      ((128, 96), 100), ((512, 512), 10), ((1024, 1024), 2)])
def test_scipy_cross_check(hw, count, conn):
    h, w = hw
    for seed in range(count):
        p = [0.1, 0.3, 0.45, 0.5, 0.6, 0.8][seed % 6]
        img = synthetic.bernoulli(h, w, p, seed, cfg_id=9)
        np.testing.assert_array_equal(oracle.label(img, conn), scipy_canonical(img, conn))


@pytest.mark.parametrize("conn", [4, 8])
def test_invariants_and_two_pass_count(conn):
    for seed in range(12):
        h, w = 40 + seed * 7, 31 + seed * 5
        p = 0.2 + 0.05 * seed
        img = synthetic.bernoulli(h, w, p, seed, cfg_id=8)
        lab = oracle.label(img, conn)
        check_invariants(img, lab, conn)
        assert len(np.unique(lab[lab > 0])) == two_pass_count(img, conn)


def test_fg_byte_value_irrelevant():
    img = synthetic.bernoulli(50, 70, 0.5, 1)
    for conn in (4, 8):
        np.testing.assert_array_equal(oracle.label(img * 255, conn), oracle.label(img, conn))
        np.testing.assert_array_equal(oracle.label(img * 7, conn), oracle.label(img, conn))


def test_invariants_catch_a_planted_mistake():
    """A plausible oracle mistake (a dropped diagonal) must trip a pin."""
    img = load_golden("stairs4.txt")["image"]
    wrong = oracle.label(img, 4)              # 4-connected result used for 8
    with pytest.raises(AssertionError):
        check_invariants(img, wrong, 8)
    lab = oracle.label(img, 8)
    bumped = lab.copy()
    bumped[lab == 3] = 6                      # root index off by a few pixels
    with pytest.raises(AssertionError):
        check_invariants(img, bumped, 8)


def test_canonicaliser():
    lab = np.array([[0, 5, 5], [2, 0, 5], [2, 2, 0]])
    np.testing.assert_array_equal(canonical_from_arbitrary(lab),
                                  [[0, 2, 2], [4, 0, 2], [4, 4, 0]])


def test_oracle_rejects_bad_args():
    with pytest.raises(ValueError):
        oracle.label(np.zeros((3, 3), np.uint8), 6)
    with pytest.raises(ValueError):
        oracle.label(np.zeros((0, 3), np.uint8), 4)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw,tile", [((8, 8), (4, 2)), ((7, 9), (4, 2)), ((12, 10), (3, 5)),
                                     ((16, 32), (32, 4))])
def test_seam_pair_closed_form(hw, tile, conn):
    """Eq. 1-2 count the seam cells of a whole-tile grid; the exact pair count
    for any size is: all adjacent pairs minus those inside one tile."""
    h, w = hw
    tw, th = tile
    pairs = oracle.seam_pairs(h, w, conn, tw, th)
    tile_hs = [min(th, h - y) for y in range(0, h, th)]
    tile_ws = [min(tw, w - x) for x in range(0, w, tw)]

    def pairs4(a, b):
        return a * (b - 1) + b * (a - 1)

    def diag(a, b):
        return 2 * max(a - 1, 0) * max(b - 1, 0)

    want = pairs4(h, w) - sum(pairs4(a, b) for a in tile_hs for b in tile_ws)
    if conn == 8:
        want += diag(h, w) - sum(diag(a, b) for a in tile_hs for b in tile_ws)
    assert len(pairs) == want
    if conn == 4 and h % th == 0 and w % tw == 0:
        # Eq. 1-2 (with N = width, M = height), minus the image-edge seam they
        # include: P_x = (W/b_x - 1) * H, P_y = (H/b_y - 1) * W
        assert len(pairs) == (w // tw - 1) * h + (h // th - 1) * w


# ---- component statistics (size and location of each region, §I) ----

def test_component_stats_hand_example():
    # 4-connectivity: {(0,0),(0,1)} -> 1, {(0,2)} -> 3, {(2,1),(2,2)} -> 8 (x, y)
    lab = oracle.label(np.array([[1, 0, 1], [1, 0, 0], [0, 1, 1]], dtype=np.uint8), 4)
    st = oracle.component_stats(lab)
    assert st["label"].tolist() == [1, 3, 8]
    assert st["count"].tolist() == [2, 1, 2]
    assert st["xmin"].tolist() == [0, 2, 1] and st["xmax"].tolist() == [0, 2, 2]
    assert st["ymin"].tolist() == [0, 0, 2] and st["ymax"].tolist() == [1, 0, 2]
    assert st["sum_x"].tolist() == [0, 2, 3] and st["sum_y"].tolist() == [1, 0, 4]


@pytest.mark.parametrize("conn", [4, 8])
def test_component_stats_against_pixel_loop(conn):
    """Against a pixel-by-pixel Python loop on small seeded images."""
    for seed in range(6):
        img = synthetic.bernoulli(13 + seed, 17 + 2 * seed, 0.45, seed, cfg_id=60)
        lab = oracle.label(img, conn)
        acc = {}
        h, w = lab.shape
        for y in range(h):
            for x in range(w):
                L = int(lab[y, x])
                if L:
                    c = acc.setdefault(L, [0, x, y, x, y, 0, 0])
                    c[0] += 1
                    c[1] = min(c[1], x); c[2] = min(c[2], y)
                    c[3] = max(c[3], x); c[4] = max(c[4], y)
                    c[5] += x; c[6] += y
        st = oracle.component_stats(lab)
        assert st["label"].tolist() == sorted(acc)
        for k, L in enumerate(sorted(acc)):
            c = acc[L]
            got = [st[f][k] for f in ("count", "xmin", "ymin", "xmax", "ymax", "sum_x", "sum_y")]
            assert got == c, (L, got, c)
            # the root pixel (label - 1) is the component's first pixel in raster order
            assert (L - 1) // w == c[2]


def test_component_stats_closed_forms():
    h, w = 12, 20
    full = oracle.component_stats(oracle.label(synthetic.full(h, w), 8))
    assert full["label"].tolist() == [1] and full["count"].tolist() == [h * w]
    assert full["sum_x"].tolist() == [h * w * (w - 1) // 2]
    assert full["sum_y"].tolist() == [w * h * (h - 1) // 2]
    assert oracle.component_stats(oracle.label(synthetic.empty(h, w), 4))["count"].size == 0
    cb = oracle.component_stats(oracle.label(synthetic.checkerboard(h, w), 4))
    assert cb["count"].size == h * w // 2 and set(cb["count"].tolist()) == {1}


@pytest.mark.parametrize("conn", [4, 8])
def test_component_stats_against_scipy(conn):
    """Library special case: scipy.ndimage's per-label sums, bounding slices and
    centres of mass over the same labels."""
    from scipy import ndimage

    for seed in range(4):
        img = synthetic.bernoulli(150 + 7 * seed, 230, 0.3 + 0.1 * seed, seed, cfg_id=65)
        lab = oracle.label(img, conn)
        st = oracle.component_stats(lab)
        idx = st["label"]
        ones = np.ones(lab.shape, np.int64)
        np.testing.assert_array_equal(ndimage.sum_labels(ones, lab, idx).astype(np.int64),
                                      st["count"])
        ys, xs = np.indices(lab.shape)
        np.testing.assert_array_equal(ndimage.sum_labels(xs, lab, idx).astype(np.int64),
                                      st["sum_x"])
        np.testing.assert_array_equal(ndimage.sum_labels(ys, lab, idx).astype(np.int64),
                                      st["sum_y"])
        # find_objects indexes slices by label value: entry L - 1 for label L
        boxes = ndimage.find_objects(lab)
        for k, L in enumerate(idx.tolist()):
            sy, sx = boxes[L - 1]
            assert (st["ymin"][k], st["ymax"][k]) == (sy.start, sy.stop - 1)
            assert (st["xmin"][k], st["xmax"][k]) == (sx.start, sx.stop - 1)
        com = np.array(ndimage.center_of_mass(ones, lab, idx))
        np.testing.assert_allclose(com[:, 0], st["sum_y"] / st["count"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(com[:, 1], st["sum_x"] / st["count"], rtol=0, atol=1e-9)


# ---------------------------------------------------------------------------
# label_regions: every equal-value region (the paper's equality predicate,
# §II-A row/column scans and §II-B boundary tests)

@pytest.mark.parametrize("name", regions_golden_names())
@pytest.mark.parametrize("conn", [4, 8])
def test_regions_hand_worked(name, conn):
    g = load_regions_golden(name)
    np.testing.assert_array_equal(oracle.label_regions(g["image"], g["levels"], conn),
                                  g[f"conn{conn}"])
    np.testing.assert_array_equal(oracle.label_regions_py(g["image"], g["levels"], conn),
                                  g[f"conn{conn}"])


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(1, 4), (2, 2), (2, 3), (3, 2), (1, 6)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_regions_closure_all_three_level_images(hw, conn):
    """Every image over {0, 1, 2} of the size, all values and a subset labelled."""
    h, w = hw
    imgs = all_images_valued(h, w, 3)
    for levels in ([0, 1, 2], [2, 0], [1]):
        want = closure_labels_valued(imgs, conn, levels)
        for k in range(imgs.shape[0]):
            got = oracle.label_regions(imgs[k], levels, conn)
            if not np.array_equal(got, want[k]):
                raise AssertionError(f"image {k} levels {levels}: {got} vs {want[k]}")


@pytest.mark.parametrize("conn", [4, 8])
def test_regions_python_twin_and_scipy(conn):
    rng = np.random.default_rng(11)
    for t in range(24):
        h, w = (int(v) for v in rng.integers(1, 30, size=2))
        nval = int(rng.integers(2, 6))
        vals = rng.choice(256, size=nval, replace=False)
        img = synthetic.multilevel(h, w, vals, t, g=int(rng.integers(1, 4)))
        levels = list(rng.permutation(vals)[: int(rng.integers(1, nval + 1))])
        got = oracle.label_regions(img, levels, conn)
        np.testing.assert_array_equal(oracle.label_regions_py(img, levels, conn), got)
        # per level, scipy's labelling of the indicator image, canonicalised
        want = np.zeros(img.shape, np.int64)
        for v in levels:
            want += scipy_canonical(img == v, conn)
        np.testing.assert_array_equal(got, want)


def test_regions_reduce_to_binary_labelling():
    """On a binary image, labelling the nonzero level alone is the plain
    labelling, and labelling {0, v} adds the background regions of the
    complement image without touching the foreground labels."""
    for conn in (4, 8):
        for seed in range(6):
            img = synthetic.bernoulli(37 + seed, 53, 0.3 + 0.08 * seed, seed, cfg_id=12,
                                      fg=255 if seed % 2 else 1)
            v = int(img.max()) or 1
            plain = oracle.label(img, conn)
            np.testing.assert_array_equal(oracle.label_regions(img, [v], conn), plain)
            both = oracle.label_regions(img, [0, v], conn)
            np.testing.assert_array_equal(both[img != 0], plain[img != 0])
            comp = (img == 0).astype(np.uint8)
            np.testing.assert_array_equal(both[img == 0], oracle.label(comp, conn)[img == 0])
            assert (both > 0).all()


def test_regions_level_order_irrelevant_and_bad_levels():
    img = synthetic.multilevel(40, 41, [3, 9, 200], 1, g=2)
    a = oracle.label_regions(img, [3, 9, 200], 8)
    np.testing.assert_array_equal(oracle.label_regions(img, [200, 3, 9], 8), a)
    for bad in ([], [1, 1], [256], [-1]):
        with pytest.raises(ValueError):
            oracle.label_regions(img, bad, 8)


def test_regions_catch_a_planted_mistake():
    """A labelling that ignores the value (joins neighbours of any two listed
    levels) fails the closure pin: the pin can see the mistake."""
    imgs = all_images_valued(2, 2, 3)
    want = closure_labels_valued(imgs, 4, [1, 2])
    wrong = np.stack([oracle.label(np.isin(im, [1, 2]).astype(np.uint8), 4) for im in imgs])
    assert not np.array_equal(wrong, want)
