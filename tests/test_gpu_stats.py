"""Component statistics on the GPU (ccl_component_stats) vs the oracle's plain
definition (oracle.component_stats over the oracle's labels): exact, in label
order, on random, ragged, structured and full-size images."""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402

DEV = "cuda:0"
FIELDS = ("label", "count", "xmin", "ymin", "xmax", "ymax", "sum_x", "sum_y")


def gpu_stats(img, conn):
    labels = ccl.label(torch.from_numpy(np.ascontiguousarray(img)).to(DEV), conn)
    return ccl.component_stats(labels)


def assert_stats_equal(got, want, what=""):
    assert got["label"].size == want["label"].size, (what, got["label"].size, want["label"].size)
    for f in FIELDS:
        if not np.array_equal(got[f], want[f]):
            k = int(np.argmax(got[f] != want[f]))
            raise AssertionError(f"{what}: {f} differs at component {k} (label "
                                 f"{want['label'][k]}): got {got[f][k]} want {want[f][k]}")


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(1, 1), (1, 300), (300, 1), (64, 256), (65, 257), (777, 1500),
                                (1024, 1024)])
def test_random_images(hw, conn):
    h, w = hw
    for k, p in enumerate((0.3, 0.5, 0.7)):
        img = synthetic.bernoulli(h, w, p, k, cfg_id=61)
        assert_stats_equal(gpu_stats(img, conn), oracle.component_stats(oracle.label(img, conn)),
                           f"{h}x{w} p={p}")


@pytest.mark.parametrize("conn", [4, 8])
def test_structured(conn):
    for name, img in synthetic.structured_set(1024, 1024):
        assert_stats_equal(gpu_stats(img, conn), oracle.component_stats(oracle.label(img, conn)),
                           name)


def test_full_size_8192():
    img = synthetic.bernoulli(8192, 8192, 0.5, 0)
    assert_stats_equal(gpu_stats(img, 8), oracle.component_stats(oracle.label(img, 8)), "8192")


def test_capacity_smaller_than_count():
    """max_comps below the count: the count is complete, the first max_comps
    records are exact, nothing past them is written."""
    img = synthetic.bernoulli(500, 600, 0.4, 3, cfg_id=62)
    want = oracle.component_stats(oracle.label(img, 8))
    n = want["label"].size
    labels = ccl.label(torch.from_numpy(img).to(DEV), 8)
    cap = n // 3
    comps = torch.full((cap + 16, ccl.COMPONENT_WORDS), -77, dtype=torch.int32, device=DEV)
    comps_out, ncomps = ccl.ccl_component_stats(labels, cap, comps=comps)
    ccl.ccl_sync()
    assert int(ncomps.item()) == n
    raw = comps_out.cpu().numpy()
    assert (raw[cap:] == -77).all()
    got = {f: raw[:cap, k].astype(np.int64) for k, f in enumerate(FIELDS[:6])}
    wide = raw[:cap, 6:10].copy().view(np.int64)
    got["sum_x"], got["sum_y"] = wide[:, 0], wide[:, 1]
    assert_stats_equal(got, {f: v[:cap] for f, v in want.items()}, "first records")


def test_no_components():
    img = np.zeros((100, 130), dtype=np.uint8)
    st = gpu_stats(img, 8)
    assert st["label"].size == 0


# ---- statistics gathered in the labelling pass (ccl_label_with_stats) ----

def fused(img, conn):
    """Labels and statistics from one ccl_label_with_stats call, the records
    sorted by label."""
    return ccl.label_with_stats(torch.from_numpy(np.ascontiguousarray(img)).to(DEV), conn)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(1, 1), (1, 300), (300, 1), (64, 256), (65, 257), (777, 1500),
                                (1024, 1024), (1080, 1920)])
def test_fused_random_images(hw, conn):
    h, w = hw
    for k, p in enumerate((0.1, 0.3, 0.5, 0.7)):
        img = synthetic.bernoulli(h, w, p, k, cfg_id=63)
        labels, st = fused(img, conn)
        want_labels = oracle.label(img, conn)
        assert np.array_equal(labels.cpu().numpy(), want_labels), f"{h}x{w} p={p}: labels"
        assert_stats_equal(st, oracle.component_stats(want_labels), f"fused {h}x{w} p={p}")


@pytest.mark.parametrize("conn", [4, 8])
def test_fused_structured(conn):
    cases = list(synthetic.structured_set(1024, 1024))
    # more border roots per tile than the shared tables hold: isolated pixels
    # on every even column of each tile's first and last rows and on the even
    # rows of its first column
    h = w = 1024
    yy, xx = np.indices((h, w))
    many = (((yy % 64 == 0) | (yy % 64 == 63)) & (xx % 2 == 0)) | ((xx % 256 == 0) & (yy % 2 == 0))
    cases.append(("many_border_roots", many.astype(np.uint8)))
    for name, img in cases:
        labels, st = fused(img, conn)
        want_labels = oracle.label(img, conn)
        assert np.array_equal(labels.cpu().numpy(), want_labels), name
        assert_stats_equal(st, oracle.component_stats(want_labels), f"fused {name}")


def test_fused_full_size_8192():
    img = synthetic.bernoulli(8192, 8192, 0.5, 0)
    labels, st = fused(img, 8)
    want_labels = oracle.label(img, 8)
    assert np.array_equal(labels.cpu().numpy(), want_labels)
    assert_stats_equal(st, oracle.component_stats(want_labels), "fused 8192")


def test_fused_capacity_smaller_than_count():
    """max_comps below the count: the count is complete, max_comps records are
    written, each exact, and nothing past them."""
    img = synthetic.bernoulli(500, 600, 0.4, 3, cfg_id=64)
    want = oracle.component_stats(oracle.label(img, 8))
    n = want["label"].size
    cap = n // 3
    comps = torch.full((cap + 16, ccl.COMPONENT_WORDS), -77, dtype=torch.int32, device=DEV)
    _, comps_out, ncomps = ccl.ccl_label_with_stats(torch.from_numpy(img).to(DEV), 8, cap,
                                                    comps=comps)
    ccl.ccl_sync()
    assert int(ncomps.item()) == n
    raw = comps_out.cpu().numpy()
    assert (raw[cap:] == -77).all()
    got = {f: raw[:cap, k].astype(np.int64) for k, f in enumerate(FIELDS[:6])}
    wide = raw[:cap, 6:10].copy().view(np.int64)
    got["sum_x"], got["sum_y"] = wide[:, 0], wide[:, 1]
    idx = np.searchsorted(want["label"], got["label"])
    assert np.array_equal(want["label"][idx], got["label"]), "a written record has no component"
    assert np.unique(got["label"]).size == cap, "a component was written twice"
    assert_stats_equal(got, {f: v[idx] for f, v in want.items()}, "written records")


def test_fused_no_components():
    img = np.zeros((100, 130), dtype=np.uint8)
    labels, st = fused(img, 8)
    assert st["label"].size == 0
    assert int(labels.abs().sum().item()) == 0
