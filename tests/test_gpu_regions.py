"""Every-region labelling on the GPU (ccl_label_regions) vs the oracle's
label_regions: bit-exact on multi-level and binary images, at ragged sizes,
unaligned widths and the full 8192 x 8192 size, with level subsets."""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402

DEV = "cuda:0"


def gpu_regions(img, levels, conn, out=None):
    t = torch.from_numpy(np.ascontiguousarray(img)).to(DEV)
    got = ccl.ccl_label_regions(t, levels, conn, out=out)
    return got.cpu().numpy()


def assert_equal(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {bad.shape[0]} pixels differ, first ({y},{x}): "
                             f"got {got[y, x]} want {want[y, x]}")


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(1, 1), (1, 300), (300, 1), (64, 256), (65, 257), (130, 77),
                                (777, 1500), (1024, 1024), (1000, 1003)])
def test_multilevel_random(hw, conn):
    h, w = hw
    for k, (vals, g) in enumerate((([0, 1, 2], 1), ([0, 7, 200, 255], 3), ([5, 6], 16))):
        img = synthetic.multilevel(h, w, vals, k, g=g)
        for levels in (vals, vals[1:] or vals, [vals[-1], vals[0]]):
            assert_equal(gpu_regions(img, levels, conn), oracle.label_regions(img, levels, conn),
                         f"{h}x{w} vals={vals} g={g} levels={levels}")


@pytest.mark.parametrize("conn", [4, 8])
def test_binary_every_region(conn):
    for k, p in enumerate((0.2, 0.5, 0.8)):
        img = synthetic.bernoulli(1024, 1024, p, k, cfg_id=63)
        assert_equal(gpu_regions(img, [0, 1], conn), oracle.label_regions(img, [0, 1], conn),
                     f"p={p}")


@pytest.mark.parametrize("conn", [4, 8])
def test_structured_background(conn):
    for name, img in synthetic.structured_set(1024, 1024):
        assert_equal(gpu_regions(img, [0], conn), oracle.label_regions(img, [0], conn), name)


def test_full_size_8192():
    img = synthetic.bernoulli(8192, 8192, 0.5, 0)
    assert_equal(gpu_regions(img, [0, 1], 8), oracle.label_regions(img, [0, 1], 8), "8192")


def test_output_fully_written_and_level_order():
    """The first pass writes every pixel (stale contents vanish); the level
    order changes nothing."""
    img = synthetic.multilevel(333, 517, [10, 20, 30, 40], 2, g=2)
    want = oracle.label_regions(img, [20, 40], 8)
    out = torch.full((333, 517), -5, dtype=torch.int32, device=DEV)
    assert_equal(gpu_regions(img, [20, 40], 8, out=out), want, "prefilled")
    assert_equal(gpu_regions(img, [40, 20], 8), want, "order")


def test_single_level_equals_plain_label():
    img = synthetic.bernoulli(900, 1100, 0.45, 5, cfg_id=64, fg=255)
    t = torch.from_numpy(img).to(DEV)
    plain = ccl.label(t, 8).cpu().numpy()
    assert_equal(gpu_regions(img, [255], 8), plain, "level 255")


def test_rejects_bad_levels():
    t = torch.zeros((16, 16), dtype=torch.uint8, device=DEV)
    with pytest.raises(ccl.CclError):
        ccl.ccl_label_regions(t, [1, 1], 8)
    with pytest.raises(ValueError):
        ccl.ccl_label_regions(t, [], 8)
