"""Batched path: many images of different sizes in one graph replay give
exactly the single-image results (tolerance 0) and the oracle's."""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402

DEV = "cuda:0"


def to_dev(imgs):
    return [torch.from_numpy(np.ascontiguousarray(im)).to(DEV) for im in imgs]


@pytest.mark.parametrize("conn", [4, 8])
def test_small_mixed_batch(conn):
    rng = np.random.default_rng(conn)
    imgs = []
    for k in range(40):
        h, w = int(rng.integers(1, 700)), int(rng.integers(1, 700))
        imgs.append(synthetic.bernoulli(h, w, float(rng.uniform(0.2, 0.8)), k, cfg_id=30))
    outs = ccl.label_batched(to_dev(imgs), conn)
    for im, o in zip(imgs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), oracle.label(im, conn))


def test_batched_equals_plain_calls_and_oracle_full_composition():
    """The batched configuration: 256 images, sides log-uniform in 64..2048,
    p ~ U(0.3, 0.7), 8-connectivity."""
    imgs = synthetic.batch_images(seed=0)
    dimgs = to_dev(imgs)
    outs = ccl.label_batched(dimgs, 8)
    for k, (im, d, o) in enumerate(zip(imgs, dimgs, outs)):
        alone = ccl.label(d, 8)
        got = o.cpu().numpy()
        np.testing.assert_array_equal(got, alone.cpu().numpy(), err_msg=f"image {k} vs plain")
        np.testing.assert_array_equal(got, oracle.label(im, 8), err_msg=f"image {k} vs oracle")


def test_graph_reused_across_different_batches():
    """Consecutive batches of different shapes on one stream replay the same
    captured graph; every result stays exact."""
    ws = None
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        n = int(rng.integers(1, 30))
        imgs = [synthetic.bernoulli(int(rng.integers(1, 900)), int(rng.integers(1, 900)), 0.5,
                                    seed * 100 + k, cfg_id=31) for k in range(n)]
        dimgs = to_dev(imgs)
        need = ccl.ccl_batched_workspace_bytes(dimgs, 8)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need * 2, dtype=torch.uint8, device=DEV)
        outs = ccl.ccl_label_batched(dimgs, 8, ws=ws)
        ccl.ccl_sync()
        for im, o in zip(imgs, outs):
            np.testing.assert_array_equal(o.cpu().numpy(), oracle.label(im, 8))


@pytest.mark.parametrize("conn", [4, 8])
def test_all_tiny_images_in_one_batched_call(conn):
    """Every binary image up to 4x4 (74,954 images) in a single batched call,
    packed back to back (unaligned rows)."""
    from helpers import all_images

    groups = [(h, w, all_images(h, w)) for h in range(1, 5) for w in range(1, 5)]
    total = sum(g[2].size for g in groups)
    dbuf = torch.empty(total, dtype=torch.uint8, device=DEV)
    obuf = torch.empty(total, dtype=torch.int32, device=DEV)
    imgs, outs, off = [], [], 0
    host = np.concatenate([g[2].reshape(-1) for g in groups])
    dbuf.copy_(torch.from_numpy(host))
    for h, w, arr in groups:
        for k in range(arr.shape[0]):
            imgs.append(dbuf[off:off + h * w].view(h, w))
            outs.append(obuf[off:off + h * w].view(h, w))
            off += h * w
    assert len(imgs) == 74954
    ccl.ccl_label_batched(imgs, conn, outs=outs)
    ccl.ccl_sync()
    got_all = obuf.cpu().numpy()
    off = 0
    for h, w, arr in groups:
        want = oracle.label_many(arr, conn)
        got = got_all[off:off + arr.size].reshape(arr.shape)
        bad = np.nonzero(np.any(got != want, axis=(1, 2)))[0]
        assert bad.size == 0, f"{h}x{w}: images {bad[:5]} differ"
        off += arr.size


def test_batched_on_side_stream():
    s = torch.cuda.Stream()
    imgs = [synthetic.bernoulli(300 + 7 * k, 200 + 11 * k, 0.5, k, cfg_id=32) for k in range(8)]
    with torch.cuda.stream(s):
        dimgs = to_dev(imgs)
        outs = ccl.ccl_label_batched(dimgs, 8, stream=s)
    ccl.ccl_sync(s)
    for im, o in zip(imgs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(), oracle.label(im, 8))
