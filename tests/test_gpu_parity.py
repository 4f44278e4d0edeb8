"""Single-image GPU path vs the CPU oracle: bit-exact on every seeded input.

Covers every tile width, both connectivities, ragged tails and partial tiles,
unaligned image/label pointers, exhaustive tiny images, structured extremes,
the local-merge-only output, repeat runs, and the full-size headline config.
"""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402

DEV = "cuda:0"
TILES = [32, 64, 128, 256]


def gpu_label(img, conn, tile_w=0, flags=0, img_offset=0, out_offset=0):
    """Run the library on a copy of `img` placed `img_offset` bytes into a
    device buffer (to exercise unaligned rows) and return the labels."""
    h, w = img.shape
    buf = torch.empty(h * w + 64, dtype=torch.uint8, device=DEV)
    dimg = buf[img_offset:img_offset + h * w].view(h, w)
    dimg.copy_(torch.from_numpy(np.ascontiguousarray(img)))
    obuf = torch.empty(h * w + 16, dtype=torch.int32, device=DEV)
    out = obuf[out_offset:out_offset + h * w].view(h, w)
    ccl.ccl_label_tiled(dimg, conn, tile_w, flags, out=out)
    ccl.ccl_sync()
    return out.cpu().numpy()


def assert_same(got, want, what=""):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"{what}: {len(bad)} labels differ; first at y={y} x={x}: "
                             f"got {got[y, x]} want {want[y, x]}")


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("tile_w", TILES)
def test_random_sizes_all_tiles(conn, tile_w):
    rng = np.random.default_rng(1000 + tile_w + conn)
    th = (256 // (tile_w // 32)) * (2 if conn == 8 else 1)
    for k in range(6):
        h = int(rng.integers(1, 3 * th + 7))
        w = int(rng.integers(1, 4 * tile_w + 45))
        p = [0.1, 0.3, 0.45, 0.5, 0.6, 0.9][k]
        img = synthetic.bernoulli(h, w, p, k, cfg_id=20)
        assert_same(gpu_label(img, conn, tile_w), oracle.label(img, conn), f"{h}x{w} p={p}")


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("hw", [(1, 1), (1, 2), (2, 1), (1, 1000), (1000, 1), (33, 17), (3, 4097),
                                (4099, 3), (517, 300), (1080, 1920), (640, 2049)])
def test_edge_shapes(hw, conn):
    h, w = hw
    for p in (0.5, 0.95):
        img = synthetic.bernoulli(h, w, p, 1, cfg_id=21)
        assert_same(gpu_label(img, conn), oracle.label(img, conn), f"{h}x{w} p={p}")


@pytest.mark.parametrize("conn", [4, 8])
def test_unaligned_pointers(conn):
    img = synthetic.bernoulli(77, 301, 0.55, 2, cfg_id=22)
    want = oracle.label(img, conn)
    for off in (1, 2, 3, 5, 13):
        assert_same(gpu_label(img, conn, 0, 0, img_offset=off, out_offset=off % 4), want,
                    f"offset {off}")


@pytest.mark.parametrize("conn", [4, 8])
def test_exhaustive_tiny_images(conn):
    """Every binary image up to 4x4 (74,954), each through the plain path:
    packed back to back in one device buffer (unaligned starts)."""
    from helpers import all_images

    for h in range(1, 5):
        for w in range(1, 5):
            imgs = all_images(h, w)
            want = oracle.label_many(imgs, conn)
            n = imgs.shape[0]
            dimg = torch.from_numpy(imgs.reshape(-1)).to(DEV)
            dout = torch.empty(n * h * w, dtype=torch.int32, device=DEV)
            ws = torch.empty(ccl.ccl_workspace_bytes(h, w, conn), dtype=torch.uint8, device=DEV)
            for k in range(n):
                ccl.ccl_label(dimg[k * h * w:(k + 1) * h * w].view(h, w), conn,
                              out=dout[k * h * w:(k + 1) * h * w].view(h, w), ws=ws)
            ccl.ccl_sync()
            got = dout.view(n, h, w).cpu().numpy()
            bad = np.nonzero(np.any(got != want, axis=(1, 2)))[0]
            assert bad.size == 0, f"{h}x{w}: images {bad[:5]} differ"


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("tile_w", TILES)
def test_structured(conn, tile_w):
    h = w = 1024
    cases = [(n, im) for n, im in synthetic.structured_set(h, w)]
    cases.append(("checker", synthetic.checkerboard(h, w)))
    for name, img in cases:
        assert_same(gpu_label(img, conn, tile_w), oracle.label(img, conn), name)


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("tile_w", TILES)
def test_local_merge_only_matches_per_tile_oracle(conn, tile_w):
    th = (256 // (tile_w // 32)) * (2 if conn == 8 else 1)
    img = synthetic.bernoulli(2 * th + 19, 3 * tile_w + 11, 0.5, 3, cfg_id=23)
    want = oracle.label_tiles(img, conn, tile_w, th)
    assert_same(gpu_label(img, conn, tile_w, ccl.CCL_FLAG_LOCAL_ONLY), want, "local-only")


def test_foreground_byte_value_irrelevant():
    img = synthetic.bernoulli(300, 333, 0.5, 4, cfg_id=24)
    for conn in (4, 8):
        a = gpu_label(img, conn)
        assert_same(gpu_label(img * 255, conn), a, "255")
        assert_same(gpu_label(img * 7, conn), a, "7")


@pytest.mark.parametrize("conn", [4, 8])
def test_repeat_runs_identical(conn):
    """Union order varies run to run; the canonical result may not."""
    img = synthetic.bernoulli(2048, 2048, 0.6 if conn == 4 else 0.45, 5, cfg_id=25)
    want = oracle.label(img, conn)
    dimg = torch.from_numpy(img).to(DEV)
    out = torch.empty((2048, 2048), dtype=torch.int32, device=DEV)
    ws = torch.empty(ccl.ccl_workspace_bytes(2048, 2048, conn), dtype=torch.uint8, device=DEV)
    for _ in range(20):
        out.fill_(-5)
        ccl.ccl_label(dimg, conn, out=out, ws=ws)
        ccl.ccl_sync()
        assert_same(out.cpu().numpy(), want, "repeat")


@pytest.mark.parametrize("n", [1024, 2048])
@pytest.mark.parametrize("conn", [4, 8])
def test_density_sweep_full_range(n, conn):
    """The plain-path sweep at 1024^2 and 2048^2: densities 0.1 ... 0.9 in
    steps of 0.1, seeds 0-9, every image compared in full with the oracle."""
    for k in range(1, 10):
        p = k / 10
        for seed in range(10):
            img = synthetic.bernoulli(n, n, p, seed)
            assert_same(gpu_label(img, conn), oracle.label(img, conn), f"{n} p={p} seed={seed}")


@pytest.mark.parametrize("p", [k / 10 for k in range(1, 10)])
@pytest.mark.parametrize("conn", [4, 8])
def test_density_sweep_4096(p, conn):
    """4096^2 at every density of the sweep; seeds 0-9 around the
    site-percolation thresholds (p = 0.4, 0.5, 0.6: about 0.41 for
    8-connectivity, 0.59 for 4-connectivity), where the components crossing
    tile seams are largest, seed 0 elsewhere."""
    seeds = range(10) if p in (0.4, 0.5, 0.6) else (0,)
    for seed in seeds:
        img = synthetic.bernoulli(4096, 4096, p, seed)
        assert_same(gpu_label(img, conn), oracle.label(img, conn), f"4096 p={p} seed={seed}")


@pytest.fixture(scope="module")
def buffers_8192():
    n = 8192
    need = max(ccl.ccl_workspace_bytes(n, n, c) for c in (4, 8))
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    out = torch.empty((n, n), dtype=torch.int32, device=DEV)
    dimg = torch.empty((n, n), dtype=torch.uint8, device=DEV)
    return dimg, out, ws


@pytest.mark.parametrize("p", [k / 10 for k in range(1, 10)])
@pytest.mark.parametrize("conn", [4, 8])
def test_density_sweep_8192(p, conn, buffers_8192):
    """8192^2 at every density and both connectivities, in the launch
    configuration bench.py times (ccl_label, default tile, caller workspace,
    current stream), compared in full with the oracle.  Seeds 1 and 2 are
    added at the densities next to the percolation thresholds (0.4 and 0.6),
    where seam unions meet the longest chains in the global forest."""
    dimg, out, ws = buffers_8192
    seeds = (0, 1, 2) if p in (0.4, 0.6) else (0,)
    for seed in seeds:
        img = synthetic.bernoulli(8192, 8192, p, seed)
        dimg.copy_(torch.from_numpy(img))
        out.fill_(-3)
        ccl.ccl_label(dimg, conn, out=out, ws=ws)
        ccl.ccl_sync()
        assert_same(out.cpu().numpy(), oracle.label(img, conn), f"8192 p={p} conn={conn} seed={seed}")


def test_small_config_512_seeds():
    """The 512^2 workload (Bernoulli 0.5, 8-connectivity), seeds 0-9."""
    for seed in range(10):
        img = synthetic.bernoulli(512, 512, 0.5, seed, cfg_id=synthetic.CFG_SMALL)
        assert_same(gpu_label(img, 8), oracle.label(img, 8), f"512 seed={seed}")


def test_full_size_headline_8192():
    """The benchmark's workload (8192^2, p = 0.5, 8-connectivity, default tile)
    compared in full with the oracle, in the launch configuration bench.py
    times (ccl_label with a caller workspace on the current stream)."""
    img = synthetic.bernoulli(8192, 8192, 0.5, 0)
    want = oracle.label(img, 8)
    dimg = torch.from_numpy(img).to(DEV)
    ws = torch.empty(ccl.ccl_workspace_bytes(8192, 8192, 8), dtype=torch.uint8, device=DEV)
    out = ccl.ccl_label(dimg, 8, ws=ws)
    ccl.ccl_sync()
    assert_same(out.cpu().numpy(), want, "8192 headline")


@pytest.mark.parametrize("conn", [4, 8])
def test_structured_4096(conn):
    for name, img in synthetic.structured_set(4096, 4096):
        assert_same(gpu_label(img, conn), oracle.label(img, conn), name)


def test_ring_closed_form_on_gpu():
    h = w = 4096
    img = synthetic.rings(h, w)
    for conn in (4, 8):
        got = gpu_label(img, conn)
        for d in synthetic.ring_insets(h, w):
            assert got[d, d] == 1 + d * w + d
            assert got[h - 1 - d, w - 1 - d] == 1 + d * w + d


def test_invalid_args_enqueue_nothing():
    img = torch.zeros((8, 8), dtype=torch.uint8, device=DEV)
    with pytest.raises(ccl.CclError):
        ccl.ccl_label_tiled(img, 6)
    with pytest.raises(ccl.CclError):
        ccl.ccl_label_tiled(img, 8, tile_w=48)
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(ccl.CclError):
        ccl.ccl_label(img, 8, ws=small)
    ccl.ccl_sync()


def test_library_workspace_when_none_given():
    from paper_1708_08180_gb300 import _lib

    img = synthetic.bernoulli(300, 500, 0.5, 6, cfg_id=26)
    dimg = torch.from_numpy(img).to(DEV)
    out = torch.empty((300, 500), dtype=torch.int32, device=DEV)
    st = _lib.load().ccl_label(dimg.data_ptr(), out.data_ptr(), 300, 500, 8, None, 0,
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0
    ccl.ccl_sync()
    assert_same(out.cpu().numpy(), oracle.label(img, 8), "library workspace")


@pytest.mark.parametrize("n", [1024, 4096])
@pytest.mark.parametrize("conn", [4, 8])
def test_back_to_back_calls_share_workspace(n, conn):
    """Calls queued without a host sync in between, all on one workspace:
    each call's kernels start early where the launch allows it (programmatic
    dependent launch of the seam and link kernels), so the next call must not
    touch the workspace before the previous link kernel is done with it.
    1024^2 is a one-wave local merge (seam kernel launched early as well)."""
    imgs = [synthetic.bernoulli(n, n, p, 40 + k, cfg_id=27) for k, p in enumerate((0.45, 0.6, 0.3, 0.5))]
    wants = [oracle.label(im, conn) for im in imgs]
    ws = torch.empty(ccl.ccl_workspace_bytes(n, n, conn), dtype=torch.uint8, device=DEV)
    dimgs = [torch.from_numpy(im).to(DEV) for im in imgs]
    outs = [torch.full((n, n), -7, dtype=torch.int32, device=DEV) for _ in imgs]
    torch.cuda.synchronize()
    for _ in range(3):
        for d, o in zip(dimgs, outs):
            ccl.ccl_label(d, conn, out=o, ws=ws)
    ccl.ccl_sync()
    for k, (o, want) in enumerate(zip(outs, wants)):
        assert_same(o.cpu().numpy(), want, f"back-to-back call {k}")


@pytest.mark.parametrize("conn", [4, 8])
def test_workspace_bound_is_respected(conn):
    """A workspace of exactly ccl_workspace_bytes_tiled bytes, followed by a
    guard region: no call writes past the size it asked for."""
    img = synthetic.bernoulli(777, 1500, 0.5, 3, cfg_id=28)
    want = oracle.label(img, conn)
    dimg = torch.from_numpy(img).to(DEV)
    for tw in TILES:
        need = ccl.ccl_workspace_bytes_tiled(777, 1500, conn, tw)
        buf = torch.full((need + 4096,), 0xAB, dtype=torch.uint8, device=DEV)
        out = torch.empty((777, 1500), dtype=torch.int32, device=DEV)
        ccl.ccl_label_tiled(dimg, conn, tw, out=out, ws=buf[:need])
        ccl.ccl_sync()
        assert_same(out.cpu().numpy(), want, f"tile {tw}")
        assert bool((buf[need:] == 0xAB).all()), f"tile {tw}: write past the workspace"
