"""3-D labelling on the GPU (ccl_label3d) vs the oracle (oracle.label3d):
bit-exact at 6-, 18- and 26-connectivity on random, blobby and structured
volumes, ragged and brick-aligned shapes, an unaligned input, and 512^3."""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402

DEV = "cuda:0"
CONNS = (6, 18, 26)


def gpu3d(vol, conn, **kw):
    t = torch.from_numpy(np.ascontiguousarray(vol)).to(DEV)
    out = ccl.ccl_label3d(t, conn, **kw)
    ccl.ccl_sync()
    return out.cpu().numpy()


def assert_equal(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        z, y, x = bad[0]
        raise AssertionError(f"{what}: {bad.shape[0]} voxels differ, first (z={z},y={y},x={x}): "
                             f"got {got[z, y, x]} want {want[z, y, x]}")


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 300), (1, 300, 1), (300, 1, 1), (3, 17, 40),
                                   (16, 16, 32), (17, 17, 33), (20, 33, 65), (33, 18, 70),
                                   (40, 50, 130), (64, 64, 64)],
                         ids=lambda s: "x".join(map(str, s)))
def test_random_volumes(shape, conn):
    d, h, w = shape
    for k, p in enumerate((0.2, 0.31, 0.5, 0.8)):
        vol = synthetic.bernoulli3d(d, h, w, p, k)
        assert_equal(gpu3d(vol, conn), oracle.label3d(vol, conn), f"{shape} p={p}")


@pytest.mark.parametrize("conn", CONNS)
def test_blobby_volumes(conn):
    for g in (2, 4, 8):
        vol = synthetic.bernoulli3d(70, 90, 100, 0.45, g, g=g)
        assert_equal(gpu3d(vol, conn), oracle.label3d(vol, conn), f"g={g}")


@pytest.mark.parametrize("conn", CONNS)
def test_structured_volumes(conn):
    d, h, w = 40, 37, 96
    z, y, x = np.indices((d, h, w))
    vols = {
        "full": np.ones((d, h, w), np.uint8),
        "empty": np.zeros((d, h, w), np.uint8),
        "checkerboard": ((x + y + z) % 2 == 0).astype(np.uint8),
        "body_centred": (((x % 2) == (y % 2)) & ((y % 2) == (z % 2))).astype(np.uint8),
        "slabs": (z % 2 == 0).astype(np.uint8),
        "columns": ((x % 3 == 0) & (y % 3 == 0)).astype(np.uint8),
        # 16 segments per strip row and as many contacts with every neighbour strip:
        # the local merge's contact queue overflows and takes further passes
        "x_stripes": (x % 2 == 0).astype(np.uint8),
        # a 3-D serpentine: every other x-row of every slice, joined at alternate ends,
        # and slices joined through one corner voxel
        "serpentine": np.zeros((d, h, w), np.uint8),
    }
    s = vols["serpentine"]
    s[:, 0::2, :] = 1
    s[:, 1::4, w - 1] = 1
    s[:, 3::4, 0] = 1
    for name, vol in vols.items():
        assert_equal(gpu3d(vol, conn), oracle.label3d(vol, conn), name)


@pytest.mark.parametrize("conn", CONNS)
def test_256_cubed(conn):
    for p in (0.3, 0.5):
        vol = synthetic.bernoulli3d(256, 256, 256, p, 7)
        assert_equal(gpu3d(vol, conn), oracle.label3d(vol, conn), f"256^3 p={p}")


def test_512_cubed_26():
    vol = synthetic.bernoulli3d(512, 512, 512, 0.5, 0)
    assert_equal(gpu3d(vol, 26), oracle.label3d(vol, 26), "512^3")


def test_unaligned_input_and_reused_workspace():
    d, h, w = 33, 20, 64
    vol = synthetic.bernoulli3d(d, h, w, 0.4, 3)
    buf = torch.zeros(d * h * w + 1, dtype=torch.uint8, device=DEV)
    buf[1:] = torch.from_numpy(vol.ravel()).to(DEV)
    view = buf[1:].view(d, h, w)                       # 1-byte offset: unaligned loads
    need = max(ccl.ccl_workspace_bytes3d(d, h, w, c) for c in CONNS)
    guard = 4096
    ws = torch.full((need + guard,), 0xA5, dtype=torch.uint8, device=DEV)
    for conn in CONNS:
        out = ccl.ccl_label3d(view, conn, ws=ws[:need])
        ccl.ccl_sync()
        assert_equal(out.cpu().numpy(), oracle.label3d(vol, conn), f"unaligned conn={conn}")
    assert (ws[need:] == 0xA5).all(), "a kernel wrote past its workspace"


def test_rejects_bad_arguments():
    vol = torch.zeros((4, 4, 4), dtype=torch.uint8, device=DEV)
    with pytest.raises(ccl.CclError):
        ccl.ccl_label3d(vol, 8)
    with pytest.raises(TypeError):
        ccl.ccl_label3d(vol[0], 6)
