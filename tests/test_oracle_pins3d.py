"""Pins for the 3-D oracle (``oracle.label3d``, no GPU): exhaustive transitive
closure on every binary volume of up to 12 voxels, hand-worked examples, the
reduction to the 2-D labelling on one-voxel-thick volumes, scipy.ndimage.label
with the matching 3-D structuring element, invariants, and the pure-Python
twin."""
import numpy as np
import pytest

import oracle
from helpers import canonical_from_arbitrary

CONNS = (6, 18, 26)


def all_volumes(d, h, w):
    n = d * h * w
    k = np.arange(1 << n, dtype=np.int64)
    bits = (k[:, None] >> np.arange(n)[None, :]) & 1
    return bits.reshape(-1, d, h, w).astype(np.uint8)


def closure_labels3d(vols, conn):
    """1 + the first voxel reachable from each foreground voxel, by squaring the
    adjacency relation (restricted to foreground) until it stops changing."""
    cnt, d, h, w = vols.shape
    n = d * h * w
    idx = np.arange(n)
    zs, ys, xs = idx // (h * w), (idx // w) % h, idx % w
    ad = [np.abs(c[:, None] - c[None, :]) for c in (xs, ys, zs)]
    cheb = np.maximum(np.maximum(ad[0], ad[1]), ad[2])
    manh = ad[0] + ad[1] + ad[2]
    adj = (cheb <= 1) & (manh <= {6: 1, 18: 2, 26: 3}[conn])
    fg = vols.reshape(cnt, n).astype(bool)
    r = (adj[None] & fg[:, :, None] & fg[:, None, :]).astype(np.float32)
    for _ in range(max(1, int(np.ceil(np.log2(max(n, 2)))) + 1)):
        r2 = (np.matmul(r, r) > 0).astype(np.float32)
        if np.array_equal(r2, r):
            break
        r = r2
    first = np.argmax(r > 0, axis=2)
    return np.where(fg, first + 1, 0).reshape(cnt, d, h, w).astype(np.int32)


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("shape", [(2, 2, 2), (2, 2, 3), (2, 3, 2), (3, 2, 2), (1, 3, 4),
                                   (3, 1, 3)], ids=lambda s: "x".join(map(str, s)))
def test_closure_every_small_volume(shape, conn):
    vols = all_volumes(*shape)
    want = closure_labels3d(vols, conn)
    for k in range(vols.shape[0]):
        got = oracle.label3d(vols[k], conn)
        if not np.array_equal(got, want[k]):
            raise AssertionError(f"volume {k}: {got.ravel()} vs {want[k].ravel()}")


def _vol(shape, voxels):
    v = np.zeros(shape, np.uint8)
    for z, y, x in voxels:
        v[z, y, x] = 1
    return v


# Hand-worked: two voxels of a 2x2x2 cube, index (z*2 + y)*2 + x.
#   corner diagonal (0,0,0)-(1,1,1): offset (1,1,1), |d|_1 = 3: joined only at 26
#   edge diagonal   (0,0,0)-(1,1,0): offset (0,1,1), |d|_1 = 2: joined at 18 and 26
#   in-plane diagonal (0,0,0)-(0,1,1): same as the edge case, inside one slice
#   face neighbours (0,0,1)-(1,0,1): joined everywhere, label 1 + 1 = 2
HAND = [
    ([(0, 0, 0), (1, 1, 1)], {6: (1, 8), 18: (1, 8), 26: (1, 1)}),
    ([(0, 0, 0), (1, 1, 0)], {6: (1, 7), 18: (1, 1), 26: (1, 1)}),
    ([(0, 0, 0), (0, 1, 1)], {6: (1, 4), 18: (1, 1), 26: (1, 1)}),
    ([(0, 0, 1), (1, 0, 1)], {6: (2, 2), 18: (2, 2), 26: (2, 2)}),
]


@pytest.mark.parametrize("case", range(len(HAND)))
@pytest.mark.parametrize("conn", CONNS)
def test_hand_worked(case, conn):
    voxels, want = HAND[case]
    v = _vol((2, 2, 2), voxels)
    for fn in (oracle.label3d, oracle.label3d_py):
        lab = fn(v, conn)
        assert tuple(int(lab[z, y, x]) for z, y, x in voxels) == want[conn]
        assert int((lab > 0).sum()) == 2


def test_closed_forms():
    for shape in ((1, 1, 1), (3, 4, 5), (17, 9, 33)):
        for conn in CONNS:
            assert (oracle.label3d(np.zeros(shape, np.uint8), conn) == 0).all()
            assert (oracle.label3d(np.ones(shape, np.uint8), conn) == 1).all()
    # 3-D checkerboard (x+y+z even): no two foreground voxels share a face, so at
    # 6-connectivity every voxel is its own component; every pair at |d|_1 = 2
    # is an edge neighbour, so at 18 and 26 all of them form one component
    d, h, w = 6, 7, 8
    z, y, x = np.indices((d, h, w))
    cb = ((x + y + z) % 2 == 0).astype(np.uint8)
    idx = (z * h + y) * w + x
    np.testing.assert_array_equal(oracle.label3d(cb, 6), np.where(cb == 1, idx + 1, 0))
    for conn in (18, 26):
        np.testing.assert_array_equal(oracle.label3d(cb, conn), cb.astype(np.int32))
    # body-centred lattice (x, y, z all even, or all odd): only corner contacts
    bc = (((x % 2) == (y % 2)) & ((y % 2) == (z % 2))).astype(np.uint8)
    for conn in (6, 18):
        np.testing.assert_array_equal(oracle.label3d(bc, conn), np.where(bc == 1, idx + 1, 0))
    np.testing.assert_array_equal(oracle.label3d(bc, 26), bc.astype(np.int32))
    # slabs z = 0, 2, 4: slab k is labelled 1 + the index of its first voxel
    sl = (z % 2 == 0).astype(np.uint8)
    for conn in CONNS:
        np.testing.assert_array_equal(oracle.label3d(sl, conn),
                                      np.where(sl == 1, z * h * w + 1, 0))


@pytest.mark.parametrize("conn2,conns3", [(4, (6,)), (8, (18, 26))])
def test_thin_volumes_reduce_to_2d(conn2, conns3):
    """One slice (d = 1) or one row per slice (h = 1) is a 2-D image whose raster
    index equals the voxel index; in-plane neighbours are 4-neighbours at 6 and
    8-neighbours at 18 and 26."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        a, b = (int(v) for v in rng.integers(1, 40, size=2))
        img = (rng.random((a, b)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        want = oracle.label(img, conn2)
        for conn in conns3:
            np.testing.assert_array_equal(oracle.label3d(img[None, :, :], conn)[0], want)
            np.testing.assert_array_equal(oracle.label3d(img[:, None, :], conn)[:, 0, :], want)


@pytest.mark.parametrize("conn", CONNS)
def test_scipy_cross_check(conn):
    from scipy import ndimage

    st = ndimage.generate_binary_structure(3, {6: 1, 18: 2, 26: 3}[conn])
    rng = np.random.default_rng(17)
    for t in range(40):
        shape = tuple(int(v) for v in rng.integers(1, 36, size=3))
        p = (0.15, 0.25, 0.31, 0.4, 0.5, 0.7)[t % 6]
        vol = (rng.random(shape) < p).astype(np.uint8)
        lab, _ = ndimage.label(vol, structure=st)
        np.testing.assert_array_equal(oracle.label3d(vol, conn), canonical_from_arbitrary(lab))


@pytest.mark.parametrize("conn", CONNS)
def test_python_twin_and_invariants(conn):
    offs = [o for o in oracle._offsets3(conn)]
    rng = np.random.default_rng(23)
    for _ in range(12):
        shape = tuple(int(v) for v in rng.integers(1, 12, size=3))
        vol = (rng.random(shape) < rng.uniform(0.2, 0.7)).astype(np.uint8)
        lab = oracle.label3d(vol, conn)
        np.testing.assert_array_equal(oracle.label3d_py(vol, conn), lab)
        d, h, w = shape
        idx = np.arange(d * h * w).reshape(shape)
        fg = vol != 0
        assert np.all((lab == 0) == ~fg)
        assert np.all(lab[fg] - 1 <= idx[fg])
        flat = lab.ravel()
        vals = np.unique(lab[fg])
        assert np.all(flat[vals - 1] == vals)
        for dx, dy, dz in offs:
            # voxel p and its neighbour p + (dx, dy, dz), both inside the volume
            src = tuple(slice(max(0, -o), n - max(0, o)) for o, n in ((dz, d), (dy, h), (dx, w)))
            dst = tuple(slice(max(0, o), n - max(0, -o)) for o, n in ((dz, d), (dy, h), (dx, w)))
            both = fg[src] & fg[dst]
            la, lb = lab[src], lab[dst]
            assert np.array_equal(la[both], lb[both])


def test_closure_pin_catches_a_planted_mistake():
    """Labels computed at 6-connectivity fail the 26-connected closure pin."""
    vols = all_volumes(2, 2, 2)
    want = closure_labels3d(vols, 26)
    wrong = np.stack([oracle.label3d(v, 6) for v in vols])
    assert not np.array_equal(wrong, want)


def test_rejects_bad_args():
    with pytest.raises(ValueError):
        oracle.label3d(np.zeros((2, 2, 2), np.uint8), 8)
    with pytest.raises(ValueError):
        oracle.label3d(np.zeros((2, 2), np.uint8), 6)
