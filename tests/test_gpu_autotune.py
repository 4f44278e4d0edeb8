"""The autotuner measures every admissible tile width per size class and
installs the fastest; labels stay bit-exact under any table."""
import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402


@pytest.mark.parametrize("conn", [4, 8])
def test_autotune_installs_valid_table_and_results_stay_exact(conn):
    saved = ccl.ccl_get_tile_table(conn)
    try:
        table = ccl.ccl_autotune(conn, reps=1)
        assert all(w in (32, 64, 128, 256) for row in table for w in row)
        for h, w in ((64, 3000), (700, 90), (2100, 2100), (5000, 40)):
            img = synthetic.bernoulli(h, w, 0.5, 7, cfg_id=60)
            got = ccl.label(torch.from_numpy(img).cuda(), conn).cpu().numpy()
            np.testing.assert_array_equal(got, oracle.label(img, conn))
    finally:
        ccl.ccl_set_tile_table(conn, saved)
