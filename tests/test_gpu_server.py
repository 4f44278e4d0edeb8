"""Server: continuous batching of host-memory requests.  Every result equals
the same image labelled alone (tolerance 0) and the oracle; admission by HBM
budget; shutdown drains admitted work."""
import threading

import numpy as np
import pytest

import oracle
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1708_08180_gb300 as ccl  # noqa: E402


def pinned(arr):
    t = torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
    return t


def mixed_requests(n, seed):
    rng = np.random.default_rng(seed)
    frames = synthetic.video_frames(4, seed, h=270, w=480)
    reqs = []
    for k in range(n):
        if k % 2 == 0:
            reqs.append(frames[(k // 2) % len(frames)])
        else:
            s = int(round(np.exp(rng.uniform(np.log(32), np.log(700)))))
            reqs.append(synthetic.bernoulli(s, s, 0.5, k, cfg_id=40))
    return reqs


def test_results_same_alone_and_in_the_mix():
    reqs = mixed_requests(60, 0)
    outs = [pinned(np.zeros(r.shape, np.int32)) for r in reqs]
    ins = [pinned(r) for r in reqs]
    with ccl.Server(conn=8, hbm_budget_bytes=1 << 30, max_batch=16, max_inflight=2) as srv:
        ids = [srv.submit(i, o) for i, o in zip(ins, outs)]
        for rid in ids:
            srv.wait(rid, timeout_ms=60000)
        st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for r, o in zip(reqs, outs):
        alone = ccl.label(torch.from_numpy(r).cuda(), 8).cpu().numpy()
        np.testing.assert_array_equal(o.numpy(), alone)
        np.testing.assert_array_equal(o.numpy(), oracle.label(r, 8))


def test_concurrent_submitters_and_poll():
    reqs = mixed_requests(40, 1)
    outs = [pinned(np.zeros(r.shape, np.int32)) for r in reqs]
    ins = [pinned(r) for r in reqs]
    ids = [None] * len(reqs)
    with ccl.Server(conn=4, hbm_budget_bytes=256 << 20, max_batch=8, max_inflight=3) as srv:
        def go(part):
            for k in part:
                ids[k] = srv.submit(ins[k], outs[k])
        ts = [threading.Thread(target=go, args=(range(j, len(reqs), 2),)) for j in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        pending = set(ids)
        while pending:
            pending = {rid for rid in pending if not srv.poll(rid)}
    for r, o in zip(reqs, outs):
        np.testing.assert_array_equal(o.numpy(), oracle.label(r, 4))


def test_budget_admission_and_rejection():
    big = np.zeros((2048, 2048), np.uint8)
    out = np.zeros((2048, 2048), np.int32)
    with ccl.Server(conn=8, hbm_budget_bytes=8 << 20, max_batch=4, max_inflight=2) as srv:
        with pytest.raises(ccl.CclError) as ei:
            srv.submit(big, out)
        assert ei.value.status == 5   # CCL_ERR_REJECTED
        # requests that fit only one at a time still all complete
        reqs = [synthetic.bernoulli(700, 700, 0.5, k, cfg_id=41) for k in range(6)]
        outs = [np.zeros(r.shape, np.int32) for r in reqs]
        ids = [srv.submit(r, o) for r, o in zip(reqs, outs)]
        for rid in ids:
            srv.wait(rid, timeout_ms=60000)
        assert srv.stats()["rejected"] == 1
    for r, o in zip(reqs, outs):
        np.testing.assert_array_equal(o, oracle.label(r, 8))


def test_destroy_drains_admitted_work():
    reqs = [synthetic.bernoulli(512, 512, 0.5, k, cfg_id=42) for k in range(12)]
    outs = [np.zeros(r.shape, np.int32) for r in reqs]
    srv = ccl.Server(conn=8, hbm_budget_bytes=1 << 30, max_batch=4, max_inflight=2)
    for r, o in zip(reqs, outs):
        srv.submit(r, o)
    srv.close()
    for r, o in zip(reqs, outs):
        np.testing.assert_array_equal(o, oracle.label(r, 8))


def test_wait_timeout_and_unknown_id():
    with ccl.Server(conn=8, hbm_budget_bytes=1 << 30) as srv:
        with pytest.raises(ccl.CclError) as ei:
            srv.wait(123456, timeout_ms=10)
        assert ei.value.status == 7   # CCL_ERR_NOT_FOUND
