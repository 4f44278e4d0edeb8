"""Host-side logic of bench.py on CPU: max-over-ranks timing and the barrier
with two gloo ranks, and the reference arm's JSON line (oracle on host cores)."""
import json
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, values, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.reduce_max(values[rank], world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, got))


def test_reduce_max_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    values = [3.5, 7.25]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 7.25, 1: 7.25}


def test_reduce_max_single_rank_is_identity():
    assert bench.reduce_max(2.5, 1) == 2.5
    bench.barrier(1)


def test_reference_arm_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "H", 256)
    monkeypatch.setattr(bench, "W", 256)
    args = bench.argparse.Namespace(steps=3, warmup=3)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "Gpixels/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # non-zero ranks do no work and print nothing
    assert bench.run_reference(args, 1, 2) == 0
    assert capsys.readouterr().out == ""


def test_clock_sampler_summary_parsing():
    s = bench.ClockSampler("00000000:01:00.0")
    row = ["2026/12/03 10:00:00.000", "00000000:01:00.0", "1900", "2070", "800.5", "0x0",
           "Not Active", "Not Active", "Not Active", "Active"]
    s.rows = [(1.0, row), (2.0, row), (9.0, row)]
    out = s.summary(0.5, 2.5)
    assert out["samples"] == 2
    assert out["sm_mhz"] == 1900.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
