#!/usr/bin/env python3
"""Benchmark: union-find CCL of an 8192 x 8192 uint8 Bernoulli(p=0.5) image,
8-connectivity, plain single-image path (``ccl_label``), on N GPUs.

One step = one ``ccl_label`` call (local merge, seam unions, link) on one
resident 8192^2 image.  Each rank rotates over 3 distinct inputs (and outputs
and workspaces) so that consecutive steps never find their data in L2
(3 x (64 MiB in + 256 MiB out) > 129 MB L2).  W warm-up steps, then exactly K
timed steps bracketed by a barrier and a device synchronise on both sides,
timed with CUDA events on the launching stream; the max over ranks is used.
N > 1: independent replicas (images are independent; no collective on the
data path), weak scaling.

Also reported:
  roofline      per-kernel CUDA-event time of the dominant kernel (the link
                kernel, 4 B/px algorithmic) against the measured HBM peak;
                ``path`` gives the whole step against 5 B/px;
  e2e           the same metric through the server's C ABI with pinned HOST
                buffers: host-to-device copy + labelling + device-to-host copy;
  cpu_baseline  the CPU oracle (single-threaded BFS) on a bounded sample;
  clocks        nvidia-smi samples taken during the timed region;
  batched       256 images of 64..2048: one batched call vs 256 plain calls;
  served        Poisson request streams: the server vs one plain call per
                request, p50/p99 latency and throughput.

``--impl reference`` times the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("Gpixels/s & % HBM roofline (8192² p=0.5, 8-conn); batched/served vs plain, p99")
UNIT = "Gpixels/s"
H = W = 8192
P = 0.5
CONN = 8
ROTATE = 3
FALLBACK_HBM_GBS = 6800.0
KERNELS = ("local_merge", "seam_union", "link")
ALG_BYTES_PER_PX = {"local_merge": 1.0, "seam_union": 0.0, "link": 4.0}
PATH_BYTES_PER_PX = 5.0


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None) -> None:
    if world <= 1:
        return
    import torch.distributed as dist

    if device is not None and dist.get_backend() == "nccl":
        dist.barrier(device_ids=[device.index])
    else:
        dist.barrier()


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources of the profiled kernels (k_merge, k_seams, k_link and their launch)
PROFILED_SOURCES = ("ccl_core.cuh", "ccl_tile.cuh", "ccl_plain.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1708_08180_gb300", "csrc")
    for name in PROFILED_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d["kernels"][kernel]
        if d.get("source_hash") != kernel_source_hash():
            return None
        return float(ent["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


def ncu_warp_inst(kernel: str):
    """Warp instructions per launch of `kernel` from the committed ncu summary,
    if it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != kernel_source_hash():
            return None
        v = d["kernels"][kernel].get("warp_inst_per_launch")
        return float(v) if v else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples every 100 ms; keeps those inside [t0, t1]."""

    FIELDS = ("timestamp,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        rows = [r for (t, r) in self.rows if t0 <= t <= t1 and len(r) >= 10]
        if self.bus_id:
            mine = [r for r in rows if self.bus_id.endswith(r[1].lower()[-12:]) or
                    r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[4]) or 0.0) for r in rows)}


def cpu_baseline(img, budget_s: float = 15.0):
    """Time the CPU oracle (as it stands) on the benchmark image, single
    thread, for about `budget_s` seconds (at least 2 runs)."""
    import oracle

    oracle.label(img[:64], CONN)                      # build/load outside the timing
    times = []
    t_end = time.perf_counter() + budget_s
    while len(times) < 2 or (time.perf_counter() < t_end and len(times) < 20):
        t0 = time.perf_counter()
        oracle.label(img, CONN)
        times.append(time.perf_counter() - t0)
    med = statistics.median(times)
    return {"value": img.size / med / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle BFS on the full {H}x{W} p={P} {CONN}-conn image, {len(times)} runs, "
                      f"median {med:.3f} s", "runs": len(times)}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on host cores, rank 0 only."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import synthetic

    img = synthetic.bernoulli(H, W, P, seed=0)
    oracle.label(img[:64], CONN)
    # size each step's sample (whole rows of the benchmark image) so that the
    # run takes about two minutes in total
    t0 = time.perf_counter()
    oracle.label(img[:1024], CONN)
    px_per_s = 1024 * W / max(time.perf_counter() - t0, 1e-6)
    total_steps = max(1, args.steps + args.warmup)
    rows = int(max(1, min(H, 90.0 * px_per_s / total_steps / W)))
    sample = np.ascontiguousarray(img[:rows])
    for _ in range(args.warmup):
        oracle.label(sample, CONN)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.label(sample, CONN)
    dt = time.perf_counter() - t0
    value = sample.size * args.steps / dt / 1e9
    desc = (f"oracle BFS (single thread) on the first {rows} rows ({rows}x{W}) of the "
            f"{H}x{W} p={P} {CONN}-conn benchmark image per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{H}x{W} uint8 Bernoulli(p={P}), {CONN}-connectivity, CPU oracle",
                   "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def host_link_gbs(device_index: int, reps: int = 5):
    """The host link's bandwidth: one 256 MiB device-to-host and one 64 MiB
    host-to-device copy of pinned memory (CUDA events, best of `reps`), and
    both directions at once."""
    import torch

    dev = torch.device("cuda", device_index)
    d_big = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    d_small = torch.empty(64 << 20, dtype=torch.uint8, device=dev)
    h_big = torch.empty(256 << 20, dtype=torch.uint8).pin_memory()
    h_small = torch.empty(64 << 20, dtype=torch.uint8).pin_memory()
    s = torch.cuda.Stream(dev)

    def best(fn):
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            with torch.cuda.stream(s):
                fn()
            e1.record(s)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    d2h = best(lambda: h_big.copy_(d_big, non_blocking=True))
    h2d = best(lambda: d_small.copy_(h_small, non_blocking=True))
    both = best(lambda: (h_big.copy_(d_big, non_blocking=True), d_small.copy_(h_small, non_blocking=True)))
    return {"d2h_gb_s": round((256 << 20) / d2h / 1e6, 1), "h2d_gb_s": round((64 << 20) / h2d / 1e6, 1),
            "both_gb_s": round((320 << 20) / both / 1e6, 1)}


def e2e_server(img_np, steps: int, device_index: int):
    """Same metric through the server's C ABI with pinned host buffers: every
    request copies its image host-to-device and its labels device-to-host."""
    import torch

    import paper_1708_08180_gb300 as ccl

    n = max(4, min(steps, 48))
    ins = [torch.from_numpy(img_np).pin_memory() for _ in range(2)]
    window = 6
    outs = [torch.empty((H, W), dtype=torch.int32).pin_memory() for _ in range(window)]
    with ccl.Server(conn=CONN, max_batch=1, max_inflight=3, device=device_index) as srv:
        # warm-up (graph capture, pool growth)
        for k in range(3):
            srv.wait(srv.submit(ins[k % 2], outs[k % window]))
        t0 = time.perf_counter()
        ids = []
        for k in range(n):
            if len(ids) >= window:
                srv.wait(ids.pop(0))
            ids.append(srv.submit(ins[k % 2], outs[k % window]))
        for rid in ids:
            srv.wait(rid)
        dt = time.perf_counter() - t0
        stats = srv.stats()
        split = srv.timing()
    return {"value": n * H * W / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": H * W,
            "d2h_bytes_per_step": 4 * H * W, "requests": n,
            "server_p50_ms": stats["p50_ms"], "server_p99_ms": stats["p99_ms"],
            "per_request_ms": {"h2d": round(split["h2d_ms"], 4), "label": round(split["label_ms"], 4),
                               "d2h": round(split["d2h_ms"], 4)},
            "copy_gb_s": {"h2d": round(H * W / max(split["h2d_ms"], 1e-9) / 1e6, 1),
                          "d2h": round(4 * H * W / max(split["d2h_ms"], 1e-9) / 1e6, 1)},
            "what": "each request: host-to-device copy, labelling, device-to-host copy on one "
                    "worker stream (CUDA events); three workers overlap requests"}


def batched_vs_plain(device_index: int, seed: int = 0, reps: int = 10):
    """The batched configuration: 256 images, sides log-uniform in 64..2048,
    p ~ U(0.3, 0.7), 8-connectivity.  One batched call (graph replay) against
    256 plain ccl_label calls on one stream.  Both go through the C ABI with
    their arguments built beforehand (a C caller's cost, not the Python
    binding's), `reps` batches back to back between CUDA events, so that the
    device time is not diluted by host preparation; also the host latency of
    one synchronised batched call."""
    import ctypes

    import torch

    import paper_1708_08180_gb300 as ccl
    from paper_1708_08180_gb300 import _lib
    import synthetic

    lib = _lib.load()
    dev = torch.device("cuda", device_index)
    host = synthetic.batch_images(seed)
    imgs = [torch.from_numpy(h).to(dev) for h in host]
    outs = [torch.empty(tuple(i.shape), dtype=torch.int32, device=dev) for i in imgs]
    px = sum(h.size for h in host)
    ws_b = torch.empty(ccl.ccl_batched_workspace_bytes(imgs, 8), dtype=torch.uint8, device=dev)
    ws_p = torch.empty(max(ccl.ccl_workspace_bytes(*h.shape, 8) for h in host),
                       dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sh = ctypes.c_void_p(stream.cuda_stream)
    arr = (_lib.ccl_image * len(imgs))()
    for k, (im, o) in enumerate(zip(imgs, outs)):
        arr[k].d_img, arr[k].d_labels = im.data_ptr(), o.data_ptr()
        arr[k].height, arr[k].width = im.shape[0], im.shape[1]
    plain_args = [(ctypes.c_void_p(im.data_ptr()), ctypes.c_void_p(o.data_ptr()), im.shape[0],
                   im.shape[1]) for im, o in zip(imgs, outs)]
    wsb_p, wsb_n = ctypes.c_void_p(ws_b.data_ptr()), ws_b.numel()
    wsp_p, wsp_n = ctypes.c_void_p(ws_p.data_ptr()), ws_p.numel()

    def batched():
        st = lib.ccl_label_batched(arr, len(imgs), 8, wsb_p, wsb_n, sh)
        if st:
            raise ccl.CclError(st, "ccl_label_batched")

    def plain():
        for a, b, h, w in plain_args:
            st = lib.ccl_label(a, b, h, w, 8, wsp_p, wsp_n, sh)
            if st:
                raise ccl.CclError(st, "ccl_label")

    def time_it(fn):
        fn()
        fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    tb = time_it(batched)
    tp = time_it(plain)
    lat = []
    for _ in range(reps):
        t0 = time.perf_counter()
        batched()
        stream.synchronize()
        lat.append((time.perf_counter() - t0) * 1e3)
    ccl.ccl_sync(stream)
    lat.sort()
    peak, _ = hbm_peak()
    return {"images": len(host), "pixels": px,
            "batched_gpix_s": px / (tb / 1e3) / 1e9, "batched_ms": tb,
            "batched_path_frac_5B": round(5 * px / (tb / 1e3) / 1e9 / peak, 4),
            "batched_sync_latency_ms_p50": lat[len(lat) // 2], "batched_sync_latency_ms_max": lat[-1],
            "plain_gpix_s": px / (tp / 1e3) / 1e9, "plain_ms": tp,
            "speedup": tp / tb,
            "what": "device time per batch (CUDA events around %d back-to-back batches), "
                    "C ABI with prebuilt arguments; sync latency = one call + stream synchronise "
                    "on the host clock" % reps}


def served_vs_plain(device_index: int, rates=(1000.0, 5000.0, 20000.0), seconds: float = 1.0,
                    seed: int = 0, max_requests: int = 0):
    """Serving: Poisson arrivals; 50 % 1920x1080 smoothed-noise video frames,
    50 % squares log-uniform 128..4096, Bernoulli 0.5, 8-connectivity.  The
    continuous-batching server against one plain call per request (H2D,
    ccl_label, D2H, synchronise) replaying the same trace.  Latency = scheduled
    arrival -> labels in pinned host memory."""
    import numpy as np
    import torch

    import paper_1708_08180_gb300 as ccl
    import synthetic

    dev = torch.device("cuda", device_index)
    frames = synthetic.video_frames(16, seed)
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(128), np.log(4096), 16))).astype(int)
    squares = [synthetic.bernoulli(int(sd), int(sd), 0.5, k, cfg_id=synthetic.CFG_SERVE)
               for k, sd in enumerate(sides)]
    pool = {"frame": [torch.from_numpy(f).pin_memory() for f in frames],
            "square": [torch.from_numpy(q).pin_memory() for q in squares]}
    pool_out = {k: [torch.empty(tuple(t.shape), dtype=torch.int32).pin_memory() for t in v]
                for k, v in pool.items()}
    out = {}
    for rate in rates:
        count = max(1, int(rate * seconds))
        if max_requests > 0:
            count = min(count, max_requests)
        trace = synthetic.serving_trace(rate, count, seed)
        items = []
        for k, (t_arr, kind, h, w) in enumerate(trace):
            j = k % 16
            items.append((t_arr, pool[kind][j], pool_out[kind][j]))
        px = sum(int(i[1].numel()) for i in items)

        # server
        lat = [0.0] * len(items)
        with ccl.Server(conn=8, max_batch=64, max_inflight=3, device=device_index) as srv:
            srv.wait(srv.submit(items[0][1], items[0][2]))          # warm-up
            ids = [None] * len(items)
            done_t = [0.0] * len(items)
            t0 = time.perf_counter()

            def waiter():
                for k in range(len(items)):
                    while ids[k] is None:
                        time.sleep(2e-5)
                    srv.wait(ids[k])
                    done_t[k] = time.perf_counter() - t0

            th = threading.Thread(target=waiter)
            th.start()
            for k, (t_arr, src, dst) in enumerate(items):
                now = time.perf_counter() - t0
                if t_arr > now:
                    time.sleep(t_arr - now)
                ids[k] = srv.submit(src, dst)
            th.join()
            for k in range(len(items)):
                lat[k] = (done_t[k] - items[k][0]) * 1e3
            span = max(done_t) - items[0][0]
            native = srv.stats()
            split = srv.timing()
        # client side: scheduled arrival -> labels in host memory, seen by a
        # Python thread that waits in arrival order; native: the server's own
        # submit -> completion clock (C++ steady_clock, no interpreter in it)
        srv_res = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "gpix_s": px / span / 1e9,
                   "native_p50_ms": native.get("p50_ms"), "native_p99_ms": native.get("p99_ms"),
                   "per_batch_ms": {k: round(v, 4) for k, v in split.items() if k != "batches"},
                   "batches": split["batches"]}

        # plain: one ccl_label per request, in arrival order, one stream
        stream = torch.cuda.Stream(dev)
        maxpx = max(int(i[1].numel()) for i in items)
        d_in = torch.empty(maxpx, dtype=torch.uint8, device=dev)
        d_out = torch.empty(maxpx, dtype=torch.int32, device=dev)
        ws = torch.empty(max(ccl.ccl_workspace_bytes(*i[1].shape, 8) for i in items),
                         dtype=torch.uint8, device=dev)
        lat_p = []
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for t_arr, src, dst in items:
                now = time.perf_counter() - t0
                if t_arr > now:
                    time.sleep(t_arr - now)
                h, w = src.shape
                di = d_in[:h * w].view(h, w)
                do = d_out[:h * w].view(h, w)
                di.copy_(src, non_blocking=True)
                ccl.ccl_label(di, 8, out=do, ws=ws, stream=stream)
                dst.copy_(do, non_blocking=True)
                stream.synchronize()
                lat_p.append((time.perf_counter() - t0 - t_arr) * 1e3)
        span_p = time.perf_counter() - t0 - items[0][0]
        ccl.ccl_sync(stream)
        out[str(int(rate))] = {
            "requests": len(items), "offered_gpix_s": px / (items[-1][0] - items[0][0] + 1e-9) / 1e9,
            "server": srv_res,
            "plain": {"p50_ms": float(np.percentile(lat_p, 50)),
                      "p99_ms": float(np.percentile(lat_p, 99)), "gpix_s": px / span_p / 1e9}}
    return out


def flush_l2(buf):
    """Overwrite a buffer larger than L2 so that the next call reads from HBM."""
    buf.add_(1)


def small_leg(dev, stream, reps: int = 200):
    """The 512 x 512 workload (Bernoulli 0.5, 8-connectivity), seeds 0-9:
    back-to-back calls on one stream (throughput, CUDA events around `reps`
    calls per image) and single calls each followed by a device synchronise
    (latency, wall clock).  The inputs fit in L2 at this size, so the roofline
    fraction is informational only."""
    import torch

    import paper_1708_08180_gb300 as ccl
    import synthetic

    n = 512
    imgs = [torch.from_numpy(synthetic.bernoulli(n, n, 0.5, sd, cfg_id=synthetic.CFG_SMALL)).to(dev)
            for sd in range(10)]
    out = torch.empty((n, n), dtype=torch.int32, device=dev)
    ws = torch.empty(ccl.ccl_workspace_bytes(n, n, 8), dtype=torch.uint8, device=dev)
    per_img, lat = [], []
    for im in imgs:
        for _ in range(5):
            ccl.ccl_label(im, 8, out=out, ws=ws, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ccl.ccl_label(im, 8, out=out, ws=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        per_img.append(e0.elapsed_time(e1) / reps)
        for _ in range(20):
            t0 = time.perf_counter()
            ccl.ccl_label(im, 8, out=out, ws=ws, stream=stream)
            stream.synchronize()
            lat.append((time.perf_counter() - t0) * 1e3)
    ccl.ccl_sync(stream)
    ms = statistics.median(per_img)
    peak, _ = hbm_peak()
    return {"shape": [n, n], "density": 0.5, "conn": 8, "seeds": 10,
            "back_to_back_us": round(ms * 1e3, 2), "gpix_s": round(n * n / (ms / 1e3) / 1e9, 3),
            "path_frac_5B": round(5 * n * n / (ms / 1e3) / 1e9 / peak, 5),
            "sync_latency_p50_us": round(statistics.median(lat) * 1e3, 1),
            "sync_latency_p99_us": round(sorted(lat)[int(0.99 * (len(lat) - 1))] * 1e3, 1),
            "what": "per-call device time back to back (events) and host-synchronised latency"}


def structured_leg(dev, stream, reps: int = 10):
    """The structured 4096 x 4096 workload at both connectivities: block noise
    with g in {1, 2, 4, 8, 16}, the serpentine and its transpose, 64 concentric
    rings, full and empty.  Each image: `reps` calls, each timed with CUDA
    events after an L2 flush (a 256 MiB buffer overwritten), median."""
    import torch

    import paper_1708_08180_gb300 as ccl
    import synthetic

    n = 4096
    flush = torch.zeros(64 << 20, dtype=torch.int32, device=dev)
    out = torch.empty((n, n), dtype=torch.int32, device=dev)
    res = {}
    for name, img in synthetic.structured_set(n, n):
        dimg = torch.from_numpy(img).to(dev)
        for conn in (4, 8):
            ws = torch.empty(ccl.ccl_workspace_bytes(n, n, conn), dtype=torch.uint8, device=dev)
            ccl.ccl_label(dimg, conn, out=out, ws=ws, stream=stream)
            ts = []
            for _ in range(reps):
                flush_l2(flush)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ccl.ccl_label(dimg, conn, out=out, ws=ws, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            res[f"{name}_conn{conn}"] = {"ms": round(ms, 4),
                                         "gpix_s": round(n * n / (ms / 1e3) / 1e9, 2)}
    ccl.ccl_sync(stream)
    return {"shape": [n, n], "images": res,
            "what": "device time per call after an L2 flush, median of %d" % reps}


def stats_leg(labels, stream, reps: int = 50):
    """ccl_component_stats on the headline image's labels (count, bounding box
    and coordinate sums of every component, in label order): device time per
    call (CUDA events, after warm-up) and the number of components."""
    import torch

    import paper_1708_08180_gb300 as ccl

    h, w = labels.shape
    _, ncomps = ccl.ccl_component_stats(labels, 0, stream=stream)
    torch.cuda.synchronize()
    n = int(ncomps.item())
    ws = torch.empty(ccl.ccl_stats_workspace_bytes(h, w, n), dtype=torch.uint8,
                     device=labels.device)
    comps = torch.empty((max(n, 1), ccl.COMPONENT_WORDS), dtype=torch.int32, device=labels.device)
    for _ in range(3):
        ccl.ccl_component_stats(labels, n, comps=comps, ncomps=ncomps, ws=ws, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ccl.ccl_component_stats(labels, n, comps=comps, ncomps=ncomps, ws=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ccl.ccl_sync(stream)
    ms = e0.elapsed_time(e1) / reps
    return {"components": n, "ms": round(ms, 5), "gpix_s": round(h * w / (ms / 1e3) / 1e9, 2),
            "what": "pixel count, bounding box and coordinate sums of every component"}


def fused_stats_leg(imgs, outs, label_ms: float, stream, reps: int = 50):
    """ccl_label_with_stats on the headline images (labels and every
    component's statistics in one pass): device time per call (CUDA events,
    inputs rotated as in the headline loop), against the labelling alone."""
    import torch

    import paper_1708_08180_gb300 as ccl

    h, w = imgs[0].shape
    dev = imgs[0].device
    _, _, nc = ccl.ccl_label_with_stats(imgs[0], CONN, 0, out=outs[0], stream=stream)
    torch.cuda.synchronize()
    n = int(nc.item())
    cap = n + n // 4 + 1024
    comps = torch.empty((cap, ccl.COMPONENT_WORDS), dtype=torch.int32, device=dev)
    ncomps = torch.empty(1, dtype=torch.int32, device=dev)
    wss = [torch.empty(ccl.ccl_workspace_bytes_with_stats(h, w, CONN), dtype=torch.uint8,
                       device=dev) for _ in imgs]
    for k in range(3):
        ccl.ccl_label_with_stats(imgs[k % len(imgs)], CONN, cap, out=outs[k % len(imgs)], comps=comps,
                                 ncomps=ncomps, ws=wss[k % len(imgs)], stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(reps):
        ccl.ccl_label_with_stats(imgs[k % len(imgs)], CONN, cap, out=outs[k % len(imgs)], comps=comps,
                                 ncomps=ncomps, ws=wss[k % len(imgs)], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ccl.ccl_sync(stream)
    ms = e0.elapsed_time(e1) / reps
    return {"components": n, "ms": round(ms, 5), "gpix_s": round(h * w / (ms / 1e3) / 1e9, 2),
            "ratio_to_labelling": round(ms / label_ms, 3), "gpu_launches_per_call": 4,
            "what": "labels plus count, bounding box and coordinate sums of every component, "
                    "gathered in the link pass (ccl_label_with_stats)"}


def regions_leg(img, out, ws, stream, reps: int = 50):
    """ccl_label_regions on the headline image with levels {0, 1}: every
    region, background included (one three-phase pass per level).  Device
    time per call (CUDA events, after warm-up) and its pixel rate."""
    import torch

    import paper_1708_08180_gb300 as ccl

    h, w = img.shape
    for _ in range(3):
        ccl.ccl_label_regions(img, (0, 1), CONN, out=out, ws=ws, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ccl.ccl_label_regions(img, (0, 1), CONN, out=out, ws=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ccl.ccl_sync(stream)
    ms = e0.elapsed_time(e1) / reps
    return {"levels": [0, 1], "ms": round(ms, 5), "gpix_s": round(h * w / (ms / 1e3) / 1e9, 2),
            "gpu_launches_per_call": 6,
            "what": "every equal-value region (foreground and background) of the headline image"}


def volume_leg(dev, stream, reps: int = 20, side: int = 512, p: float = 0.5,
               conns=(6, 18, 26)):
    """ccl_label3d on a side^3 Bernoulli(p) volume at 6-, 18- and 26-connectivity:
    device time per call (CUDA events, after warm-up; input 128 MiB and labels
    512 MiB, both larger than L2) and its voxel rate."""
    import torch

    import paper_1708_08180_gb300 as ccl
    import synthetic

    vol = torch.from_numpy(synthetic.bernoulli3d(side, side, side, p, 0)).to(dev)
    out = torch.empty((side, side, side), dtype=torch.int32, device=dev)
    res = {"shape": [side, side, side], "density": p,
           "what": "3-D labelling (bricks of 16x16 strips of 1, 2 or 2x2 rows by 32 voxels), "
                   "labels 1 + smallest voxel index"}
    for conn in conns:
        ws = torch.empty(ccl.ccl_workspace_bytes3d(side, side, side, conn), dtype=torch.uint8,
                         device=dev)
        for _ in range(3):
            ccl.ccl_label3d(vol, conn, out=out, ws=ws, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ccl.ccl_label3d(vol, conn, out=out, ws=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ccl.ccl_sync(stream)
        ms = e0.elapsed_time(e1) / reps
        peak, _ = hbm_peak()
        res[f"conn{conn}"] = {"ms": round(ms, 4),
                              "gvox_s": round(side ** 3 / (ms / 1e3) / 1e9, 2),
                              "path_frac_5B": round(5 * side ** 3 / (ms / 1e3) / 1e9 / peak, 4)}
        del ws
    return res


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import paper_1708_08180_gb300 as ccl
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    ccl.load()

    host_imgs = [synthetic.bernoulli(H, W, P, seed=rank * ROTATE + r) for r in range(ROTATE)]
    imgs = [torch.from_numpy(h).to(dev) for h in host_imgs]
    outs = [torch.empty((H, W), dtype=torch.int32, device=dev) for _ in range(ROTATE)]
    wsb = ccl.ccl_workspace_bytes(H, W, CONN)
    wss = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(ROTATE)]
    stream = torch.cuda.current_stream(dev)

    for k in range(args.warmup):
        ccl.ccl_label(imgs[k % ROTATE], CONN, out=outs[k % ROTATE], ws=wss[k % ROTATE],
                      stream=stream)
    ccl.ccl_sync(stream)

    K = args.steps
    # Per-kernel times come from a second loop with events recorded between
    # the kernels; an event between two kernels stops the link kernel from
    # starting early (programmatic dependent launch), so the headline loop
    # records none.
    KP = min(K, args.phase_steps) if args.phase_steps > 0 else 0
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(max(KP, 1))]
    for e4 in ev:                      # materialise the CUDA events outside the timing
        for e in e4:
            e.record(stream)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    if bus is not None and not isinstance(bus, str):
        bus = f"{getattr(props, 'pci_domain_id', 0):08x}:{int(bus):02x}:{getattr(props, 'pci_device_id', 0):02x}.0"
    sampler = ClockSampler(bus)
    sampler.start()
    time.sleep(0.3)

    # The K timed steps are repeated back to back until the timed region spans
    # at least --min-timed-s of wall time, so that the clock sampler (100 ms
    # period) sees it; ms_per_step is the median repetition's K-step time / K.
    start.record(stream)
    for k in range(K):
        ccl.ccl_label(imgs[k % ROTATE], CONN, out=outs[k % ROTATE], ws=wss[k % ROTATE],
                      stream=stream)
    end.record(stream)
    torch.cuda.synchronize(dev)
    est_ms = max(start.elapsed_time(end), 1e-3)
    reps = max(1, min(100000, int(-(-args.min_timed_s * 1e3 // est_ms))))
    rep_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    for e0, e1 in rep_ev:
        e0.record(stream)
        for k in range(K):
            ccl.ccl_label(imgs[k % ROTATE], CONN, out=outs[k % ROTATE], ws=wss[k % ROTATE],
                          stream=stream)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    t_wall1 = time.time()
    barrier(world, dev)
    ccl.ccl_sync(stream)
    rep_ms = sorted(e0.elapsed_time(e1) for e0, e1 in rep_ev)
    # the per-kernel loop, same work, events around each kernel
    for k in range(KP):
        ccl.ccl_set_phase_events(ev[k])
        ccl.ccl_label(imgs[k % ROTATE], CONN, out=outs[k % ROTATE], ws=wss[k % ROTATE],
                      stream=stream)
    torch.cuda.synchronize(dev)
    t_wall2 = time.time()
    ccl.ccl_sync(stream)
    sampler.stop()

    ms_local = rep_ms[len(rep_ms) // 2]
    ms_total = reduce_max(ms_local, world, dev)
    phase = {name: [] for name in KERNELS}
    for k in range(KP):
        e = ev[k]
        phase["local_merge"].append(e[0].elapsed_time(e[1]))
        phase["seam_union"].append(e[1].elapsed_time(e[2]))
        phase["link"].append(e[2].elapsed_time(e[3]))
    phase_ms = {n: (statistics.mean(v) if v else 0.0) for n, v in phase.items()}
    phase_ms = {n: reduce_max(v, world, dev) for n, v in phase_ms.items()}
    clocks = sampler.summary(t_wall0, t_wall1)

    px = H * W
    ms_per_step = ms_total / K
    value = world * px * K / (ms_total / 1e3) / 1e9
    peak, peak_src = hbm_peak()
    dominant = max(phase_ms, key=lambda n: phase_ms[n])
    alg = ALG_BYTES_PER_PX[dominant] * px
    achieved = alg / (phase_ms[dominant] / 1e3) / 1e9 if phase_ms[dominant] > 0 else 0.0
    path_gbs = PATH_BYTES_PER_PX * px / (ms_per_step / 1e3) / 1e9
    traffic = ncu_traffic(dominant)
    roofline = {
        "bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1), "peak": peak,
        "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
        "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
        else "fallback 6.8 TB/s",
        "algorithmic_bytes_per_launch": alg,
        "kernel_ms": {n: round(v, 5) for n, v in phase_ms.items()},
        "kernel_ms_source": f"second timed loop of {KP} steps, CUDA events between the kernels "
                            "on the launching stream",
        "path": {"bytes_per_px": PATH_BYTES_PER_PX, "achieved": round(path_gbs, 1),
                 "frac": round(path_gbs / peak, 4)},
    }

    # The local merge is bound by instruction issue, not by HBM: its issue
    # roofline is warp instructions per launch (ncu, same sources) over the
    # launch time, against SMs x 4 schedulers x the median SM clock sampled
    # during the timed loop.
    winst = ncu_warp_inst("local_merge")
    sm_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
    if winst and sm_mhz and phase_ms["local_merge"] > 0:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ach = winst / (phase_ms["local_merge"] / 1e3) / 1e12
        pk = sms * 4 * sm_mhz * 1e6 / 1e12
        roofline["issue"] = {"kernel": "local_merge", "bound": "issue",
                             "achieved": round(ach, 4), "peak": round(pk, 4),
                             "unit": "T warp-inst/s", "frac": round(ach / pk, 4),
                             "warp_inst_per_launch": winst,
                             "peak_source": f"{sms} SMs x 4 issue slots x {sm_mhz:.0f} MHz"}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{H}x{W} uint8 Bernoulli(p={P}) image, {CONN}-connectivity, "
                               "plain single-image path (ccl_label)",
                   "tile": f"{ccl.ccl_default_tile_width(H, W, CONN)} px wide",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"{ROTATE} distinct inputs/outputs/workspaces rotated per step "
                         f"({ROTATE} x 320 MiB > 129 MB L2), no flush"},
        "roofline": roofline,
        "gpu_launches": 3 * K * reps,
        "clocks": clocks,
        "timing": {"repetitions_of_K_steps": reps, "rep_ms_min": round(rep_ms[0], 5),
                   "rep_ms_median": round(ms_local, 5), "rep_ms_max": round(rep_ms[-1], 5),
                   "timed_region_s": round(t_wall1 - t_wall0, 3),
                   "what": "the K timed steps repeated back to back so that the clock samples "
                           "cover the timed region; ms_per_step = median repetition / K"},
    }
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_server(host_imgs[0], K, local)
        link = host_link_gbs(local)
        ceiling = link["both_gb_s"] / PATH_BYTES_PER_PX   # Gpx/s the link allows at 5 B/px
        line["e2e"]["host_link"] = dict(link, gpix_s_ceiling=round(ceiling, 2),
                                        frac=round(line["e2e"]["value"] / ceiling, 3),
                                        what="pinned copies, CUDA events; the ceiling moves "
                                             "1 B/px in and 4 B/px out over the measured link")
    if rank == 0 and not args.no_small:
        line["small_512"] = small_leg(dev, stream)
    if rank == 0 and not args.no_structured:
        line["structured_4096"] = structured_leg(dev, stream)
    if rank == 0 and not args.no_stats:
        line["component_stats"] = stats_leg(outs[0], stream)
        line["label_with_stats"] = fused_stats_leg(imgs, outs, ms_per_step, stream)
    if rank == 0 and not args.no_volume:
        line["volume"] = volume_leg(dev, stream, side=args.volume_side)
    if rank == 0 and not args.no_regions:
        line["label_regions"] = regions_leg(imgs[1 % ROTATE], outs[1 % ROTATE], wss[1 % ROTATE],
                                            stream)
    if rank == 0 and not args.no_batched:
        line["batched"] = batched_vs_plain(local)
    if rank == 0 and not args.no_served:
        line["served"] = served_vs_plain(local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(host_imgs[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stats", action="store_true", help="skip the component-statistics leg")
    ap.add_argument("--no-small", action="store_true", help="skip the 512x512 leg")
    ap.add_argument("--no-structured", action="store_true",
                    help="skip the structured 4096x4096 leg")
    ap.add_argument("--no-volume", action="store_true", help="skip the 3-D volume leg")
    ap.add_argument("--served-full", action="store_true",
                    help="run only the serving sweep (1k-20k req/s, 10 s or 20k requests each)")
    ap.add_argument("--stats-only", action="store_true",
                    help="run only the component-statistics legs (one JSON line)")
    ap.add_argument("--cpu-sweep", action="store_true",
                    help="run only the CPU oracle over the density sweep and structured set")
    ap.add_argument("--volume-only", action="store_true",
                    help="run only the 3-D volume leg (one JSON line), e.g. for profiling")
    ap.add_argument("--volume-side", type=int, default=512, help="volume side (default 512)")
    ap.add_argument("--volume-conn", type=int, choices=(6, 18, 26), default=None,
                    help="one volume connectivity (default: 6, 18 and 26)")
    ap.add_argument("--volume-reps", type=int, default=20)
    ap.add_argument("--no-regions", action="store_true",
                    help="skip the every-region (levels 0 and 1) leg")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-vs-plain leg (256 images of 64..2048)")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served-vs-plain leg (Poisson arrivals)")
    ap.add_argument("--min-timed-s", type=float, default=1.5,
                    help="repeat the K timed steps until the timed region lasts this long "
                         "(clock samples need it); the median repetition is reported")
    ap.add_argument("--phase-steps", type=int, default=1000,
                    help="steps of the second, per-kernel timed loop (0: skip it)")
    ap.add_argument("--size", type=int, default=8192, help="image side (default 8192)")
    ap.add_argument("--density", type=float, default=0.5, help="Bernoulli p (default 0.5)")
    ap.add_argument("--conn", type=int, choices=(4, 8), default=8)
    ap.add_argument("--rotate", type=int, default=3,
                    help="distinct input/output/workspace sets cycled per step (default 3)")
    args = ap.parse_args(argv)
    global H, W, P, CONN, ROTATE
    H = W = args.size
    P = args.density
    CONN = args.conn
    ROTATE = max(1, args.rotate)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.volume_only:
        return run_volume_only(args, local)
    if args.served_full:
        return run_served_full(args, local)
    if args.stats_only:
        return run_stats_only(args, local)
    if args.cpu_sweep:
        return run_cpu_sweep(args)
    return run_ours(args, rank, world, local)


def run_served_full(args, local) -> int:
    """The serving workload at every rate of its sweep (1k, 2k, 5k, 10k, 20k
    requests/s), each run for 10 s of arrivals or 20,000 requests, whichever
    comes first: server vs one plain call per request, one JSON line."""
    import torch

    import paper_1708_08180_gb300 as ccl

    torch.cuda.set_device(local)
    ccl.load()
    res = served_vs_plain(local, rates=(1000.0, 2000.0, 5000.0, 10000.0, 20000.0),
                          seconds=10.0, max_requests=20000)
    print(json.dumps({"served_full": res}), flush=True)
    return 0


def run_cpu_sweep(args) -> int:
    """The CPU oracle (single-threaded breadth-first labelling) over the
    plain-path sweep -- 1024^2 ... 8192^2 x p = 0.1 ... 0.9 x 4/8-connectivity,
    seed 0 -- and the structured 4096^2 set, each the median of 3 runs, in
    Mpixels/s; with the host's core count and CPU model."""
    import platform

    import oracle
    import synthetic

    oracle.label(synthetic.bernoulli(64, 64, 0.5, 0), 8)     # build/load outside the timing

    def med3(img, conn):
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            oracle.label(img, conn)
            ts.append(time.perf_counter() - t0)
        return img.size / statistics.median(ts) / 1e6

    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    out = {"cores_used": 1, "nproc": os.cpu_count(), "cpu": model, "machine": platform.machine(),
           "unit": "Mpixels/s", "sweep": {}, "structured_4096": {}}
    for n in (1024, 2048, 4096, 8192):
        for k in range(1, 10):
            p = k / 10
            img = synthetic.bernoulli(n, n, p, 0)
            for conn in (4, 8):
                out["sweep"][f"{n}_p{p:.1f}_conn{conn}"] = round(med3(img, conn), 2)
    for name, img in synthetic.structured_set(4096, 4096):
        for conn in (4, 8):
            out["structured_4096"][f"{name}_conn{conn}"] = round(med3(img, conn), 2)
    print(json.dumps({"cpu_sweep": out}), flush=True)
    return 0


def run_stats_only(args, local) -> int:
    """Only the statistics legs on the headline images (ccl_component_stats
    after labelling, and ccl_label_with_stats), one JSON line."""
    import torch

    import paper_1708_08180_gb300 as ccl
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ccl.load()
    stream = torch.cuda.current_stream(dev)
    imgs = [torch.from_numpy(synthetic.bernoulli(H, W, P, seed=r)).to(dev) for r in range(ROTATE)]
    outs = [torch.empty((H, W), dtype=torch.int32, device=dev) for _ in range(ROTATE)]
    ws = torch.empty(ccl.ccl_workspace_bytes(H, W, CONN), dtype=torch.uint8, device=dev)
    for k in range(3):
        ccl.ccl_label(imgs[k % ROTATE], CONN, out=outs[k % ROTATE], ws=ws, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(20):
        ccl.ccl_label(imgs[k % ROTATE], CONN, out=outs[k % ROTATE], ws=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    label_ms = e0.elapsed_time(e1) / 20
    res = {"label_ms": round(label_ms, 5), "component_stats": stats_leg(outs[0], stream),
           "label_with_stats": fused_stats_leg(imgs, outs, label_ms, stream)}
    print(json.dumps(res), flush=True)
    return 0


def run_volume_only(args, local) -> int:
    import torch

    import paper_1708_08180_gb300 as ccl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ccl.load()
    conns = (args.volume_conn,) if args.volume_conn else (6, 18, 26)
    res = volume_leg(dev, torch.cuda.current_stream(dev), reps=args.volume_reps,
                     side=args.volume_side, p=args.density, conns=conns)
    print(json.dumps({"volume": res}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
