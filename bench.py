#!/usr/bin/env python
"""Benchmark: exact 2D median of a 4096x4096 uint16 (12-bit x-ray-like) image
at radii 1, 5, 15 and 50 -- output Mpix/s against radius, fraction of the HBM
roofline, p50/p99 per launch.

One step filters the image once at every radius (the whole hot path: the
selection network at r = 1, the level pre-pass plus the hierarchical
histogram kernel at r >= 3).  L2 is flushed (a 512 MiB write) before every
launch; launches are timed with CUDA events on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hrm|reference]

Multi-GPU (torchrun, one process per GPU): every rank filters its own image
(weak scaling, no data-path collective); the timing is the max over ranks.
``--impl reference`` times the brute-force CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "output Mpix/s vs radius (uint16 4096^2, bit-exact) and % HBM roofline; p50/p99 ms"
UNIT = "Mpix/s"
RADII = (1, 5, 15, 50)
SIDE = 4096
SORTNET_MAX_R = 5  # 2D radii served by the selection networks (one launch, no pre-pass)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- clocks ------------------------------------------------------------------

REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, index: str):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(REASONS, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- roofline traffic from a committed ncu summary ----------------------------

def csrc_hash() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1105_3829_gb300", "csrc", "*"))):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, key: str = "kernels"):
    """Per-launch figures recorded by profiles/traffic.json for the current
    kernel sources (DRAM bytes by default; null when the sources changed
    since the capture)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("csrc_hash") != csrc_hash():
        return None
    return d.get(key, {}).get(kernel)


# ---- multi-GPU host logic (weak scaling: every rank filters its own image) ----

def rank_seed(rank: int) -> int:
    """Seed of rank's image: each rank gets a distinct image of the same recipe."""
    from paper_1105_3829_gb300 import inputs
    return inputs.seed_for(2, rank)


def max_over_ranks(dist, vals, device):
    """Element-wise max of per-rank floats (the slowest rank sets the time)."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_value(ws: int, nradii: int, npx: int, ms_per_step: float) -> float:
    """Whole-job Mpix/s: every rank's outputs of one step over the max step time."""
    return ws * nradii * npx / (ms_per_step * 1e-3) / 1e6


def bench_config(ws: int, img=None) -> dict:
    """The benchmark workload, shared by both arms' JSON lines (with the
    SHA-256 prefix of rank 0's input image when it is given)."""
    extra = {} if img is None else {"input_sha256": hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest()[:16]}
    return extra | {"workload": "2D median, 4096x4096 uint16 12-bit x-ray mixture (0.6 N(800,150) + "
                        "0.4 N(3000,400), 1% salt/pepper), radii 1/5/15/50, replicate border",
            "radii": list(RADII), "width": SIDE, "height": SIDE, "parallelism": "dp%d" % ws,
            "l2": "flushed (512 MiB write) before every launch; ms_per_step is the sum of the "
                  "launches' CUDA-event times, flushes excluded"}


# ---- CPU oracle on a bounded sample ---------------------------------------------

def oracle_sample(img, budget_s: float, radii=RADII):
    """Time the oracle on the same number P of random output points at every
    radius (the GPU metric weights the radii equally), with P chosen so the
    whole sample takes about budget_s seconds.  Returns (points, seconds,
    threads)."""
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    rng = np.random.default_rng(12345)
    # calibration: grow the probe until it takes a measurable time, so the
    # per-call thread start-up does not dominate the per-point cost
    n0 = 16 * threads
    while True:
        spent = 0.0
        for r in radii:
            ys, xs = rng.integers(0, img.shape[0], n0), rng.integers(0, img.shape[1], n0)
            t0 = time.perf_counter()
            oracle.points(img, r, ys, xs, threads=threads)
            spent += time.perf_counter() - t0
        if spent >= min(0.5, budget_s / 8) or n0 >= 1_000_000:
            break
        n0 *= 4
    cost = spent / n0
    P = int(max(16 * threads, min(20_000_000, budget_s / max(cost, 1e-9))))
    tot_s = 0.0
    for r in radii:
        ys, xs = rng.integers(0, img.shape[0], P), rng.integers(0, img.shape[1], P)
        t0 = time.perf_counter()
        oracle.points(img, r, ys, xs, threads=threads)
        tot_s += time.perf_counter() - t0
    return P * len(radii), tot_s, threads


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from paper_1105_3829_gb300 import inputs
    img = inputs.xray12_u16(SIDE, SIDE)
    step_budget = args.ref_step_seconds or max(2.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(img, step_budget / 4, radii=RADII)
    pts, secs = 0, 0.0
    threads = 1
    for _ in range(args.steps):
        p, s, threads = oracle_sample(img, step_budget, radii=RADII)
        pts += p
        secs += s
    value = pts / secs / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic",
        "config": bench_config(args.gpus, img),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "per step: random output points at each radius, ~%.0f s of CPU work "
                                   "(brute-force gather + Quickselect per point)" % step_budget},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---- secondary workloads (one JSON line each; not the benchmark headline) --------------

def _timed(fn, flush, reps=5, warm=2):
    """CUDA-event time (ms) of fn() per call, L2 flushed before each call."""
    import torch
    for _ in range(warm):
        fn()
    out = []
    for _ in range(reps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return np.array(out)


def _line(metric, unit, value, extra, args, hib=True, clk=None):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
         "higher_is_better": hib, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    d.update(extra)
    if clk is not None:
        d["clocks"] = clk.summary()
    print(json.dumps(d))


def _smi_index(local: int = 0) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    return vis.split(",")[local].strip() if vis else str(local)


def run_secondary(args):
    import torch
    from __graft_entry__ import build
    from paper_1105_3829_gb300 import hrm, inputs
    build()
    dev = torch.device("cuda", 0)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    reps = max(3, args.steps)
    if args.workload == "volume3d":
        vol_np = inputs.xray12_volume()
        vol = torch.from_numpy(vol_np).to(dev)
        octs = [torch.from_numpy(o).to(dev) for o in inputs.octants(vol_np)]
        nvox = vol.numel()
        res = {}
        clk = ClockSampler(_smi_index()).__enter__()
        for r in (1, 3, 7):
            out = torch.empty_like(vol)
            outs = [torch.empty_like(o) for o in octs]
            jobs = [hrm.make_job(o, d_, r) for o, d_ in zip(octs, outs)]
            g = hrm.BatchGraph(jobs)
            t_single = _timed(lambda: hrm.filter3d(vol, r, out=out), flush, reps)
            t_batch = _timed(lambda: hrm.filter_batch(jobs), flush, reps)
            t_graph = _timed(lambda: g.launch(), flush, reps)
            t_sep = _timed(lambda: [hrm.filter3d(o, r, out=d_) for o, d_ in zip(octs, outs)], flush, reps)
            g.close()
            med = lambda t: float(np.median(t))
            res[str(r)] = {"volume_256_mvox_s": nvox / med(t_single) / 1e3,
                           "octants_one_launch_mvox_s": nvox / med(t_batch) / 1e3,
                           "octants_graph_replay_mvox_s": nvox / med(t_graph) / 1e3,
                           "octants_8_launches_mvox_s": nvox / med(t_sep) / 1e3,
                           "p50_ms": {"single": med(t_single), "batch": med(t_batch), "graph": med(t_graph),
                                      "separate": med(t_sep)},
                           "p99_ms_batch": float(np.percentile(t_batch, 99))}
        clk.__exit__()
        value = float(np.mean([v["octants_one_launch_mvox_s"] for v in res.values()]))
        _line("3D median, uint16 256^3 as 8 x 128^3 in one launch: output Mvox/s (mean over r=1,3,7)", "Mvox/s",
              value, {"dtype": "u16", "per_radius": res,
                      "config": {"workload": "3D median 256^3 uint16 x-ray mixture + 3D low-frequency noise; "
                                             "8 octant volumes in one persistent launch vs one 256^3 volume vs 8 "
                                             "launches", "l2": "flushed before every timed call"}}, args, clk=clk)
    elif args.workload in ("lowkey2d", "u8small"):
        if args.workload == "lowkey2d":
            img_np, radii, dt = inputs.lowkey16_u16(), (15, 50), "u16"
        else:
            img_np, radii, dt = inputs.uniform_u8(), (3,), "u8"
        img = torch.from_numpy(img_np).to(dev)
        out = torch.empty_like(img)
        res = {}
        clk = ClockSampler(_smi_index()).__enter__()
        for r in radii:
            for ad in ((False, True) if args.workload == "lowkey2d" else (False,)):
                t = _timed(lambda: hrm.filter2d(img, r, adaptive=ad, out=out), flush, reps)
                case = {"mpix_s": img.numel() / float(np.median(t)) / 1e3, "p50_ms": float(np.median(t)),
                        "p99_ms": float(np.percentile(t, 99))}
                if args.workload == "lowkey2d":  # the same call after hrm_autotune picked the plan
                    plan = hrm.autotune(img, r, adaptive=ad)
                    t2 = _timed(lambda: hrm.filter2d(img, r, adaptive=ad, out=out), flush, reps)
                    case["autotuned"] = {"p50_ms": float(np.median(t2)),
                                         "mpix_s": img.numel() / float(np.median(t2)) / 1e3,
                                         "plan": {"tile_width": plan.tile_width, "strip_height": plan.strip_height,
                                                  "slot_kbytes": plan.slot_kbytes, "path": plan.path,
                         "tree": ("uniform", "adaptive")[plan.tree - 1] if plan.tree else None}}
                res["r%d%s" % (r, "_adaptive" if ad else "")] = case
        clk.__exit__()
        value = float(np.mean([v.get("autotuned", v)["mpix_s"] for v in res.values()]))
        _line("2D median %s: output Mpix/s (mean over cases%s)" % ("8192^2 uint16 low-key" if dt == "u16" else
                                                               "512^2 uint8 uniform r=3",
                                                               ", autotuned plans" if dt == "u16" else ""),
              "Mpix/s", value, {"dtype": dt, "cases": res,
                                "config": {"workload": args.workload, "l2": "flushed before every timed call"}}, args,
              clk=clk)
    elif args.workload == "video":
        run_video(args, hrm, inputs, torch, dev, flush)
    elif args.workload == "paper":
        run_paper(args, hrm, inputs, torch, dev, flush)
    else:
        run_serve(args, hrm, inputs, torch, dev)
    return 0


def run_video(args, hrm, inputs, torch, dev, flush):
    """Frame stream (8 frames of 4096^2 uint16 low-key content with blobs
    drifting 4 px per frame): per-frame time of the uniform tree, the
    image-based adaptive tree, and the topology carried from the previous
    frame's medians (Section III-C).  Outputs are identical in all three."""
    frames = [torch.from_numpy(f).to(dev) for f in inputs.video_frames(8, 4096, 4096, drift=4)]
    out = torch.empty_like(frames[0])
    res = {}
    clk = ClockSampler(_smi_index()).__enter__()
    for r in (15, 50):
        row = {}
        for mode in ("uniform", "adaptive", "video"):
            topo = hrm.Topology() if mode == "video" else None
            times = []
            for rep in range(2):  # the first pass warms up the plan (and the topology)
                for f in frames:
                    flush.fill_(1)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    if mode == "video":
                        hrm.filter2d_video(f, r, topo, out=out)
                    else:
                        hrm.filter2d(f, r, adaptive=(mode == "adaptive"), out=out)
                    e1.record()
                    torch.cuda.synchronize()
                    if rep:
                        times.append(e0.elapsed_time(e1))
            if topo:
                topo.close()
            row[mode] = {"ms_per_frame": float(np.mean(times)), "mpix_s": out.numel() / float(np.mean(times)) / 1e3}
        res["r%d" % r] = row
    value = float(np.mean([res[k]["video"]["mpix_s"] for k in res]))
    res["served"] = _served_streams(hrm, inputs, torch, dev)
    clk.__exit__()
    _line("frame stream: output Mpix/s with the previous frame's topology (mean over r=15,50)", "Mpix/s", value,
          {"dtype": "u16", "cases": res, "config": {"workload": "video: 8 frames 4096^2 uint16 low-key, blobs "
                                                    "drifting 4 px/frame; served: 4 streams x 8 frames 2048^2 "
                                                    "through the server", "l2": "flushed before every timed call "
                                                    "(served: host wall clock, submit of the first frame to the "
                                                    "poll of the last)"}},
          args, clk=clk)


def _served_streams(hrm, inputs, torch, dev, nstreams=4, nframes=8, side=2048, r=15):
    """Several frame streams through the serving loop, all frames submitted
    at once: each stream keeps its order (one frame per wave) while frames of
    different streams share waves.  Wall-clock throughput with a topology per
    stream vs the same frames as plain requests (uniform tree)."""
    import time
    streams = [[torch.from_numpy(f).to(dev) for f in inputs.video_frames(nframes, side, side, drift=4,
                                                                          seed=inputs.seed_for(6, 10 + k))]
               for k in range(nstreams)]
    outs = [[torch.empty_like(f) for f in s] for s in streams]
    arena = torch.empty(4 << 30, dtype=torch.uint8, device=dev)
    row = {}
    for mode in ("plain", "topology"):
        best = waves = None
        for rep in range(2):  # the first pass warms up plans and topologies
            srv = hrm.Server(arena, max_inflight=4096, max_queue=16384)
            topos = [hrm.Topology() for _ in range(nstreams)] if mode == "topology" else [None] * nstreams
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tickets = [srv.submit(streams[k][f], outs[k][f], r, topo=topos[k])
                       for f in range(nframes) for k in range(nstreams)]
            for i, t in enumerate(tickets):
                rc = srv.poll(t, 60_000_000)  # bounded: a lost wave fails the run instead of hanging it
                if rc != hrm.HRM_OK:
                    raise RuntimeError("served frame %d (%s) failed: %d" % (i, mode, rc))
            dt = time.perf_counter() - t0
            waves = int(srv.stats().waves)
            srv.close()
            for t in topos:
                if t is not None:
                    t.close()
            if rep:
                best = dt
        npx = nstreams * nframes * side * side
        row[mode] = {"wall_ms": best * 1e3, "mpix_s": npx / best / 1e6, "waves": waves}
    row["config"] = "%d streams x %d frames %d^2 uint16 low-key, r=%d" % (nstreams, nframes, side, r)
    return row


def run_paper(args, hrm, inputs, torch, dev, flush):
    """The paper's synthetic workloads at its window n = 51 (r = 25),
    4096^2: random normal (mid-range mean, 3 sigma = half range) and diagonal
    sines of period 100 / 25 px, 8-bit and 16-bit, uniform and adaptive tree.
    The paper's single-core CPU figures (Tables I/II) are context only."""
    cases = {"normal8": inputs.paper_normal(4096, 4096, 8, seed=inputs.seed_for(7, 1)),
             "sine100_8": inputs.paper_sine(4096, 4096, 100, 8),
             "sine25_8": inputs.paper_sine(4096, 4096, 25, 8),
             "normal16": inputs.paper_normal(4096, 4096, 16, seed=inputs.seed_for(7, 2)),
             "sine100_16": inputs.paper_sine(4096, 4096, 100, 16)}
    res = {}
    clk = ClockSampler(_smi_index()).__enter__()
    imgs = {name: torch.from_numpy(a).to(dev) for name, a in cases.items()}
    for name, img in imgs.items():
        out = torch.empty_like(img)
        for ad in (False, True):
            t = _timed(lambda: hrm.filter2d(img, 25, adaptive=ad, out=out), flush, max(3, args.steps))
            ms = float(np.median(t))
            res["%s%s" % (name, "_adaptive" if ad else "")] = {"p50_ms": ms, "mpix_s": img.numel() / ms / 1e3}
    # the node cache's worst case: what hrm_autotune finds for the 16-bit images (after every default
    # timing: images of one size, dtype and radius share a problem class, hence a cached plan)
    for name, img in imgs.items():
        if not name.endswith("16"):
            continue
        out = torch.empty_like(img)
        for ad in (False, True):
            plan = hrm.autotune(img, 25, adaptive=ad)
            t2 = _timed(lambda: hrm.filter2d(img, 25, adaptive=ad, out=out), flush, max(3, args.steps))
            res["%s%s" % (name, "_adaptive" if ad else "")]["autotuned"] = {
                "p50_ms": float(np.median(t2)), "mpix_s": img.numel() / float(np.median(t2)) / 1e3,
                "plan": {"tile_width": plan.tile_width, "strip_height": plan.strip_height,
                         "slot_kbytes": plan.slot_kbytes, "path": plan.path,
                         "tree": ("uniform", "adaptive")[plan.tree - 1] if plan.tree else None}}
    clk.__exit__()
    value = float(np.mean([v["mpix_s"] for v in res.values()]))
    _line("paper synthetic workloads at r=25 (4096^2): output Mpix/s (mean over cases)", "Mpix/s", value,
          {"dtype": "u8+u16", "cases": res, "config": {"workload": "paper: random normal and diagonal sines, "
                                                       "8/16-bit, r=25", "l2": "flushed before every timed call"}},
          args, clk=clk)


def run_serve(args, hrm, inputs, torch, dev):
    """Continuous batching (hrm server) vs plain per-image launches on the same
    Poisson request stream: latency from arrival to result, and throughput.
    After the timing, every served output is compared bit for bit with the
    plain launch of the same request; any difference fails the run."""
    pool = {"u8": torch.from_numpy(inputs.uniform_u8(4096, 4096)).to(dev),
            "u16": torch.from_numpy(inputs.xray12_u16(4096, 4096)).to(dev)}
    arena = torch.empty(16 << 30, dtype=torch.uint8, device=dev)  # the 16 GB admission budget
    results = {}
    clk = ClockSampler(_smi_index()).__enter__()
    for rate in [float(x) for x in args.rates.split(",")]:
        n = int(min(args.requests, rate * 10))
        reqs = inputs.request_stream(n, rate=rate, seed=inputs.seed_for(5, int(rate)))
        rng = np.random.default_rng(int(rate))
        views = []
        for q in reqs:
            y0, x0 = rng.integers(0, 4097 - q["h"]), rng.integers(0, 4097 - q["w"])
            views.append(pool[q["dtype"]][y0:y0 + q["h"], x0:x0 + q["w"]])
        npx = sum(q["w"] * q["h"] for q in reqs)
        outs = [torch.empty_like(v) for v in views]
        plain_outs = [torch.empty_like(v) for v in views]
        torch.cuda.synchronize()
        # (a) server: continuous batching
        srv = hrm.Server(arena, max_inflight=4096, max_queue=16384)
        tick = [0] * n
        t0 = time.perf_counter()
        for i, q in enumerate(reqs):
            while time.perf_counter() - t0 < q["t"]:
                pass
            tick[i] = srv.submit(views[i], outs[i], q["r"])
        for i in range(n):
            rc = srv.poll(tick[i], 600_000_000)  # bounded: a lost wave fails the run instead of hanging it
            if rc != hrm.HRM_OK:
                raise SystemExit("served request %d failed with status %d" % (i, rc))
        t_srv = time.perf_counter() - t0
        lat_srv = np.array([srv.latency_us(t) for t in tick]) / 1e3
        st = srv.stats()
        srv.close()
        # (b) plain launches: one hrm_filter2d per request, in arrival order
        stream = torch.cuda.current_stream()
        lat_plain = np.zeros(n)
        t0 = time.perf_counter()
        for i, q in enumerate(reqs):
            while time.perf_counter() - t0 < q["t"]:
                pass
            hrm.filter2d(views[i], q["r"], out=plain_outs[i])
            stream.synchronize()
            lat_plain[i] = (time.perf_counter() - t0 - q["t"]) * 1e3
        t_plain = time.perf_counter() - t0
        # (c) bit-exact: every served output equals its plain launch
        diff = [i for i in range(n) if not torch.equal(outs[i], plain_outs[i])]
        if diff:
            raise SystemExit("serving at %g req/s: %d of %d served outputs differ from their plain launches "
                             "(first: request %d)" % (rate, len(diff), n, diff[0]))
        results[str(int(rate))] = {
            "requests": n, "mpix": npx / 1e6, "bit_identical_to_plain_launches": True,
            "server": {"mpix_s": npx / t_srv / 1e6, "p50_ms": float(np.percentile(lat_srv, 50)),
                       "p99_ms": float(np.percentile(lat_srv, 99)), "waves": int(st.waves),
                       "bytes_high_water": int(st.bytes_high_water)},
            "plain": {"mpix_s": npx / t_plain / 1e6, "p50_ms": float(np.percentile(lat_plain, 50)),
                      "p99_ms": float(np.percentile(lat_plain, 99))}}
        del outs, plain_outs
    clk.__exit__()
    top = results[max(results, key=float)]
    _line("serving: output Mpix/s and p50/p99 latency, continuous batching vs plain launches", "Mpix/s",
          top["server"]["mpix_s"], {"dtype": "u8+u16", "per_rate": results,
                                    "config": {"workload": "Poisson request stream, side log-uniform 64..4096, "
                                                           "50% uint8 / 50% uint16, radius 1..50, 16 GB budget",
                                               "value_is": "server Mpix/s at the highest rate",
                                               "parity": "every served output compared bit for bit with the "
                                                         "plain launch of the same request (the run fails on "
                                                         "any difference)"}}, args, clk=clk)


# ---- GPU arm ------------------------------------------------------------------------

def main():
    global RADII
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hrm", choices=["hrm", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=16.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-step-seconds", type=float, default=None,
                    help="--impl reference: seconds of oracle work per step (default: 90 s over all steps, 2..20 s)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--workload", default="xray2d",
                    choices=["xray2d", "volume3d", "lowkey2d", "u8small", "serve", "video", "paper"],
                    help="xray2d (default) is the benchmark workload; the others are the secondary configs")
    ap.add_argument("--rates", default="100,300,1000,3000,5000", help="serve: Poisson arrival rates (1/s)")
    ap.add_argument("--requests", type=int, default=10000, help="serve: requests per rate (capped at rate x 10 s)")
    ap.add_argument("--radii", default=",".join(map(str, RADII)),
                    help="comma list; the default is the benchmark workload (profiling runs may narrow it)")
    args = ap.parse_args()
    RADII = tuple(int(x) for x in args.radii.split(","))
    ws, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != "xray2d":
        return run_secondary(args)

    import torch
    from __graft_entry__ import build
    from paper_1105_3829_gb300 import hrm, inputs

    if rank == 0 or ws == 1:
        build()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        build()
    dev = torch.device("cuda", local)

    img_np = inputs.xray12_u16(SIDE, SIDE, seed=rank_seed(rank))
    img = torch.from_numpy(img_np).to(dev)
    outs = {r: torch.empty_like(img) for r in RADII}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    npx = SIDE * SIDE

    def step(events=None):
        for r in RADII:
            flush.fill_(r & 0xFF)
            if events is not None:
                events[r][0].record(stream)
            hrm.filter2d(img, r, out=outs[r])
            if events is not None:
                events[r][1].record(stream)

    for _ in range(args.warmup):
        step()
    hrm.device_status()

    ev = [{r: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for r in RADII}
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local].strip() if vis else str(local)
    with ClockSampler(smi_index) as clk:
        t_wall0 = time.perf_counter()
        # One untimed fill ahead of the first step: the timed steps start from
        # an empty GPU queue, and a host stall between a launch's start event
        # and the launch itself would be timed as idle GPU.  Later steps queue
        # behind the previous step's r = 50 call.
        flush.fill_(0)
        for k in range(args.steps):
            step(ev[k])
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    hrm.device_status()
    times = {r: np.array([ev[k][r][0].elapsed_time(ev[k][r][1]) for k in range(args.steps)]) for r in RADII}
    dev_ms_step = float(sum(times[r].sum() for r in RADII) / args.steps)
    if dist:
        dev_ms_step, t_wall = max_over_ranks(dist, [dev_ms_step, t_wall], dev)
    value = job_value(ws, len(RADII), npx, dev_ms_step)

    # ---- end to end through host buffers (pinned), same workload ----
    if args.no_e2e:
        e2e_ms = float("nan")
    else:
        e2e_ms = run_e2e(args, img_np, img, outs, stream, hrm, dist, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    return report(args, ws, times, dev_ms_step, value, t_wall, e2e_ms, clk, npx, dist, img_np)


def run_e2e(args, img_np, img, outs, stream, hrm, dist, dev):
    import torch
    host_in = torch.from_numpy(img_np).pin_memory()
    host_out = {r: torch.empty((SIDE, SIDE), dtype=torch.uint16).pin_memory() for r in RADII}
    dev_in = [torch.empty_like(img), torch.empty_like(img)]

    # Each step's input goes host -> device on a copy-in stream into one of two
    # buffers (the next step's upload overlaps this step's filters); each
    # output's device -> host copy runs on a copy-out stream as soon as its
    # filter finishes, overlapping the next radius.  Events order the reuse of
    # every buffer.
    cin, cout = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    uploaded = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    done = {r: torch.cuda.Event() for r in RADII}
    copied = {r: torch.cuda.Event() for r in RADII}
    state = {"k": 0}

    def e2e_step():
        b = state["k"] & 1
        state["k"] += 1
        cin.wait_event(consumed[b])
        with torch.cuda.stream(cin):
            dev_in[b].copy_(host_in, non_blocking=True)
        uploaded[b].record(cin)
        stream.wait_event(uploaded[b])
        for r in RADII:
            stream.wait_event(copied[r])
            hrm.filter2d(dev_in[b], r, out=outs[r])
            done[r].record(stream)
            cout.wait_event(done[r])
            with torch.cuda.stream(cout):
                host_out[r].copy_(outs[r], non_blocking=True)
            copied[r].record(cout)
        consumed[b].record(stream)

    for r in RADII:
        copied[r].record(cout)
    for b in (0, 1):
        consumed[b].record(stream)
    for _ in range(max(1, args.warmup)):
        e2e_step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    cin.wait_stream(stream)  # the first timed upload starts after e0
    for _ in range(args.steps):
        e2e_step()
    for r in RADII:
        stream.wait_event(copied[r])
    e1.record(stream)  # after every upload, filter and download of the timed steps
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t[0])
    ok = all(np.array_equal(host_out[r].numpy(), outs[r].cpu().numpy()) for r in RADII)
    if not ok:
        raise SystemExit("e2e outputs differ from the device outputs")
    return e2e_ms


def report(args, ws, times, dev_ms_step, value, t_wall, e2e_ms, clk, npx, dist, img_np):
    hbm_gbs, peak_kind = peaks()
    per_radius = {}
    for r in RADII:
        t = times[r]
        p50 = float(np.percentile(t, 50))
        per_radius[str(r)] = {
            "mpix_s": npx / (p50 * 1e-3) / 1e6,
            "p50_ms": p50, "p99_ms": float(np.percentile(t, 99)),
            "hbm_frac": (4.0 * npx / (p50 * 1e-3) / 1e9) / hbm_gbs,
            "path": "selection network" if r <= SORTNET_MAX_R else "levels pre-pass + hierarchical histogram",
        }
    dom = max(RADII, key=lambda r: times[r].mean())
    dom_ms = float(times[dom].mean())
    achieved = 4.0 * npx / (dom_ms * 1e-3) / 1e9
    kname = "hist2d r=%d" % dom if dom > SORTNET_MAX_R else "sortnet r=%d" % dom
    launches_per_step = sum(1 if r <= SORTNET_MAX_R else 3 for r in RADII)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": bench_config(ws, img_np),
        "value_is": "whole-job output pixels of one step (one image at each of the radii) / the summed CUDA-event "
                    "times of its launches: a time-weighted aggregate dominated by the slowest radii; "
                    "per_radius gives each radius alone",
        "ms_per_step_wall_incl_flush": 1e3 * t_wall / args.steps,
        "per_radius": per_radius,
        "roofline": {"bound": "hbm", "kernel": kname + " (the hrm_filter2d call: level pre-pass + kernel)",
                     "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
                     "peak_kind": peak_kind, "traffic": traffic_for(kname),
                     "ncu_issue_active": traffic_for(kname, "issue_active"),
                     "ncu_alu_pipe_active": traffic_for(kname, "alu_pipe_active"),
                     "note": "the histogram kernel (r >= 6) is limited by instruction issue and latency, "
                             "not by HBM; ncu_issue_active is its measured issue utilisation",
                     "algorithmic_bytes_per_launch": 4 * npx},
        "gpu_launches": launches_per_step * args.steps,
        "e2e": None if e2e_ms != e2e_ms else
               {"value": ws * len(RADII) * npx / (e2e_ms * 1e-3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": 2 * npx, "d2h_bytes_per_step": 2 * npx * len(RADII),
                "ms_per_step": e2e_ms, "path": "pinned host -> device copy of the input, hrm_filter2d at every "
                                              "radius, device -> pinned host copy of every output (uploads and "
                                              "downloads on their own streams, overlapping the filters)",
                "cache": "warm: no L2 flush in this leg; each step's input arrives by a fresh host -> device "
                         "copy, which leaves it in L2 as it would for any caller (the device-timed value "
                         "flushes L2 before every launch)"},
        "clocks": clk.summary(),
    }
    if ws == 1 and not args.no_cpu_baseline:
        pts, secs, threads = oracle_sample(img_np, args.cpu_budget, radii=RADII)
        line["cpu_baseline"] = {"value": pts / secs / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": "%d random output points spread over radii 1/5/15/50 (~%.0f s): "
                                          "brute-force gather + Quickselect per point" % (pts, secs)}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
