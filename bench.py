#!/usr/bin/env python
"""Benchmark of the exact point-in-polygon join (SPADE §5.2 polygon x point join).

Default workload (the join at scale): 100M clustered points (64-component
Gaussian mixture, sigma 0.5-5 % of the box, 10 % uniform background) in int32
fixed point, joined against a 2000-cell tessellation of jittered quads with
noisily subdivided edges (52-2000 vertices per cell); output: (point, polygon)
pairs sorted by point id plus per-polygon counts.

One step = one join of the whole resident point table against the resident
grid index (point -> cell, candidate dispatch, exact crossing tests with the
FP32 filter, order-preserving compaction, per-polygon counts).  The index is
built once before timing; its build time is reported separately.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle instead
(the reference arm), on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "billion points joined/sec and % HBM roofline; serving p50/p99 ms vs plain kernel"
UNIT = "Gpoints/s"
L2_BYTES = 129 * 1024 * 1024
# DRAM bytes (read + write) per point of the polygon join's kernels from one
# ncu capture of a 20M-point run of the default workload (16-bit per-point
# results), scaled per point, keyed by the index's (grid_log2, sub_log2); only
# valid for those kernel versions and the default workload.  A missing entry:
# not captured.
RESOLVE_TRAFFIC_BYTES_PER_POINT = {(12, 3): {"k_resolve": (272.762368e6 + 30.259712e6) / 20e6,
                                             "k_walk": (62.574336e6 + 1.225728e6) / 20e6,
                                             "k_wemit": (43.166720e6 + 98.548992e6) / 20e6}}
# The same for the distance join's pass 1 (k_dwarp<resolve>), from one capture
# of a 20M-point run of the 1024-disk workload at its default grid (g = 12).
DISK_RESOLVE_TRAFFIC_BYTES_PER_POINT = (167.498496e6 + 25.302784e6) / 20e6
SERVE_SEED = 0x2203143620 + 4  # request indexes of the serving measurement


# ------------------------------------------------------------------ workloads
def make_workload(name: str, n_override: int | None, rank: int):
    from paper_2203_14362_gb300 import datagen as g

    if name == "tess2000_100m":
        n = n_override or 100_000_000
        seed = g.SEED_BASE + 2
        nx, ny = g.tessellation_shape(2000)
        t = g.quad_tessellation(nx, ny, seed, kmin=12, kmax=499)
        mix = g.make_mixture(seed)
        pts = g.mixture_points_parallel(n, seed, mix, start=shard_start(rank, n))
        desc = (f"{n} mixture points (64 Gaussians, sigma 0.5-5% of box, 10% uniform) x 2000-cell tessellation "
                f"(jittered quads, noisy edges, 52-2000 vertices/cell); pairs + counts")
        return pts, t.verts, t.ring_off, desc
    if name == "select256_500m":
        n = n_override or 500_000_000
        seed = g.SEED_BASE + 3
        mix = g.make_mixture(seed)
        v, o = g.query_polygons(256, seed, mix)
        pts = g.mixture_points_parallel(n, seed, mix, start=shard_start(rank, n))
        desc = (f"batched selection: {n} mixture points x 256 query polygons (lognormal 8-5000 vertices, "
                f"concave, overlapping); per-query ascending id lists")
        return pts, v, o, desc
    if name == "dist1024_100m":
        n = n_override or 100_000_000
        seed = g.SEED_BASE + 6
        mix = g.make_mixture(seed)
        pts = g.mixture_points_parallel(n, seed, mix, start=shard_start(rank, n))
        centers = g.mixture_points(1024, seed + 1, mix)
        rng = np.random.default_rng(seed)
        radii = np.clip(np.exp(rng.normal(np.log(0.001 * (1 << 30)), 0.8, 1024)), 1e4, 2e7).astype(np.int32)
        desc = (f"distance join: {n} mixture points x 1024 disks (centres from the point mixture, radius "
                f"lognormal, median 0.1% of the box); pairs (point, disk) with distance <= r + counts")
        return pts, centers, radii, desc
    if name == "buffer256_100m":
        n = n_override or 100_000_000
        seed = g.SEED_BASE + 8
        mix = g.make_mixture(g.SEED_BASE + 3)
        v, o = g.query_polygons(256, g.SEED_BASE + 3, mix)
        pts = g.mixture_points_parallel(n, seed, mix, start=shard_start(rank, n))
        rng = np.random.default_rng(seed)
        radii = np.clip(np.exp(rng.normal(np.log(1 << 20), 0.7, 256)), 1 << 16, 1 << 23).astype(np.int32)
        desc = (f"buffered-polygon join: {n} mixture points x the 256 query polygons of the selection workload, "
                f"each grown by a radius (lognormal, median 2^20 = 0.1% of the box side); pairs (point, polygon) "
                f"with distance <= r + counts")
        return pts, (v, o), radii, desc
    if name == "serve_1b":
        n = n_override or 1_000_000_000
        seed = g.SEED_BASE + 4
        mix = g.make_mixture(seed)
        pts = g.mixture_points_parallel(n, seed, mix, start=shard_start(rank, n))
        desc = (f"serving: {n} resident mixture points; Poisson stream of 70% selections (1-64 query polygons) "
                f"and 30% joins vs 500/1000/2500/5000-cell tessellations")
        return pts, None, None, desc
    if name == "stars_1m":
        n = n_override or 1_000_000
        seed = g.SEED_BASE + 1
        v, o = g.star_polygons(seed)
        pts = g.uniform_points(n * (rank + 1), seed)[rank * n:]
        return pts, v, o, f"{n} uniform points x 256 star polygons (16-64 vertices); pairs + counts"
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples with host timestamps."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int, period_ms: int = 20):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", str(period_ms),
                 "-i", str(gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [c.strip() for c in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        win = [s for t, s in self.samples if t0 <= t <= t1]
        if not win and self.samples:  # timed region shorter than the sampling period: nearest samples
            mid = 0.5 * (t0 + t1)
            win = [min(self.samples, key=lambda ts: abs(ts[0] - mid))[1]]
        if not win:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(s[1]) for s in win if len(s) > 8 and num(s[1]) is not None]
        mx = [num(s[2]) for s in win if len(s) > 8 and num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in win if len(s) > 8 for k in range(4) if s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(win)}


# -------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, local: int, torch):
    """One process per GPU (NCCL); gloo where there is no GPU (tests)."""
    if world == 1:
        return
    import torch.distributed as dist
    if dist.is_initialized():
        return
    if torch.cuda.is_available():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group("gloo")


def _dist_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float, world: int, torch):
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_dist_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_counts_over_ranks(counts, world: int):
    """Per-polygon counts of the whole table: each rank joins its own range of
    points, so the counts are summed over ranks (the path's one exchange)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(counts, op=dist.ReduceOp.SUM)
    return counts


def join_launches(n: int, plain: bool, dist: bool = False) -> int:
    """Kernels one spx_join launches: pass 1 (two kernels; the distance join:
    one), the scan (one kernel up to 32768 values, else three), pass 3
    (256-point chunks; plain: 256-point blocks and the one-block scan)."""
    if plain:
        return 3
    chunks = (n + 255) // 256
    return (2 if dist else 3) + (1 if chunks <= 4 * 8192 else 3)


def shard_start(rank: int, n_per_rank: int) -> int:
    """First global point index of a rank's range (weak scaling)."""
    return rank * n_per_rank


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------- CPU baseline
def cpu_baseline(pts, verts, ring_off, budget_s: float = 12.0, chunk: int = 1_000_000, single_s: float = 4.0):
    """The fast oracle on the first points of the table: all host cores for
    budget_s, then one thread for single_s (reported as single_thread)."""
    import oracle
    pr = oracle.Prepared(verts, ring_off)

    def timed(threads, budget, step):
        done, t0 = 0, time.perf_counter()
        while done < pts.shape[0] and time.perf_counter() - t0 < budget:
            m = min(step, pts.shape[0] - done)
            pr.join(pts[done:done + m], threads=threads)
            done += m
        return done, time.perf_counter() - t0

    threads = oracle.default_threads()
    done, el = timed(threads, budget_s, chunk)
    out = {"value": done / el / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {done} points of the same table (pairs + counts, fast oracle, {el:.1f} s)"}
    if single_s > 0:
        d1, e1 = timed(1, single_s, max(chunk // 10, 1))
        out["single_thread"] = {"value": d1 / e1 / 1e9, "unit": UNIT, "cores": 1,
                                "sample": f"first {d1} points ({e1:.1f} s)"}
    pr.close()
    return out


def disk_cpu_baseline(pts, centers, radii, budget_s: float = 12.0, chunk: int = 200_000):
    """The oracle's distance join (every disk for every point) on the first points."""
    import oracle
    done, t0 = 0, time.perf_counter()
    while done < pts.shape[0] and time.perf_counter() - t0 < budget_s:
        m = min(chunk, pts.shape[0] - done)
        oracle.disk_join(pts[done:done + m], centers, radii)
        done += m
    el = time.perf_counter() - t0
    return {"value": done / el / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} points (distance join, brute force over all disks, {el:.1f} s)"}


# ------------------------------------------------------------ reference arm
def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_2203_14362_gb300 import datagen as g

    sample = args.ref_sample
    if args.workload in ("serve_1b", "count_4b"):
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the oracle on the join "
                          "workloads; this workload reports its oracle sample in cpu_baseline"}), flush=True)
        return 0
    pts, v, o, desc = make_workload(args.workload, sample, 0)
    if args.workload.startswith("dist"):
        threads = 1

        def step():
            oracle.disk_join(pts, v, o)
    elif args.workload.startswith("buffer"):
        threads = oracle.default_threads()
        (bv, bo), radii = v, o

        def step():
            oracle.buffer_join(pts, bv, bo, radii, threads=threads)
    else:
        pr = oracle.Prepared(v, o)
        threads = oracle.default_threads()

        def step():
            pr.join(pts, threads=threads)
    for _ in range(max(args.warmup, 0)):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    val = sample / sec / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "sample_points_per_step": sample,
                   "polygons": (int(v.shape[0]) if args.workload.startswith("dist") else
                                int(v[1].shape[0] - 1) if args.workload.startswith("buffer") else int(o.shape[0] - 1))},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": (f"first {sample} points of the workload per step (distance join, brute force "
                                    "over all disks)" if args.workload.startswith("dist") else
                                    f"first {sample} points of the workload per step (buffered-polygon join, every "
                                    "edge of each polygon whose grown bbox holds the point)"
                                    if args.workload.startswith("buffer") else
                                    f"first {sample} points of the workload per step (pairs + counts, fast oracle)")},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- GPU arm
def run_spx(args, world, rank, local):
    import torch

    from paper_2203_14362_gb300 import spx

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist_init(world, local, torch)
    if args.workload == "count_4b":
        line = count_measure(args, world, rank, local, torch, args.steps, args.warmup, args.points, e2e=not args.no_e2e)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    if args.workload.startswith("select"):
        line = select_measure(args, world, rank, local, torch, args.steps, args.warmup, args.points)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    if args.workload.startswith("buffer"):
        line = buffer_measure(args, world, rank, local, torch, args.steps, args.warmup, args.points)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    clocks = ClockSampler(local)
    pts, v, o, desc = make_workload(args.workload, args.points, rank)
    N = pts.shape[0]

    eng = spx.Engine(local)
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    if args.workload == "serve_1b":
        return run_serve_bench(args, world, rank, eng, ph, dpts, N, desc, clocks, torch)
    dist = args.workload.startswith("dist")
    P = int(v.shape[0]) if dist else int(o.shape[0] - 1)
    gh = None if dist else eng.load_polygons(v, o)
    tune = None
    device_build_ms = None
    if dist:
        ih = eng.build_disk_index(v, o, args.grid)
        # the same index built on the device (the second build: the first loads the kernels)
        for _ in range(2):
            ih_dev = eng.build_disk_index(v, o, args.grid, on_device=True)
            device_build_ms = eng.index_info(ih_dev)["build_ms"]
            eng.free(ih_dev)
    elif args.autotune:
        t0 = time.perf_counter()
        params, trials, ih = eng.autotune(ph, gh, fp32_filter=bool(args.fp32))
        tune = {"picked": [params["grid_log2"], params["sub_log2"]], "seconds": round(time.perf_counter() - t0, 2),
                "trials": [[t["grid_log2"], t["sub_log2"], round(t["ms"], 4)] for t in trials],
                "sample": "every (N / m)-th point, m = max(N / 100, min(N, 2^22)); count-only launches"}
    else:
        ih = eng.build_index(gh, grid_log2=args.grid, fp32_filter=bool(args.fp32), sub_log2=args.sub)
    info = eng.index_info(ih)
    if not dist:
        # the same index built on the device (the second build: the first loads the kernels)
        for _ in range(2):
            ih_dev = eng.build_index(gh, grid_log2=info["grid_log2"], fp32_filter=bool(args.fp32),
                                     sub_log2=info["sub_log2"], on_device=True)
            device_build_ms = eng.index_info(ih_dev)["build_ms"]
            eng.free(ih_dev)
    cap = N if args.cap is None else args.cap
    pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    counts = torch.zeros(max(P, 1), dtype=torch.int64, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    try:
        n_pairs = eng.join(ph, ih, pairs, counts, total, sync=True, plain=args.plain)
    except spx.SpxError as e:  # the two-call pattern: the first call reports the size
        if e.status != spx.SPX_ECAPACITY:
            raise
        cap = int(str(e).split("needs ")[1].split(" ")[0])
        pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
        n_pairs = eng.join(ph, ih, pairs, counts, total, sync=True, plain=args.plain)
    assert int(counts.sum().item()) == n_pairs

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        eng.join(ph, ih, pairs, counts, total, sync=False, stream=stream, plain=args.plain)
    torch.cuda.synchronize()
    eng.stats(reset=True)
    barrier(world)
    torch.cuda.synchronize()
    # one event per step boundary (the first and last bracket the whole timed region)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = ev[0], ev[-1]
    t_host0 = time.time()
    e0.record(stream)
    for k in range(args.steps):
        eng.join(ph, ih, pairs, counts, total, sync=False, stream=stream, plain=args.plain)
        sum_counts_over_ranks(counts, world)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    st = eng.stats(reset=True)
    ms_max = max_over_ranks(ms, world, torch)
    clk = clocks.summary(t_host0, t_host1)

    # per-kernel device times, live: CUDA events around each pass on the same stream
    eng.set_phase_timing(True)
    k_phase = max(1, min(args.steps, 10))
    for _ in range(k_phase):
        eng.join(ph, ih, pairs, counts, total, sync=False, stream=stream, plain=args.plain)
    torch.cuda.synchronize()
    ph_st = eng.stats(reset=True)
    eng.set_phase_timing(False)
    nt = max(ph_st["timed_joins"], 1)
    phase_ms = {"resolve": ph_st["ms_resolve"] / nt, "walk": ph_st["ms_walk"] / nt, "scan": ph_st["ms_scan"] / nt,
                "emit": ph_st["ms_emit"] / nt}

    # end to end through the C ABI on pinned host buffers (H2D points, join, D2H pairs + counts)
    e2e = None
    if not args.no_e2e and not dist:  # spx_join_host takes polygon indexes
        hx = torch.empty((N, 2), dtype=torch.int32, pin_memory=True)
        hx.numpy()[:] = pts
        hp = torch.empty((cap, 2), dtype=torch.int32, pin_memory=True)
        hc = torch.empty(max(P, 1), dtype=torch.int64, pin_memory=True)
        hxn, hpn, hcn = hx.numpy(), hp.numpy().view(np.uint32), hc.numpy().view(np.uint64)
        eng.join_host(hxn, ih, cap, P, pairs_out=hpn, counts_out=hcn)
        k_e2e = max(1, min(args.steps, args.e2e_steps))
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            _, _, m = eng.join_host(hxn, ih, cap, P, pairs_out=hpn, counts_out=hcn)
        sec = (time.perf_counter() - t0) / k_e2e
        sec = max_over_ranks(sec, world, torch)
        e2e = {"value": world * N / sec / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(N * 8),
               "d2h_bytes_per_step": int(m * 8 + P * 8 + 8), "ms_per_step": sec * 1e3}
    clocks.stop()

    serving = None
    if not args.no_serve and not args.plain and not dist:
        serving = run_serving(eng, ph, N, SERVE_SEED, timed=args.serve_timed, warm=args.serve_warmup,
                              burst=args.serve_burst)

    idx_bytes = int(info["device_bytes"])
    step_bytes = 8 * N + 8 * n_pairs + 8 * P + idx_bytes  # algorithmic bytes of one join
    peak, peak_kind = peaks()
    # dominant kernel: the resolve pass (reads every point once, writes the counts)
    # the dominant kernel: the longest pass of the step, with its algorithmic
    # bytes (pass 1a / the distance join's pass 1: every point read once, the
    # counts written, the index read once; pass 1b: the points it tests and
    # their results; pass 3: 8 B per pair written)
    if args.plain:
        dom, dom_ms, dom_bytes = "plain join (3 kernels)", ms, step_bytes
    else:
        cand = {"resolve": (phase_ms["resolve"], 8 * N + 8 * P + idx_bytes),
                "emit": (phase_ms["emit"], 8 * n_pairs)}
        if not dist:  # pass 1b re-reads what pass 1a read: no algorithmic bytes of its own
            cand["walk"] = (phase_ms["walk"], 0)
        key = max(cand, key=lambda k: cand[k][0])
        dom_ms, dom_bytes = cand[key]
        names = {"resolve": "k_dwarp<resolve> (distance join pass 1)" if dist else "k_resolve (join pass 1a)",
                 "walk": "k_walk (join pass 1b: exact tests)",
                 "emit": "k_dwemit (distance join pass 3)" if dist else "k_wemit (join pass 3)"}
        dom = names[key]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = args.traffic
    if (traffic is None and not args.plain and not dist and args.workload == "tess2000_100m"
            and (info["grid_log2"], info["sub_log2"]) in RESOLVE_TRAFFIC_BYTES_PER_POINT):
        per_pt = RESOLVE_TRAFFIC_BYTES_PER_POINT[(info["grid_log2"], info["sub_log2"])].get(dom.split(" ")[0])
        traffic = None if per_pt is None else per_pt * N
    if traffic is None and dist and info["grid_log2"] == 12 and dom.startswith("k_dwarp"):
        traffic = DISK_RESOLVE_TRAFFIC_BYTES_PER_POINT * N
    out = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = disk_cpu_baseline(pts, v, o, args.cpu_budget) if dist else cpu_baseline(pts, v, o, args.cpu_budget)
        out = {
            "metric": METRIC, "value": world * N / (ms_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {
                "workload": args.workload, "desc": desc, "points_per_gpu": N, "polygons": P,
                "vertices": 0 if dist else int(v.shape[0]), "pairs": int(n_pairs), "grid_log2": info["grid_log2"],
                "sub_log2": info["sub_log2"], "fp32_filter": bool(args.fp32),
                "kernel": ("distance join: resolve (k_dwarp) + scan + emit (k_dwemit)" if dist else
                           "plain two-pass" if args.plain else
                           "resolve (k_resolve) + exact tests (k_walk) + scan + emit (k_wemit): cached two-pass Map"),
                "index_build_ms": round(info["build_ms"], 1), "index_device_bytes": int(info["device_bytes"]),
                "index_build_on_device_ms": None if device_build_ms is None else round(device_build_ms, 2),
                "l2": "inputs larger than L2 (points 8 B x N + pairs 8 B x N >> 129 MB); no flush",
                "edge_tests_per_point": st["edge_tests"] / max(st["points_scanned"], 1),
                "fp32_escalation_fraction": st["fp32_escalations"] / max(st["edge_tests"], 1),
                "parallelism": f"points sharded by rank, index replicated, dp{world}",
                "autotune": tune,
            },
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": dom,
                         "kernel_ms": dom_ms, "algorithmic_bytes_per_launch": int(dom_bytes),
                         "step": {"algorithmic_bytes": int(step_bytes), "ms": ms,
                                  "achieved_gbs": step_bytes / (ms * 1e-3) / 1e9,
                                  "frac": step_bytes / (ms * 1e-3) / 1e9 / peak},
                         "phase_ms": phase_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "step_ms": {"mean": ms, "best": min(per_step), "median": statistics.median(per_step),
                        "worst": max(per_step), "rank": 0},
            "gpu_launches": args.steps * join_launches(N, args.plain, dist),
            "clocks": clk,
            "serving": serving,
        }
    eng.free(ih)
    if gh is not None:
        eng.free(gh)
    eng.free(ph)
    eng.close()
    del dpts, pairs, counts, total
    torch.cuda.empty_cache()
    if args.workload == "tess2000_100m" and world == 1 and not args.no_extra and not args.plain:
        # the batched selection (500M points) and the count-only aggregate (4B
        # points) at their full sizes, each with its own roofline, CPU
        # baseline and clocks
        k, w = max(1, min(args.steps, 10)), max(3, min(args.warmup, 5))
        sel = select_measure(args, world, rank, local, torch, k, w, None)
        torch.cuda.empty_cache()
        cnt = count_measure(args, world, rank, local, torch, k, w, None, e2e=False)
        torch.cuda.empty_cache()
        sv1b = None if args.no_serve else serve_capacity_measure(args, local, torch)
        if rank == 0:
            out["select"] = sel
            out["count"] = cnt
            out["serving_1b"] = sv1b
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# -------------------------------------------------------------------- serving
def serve_indexes(eng, seed: int, pool: int = 32):
    """Prebuilt request indexes: 4 tessellations (joins) and a pool of query
    polygon sets of 1-64 polygons (selections)."""
    from paper_2203_14362_gb300 import datagen as g
    from paper_2203_14362_gb300 import spx
    out = []  # (kind, polys handle, index handle, polygons, vertices, ring offsets)
    for k, cells in enumerate((500, 1000, 2500, 5000)):
        nx, ny = g.tessellation_shape(cells)
        t = g.quad_tessellation(nx, ny, seed + 100 + k)
        gh = eng.load_polygons(t.verts, t.ring_off)
        out.append((spx.SPX_REQ_JOIN, gh, eng.build_index(gh), cells, t.verts, t.ring_off))
    mix = g.make_mixture(seed)
    rng = np.random.default_rng(seed)
    for k in range(pool):
        q = int(rng.integers(1, 65))
        v, o = g.query_polygons(q, seed + 200 + k, mix)
        gh = eng.load_polygons(v, o)
        out.append((spx.SPX_REQ_SELECT, gh, eng.build_index(gh), q, v, o))
    return out


def serve_stream(idx, n: int, seed: int):
    """n requests: 70 % selections (uniform over the pool), 30 % joins."""
    from paper_2203_14362_gb300 import spx
    rng = np.random.default_rng(seed)
    joins = [i for i, x in enumerate(idx) if x[0] == spx.SPX_REQ_JOIN]
    sels = [i for i, x in enumerate(idx) if x[0] == spx.SPX_REQ_SELECT]
    out = []
    for _ in range(n):
        pos = int(rng.choice(sels)) if rng.random() < 0.7 else int(rng.choice(joins))
        out.append((idx[pos][0], pos))
    return out


def serve_run(srv, reqs, rate, warm: int, seed: int = 7, polys=None):
    """Submit reqs at Poisson arrivals of `rate` per second (None: all at once);
    a collector waits for each result and releases it.  Latency = completion on
    the device - submission, both on the server's clock.  polys (or None):
    per index position its (vertices, ring offsets): every request then brings
    its polygons, indexed on the device when its batch starts."""
    ids = [None] * len(reqs)
    res = [None] * len(reqs)
    ready = threading.Semaphore(0)

    def collect():
        for i in range(len(reqs)):
            ready.acquire()
            res[i] = srv.wait(ids[i], -1.0)
            srv.release(ids[i])

    th = threading.Thread(target=collect)
    th.start()
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    t0, t = time.perf_counter(), 0.0
    for i, (kind, pos) in enumerate(reqs):
        t += gaps[i]
        d = t0 + t - time.perf_counter()
        if d > 0:
            time.sleep(d)
        ids[i] = srv.submit(kind, pos, tag=i) if polys is None else srv.submit_polygons(kind, *polys[pos], tag=i)
        ready.release()
    th.join()
    timed = res[warm:]
    serve_run.last = timed
    bad = sum(1 for r in timed if r["status"] != 0)
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in timed])
    span = (max(r["t_done_ms"] for r in timed) - min(r["t_submit_ms"] for r in timed)) / 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "throughput_rps": len(timed) / span,
            "mean_batch": float(np.mean([r["batch_size"] for r in timed])), "failed": bad}


def serve_capacity(eng, ph, N: int, idx, burst: int, seed: int, plain_burst: int = 0):
    """Capacity (requests/s over a burst submitted at once, after a warm-up
    burst) of the batching server, of its fused one-pass mode, of the plain
    comparison and of the batching server with every request bringing its
    polygons (batched_own: each index built on the device in the request's
    latency), and the batching server's served roofline over its burst: the
    algorithmic bytes of every request (8 B per scanned point, 8 B per pair or
    4 B per id, its index once) over the burst's span."""
    from paper_2203_14362_gb300 import spx
    handles = [x[2] for x in idx]
    peak, peak_kind = peaks()
    ix_bytes = [eng.index_info(h)["device_bytes"] for h in handles]
    cap, roof = {}, None
    arms = (("batched", dict(max_batch=8, slots=2)), ("fused", dict(max_batch=8, slots=2, fused=True)),
            ("plain", dict(plain=True)), ("batched_own", dict(max_batch=8, slots=2)))
    polys = [(x[4], x[5]) for x in idx]
    for name, kw in arms:
        n = plain_burst if name == "plain" and plain_burst else burst
        own = polys if name == "batched_own" else None  # every request brings its polygons
        srv = spx.Server(eng, ph, handles, **kw)
        serve_run(srv, serve_stream(idx, max(4, n // 4), seed + 1), None, 0, polys=own)  # warm-up
        b0 = srv.stats()["batches"]
        reqs = serve_stream(idx, n, seed + 2)
        r = serve_run(srv, reqs, None, 0, polys=own)
        nb = srv.stats()["batches"] - b0
        cap[name] = r["throughput_rps"]
        if name == "batched":
            span = n / r["throughput_rps"]
            outb = sum((8 if x["kind"] == spx.SPX_REQ_JOIN else 4) * x["total"] for x in serve_run.last)
            alg = 8 * N * n + outb + sum(ix_bytes[pos] for _, pos in reqs)
            gbs = alg / span / 1e9
            roof = {"batches": nb, "requests": n, "seconds": span, "algorithmic_bytes": alg, "output_bytes": outb,
                    "achieved_gbs": gbs, "peak": peak, "frac": gbs / peak, "peak_source": f"{peak_kind} hbm_gbs",
                    "note": "8 B per scanned point per request + outputs (8 B per pair, 4 B per id) + each "
                            "request's index once, over the burst's span"}
        srv.close()
    return cap, roof


def run_serving(eng, ph, N: int, seed: int, timed: int, warm: int, burst: int):
    """Capacity (a burst) of the batching server, of its fused mode and of
    the plain comparison (one request per launch), then latency at 0.5 / 0.8
    / 0.95 x the batching server's capacity and at 0.5 / 0.8 x the plain
    server's (rates both arms sustain), `timed` requests per rate and arm
    after `warm` warm-up requests; the served roofline over the batching
    server's burst."""
    from paper_2203_14362_gb300 import spx
    t_build = time.perf_counter()
    idx = serve_indexes(eng, seed)
    build_s = time.perf_counter() - t_build
    handles = [x[2] for x in idx]
    out = {"points": N, "requests_timed": timed, "requests_warmup": warm, "burst": burst,
           "mix": "70% selection (1-64 query polygons, pool of 32 prebuilt indexes), "
                  "30% join vs 4 tessellations (500/1000/2500/5000 cells)",
           "index_build_s": round(build_s, 1), "server": {"max_batch": 8, "slots": 2},
           "latency": "device completion (stream callback) - submission, server clock", "rates": []}
    arms = {"batched": dict(max_batch=8, slots=2), "plain": dict(plain=True)}
    batches = 0
    cap, out["served_roofline"] = serve_capacity(eng, ph, N, idx, burst, seed)
    out["capacity_rps"] = cap
    plan = [("batched", x) for x in (0.5, 0.8, 0.95)] + [("plain", x) for x in (0.5, 0.8)]
    for ref, x in plan:
        rate = x * cap[ref]
        row = {"x_capacity": x, "capacity_of": ref, "rate_rps": rate}
        for name, kw in arms.items():
            srv = spx.Server(eng, ph, handles, **kw)
            row[name] = serve_run(srv, serve_stream(idx, warm + timed, seed + 10 + int(100 * x) + len(out["rates"])),
                                  rate, warm)
            batches += srv.stats()["batches"]
            srv.close()
        out["rates"].append(row)
    for _, gh, ih, *_ in idx:
        eng.free(ih)
        eng.free(gh)
    out["value_gpts"] = cap["batched"] * N / 1e9
    out["batches"] = batches
    return out


def serve_capacity_measure(args, local, torch, N: int = 1_000_000_000):
    """Serving capacity at the resident table of 1B points (the serving
    workload's size): the point table generated chunk by chunk straight into
    device memory, the same request indexes and mix as the latency sweeps, a
    burst per server (batching, fused, plain) and the batching server's
    served roofline."""
    from paper_2203_14362_gb300 import datagen as g
    from paper_2203_14362_gb300 import spx
    seed = g.SEED_BASE + 4
    mix = g.make_mixture(seed)
    t0 = time.perf_counter()
    dpts = torch.empty((N, 2), dtype=torch.int32, device="cuda")
    chunk = 1 << 28
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        dpts[lo:hi].copy_(torch.from_numpy(g.mixture_points_parallel(hi - lo, seed, mix, start=lo)))
    gen_s = time.perf_counter() - t0
    eng = spx.Engine(local)
    ph = eng.load_points(dpts)
    t1 = time.perf_counter()
    idx = serve_indexes(eng, SERVE_SEED)
    build_s = time.perf_counter() - t1
    clocks = ClockSampler(local)
    th0 = time.time()
    cap, roof = serve_capacity(eng, ph, N, idx, args.serve_burst, SERVE_SEED, plain_burst=12)
    clk = clocks.summary(th0, time.time())
    clocks.stop()
    for _, gh, ih, *_ in idx:
        eng.free(ih)
        eng.free(gh)
    eng.free(ph)
    eng.close()
    del dpts
    torch.cuda.empty_cache()
    return {"points": N, "data": "synthetic", "generate_s": round(gen_s, 1), "index_build_s": round(build_s, 1),
            "mix": "70% selection (1-64 query polygons, pool of 32 prebuilt indexes), "
                   "30% join vs 4 tessellations (500/1000/2500/5000 cells)",
            "burst": {"batched": args.serve_burst, "fused": args.serve_burst, "plain": 12},
            "capacity_rps": cap, "value_gpts": cap["batched"] * N / 1e9, "served_roofline": roof, "clocks": clk}


def run_serve_bench(args, world, rank, eng, ph, dpts, N, desc, clocks, torch):
    """Serving at scale: one JSON line whose value is the batching server's
    capacity in point evaluations per second (requests/s x resident points)."""
    t_host0 = time.time()
    sv = run_serving(eng, ph, N, SERVE_SEED, timed=args.serve_timed, warm=args.serve_warmup, burst=args.serve_burst)
    t_host1 = time.time()
    clk = clocks.summary(t_host0, t_host1)
    clocks.stop()
    cap = sv["capacity_rps"]["batched"]
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": world * sv["value_gpts"], "unit": UNIT, "n_gpus": world,
            "steps": args.serve_timed, "warmup": args.serve_warmup, "ms_per_step": 1e3 / cap,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc, "points_per_gpu": N,
                       "step": "one request at the batching server's capacity",
                       "l2": "point table (8 B x N) larger than L2; no flush"},
            "roofline": None, "cpu_baseline": None, "e2e": None,
            # two batch-kernel launches (count, emit) per batch of the timed runs;
            # scans and selection partitions add more
            "gpu_launches": 2 * sv["batches"], "gpu_launches_note": "lower bound: k_multi launches only",
            "clocks": clk, "serving": sv,
        }), flush=True)
    eng.free(ph)
    eng.close()
    del dpts
    return 0


def count_measure(args, world, rank, local, torch, steps, warmup, n_override, e2e: bool):
    """Count-only aggregate at scale (returns the JSON object): 4B
    Zipf-weighted mixture points against a 40000-cell tessellation (10-10000
    vertices per cell); per-polygon counts only.  The point table is generated
    chunk by chunk straight into device memory (32 GB); the first chunk stays
    on the host for the oracle checks and the CPU baseline."""
    import oracle
    from paper_2203_14362_gb300 import datagen as g
    from paper_2203_14362_gb300 import spx
    clocks = ClockSampler(local)
    N = n_override or 4_000_000_000
    seed = g.SEED_BASE + 5
    mix = g.make_mixture(seed, zipf_s=1.1)
    nx, ny = g.tessellation_shape(40000)
    t_gen = time.perf_counter()
    t = g.quad_tessellation(nx, ny, seed, kmin=2, kmax=2499)
    v, o = t.verts, t.ring_off
    P = int(o.shape[0] - 1)
    dpts = torch.empty((N, 2), dtype=torch.int32, device="cuda")
    chunk = 1 << 28
    head = None
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        c = g.mixture_points_parallel(hi - lo, seed, mix, start=shard_start(rank, N) + lo)
        if head is None:
            head = c[:min(c.shape[0], 20_000_000)].copy()
        dpts[lo:hi].copy_(torch.from_numpy(c))
        del c
    gen_s = time.perf_counter() - t_gen
    eng = spx.Engine(local)
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    tune = None
    if args.autotune:
        t0 = time.perf_counter()
        params, trials, ih = eng.autotune(ph, gh, fp32_filter=bool(args.fp32))
        tune = {"picked": [params["grid_log2"], params["sub_log2"]], "seconds": round(time.perf_counter() - t0, 2),
                "trials": [[x["grid_log2"], x["sub_log2"], round(x["ms"], 4)] for x in trials]}
    else:
        # g = 13 by default: with the directory at 2^13 only 7 % of the points are read
        # (11.8 ms against 15.2 ms at the automatic g = 12, directory at 2^12)
        ih = eng.build_index(gh, grid_log2=args.grid or 13, fp32_filter=bool(args.fp32), sub_log2=args.sub)
    info = eng.index_info(ih)
    # the same index built on the device (the second build: the first loads the kernels)
    device_build_ms = None
    for _ in range(2):
        ih_dev = eng.build_index(gh, grid_log2=info["grid_log2"], fp32_filter=bool(args.fp32),
                                 sub_log2=info["sub_log2"], on_device=True)
        device_build_ms = eng.index_info(ih_dev)["build_ms"]
        eng.free(ih_dev)
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    eng.aggregate(ph, ih, counts, stream=stream)
    torch.cuda.synchronize()
    # properties that hold at any size: the tessellation covers the box, so
    # every point lies in exactly one cell
    assert int(counts.sum().item()) == N, "sum of counts != number of points"
    cluster = None
    ph_run = ph
    cl = info["grid_log2"] if args.cluster < 0 else args.cluster  # default: the directory grid = the coarse grid
    if cl:
        # one-off: a copy grouped by grid cell (load time, outside the timed steps)
        t0 = time.perf_counter()
        ph_run = eng.cluster_points(ph, cl)
        cl_s = time.perf_counter() - t0
        c2 = torch.zeros(P, dtype=torch.int64, device="cuda")
        eng.aggregate(ph_run, ih, c2, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(c2, counts), "clustered counts differ from the row-order counts"
        cluster = {"grid_log2": cl, "seconds": round(cl_s, 3),
                   "check": "counts on the clustered copy == counts on the row-order table"}
        del c2
    # the first points' counts against the oracle
    m = min(head.shape[0], 2_000_000)
    ph_head = eng.load_points(dpts[:m])
    c_head = torch.zeros(P, dtype=torch.int64, device="cuda")
    eng.aggregate(ph_head, ih, c_head, stream=stream)
    torch.cuda.synchronize()
    pr = oracle.Prepared(v, o)
    ref = pr.counts(head[:m])
    assert np.array_equal(c_head.cpu().numpy().view(np.uint64), ref), "prefix counts differ from the oracle"
    eng.free(ph_head)
    for _ in range(warmup):
        eng.aggregate(ph_run, ih, counts, stream=stream)
    torch.cuda.synchronize()
    eng.stats(reset=True)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        eng.aggregate(ph_run, ih, counts, stream=stream)
        sum_counts_over_ranks(counts, world)
    e1.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    barrier(world)
    ms = e0.elapsed_time(e1) / steps
    st = eng.stats(reset=True)
    ms_max = max_over_ranks(ms, world, torch)
    clk = clocks.summary(t_host0, t_host1)
    eng.set_phase_timing(True)
    for _ in range(max(1, min(steps, 5))):
        eng.aggregate(ph_run, ih, counts, stream=stream)
    torch.cuda.synchronize()
    ph_st = eng.stats(reset=True)
    eng.set_phase_timing(False)
    # end to end from host memory: the table in pinned host memory, streamed
    # through the device every step (host-to-device copies inside the timing)
    e2e_out = None
    if e2e:
        hx = torch.empty((N, 2), dtype=torch.int32, pin_memory=True)
        hx.copy_(dpts)
        hxn = hx.numpy()
        hc = np.zeros(P, np.uint64)
        eng.aggregate_host(hxn, ih, P, counts_out=hc)
        assert np.array_equal(hc, counts.cpu().numpy().view(np.uint64)), "streamed counts differ"
        k_e2e = max(1, min(steps, args.e2e_steps))
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            eng.aggregate_host(hxn, ih, P, counts_out=hc)
        sec = max_over_ranks((time.perf_counter() - t0) / k_e2e, world, torch)
        e2e_out = {"value": world * N / sec / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(N * 8),
                   "d2h_bytes_per_step": int(P * 8), "ms_per_step": sec * 1e3,
                   "path": "spx_aggregate_host: the row-order table streamed from pinned host memory"}
        del hx, hxn
    clocks.stop()
    k_ms = ph_st["ms_aggregate"] / max(ph_st["timed_aggregates"], 1)
    idx_bytes = int(info["device_bytes"])
    # algorithmic bytes: the points that must be read (with a cell directory,
    # those of cells in mixed coarse cells; the others are counted from their
    # cell's row range), the directory, the index once, the counts
    n_dir = ph_st["points_from_directory"] // max(ph_st["timed_aggregates"], 1)
    dir_bytes = 8 * ((1 << (2 * cluster["grid_log2"])) + 1) if cluster and n_dir else 0
    alg = 8 * (N - n_dir) + dir_bytes + 8 * P + idx_bytes
    peak, peak_kind = peaks()
    achieved = alg / (k_ms * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        done = 0
        while done < head.shape[0] and time.perf_counter() - t0 < args.cpu_budget:
            k = min(1_000_000, head.shape[0] - done)
            pr.counts(head[done:done + k])
            done += k
        el = time.perf_counter() - t0
        cpu = {"value": done / el / 1e9, "unit": UNIT, "cores": oracle.default_threads(), "kind": "oracle",
               "sample": f"first {done} points of the table, counts only (fast oracle, {el:.1f} s)"}
    line = {
        "metric": METRIC, "value": world * N / (ms_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "count_4b",
                   "desc": f"{N} mixture points (64 Gaussians, Zipf(1.1) weights, 10% uniform) x 40000-cell "
                           f"tessellation (10-10000 vertices per cell); per-polygon counts only",
                   "points_per_gpu": N, "polygons": P, "vertices": int(v.shape[0]),
                   "grid_log2": info["grid_log2"], "sub_log2": info["sub_log2"],
                   "index_build_ms": round(info["build_ms"], 1), "index_device_bytes": idx_bytes,
                   "index_build_on_device_ms": round(device_build_ms, 2), "generation_s": round(gen_s, 1), "autotune": tune, "clustered_table": cluster,
                   "checks": "sum(counts) == N; counts of the first %d points == oracle" % m,
                   "counting": "global atomics (P > shared-memory histogram)" if P > 11776 else "shared memory",
                   "edge_tests_per_point": st["edge_tests"] / max(st["points_scanned"], 1),
                   "fp32_escalation_fraction": st["fp32_escalations"] / max(st["edge_tests"], 1),
                   "l2": "inputs larger than L2 (32 GB of points); no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": ("k_agg_cells + k_warp<aggregate, directory>" if n_dir else "k_warp<aggregate>"),
                     "kernel_ms": k_ms, "algorithmic_bytes_per_launch": int(alg),
                     "points_read": int(N - n_dir), "points_from_directory": int(n_dir)},
        "cpu_baseline": cpu, "e2e": e2e_out, "gpu_launches": steps, "clocks": clk,
    }
    pr.close()
    eng.free(ih)
    eng.free(gh)
    if ph_run != ph:
        eng.free(ph_run)
    eng.free(ph)
    eng.close()
    del dpts, counts
    return line


def select_measure(args, world, rank, local, torch, steps, warmup, n_override):
    """Batched selection (returns the JSON object): one step = all 256 query
    polygons answered over the resident 500M-point table in one graph-captured
    launch sequence (the join, then the partition by query)."""
    from paper_2203_14362_gb300 import spx
    clocks = ClockSampler(local)
    pts, v, o, desc = make_workload("select256_500m", n_override, rank)
    N, Q = pts.shape[0], int(o.shape[0] - 1)
    eng = spx.Engine(local)
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    tune = None
    if args.autotune:
        t0 = time.perf_counter()
        params, trials, ih = eng.autotune(ph, gh, fp32_filter=bool(args.fp32))
        tune = {"picked": [params["grid_log2"], params["sub_log2"]], "seconds": round(time.perf_counter() - t0, 2),
                "trials": [[x["grid_log2"], x["sub_log2"], round(x["ms"], 4)] for x in trials]}
    else:
        ih = eng.build_index(gh, grid_log2=args.grid, fp32_filter=bool(args.fp32), sub_log2=args.sub)
    info = eng.index_info(ih)
    # the same index built on the device (the second build: the first loads the kernels)
    device_build_ms = None
    for _ in range(2):
        ih_dev = eng.build_index(gh, grid_log2=info["grid_log2"], fp32_filter=bool(args.fp32),
                                 sub_log2=info["sub_log2"], on_device=True)
        device_build_ms = eng.index_info(ih_dev)["build_ms"]
        eng.free(ih_dev)
    offs = torch.zeros(Q + 1, dtype=torch.int64, device="cuda")
    probe = torch.empty(1, dtype=torch.int32, device="cuda")
    try:
        total = eng.select(ph, ih, probe, offs)
    except spx.SpxError as e:  # the two-call pattern: the first call reports the size
        total = int(str(e).split("needs ")[1].split(" ")[0])
    ids = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    assert eng.select(ph, ih, ids, offs) == total
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        eng.select(ph, ih, ids, offs, sync=False, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        eng.select(ph, ih, ids, offs, sync=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, torch)
    clk = clocks.summary(t_host0, t_host1)
    clocks.stop()
    peak, peak_kind = peaks()
    alg = 8 * N + 4 * total + 8 * (Q + 1) + int(info["device_bytes"])
    achieved = alg / (ms * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pts, v, o, min(args.cpu_budget, 8.0), single_s=0)
    line = {
        "metric": METRIC, "value": world * N / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "select256_500m", "desc": desc, "points_per_gpu": N, "queries": Q,
                   "vertices": int(v.shape[0]), "selected_ids": int(total), "grid_log2": info["grid_log2"],
                   "sub_log2": info["sub_log2"], "block_summary": bool(info["use_sum"]),
                   "point_query_evals_per_s": world * N * Q / (ms * 1e-3),
                   "launch": "one CUDA graph per step (pass 1a, pass 1b, scan, pass 3, count table, scan, emit)",
                   "index_build_ms": round(info["build_ms"], 1),
                   "index_build_on_device_ms": round(device_build_ms, 2), "autotune": tune,
                   "l2": "inputs larger than L2 (4 GB of points); no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "whole selection step", "algorithmic_bytes_per_launch": int(alg)},
        "cpu_baseline": cpu, "e2e": None, "clocks": clk,
        # the join (pass 1a, 1b, scan, pass 3), then the partition: count table, its scan, offsets, emit
        "gpu_launches": steps * (join_launches(N, False) + 3 +
                                 (1 if Q * max(1, -(-total // 32768)) <= 4 * 8192 else 3)),
    }
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    eng.close()
    del dpts, ids, offs
    return line


def buffer_measure(args, world, rank, local, torch, steps, warmup, n_override):
    """Buffered-polygon join (returns the JSON object): one step = spx_join of
    the resident table against the 256 buffered query polygons (count pass,
    scan, write pass), pairs + counts."""
    import oracle
    from paper_2203_14362_gb300 import spx
    clocks = ClockSampler(local)
    pts, (v, o), radii, desc = make_workload("buffer256_100m", n_override, rank)
    N, P = pts.shape[0], int(o.shape[0] - 1)
    eng = spx.Engine(local)
    dpts = torch.from_numpy(pts).cuda()
    ph = eng.load_points(dpts)
    gh = eng.load_polygons(v, o)
    ih = eng.build_buffer_index(gh, radii, grid_log2=args.grid, fp32_filter=bool(args.fp32))
    info = eng.index_info(ih)
    counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    try:
        total = eng.join(ph, ih, None, counts)
    except spx.SpxError as e:  # the two-call pattern: the first call reports the size
        total = int(str(e).split("needs ")[1].split(" ")[0])
    pairs = torch.empty((max(total, 1), 2), dtype=torch.int32, device="cuda")
    assert eng.join(ph, ih, pairs, counts) == total
    # a seeded sample of points against the oracle, one by one (any size)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(N, size=min(N, 100_000), replace=False))
    want, _ = oracle.buffer_join(pts[sample], v, o, radii)
    host = pairs[:total].cpu().numpy().view(np.uint32)
    lo = np.searchsorted(host[:, 0], sample, "left")
    hi = np.searchsorted(host[:, 0], sample, "right")
    got = np.concatenate([np.stack([np.searchsorted(sample, host[a:b, 0]), host[a:b, 1]], 1)
                          for a, b in zip(lo, hi) if b > a] or [np.zeros((0, 2), np.int64)]).astype(np.uint32)
    assert np.array_equal(got, want), "sampled points differ from the oracle"
    assert int(counts.sum().item()) == total
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        eng.join(ph, ih, pairs, counts, sync=False, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        eng.join(ph, ih, pairs, counts, sync=False, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world, torch)
    clk = clocks.summary(t_host0, t_host1)
    clocks.stop()
    peak, peak_kind = peaks()
    alg = 8 * N + 8 * total + 8 * P + int(info["device_bytes"])
    achieved = alg / (ms * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        m = min(N, 1_000_000)
        th = oracle.default_threads()
        t0 = time.perf_counter()
        oracle.buffer_join(pts[:m], v, o, radii, threads=th)
        sec = time.perf_counter() - t0
        cpu = {"value": m / sec / 1e9, "unit": UNIT, "cores": th, "kind": "oracle",
               "sample": f"first {m} points of the same table (buffered-polygon join, {sec:.1f} s)"}
    line = {
        "metric": METRIC, "value": world * N / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "buffer256_100m", "desc": desc, "points_per_gpu": N, "polygons": P,
                   "vertices": int(v.shape[0]), "pairs": int(total), "grid_log2": info["grid_log2"],
                   "edge_grid_log2": info["edge_grid_log2"], "edge_items": int(info["n_edge_items"]),
                   "index_build_ms": round(info["build_ms"], 1), "index_device_bytes": int(info["device_bytes"]),
                   "check": "100k sampled points == oracle; sum of counts == pairs",
                   "l2": "inputs larger than L2 (0.8 GB of points); no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": f"{peak_kind} hbm_gbs",
                     "kernel": "whole buffered join (k_buf_count, scan, k_buf_write)",
                     "algorithmic_bytes_per_launch": int(alg)},
        "cpu_baseline": cpu, "e2e": None, "clocks": clk,
        "gpu_launches": steps * (2 + (1 if -(-N // 256) <= 4 * 8192 else 3)),
    }
    eng.free(ih)
    eng.free(gh)
    eng.free(ph)
    eng.close()
    del dpts, pairs, counts
    return line


def spx_error():
    from paper_2203_14362_gb300 import spx
    return spx.SpxError


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["spx", "reference"], default="spx")
    ap.add_argument("--workload", default="tess2000_100m",
                    choices=["tess2000_100m", "stars_1m", "select256_500m", "serve_1b", "count_4b", "dist1024_100m",
                             "buffer256_100m"])
    ap.add_argument("--points", type=int, default=None, help="points per GPU (default: the workload's)")
    ap.add_argument("--grid", type=int, default=0, help="grid_log2 (0 = automatic)")
    ap.add_argument("--sub", type=int, default=0, help="sub_log2 (0 = default, 3)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture (reported as is)")
    ap.add_argument("--fp32", type=int, default=1)
    ap.add_argument("--autotune", action="store_true", help="choose grid_log2 / sub_log2 with spx_autotune")
    ap.add_argument("--cluster", type=int, default=-1,
                    help="count_4b: aggregate over a copy clustered by the cells of a 2^G grid, with its cell "
                         "directory (-1: G = the index's coarse grid, the default; 0: the table in row order)")
    ap.add_argument("--plain", action="store_true", help="time the plain two-pass comparison kernels")
    ap.add_argument("--cap", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-sample", type=int, default=2_000_000, help="points per reference-arm step")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement of the join workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload: skip the selection (500M points) and count (4B points) sub-measurements")
    ap.add_argument("--serve-timed", type=int, default=1000, help="timed requests per arrival rate and arm")
    ap.add_argument("--serve-warmup", type=int, default=50)
    ap.add_argument("--serve-burst", type=int, default=48, help="requests of the capacity burst")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "spx":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_spx(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
