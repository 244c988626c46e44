"""Benchmark of the SGM hot path (arXiv 1610.04121) on GB300.

One step = the whole path (Census, matching cost, path aggregation, sum,
winner-take-all, 3x3 median) over one synthetic stereo pair already resident
in HBM.  Default workload: 640x480, D = 128, 4 paths, P1 = 7, P2 = 84 (the
paper's headline shape, Section 4).  The metric is MDE/s = W*H*D per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun (N > 1) every rank processes its own pairs (replicas: pairs are
independent and one pair does not shard), so per-GPU work is fixed and the
scaling is weak.  ``--impl reference`` times the CPU oracle on the host cores
instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import stereo_synth as synth  # noqa: E402

DEFAULT_WORKLOAD = "sgm_640x480_d128_p4"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SM_COUNT_GB300 = 152
SM_MAX_MHZ_GB300 = 2070.0
# Algorithmic integer operations per disparity evaluation (DE) and path of
# Eq. 3: two "+P1", three minima, "+MC", "-m" and one minimum of the
# reduction over d; the winner-take-all adds one add per extra term and one
# minimum.  Packed u16x2 arithmetic does two of them per lane instruction.
OPS_PER_DE_PATH = 8
L2_FLUSH_BYTES = 256 << 20
SERVED_RATE_HZ = 2000.0
SERVED_LINE_SECONDS = 2.5      # the served object of the default line
SERVED_LINE_BOUND_US = 100000  # its admission bound (estimated wait)
BATCHED_LINE_STEPS = 5         # timed steps of the batched object of the default line
SERVED_OUT_RING = 4  # output buffers per pool pair (a pair can be in flight more than once)
# DRAM bytes (read + write) per launch of a kernel, from the ncu captures summarised
# under profiles/, with the fingerprint of the kernel sources they were taken on;
# reported as null once those sources have changed since the capture.  The
# 640x480 frame's figures come from the in-sequence capture (--cache-control
# none: the L2 flushed once before the frame, as in the timed steps); the
# 8-path frame's from a capture with ncu's default per-launch cache flush.
MEASURED_TRAFFIC = {
    # the paired schedule's second stage is two kernels side by side: their sum
    ("sgm_640x480_d128_p4", "pairs_vh"): (131189248, "f7a7031745fff723"),
    ("sgm_640x480_d128_p4", "pairs_h_wta"): (59698176 + 73417984, "f7a7031745fff723"),
    ("sgm_1242x375_d128_p8", "sweep_h"): (585012992, "f7a7031745fff723"),
    ("sgm_1242x375_d128_p8", "sweep_diag+"): (311625472, "f7a7031745fff723"),
    ("sgm_1242x375_d128_p8", "sweep_diag-"): (311849088, "f7a7031745fff723"),
    ("sgm_1242x375_d128_p8", "sweep_v"): (241643136, "f7a7031745fff723"),
}
KERNEL_SOURCES = ("sgm_sweeps.cuh", "sgm_pairs.cuh", "sgm_device.cuh", "sgm_internal.h")


def kernel_fingerprint():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1610_04121_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel):
    t = MEASURED_TRAFFIC.get((workload, kernel))
    if t is None or t[1] != kernel_fingerprint():
        return None
    return t[0]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(synth.WORKLOADS) + ["batch64", "served"])
    ap.add_argument("--duration", type=float, default=10.0, help="served: seconds of Poisson arrivals")
    ap.add_argument("--rate", type=float, default=SERVED_RATE_HZ, help="served: arrivals per second")
    ap.add_argument("--admission-us", type=float, default=0.0,
                    help="served: admission bound on the estimated wait (us); 0 = none")
    ap.add_argument("--no-batched", action="store_true", help="default line: skip the batched object")
    ap.add_argument("--no-served", action="store_true", help="default line: skip the served object")
    ap.add_argument("--served-seconds", type=float, default=SERVED_LINE_SECONDS,
                    help="default line: seconds of Poisson arrivals of the served object")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--post", type=int, default=0,
                    help="post-filters of sgm_compute_ex (1 sub-pixel | 2 LR check | 4 adaptive P2); "
                         "times that entry point instead of the plain path")
    ap.add_argument("--inflight", type=int, default=1,
                    help="frames in flight: N contexts on N streams take the steps in turn (a video stream's "
                         "throughput); 1 is the headline, one frame at a time")
    ap.add_argument("--schedule", type=int, default=-1,
                    help="4-path sweep schedule (0 vertical pair first, 1 horizontal pair first, 2 paired lines); "
                         "-1 lets the library autotune it (the default)")
    ap.add_argument("--census", default="csct", choices=["csct", "full"],
                    help="features: the CSCT of Eq. 1 or the full 9x7 Census (SGM_FLAG_CENSUS_FULL)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": SM_MAX_MHZ_GB300}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].strip()
                                                         .replace('.', '', 1).isdigit()) if rows else None}


def oracle_census(args):
    return "ct62" if args.census == "full" else "csct"


def oracle_mdes(w, max_seconds: float, rows: int = 0, census: str = "csct"):
    """Time the CPU oracle (single thread, as it stands) on the workload."""
    import oracle

    oracle.build()
    pair = synth.workload_pair(w.name)
    left, right = pair.left, pair.right
    if rows:
        left, right = left[:rows].copy(), right[:rows].copy()
    H, W = left.shape
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.sgm(left, right, w.spec.D, w.P1, w.P2, w.n_paths, census=census)
        n += 1
        if time.perf_counter() - t0 >= max_seconds:
            break
    dt = time.perf_counter() - t0
    return W * H * w.spec.D * n / dt / 1e6, n, (W, H)


def host_cores():
    """(usable cores, hardware threads): the affinity mask, like nproc, and os.cpu_count()."""
    try:
        usable = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        usable = os.cpu_count() or 1
    return usable, os.cpu_count() or usable


def oracle_baseline(w, census: str = "csct", seconds: float = 8.0):
    """The oracle timed on the host: single thread as it stands, and (CSCT)
    the thread-parallel driver on every usable core."""
    import oracle

    oracle.build()
    v1, n1, (bw, bh) = oracle_mdes(w, max_seconds=seconds, census=census)
    single = {"value": v1, "unit": "MDE/s", "cores": 1,
              "sample": f"{n1} full {bw}x{bh} D={w.spec.D} {w.n_paths}-path frames, one thread, ~{seconds:.0f} s"}
    usable, hw = host_cores()
    if census != "csct" or usable < 2:
        return dict(single, kind="oracle", nproc=usable, hardware_concurrency=hw, single_thread=single)
    pair = synth.workload_pair(w.name)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.sgm_threads(pair.left, pair.right, w.spec.D, w.P1, w.P2, w.n_paths, usable)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    de = w.spec.W * w.spec.H * w.spec.D
    return {"value": de * n / dt / 1e6, "unit": "MDE/s", "cores": usable, "kind": "oracle",
            "sample": f"{n} full {w.spec.W}x{w.spec.H} D={w.spec.D} {w.n_paths}-path frames on {usable} threads "
                      f"(rows, columns and directions of Eq. 1-4 in parallel), ~{seconds:.0f} s",
            "nproc": usable, "hardware_concurrency": hw, "single_thread": single}


def run_reference(args, w, ws, rank):
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    pair = synth.workload_pair(w.name)
    census = oracle_census(args)
    usable, hw = host_cores()
    threads = usable if census == "csct" else 1  # the thread-parallel driver computes the CSCT
    # each step is a bounded sample: a band of rows of the frame (the whole
    # frame for short runs), sized so the whole run stays within a few minutes
    per_frame_steps = 200 if threads > 1 else 40
    rows = min(w.spec.H, max(16, int(w.spec.H * per_frame_steps / max(args.steps + args.warmup, 1))))
    left, right = pair.left[:rows].copy(), pair.right[:rows].copy()

    def run(nt):
        if nt > 1:
            return oracle.sgm_threads(left, right, w.spec.D, w.P1, w.P2, w.n_paths, nt)
        return oracle.sgm(left, right, w.spec.D, w.P1, w.P2, w.n_paths, census=census)

    for _ in range(args.warmup):
        run(threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(threads)
    dt = time.perf_counter() - t0
    de = w.spec.W * rows * w.spec.D
    value = de * args.steps / dt / 1e6
    t1 = time.perf_counter()
    run(1)
    single = de / (time.perf_counter() - t1) / 1e6
    sample = (f"{w.spec.W}x{rows} band (rows 0..{rows - 1}) of the {w.spec.W}x{w.spec.H} D={w.spec.D} frame per "
              f"step on {threads} thread(s)")
    line = {
        "impl": "reference", "metric": "MDE/s", "value": value, "unit": "MDE/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded stereo_synth pair)",
        "config": workload_config(w, args),
        "cpu_baseline": {"value": value, "unit": "MDE/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "nproc": usable, "hardware_concurrency": hw,
                         "single_thread": {"value": single, "unit": "MDE/s", "cores": 1,
                                           "sample": "one step of the same band on one thread"}},
        "e2e": {"value": value, "unit": "MDE/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def max_over_ranks(x: float, pg, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_mdes(world_size: int, steps: int, de_per_step: int, max_ms: float) -> float:
    """Whole-job MDE/s: every rank ran `steps` pairs; time = slowest rank."""
    return world_size * steps * de_per_step / (max_ms / 1e3) / 1e6


def workload_config(w, args):
    return {"workload": w.name, "W": w.spec.W, "H": w.spec.H, "D": w.spec.D, "P1": w.P1, "P2": w.P2,
            "n_paths": w.n_paths, "pairs_per_step": 1,
            "census": "full 9x7 (62 bits)" if args.census == "full" else "CSCT (31 bits, Eq. 1)"}


def run_post_bench(args, w, ws, rank, local):
    """The path with post-filters (sgm_compute_ex_async, the captured graph)
    on the workload's pair, resident in HBM."""
    import torch
    from paper_1610_04121_gb300 import sgm

    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W, H, D = w.spec.W, w.spec.H, w.spec.D
    pair = synth.make_pair(w.spec, synth.BASE_SEED + synth.WORKLOAD_INDEX[w.name] + 7919 * rank)
    L = torch.from_numpy(pair.left).to(dev)
    R = torch.from_numpy(pair.right).to(dev)
    out = torch.empty((H, W), dtype=torch.int16, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    cflag = sgm.SGM_FLAG_CENSUS_FULL if args.census == "full" else 0
    ctx = sgm.Context(local, flags=cflag)
    sgm.sgm_set_stream(ctx.handle, stream)

    def step():
        sgm.sgm_compute_ex_async(ctx.handle, L, R, W, H, D, w.P1, w.P2, w.n_paths, args.post, out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ctx.launches
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            ev0[k].record(stream)
            step()
            ev1[k].record(stream)
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    launches = ctx.launches - launches0
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)), pg, dev)
    ms_per_step = total_ms / args.steps
    de = W * H * D
    value = job_mdes(ws, args.steps, de, total_ms)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        census = oracle_census(args)
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < 10.0:
            oracle.sgm_ex(pair.left, pair.right, D, w.P1, w.P2, w.n_paths, args.post, census)
            n += 1
        dt = time.perf_counter() - t0
        cpu = {"value": de * n / dt / 1e6, "unit": "MDE/s", "cores": 1, "kind": "oracle",
               "sample": f"{n} full {W}x{H} D={D} {w.n_paths}-path frames with post={args.post}, single thread"}
    if rank == 0:
        peaks, peak_kind = load_peaks()
        hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
        passes = 2 if args.post & 2 else 1
        frame_bytes = passes * (2 * W * H + W * H + 4 * de) + 2 * W * H
        frame_gbs = frame_bytes / (ms_per_step / 1e3) / 1e9
        line = {
            "metric": "MDE/s", "value": value, "unit": "MDE/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic (seeded stereo_synth pair, resident in HBM)",
            "config": dict(workload_config(w, args), parallelism=f"replicas x{ws}", post=args.post,
                           post_names=[n for b, n in ((1, "subpixel"), (2, "lr_check"), (4, "adaptive_p2"))
                                       if args.post & b],
                           l2="flushed between timed steps (256 MiB write)", fps=1e3 / ms_per_step,
                           de_counts="W*H*D once per frame, although the LR check runs a second matching pass"),
            "roofline": None,
            "frame_roofline": {"bound": "hbm", "achieved": frame_gbs, "peak": hbm, "unit": "GB/s",
                               "frac": frame_gbs / hbm, "algorithmic_bytes_per_frame": frame_bytes,
                               "peak_source": f"{peak_kind} hbm_gbs"},
            "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
        }
        print(json.dumps(line))
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


def run_inflight_bench(args, w, ws, rank, local):
    """Frames of one shape in flight together: context i (own stream, own
    arena, own pair) takes steps i, i + N, ...; the K steps are timed as one
    region from the first stream's start to the last stream's end.  Each
    frame's records (about 200 MB at 640x480x128) exceed L2, and the frames
    in flight use different pairs and arenas."""
    import torch
    from paper_1610_04121_gb300 import sgm

    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W, H, D, N = w.spec.W, w.spec.H, w.spec.D, args.inflight
    lanes = []
    for i in range(N):
        pair = synth.make_pair(w.spec, synth.BASE_SEED + synth.WORKLOAD_INDEX[w.name] + 7919 * rank + 101 * i)
        L = torch.from_numpy(pair.left).to(dev)
        R = torch.from_numpy(pair.right).to(dev)
        out = torch.empty((H, W), dtype=torch.uint8, device=dev)
        st = torch.cuda.Stream(dev)
        c = sgm.Context(local)
        sgm.sgm_set_stream(c.handle, st)
        if args.schedule >= 0:
            sgm.sgm_set_schedule(c.handle, args.schedule)
        lanes.append((c, st, L, R, out))

    def step(k):
        c, st, L, R, out = lanes[k % N]
        sgm.sgm_compute_async(c.handle, L, R, W, H, D, w.P1, w.P2, w.n_paths, out)

    for k in range(max(args.warmup, 3) * N):
        step(k)
    torch.cuda.synchronize(dev)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(N)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(N)]
    launches0 = sum(l[0].launches for l in lanes)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for i in range(N):
            ev0[i].record(lanes[i][1])
        for k in range(args.steps):
            step(k)
        for i in range(N):
            ev1[i].record(lanes[i][1])
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    launches = sum(l[0].launches for l in lanes) - launches0
    # the region from the earliest start to the latest end over the streams
    t_ms = max(ev0[0].elapsed_time(ev1[i]) for i in range(N)) - min(ev0[0].elapsed_time(ev0[i]) for i in range(N))
    total_ms = max_over_ranks(t_ms, pg, dev)
    ms_per_step = total_ms / args.steps
    value = job_mdes(ws, args.steps, W * H * D, total_ms)
    if rank == 0:
        line = {
            "metric": "MDE/s", "value": value, "unit": "MDE/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic (seeded stereo_synth pairs, resident in HBM)",
            "config": dict(workload_config(w, args), parallelism=f"replicas x{ws}", frames_in_flight=N,
                           l2="records of each frame (~200 MB at 640x480x128) exceed L2; frames in flight use "
                              "different pairs and arenas", fps=1e3 / ms_per_step),
            "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
        }
        print(json.dumps(line))
    for l in lanes:
        l[0].close()
    if pg:
        pg.destroy_process_group()
    return 0


def measure_batched(args, ws, rank, local, pg, steps, warmup, cpu_sample=False):
    """64 uneven pairs per step through sgm_compute_batch (persistent per-stage
    grids over device work lists, one graph per wave), against the same pairs
    as plain per-pair launches (sgm_compute_async, one after another)."""
    import torch
    from paper_1610_04121_gb300 import sgm

    dev = torch.device("cuda", local)
    recipe = synth.batch_recipe(64)
    pairs = [synth.make_pair(w.spec, synth.BASE_SEED + 3000 + i + 7919 * rank) for i, w in enumerate(recipe)]
    tuples, host_tuples = [], []
    for w, p in zip(recipe, pairs):
        W, H, D = w.spec.W, w.spec.H, w.spec.D
        L, R = torch.from_numpy(p.left).to(dev), torch.from_numpy(p.right).to(dev)
        O = torch.empty((H, W), dtype=torch.uint8, device=dev)
        tuples.append((L, R, O, W, H, D, w.P1, w.P2, w.n_paths))
        host_tuples.append((torch.from_numpy(p.left).pin_memory(), torch.from_numpy(p.right).pin_memory(),
                            torch.empty((H, W), dtype=torch.uint8).pin_memory(), W, H, D, w.P1, w.P2, w.n_paths))
    de = sum(t[3] * t[4] * t[5] for t in tuples)
    stream = torch.cuda.Stream(dev)
    ctx = sgm.Context(local)
    sgm.sgm_set_stream(ctx.handle, stream)
    for _ in range(max(warmup, 3)):  # the first call autotunes the sweep grid of the wave
        sgm.sgm_compute_batch(ctx.handle, tuples)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launches
    with ClockSampler(local) as clk:
        for a, b in ev:
            a.record(stream)
            sgm.sgm_compute_batch(ctx.handle, tuples)  # inputs (~58 GB of buffers) far exceed L2
            b.record(stream)
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
    launches = ctx.launches - launches0
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), pg, dev)
    value = job_mdes(ws, steps, de, total_ms)
    # the same pairs as plain per-pair launches
    for t in tuples:  # warm-up: tunes and captures one graph per pair
        sgm.sgm_compute_async(ctx.handle, t[0], t[1], t[3], t[4], t[5], t[6], t[7], t[8], t[2])
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for t in tuples:
        sgm.sgm_compute_async(ctx.handle, t[0], t[1], t[3], t[4], t[5], t[6], t[7], t[8], t[2])
    b.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = max_over_ranks(a.elapsed_time(b), pg, dev)
    plain = job_mdes(ws, 1, de, plain_ms)
    # end to end with pinned host buffers
    sgm.sgm_compute_batch(ctx.handle, host_tuples)
    t0 = time.perf_counter()
    sgm.sgm_compute_batch(ctx.handle, host_tuples)
    dt = max_over_ranks(time.perf_counter() - t0, pg, dev)
    h2d = sum(2 * t[3] * t[4] for t in host_tuples)
    d2h = sum(t[3] * t[4] for t in host_tuples)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    alg_bytes = sum(3 * t[3] * t[4] + 4 * t[3] * t[4] * t[5] for t in tuples)
    gbs = alg_bytes / (total_ms / steps / 1e3) / 1e9
    cpu = None
    if cpu_sample and rank == 0 and ws == 1:
        import oracle

        oracle.build()
        small = [(w, p) for w, p in zip(recipe, pairs) if w.spec.W == 320][:2]
        t0, n_de = time.perf_counter(), 0
        for w, p in small:
            oracle.sgm(p.left, p.right, w.spec.D, w.P1, w.P2, w.n_paths)
            n_de += w.spec.W * w.spec.H * w.spec.D
        cpu = {"value": n_de / (time.perf_counter() - t0) / 1e6, "unit": "MDE/s", "cores": 1, "kind": "oracle",
               "sample": f"the {len(small)} 320x240 pairs of the batch, single thread"}
    ctx.close()
    return {
        "value": value, "unit": "MDE/s", "steps": steps, "ms_per_step": total_ms / steps, "pairs_per_step": len(tuples),
        "de_per_step": de, "plain_per_pair_mdes": plain, "batched_over_plain": value / plain,
        "sizes": "320x240/640x480/1242x375/1920x1080, D 64/128/256, 4 or 8 paths (P1 = 7, P2 = 84)",
        "execution": "sgm_compute_batch: persistent per-stage grids over device work lists, one graph launch "
                     "per wave, sweep grid autotuned",
        "l2": "inputs and buffers (~58 GB) exceed L2",
        "roofline": {"bound": "hbm", "kernel": "whole batch", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                     "frac": gbs / hbm, "traffic": None, "algorithmic_bytes_per_step": alg_bytes,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "e2e": {"value": job_mdes(ws, 1, de, dt * 1e3), "unit": "MDE/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": dt * 1e3, "api": "sgm_compute_batch (pinned host buffers)"},
        "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": cpu,
    }


def run_batch_bench(args, ws, rank, local):
    import torch

    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    torch.cuda.set_device(local)
    r = measure_batched(args, ws, rank, local, pg, args.steps, args.warmup, cpu_sample=not args.no_cpu_baseline)
    if rank == 0:
        line = {
            "metric": "MDE/s", "value": r["value"], "unit": "MDE/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic (seeded stereo_synth batch, resident in HBM)",
            "config": {"workload": "batch64", "pairs_per_step": r["pairs_per_step"], "de_per_step": r["de_per_step"],
                       "sizes": r["sizes"], "parallelism": f"replicas x{ws}", "l2": r["l2"],
                       "plain_per_pair_mdes": r["plain_per_pair_mdes"], "batched_over_plain": r["batched_over_plain"]},
            "roofline": r["roofline"], "cpu_baseline": r["cpu_baseline"], "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


def measure_served(args, ws, rank, local, pg, duration, rate, bound_us):
    """Poisson arrivals of mixed pairs (sizes up to 1920x1080, D up to 256, 8
    paths) through sgm_submit / sgm_poll with pinned host buffers; the context
    batches whatever is queued and keeps two batches in flight.  With
    bound_us > 0 the admission bound sheds requests whose estimated wait
    exceeds it."""
    import threading

    import torch
    from paper_1610_04121_gb300 import sgm

    dev = torch.device("cuda", local)
    # sizes and D as the batch; 8 paths with P1 = 10, P2 = 120 ("up to 1920x1080 with D up to 256 and 8 paths")
    recipe = synth.batch_recipe(64, config=4, paths=(8,), P1=10, P2=120)
    pool = []
    for i, w in enumerate(recipe):
        p = synth.make_pair(w.spec, synth.BASE_SEED + 4000 + i + 7919 * rank)
        W, H, D = w.spec.W, w.spec.H, w.spec.D
        pool.append((torch.from_numpy(p.left).pin_memory(), torch.from_numpy(p.right).pin_memory(),
                     torch.empty((SERVED_OUT_RING, H, W), dtype=torch.uint8).pin_memory(), W, H, D, w.P1, w.P2,
                     w.n_paths))
    arrivals = synth.poisson_arrivals(rate, duration, synth.BASE_SEED + 4 + 7919 * rank)
    ctx = sgm.Context(local)

    def submit(k, ring):
        L, R, O, W, H, D, P1, P2, npth = pool[k]
        return sgm.sgm_submit(ctx.handle, L, R, W, H, D, P1, P2, npth, O[ring])

    # warm-up: every pool pair once (grows the slot arenas, measures the service rate)
    for t in [submit(k, 0) for k in range(len(pool))]:
        sgm.sgm_poll(ctx.handle, t, -1)
    sgm.sgm_served_reset_stats(ctx.handle)
    if bound_us > 0:
        sgm.sgm_set_admission_bound(ctx.handle, int(bound_us))
    launches0 = ctx.launches
    tickets = [None] * len(arrivals)
    submitted = threading.Semaphore(0)

    def producer(t0):
        for i, ta in enumerate(arrivals):
            delay = t0 + ta - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[i] = submit(i % len(pool), (i // len(pool)) % SERVED_OUT_RING)
            submitted.release()

    if pg:
        pg.barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        th = threading.Thread(target=producer, args=(t0,))
        th.start()
        for i in range(len(arrivals)):
            submitted.acquire()
            if tickets[i] is not None:  # None: shed by the admission bound
                sgm.sgm_poll(ctx.handle, tickets[i], -1)
        wall = time.perf_counter() - t0
        th.join()
    wall = max_over_ranks(wall, pg, dev)
    st = sgm.sgm_served_stats(ctx.handle)
    launches = ctx.launches - launches0
    n = len(arrivals)
    de_of = lambda i: pool[i % len(pool)][3] * pool[i % len(pool)][4] * pool[i % len(pool)][5]  # noqa: E731
    offered = sum(de_of(i) for i in range(n))
    served = sum(de_of(i) for i in range(n) if tickets[i] is not None)
    value = job_mdes(ws, 1, served, wall * 1e3)
    # the same pool as plain one-pair calls, one after another (the first pass
    # sizes the arena and captures one graph per pair)
    for timed in (False, True):
        t1 = time.perf_counter()
        for L, R, O, W, H, D, P1, P2, npth in pool:
            sgm.sgm_compute(ctx.handle, L, R, W, H, D, P1, P2, npth, O[0])
        plain_s = time.perf_counter() - t1
    pool_de = sum(t[3] * t[4] * t[5] for t in pool)
    plain = job_mdes(ws, 1, pool_de, max_over_ranks(plain_s, pg, dev) * 1e3)
    h2d = sum(2 * pool[i % len(pool)][3] * pool[i % len(pool)][4] for i in range(n)) / max(n, 1)
    ctx.close()
    return {
        "value": value, "unit": "MDE/s", "arrival_rate_hz": rate, "duration_s": duration, "requests": n,
        "admitted": n - st["shed"], "shed": st["shed"], "admission_bound_us": bound_us or None,
        "offered_mdes": offered / duration / 1e6, "served_mdes": value, "wall_s": wall,
        "pool": "64 pairs: 320x240/640x480/1242x375/1920x1080, D 64/128/256, 8 paths, P1 = 10, P2 = 120",
        "plain_per_pair_mdes": plain, "served_over_plain": value / plain if plain else None,
        "latency_us": {"p50": st["p50_us"], "p99": st["p99_us"], "max": st["max_us"]},
        "batching": {"batches": st["batches"], "mean_pairs_per_batch": st["mean_batch"],
                     "max_in_flight": st["max_in_flight"]},
        "e2e": {"value": value, "unit": "MDE/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d / 2,
                "api": "sgm_submit / sgm_poll (host buffers, copies inside)"},
        "gpu_launches": launches, "clocks": clk.summary(),
    }


def run_served_bench(args, ws, rank, local):
    import torch

    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
        pg = dist
    torch.cuda.set_device(local)
    r = measure_served(args, ws, rank, local, pg, args.duration, args.rate, args.admission_us)
    if rank == 0:
        line = {
            "metric": "MDE/s", "value": r["value"], "unit": "MDE/s", "n_gpus": ws, "steps": r["requests"],
            "warmup": args.warmup, "ms_per_step": r["wall_s"] * 1e3 / max(r["requests"], 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic (seeded stereo_synth pairs, pinned host buffers)",
            "config": {"workload": "served", "arrival_rate_hz": r["arrival_rate_hz"], "duration_s": r["duration_s"],
                       "requests": r["requests"], "admitted": r["admitted"], "shed": r["shed"],
                       "admission_bound_us": r["admission_bound_us"], "pool": r["pool"],
                       "offered_mdes": r["offered_mdes"], "step": "one request", "parallelism": f"replicas x{ws}",
                       "l2": "inputs and buffers far exceed L2", "plain_per_pair_mdes": r["plain_per_pair_mdes"],
                       "served_over_plain": r["served_over_plain"]},
            "latency_us": r["latency_us"], "batching": r["batching"], "cpu_baseline": None, "e2e": r["e2e"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
        }
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.workload in ("batch64", "served"):
        if args.impl == "reference":
            return run_reference(args, synth.WORKLOADS[DEFAULT_WORKLOAD], ws, rank)
        if args.workload == "served":
            return run_served_bench(args, ws, rank, local)
        return run_batch_bench(args, ws, rank, local)
    w = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, ws, rank)
    if args.post:
        return run_post_bench(args, w, ws, rank, local)
    if args.inflight > 1:
        return run_inflight_bench(args, w, ws, rank, local)

    import torch

    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    torch.cuda.set_device(local)
    from paper_1610_04121_gb300 import sgm

    W, H, D = w.spec.W, w.spec.H, w.spec.D
    pair = synth.make_pair(w.spec, synth.BASE_SEED + synth.WORKLOAD_INDEX[w.name] + 7919 * rank)
    dev = torch.device("cuda", local)
    L = torch.from_numpy(pair.left).to(dev)
    R = torch.from_numpy(pair.right).to(dev)
    out = torch.empty((H, W), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)
    # one explicit stream carries the path, the L2 flush and the timing events
    stream = torch.cuda.Stream(dev)
    cflag = sgm.SGM_FLAG_CENSUS_FULL if args.census == "full" else 0
    ctx = sgm.Context(local, flags=cflag)
    sgm.sgm_set_stream(ctx.handle, stream)
    # Per-kernel durations come from a second context whose captured graph
    # records an event between its kernels; those event nodes lengthen the
    # frame, so that context runs its own timed pass after the headline one.
    ctx_st = sgm.Context(local, flags=sgm.SGM_FLAG_STAGE_TIMING | cflag)
    sgm.sgm_set_stream(ctx_st.handle, stream)

    def step(c):
        sgm.sgm_compute_async(c.handle, L, R, W, H, D, w.P1, w.P2, w.n_paths, out)

    # the first call of the headline context tunes its 4-path sweep schedule
    # (unless one is forced); the timing and end-to-end contexts then run the
    # same schedule
    if args.schedule >= 0:
        sgm.sgm_set_schedule(ctx.handle, args.schedule)
    for _ in range(max(args.warmup, 3)):
        step(ctx)
    torch.cuda.synchronize(dev)
    sched = sgm.sgm_schedule_for(ctx.handle, W, H, D, w.P1, w.P2, w.n_paths)
    sgm.sgm_set_schedule(ctx_st.handle, sched)
    for _ in range(max(args.warmup, 3)):
        step(ctx_st)
    torch.cuda.synchronize(dev)

    def timed_pass(c, n, stage_ms=None):
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        if pg:
            pg.barrier()
        torch.cuda.synchronize(dev)
        for k in range(n):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)  # evict the previous step's data from L2
            ev0[k].record(stream)
            step(c)
            ev1[k].record(stream)
            if stage_ms is not None:
                for name, ms in sgm.sgm_stage_times(c.handle).items():  # waits for this step
                    stage_ms.setdefault(name, []).append(ms)
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        return [a.elapsed_time(b) for a, b in zip(ev0, ev1)]

    launches0 = ctx.launches
    with ClockSampler(local) as clk:
        step_ms = timed_pass(ctx, args.steps)
    launches = ctx.launches - launches0
    stage_steps = max(3, min(args.steps, 50))
    stage_ms = {}
    timed_pass(ctx_st, stage_steps, stage_ms)
    ctx_st.close()
    total_ms = max_over_ranks(sum(step_ms), pg, dev)
    ms_per_step = total_ms / args.steps
    de = W * H * D
    value = job_mdes(ws, args.steps, de, total_ms)

    # dominant kernel and its roofline (integer ALU: packed u16x2 lanes)
    peaks, peak_kind = load_peaks()
    clocks = clk.summary()
    mean_stage = {k: statistics.mean(v) for k, v in stage_ms.items()}
    # the dominant kernel: each stage is one kernel launch.  Path units per
    # launch (one unit = one path over every DE) and extra adds per DE:
    #   2 paths: sweep_h one path; sweep_v one path, S add and the minimum.
    #   4 paths: sweep_v+h1 the whole vertical pair (2) and the horizontal
    #     first halves (1), plus the stored-L add of the vertical second
    #     halves; sweep_h2 the horizontal second halves (1), the stored-L and
    #     S adds and the minimum.
    #   8 paths: sweep_h the horizontal pair (2) and the first halves of three
    #     vertical-type pairs (3), plus the horizontal stored-L add; every
    #     later sweep the second halves of one pair (1) with its adds.
    if w.n_paths == 2:
        kernel_stages = {"sweep_h": (1, 0), "sweep_v": (1, 2)}
    elif w.n_paths == 4:
        # the first two schedules: the whole first pair beside the other pair's
        # first halves, then that pair's second halves with the winner-take-all;
        # the paired-line schedule: the whole vertical pair beside n1 = min(W2, H2)
        # steps of each horizontal direction, then the rest of the horizontal
        # directions, and the sums and the minimum of every pixel
        W2, H2 = W + (W & 1), H + (H & 1)
        f1 = min(W2, H2) / W2
        kernel_stages = {"sweep_v+h1": (3, 1), "sweep_h2": (1, 3), "sweep_h+v1": (3, 1), "sweep_v2": (1, 3),
                         "pairs_vh": (2 + 2 * f1, 1), "pairs_h_wta": (2 * (1 - f1), 3)}
    else:
        kernel_stages = {"sweep_h": (2 + (w.n_paths - 2) // 2, 1), "sweep_v": (1, 3), "sweep_diag+": (1, 2),
                         "sweep_diag-": (1, 2)}
    dom = max((k for k in mean_stage if k in kernel_stages), key=mean_stage.get)
    units, extra = kernel_stages[dom]
    ops = de * (OPS_PER_DE_PATH * units + extra)
    sm_mhz = float(peaks.get("sm_max_mhz", SM_MAX_MHZ_GB300))
    peak_tops = SM_COUNT_GB300 * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = ops / (mean_stage[dom] / 1e3) / 1e12
    traffic = measured_traffic(w.name, dom) if args.census == "csct" else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved / peak_tops, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": f"152 SMs x 128 lanes x 2 (u16x2) x {sm_mhz:.0f} MHz (recipe unit counts, max clock)",
                "ops_per_launch": ops}
    frame_bytes = 2 * W * H + W * H + 4 * de
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    if w.n_paths == 8:
        # u16 sums: the sweeps move more bytes than their arithmetic can hide.
        # Algorithmic bytes per DE of each launch: the first stage reads MC
        # twice for the horizontal pair and once per vertical-type pair, stores
        # and reloads the horizontal stored L_r, stores the three vertical-type
        # ones and writes S (u16); each diagonal second half reads MC and its
        # stored L_r and reads and writes S; the vertical one reads all three.
        bytes_per_de = {"sweep_h": 12, "sweep_diag+": 6, "sweep_diag-": 6, "sweep_v": 4}
        alg = de * bytes_per_de[dom]
        gbs = alg / (mean_stage[dom] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "traffic": traffic,
                    "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                    "algorithmic_bytes_per_launch": alg, "peak_source": f"{peak_kind} hbm_gbs"}
    frame_gbs = frame_bytes / (ms_per_step / 1e3) / 1e9
    frame_roofline = {"bound": "hbm", "achieved": frame_gbs, "peak": hbm, "unit": "GB/s", "frac": frame_gbs / hbm,
                      "algorithmic_bytes_per_frame": frame_bytes, "peak_source": f"{peak_kind} hbm_gbs"}

    # end to end through the public C call with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        Lh = torch.from_numpy(pair.left).pin_memory()
        Rh = torch.from_numpy(pair.right).pin_memory()
        Oh = torch.empty((H, W), dtype=torch.uint8).pin_memory()
        ctx2 = sgm.Context(local, flags=cflag)
        sgm.sgm_set_schedule(ctx2.handle, sched)
        for _ in range(3):
            sgm.sgm_compute(ctx2.handle, Lh, Rh, W, H, D, w.P1, w.P2, w.n_paths, Oh)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sgm.sgm_compute(ctx2.handle, Lh, Rh, W, H, D, w.P1, w.P2, w.n_paths, Oh)
        dt = max_over_ranks(time.perf_counter() - t0, pg, dev)
        e2e = {"value": job_mdes(ws, args.e2e_steps, de, dt * 1e3), "unit": "MDE/s", "h2d_bytes_per_step": 2 * W * H,
               "d2h_bytes_per_step": W * H, "ms_per_step": dt / args.e2e_steps * 1e3, "api": "sgm_compute"}
        ctx2.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(w, census=oracle_census(args))

    # the batched and served forms of the same metric (64 uneven pairs; a
    # Poisson stream at 2000 pairs/s under an admission bound)
    batched = served = None
    if args.workload == DEFAULT_WORKLOAD and args.census == "csct" and args.schedule < 0:
        if not args.no_batched:
            batched = measure_batched(args, ws, rank, local, pg, BATCHED_LINE_STEPS, 3)
            batched.pop("cpu_baseline", None)
        if not args.no_served:
            served = measure_served(args, ws, rank, local, pg, args.served_seconds, args.rate, SERVED_LINE_BOUND_US)

    if rank == 0:
        line = {
            "metric": "MDE/s", "value": value, "unit": "MDE/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic (seeded stereo_synth pair, resident in HBM)",
            "config": dict(workload_config(w, args), parallelism=f"replicas x{ws}",
                           l2="flushed between timed steps (256 MiB write)", fps=1e3 / ms_per_step,
                           sweep_schedule={0: "V_THEN_H", 1: "H_THEN_V", 2: "PAIRS"}.get(sched, str(sched))
                           + (" (autotuned)" if w.n_paths == 4 and args.schedule < 0 else "")),
            "roofline": roofline, "frame_roofline": frame_roofline,
            "stage_ms": {k: round(v, 5) for k, v in mean_stage.items()},
            "stage_timing": f"separate pass of {stage_steps} steps with an event between kernels "
                            "(the events lengthen that pass's frames)",
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "batched": batched, "served": served,
        }
        print(json.dumps(line))
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
