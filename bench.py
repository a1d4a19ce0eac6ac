"""Benchmark: SRE+SLE update and slice close on the core-link workload.

One step = one time slice of 2^25 synthetic IP pairs (core-link trace: 16M-host Zipf(1.05)
population, 200 planted super points): sse_update() of the slice's pairs (already in
HBM) followed by sse_close_slice() (expire, hot SREs, candidate join, sort, estimation,
report copied to the host). Estimator: q=20 (RSRA 40 MiB), SLEA 2^16 SLEs x 2^12 cells,
delta'=16, window k=8, theta=1024, 8-bit stamps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Under torchrun (N > 1) every rank runs its own router's trace
(independent estimators: weak scaling, no data-path collective); the time is the max
over ranks. --impl reference times the CPU oracle (tests' checker) on the host's cores,
one oracle estimator per thread, on a bounded sample.

After the timed core-link steps the same line also carries, measured on the same GPU: the
roofs of the update's units (sse_microbench), a paced serving leg (32 routers at the offered
2e9 pairs/s: slice-close-to-report p50/p99), and, from child processes running the other
workloads, the 16-edge-router batch step and the learned correction (training samples/s,
median relative error against linear counting); --no-legs and --serve-slices 0 leave those
out. --workload selects one of the other workloads alone.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpackets/s SRE+SLE update at 1 B300 (% of L2/HBM roofline); slice-close p50/p99 ms"
UNIT = "Gpkt/s"
PAIRS_PER_SLICE = 1 << 25
PREFILL = 8          # slices scanned before warm-up so that the window is full
DISTINCT = 16        # device-resident slices the warm-up and timed steps cycle through
PAIR_BYTES = 8
CORE_LINK_WORKLOAD = ("core_link: 2^25 pairs/slice, 16M-host Zipf(1.05), 200 planted super points; "
                      "q=20, r=5, SLEA r'=5 x (2^16 SLEs, eta'=4096, delta'=16), k=8, theta=1024")
TILED8_DRAM_BYTES = 273_648_896 + 7_201_024


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 200; 27 epochs for learned)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", type=int, default=0, help="update mode: 0 auto, 1 direct, 2 tiled")
    ap.add_argument("--prefill", type=int, default=PREFILL, help="slices scanned before warm-up")
    ap.add_argument("--distinct", type=int, default=DISTINCT, help="device-resident step inputs")
    ap.add_argument("--workload", default="core_link",
                    choices=["core_link", "paper_params", "edge_routers", "serving", "learned"])
    ap.add_argument("--learn-train", type=int, default=1_000_000, help="training hosts (learned workload)")
    ap.add_argument("--learn-test", type=int, default=100_000, help="held-out hosts (learned workload)")
    ap.add_argument("--serve-seconds", type=float, default=0.5, help="virtual seconds of serving traffic")
    ap.add_argument("--routers", type=int, default=16)
    ap.add_argument("--edge-q", type=int, default=22, help="RSRA size (log2 SREs per row) for edge_routers")
    ap.add_argument("--update-variant", type=int, default=None, help="fixed update variant (no autotuning)")
    ap.add_argument("--batch-config", type=int, default=None,
                    help="fixed batch configuration item*3 + loads (no autotuning), edge_routers")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--latency-samples", type=int, default=200, help="synchronised slice closes timed after the run")
    ap.add_argument("--latency-warmup", type=int, default=400,
                    help="untimed synchronised slice closes before those samples")
    ap.add_argument("--paced", action="store_true",
                    help="serving: submit each request at its arrival time (wall clock) instead of at once")
    ap.add_argument("--serve-slices", type=int, default=200,
                    help="slice closes of the paced serving leg of the core-link run (0: no serving leg)")
    ap.add_argument("--no-legs", action="store_true",
                    help="core-link run without the edge-router and learned-correction legs")
    args = ap.parse_args(argv)
    if args.steps is None:
        args.steps = 27 if args.workload == "learned" else 200
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_ranks(world: int):
    """The process group of a multi-rank run (NCCL with GPUs, gloo without), else None."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist


def barrier(pg) -> None:
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float, device) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, value: float, device) -> float:
    """The sum of every rank's value (work done by the whole job)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def make_traffic(rank: int):
    from paper_1805_09246_b300 import synth
    return synth.Traffic(synth.core_link(seed=rank))


CPU_THREADS_MAX = 64  # host threads for the oracle timings (one oracle estimator each, ~90 MiB)


def host_cores() -> int:
    """The host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_threads(threads: int | None) -> int:
    return max(1, min(threads or host_cores(), CPU_THREADS_MAX))


def core_link_oracle_params():
    import oracle
    return oracle.Params(q=20, q2=16, eta2=4096, k=8, theta=1024, seed=0)


def run_reference(args, rank, world, threads: int | None = None):
    """The CPU oracle as it stands on the host's cores, on a bounded sample of each slice:
    one oracle estimator per thread (the data-parallel use of the unchanged oracle, one
    router per core; its C scan loop runs without Python's interpreter lock). In every step
    each thread scans the first 2^21 pairs of a core-link slice (thread i starts i slices
    further on) and advances its slice."""
    if rank != 0:
        return
    import threading

    import oracle
    tr = make_traffic(0)
    sample = 1 << 21
    n_thr = oracle_threads(threads)
    data = [tr.slice(0, t)[:sample].copy() for t in range(16)]
    orcs = [oracle.Oracle(core_link_oracle_params()) for _ in range(n_thr)]
    start, done = threading.Barrier(n_thr + 1), threading.Barrier(n_thr + 1)

    def work(i):
        try:
            o = orcs[i]
            for w in range(args.warmup):
                o.scan(data[(i + w) % len(data)])
                o.advance()
            start.wait()
            for s in range(args.steps):
                o.scan(data[(i + args.warmup + s) % len(data)])
                o.advance()
            done.wait()
        except BaseException:  # a failed thread breaks the barriers, so the run fails instead of waiting
            start.abort()
            done.abort()
            raise

    pool = [threading.Thread(target=work, args=(i,)) for i in range(n_thr)]
    for t in pool:
        t.start()
    start.wait()
    t0 = time.perf_counter()
    done.wait()
    dt = time.perf_counter() - t0
    for t in pool:
        t.join()
    value = n_thr * args.steps * sample / dt / 1e9
    desc = (f"{n_thr} oracle estimator{'s' if n_thr > 1 else ''}, one per host thread, each scanning (Alg. 3 + Alg. 6) the first {sample} "
            "pairs of a core-link slice per step plus the per-slice distance increment; detection is not "
            "timed: the oracle's tuple growth is O(|HSE|^3) at this size")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": CORE_LINK_WORKLOAD, "pairs_per_step": PAIRS_PER_SLICE,
                   "l2": "inputs larger than L2 (256 MiB per step)"},
        "sample_pairs_per_step": n_thr * sample,
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": n_thr, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline(tr_slices, min_seconds=12.0, min_slices=8, max_slices=64, threads: int | None = None):
    """The oracle's update loop on the host's cores over full slices of the workload: one
    oracle estimator per thread, each scanning the generated slices in turn (thread i
    starts i slices further on, again from the first when they run out) and advancing its
    slice after each, until min_seconds have passed and min_slices slices are done in all
    (at most max_slices per thread). The rate is all threads' pairs over the wall time from
    the common start until the last thread ends."""
    import threading

    import oracle
    n_thr = oracle_threads(threads)
    orcs = [oracle.Oracle(core_link_oracle_params()) for _ in range(n_thr)]
    pairs, slices = [0] * n_thr, [0] * n_thr
    lock = threading.Lock()
    total = [0]
    start = threading.Barrier(n_thr + 1)
    t0 = [0.0]

    def work(i):
        o = orcs[i]
        try:
            start.wait()
        except threading.BrokenBarrierError:
            return
        t = 0
        while t < max_slices:
            with lock:
                if total[0] >= min_slices and time.perf_counter() - t0[0] >= min_seconds:
                    break
                total[0] += 1
            if t:
                o.advance()
            s = tr_slices[(i + t) % len(tr_slices)]
            o.scan(s)
            pairs[i] += len(s)
            t += 1
        slices[i] = t

    pool = [threading.Thread(target=work, args=(i,)) for i in range(n_thr)]
    for t in pool:
        t.start()
    t0[0] = time.perf_counter()
    start.wait()
    for t in pool:
        t.join()
    dt = time.perf_counter() - t0[0]
    n, n_slices = sum(pairs), sum(slices)
    return {"value": round(n / dt / 1e9, 6), "unit": UNIT, "cores": n_thr, "kind": "oracle",
            "sample": f"{n_thr} oracle estimator{'s' if n_thr > 1 else ''}, one per host thread, oracle scan + slice increment over "
                      f"{n_slices} full core-link slices in all (the {len(tr_slices)} generated ones in turn; "
                      f"{n} pairs, {dt:.1f} s); detection excluded (tuple growth is O(|HSE|^3) here)"}


def main_edge_routers(args, rank, world, local):
    """16 edge routers with uneven loads (log-uniform 2^20..2^25 pairs per router and slice):
    one batch step = one persistent update launch over all routers, the merge into the global
    estimator and the global slice close, replayed from a CUDA graph."""
    import torch
    from paper_1805_09246_b300 import sse, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = init_ranks(world)
    R = args.routers
    prefill, distinct = min(args.prefill, 4), max(1, min(args.distinct, 8))
    tr = synth.Traffic(synth.edge_routers(seed=rank, n_slices=prefill + distinct, n_routers=R))
    slices = []
    for t in range(prefill + distinct):
        slices.append([torch.from_numpy(tr.slice(r, t).view(np.int32)).to(dev) for r in range(R)])
    torch.cuda.synchronize()
    # 16 routers carry about 4x the core-link aggregate: the RSRA grows 4x (q = 22) so that
    # noise keeps hot SREs rare; SLEA as in the core-link configuration
    params = sse.Params(q=args.edge_q, q2=16, eta2=4096, k=8, seed=0)
    batch = sse.Batch(params, R, 1024, use_graph=not args.no_graph)
    for t in range(prefill):
        batch.step(inputs=slices[t])

    def step_inputs(s):
        return slices[prefill + s % distinct]

    if args.batch_config is None:
        tuned, tune_ms = batch.tune(None, inputs=step_inputs(0))
    else:  # fixed configuration (profiler runs, where event timing of the candidates is distorted)
        tuned, tune_ms = args.batch_config, []
        batch.configure([1 << 18, 1 << 20, 1 << 22][tuned // 3], [2, 4, 8][tuned % 3])
    for w in range(args.warmup):
        batch.step(inputs=step_inputs(w))
    pairs_per_step = [sum(x.numel() // 2 for x in step_inputs(args.warmup + s)) for s in range(args.steps)]
    launches0 = batch.kernel_launches
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.ExternalStream(batch.stream_ptr)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    barrier(pg)
    torch.cuda.synchronize()
    # each step is enqueued before the previous step's report is read, so the device runs
    # steps back to back (sse_batch_step_async / sse_batch_step_wait)
    e0.record(stream)
    batch.step_async(inputs=step_inputs(args.warmup))
    for s in range(args.steps):
        t0 = time.perf_counter()
        if s + 1 < args.steps:
            batch.step_async(inputs=step_inputs(args.warmup + s + 1))
        batch.step_wait()
        step_ms.append((time.perf_counter() - t0) * 1e3)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    elapsed = max_over_ranks(pg, e0.elapsed_time(e1) / 1e3, dev)
    launches = batch.kernel_launches - launches0
    gstats = batch.global_estimator().stats()
    total = sum(pairs_per_step)
    total_all = sum_over_ranks(pg, float(total), dev)  # every rank scans its own routers' traces
    if pg is not None:
        pg.destroy_process_group()
    if rank != 0:
        return
    srt = sorted(step_ms)
    print(json.dumps({
        "metric": "Gpackets/s, 16-router batch step (persistent update + merge + global close)",
        "value": round(total_all / elapsed / 1e9, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"edge_routers: {R} routers, loads log-uniform 2^20..2^25 pairs per router and "
                               f"slice, super points split over 1-8 routers; estimator q={params.q}, SLEA 5 x 2^16 "
                               "x 4096, k=8, theta=1024; global detection on the merged estimator",
                   "pairs_per_step_mean": int(total / args.steps), "graph": not args.no_graph,
                   "pipelined": "each step enqueued before the previous report is read",
                   "tuned_config": tuned, "tune_ms": [round(x, 4) for x in tune_ms],
                   "l2": "inputs larger than L2"},
        "step_ms_p50": round(srt[len(srt) // 2], 4), "step_ms_p99": round(srt[min(len(srt) - 1, int(0.99 * len(srt)))], 4),
        "global_last_slice": {"hot_sre_per_row": gstats["hot"], "join_pairs": gstats["join_pairs"],
                              "candidates": gstats["n_candidates"], "super": gstats["n_super"]},
        "gpu_launches": int(launches), "clocks": clk,
    }), flush=True)


SERVE_ROUTERS = 32
SERVE_OFFERED = 2e9  # pairs/s offered by all routers together
SERVE_SLICE_PAIRS = 1 << 26  # a slice boundary every 2^26 offered pairs


def serve(rank: int, seconds: float, paced: bool, pool_pairs: int | None = None, warm: int = 200) -> dict:
    """The serving configuration: 32 routers send batches of 64K-4M pairs (log-uniform) with
    Poisson arrivals offering 2e9 pairs/s in aggregate; a slice boundary every 2^26 offered
    pairs (33.6 ms of virtual time), window k = 16, estimator memory budget 40 GB; requests
    are page-locked host memory. The first `warm` requests are submitted at once (untimed);
    the rest at once too, or with `paced`, each at its arrival time on the wall clock (the
    offered load). Returns the pairs and wall time of the timed requests and the
    slice-close-to-report latencies of the slices they closed."""
    from paper_1805_09246_b300 import sse
    from paper_1805_09246_b300.requests import poisson_requests

    R = SERVE_ROUTERS
    rs = poisson_requests(R, duration_s=seconds, offered_pps=SERVE_OFFERED, batch_min=1 << 16,
                          batch_max=1 << 22, pool_pairs=pool_pairs, seed=rank, wrap=pool_pairs is None)
    import torch
    pools = [torch.from_numpy(p.view(np.int32)).pin_memory() for p in rs.pools]  # DMA sources
    pinned = [p.numpy().view(np.uint32) for p in pools]
    params = sse.Params(q=22, q2=16, eta2=4096, k=16, seed=0)
    slice_s = SERVE_SLICE_PAIRS / SERVE_OFFERED
    srv = sse.Server(params, n_routers=R, slots=16, slot_pairs=1 << 22, memory_budget=40 << 30,
                     slice_seconds=slice_s)

    def batch(r, start, size):
        pool = pinned[r]
        if start + size <= len(pool):
            return pool[start:start + size]
        return np.take(pool, np.arange(start, start + size), axis=0, mode="wrap")

    n_warm = min(len(rs.requests) // 10, warm)
    for t, r, start, size in rs.requests[:n_warm]:
        srv.submit(r, t, batch(r, start, size))
    timed = rs.requests[n_warm:]
    first_slice = int(timed[0][0] / slice_s) if timed else 0
    total = sum(size for _, _, _, size in timed)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    v0 = timed[0][0] if timed else 0.0
    for t, r, start, size in timed:
        if paced:  # wait for the request's arrival time
            while True:
                ahead = (t - v0) - (time.perf_counter() - t0)
                if ahead <= 0:
                    break
                if ahead > 2e-3:
                    time.sleep(ahead - 1e-3)
        srv.submit(r, t, batch(r, start, size))
    srv.flush()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    reports = srv.poll()
    # slices closed by the timed requests: every slice after the one the first timed request fell in
    lat = sorted(l for rep, l in reports if rep.slice >= first_slice)
    st = srv.stats()
    srv.close()
    del pools
    return {"requests": len(rs.requests), "timed_requests": len(timed), "warm_requests": n_warm,
            "pairs_timed": total, "wall": wall, "virtual": (timed[-1][0] - v0) if timed else 0.0,
            "latencies": lat, "slices_reported": len(reports), "slot_waits": st["slot_waits"], "clocks": clk,
            "slice_s": slice_s}


def run_leg(argv: list[str], timeout: float = 900.0) -> dict:
    """Another workload of this benchmark in a child process on this rank's GPU (the
    distributed environment removed, so that it runs alone); its JSON line, or the error."""
    drop = ("RANK", "WORLD_SIZE", "LOCAL_RANK", "LOCAL_WORLD_SIZE", "GROUP_RANK", "ROLE_RANK", "MASTER_ADDR",
            "MASTER_PORT", "TORCHELASTIC_RUN_ID", "GROUP_WORLD_SIZE", "ROLE_WORLD_SIZE")
    env = {k: v for k, v in os.environ.items() if k not in drop}
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), *argv], capture_output=True, text=True,
                           timeout=timeout, env=env, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout:.0f} s"}
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": f"exit {r.returncode}: {r.stderr.strip().splitlines()[-1] if r.stderr.strip() else ''}"}
    return json.loads(lines[-1])


def pctl(xs, q):
    return round(xs[min(len(xs) - 1, int(q * len(xs)))], 4) if xs else None


def main_serving(args, rank, world, local):
    """Serving (see serve()): throughput and slice-close-to-report p50/p99; with --paced the
    requests arrive at the offered rate, otherwise as fast as the host submits them."""
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = init_ranks(world)
    barrier(pg)
    res = serve(rank, args.serve_seconds, args.paced, pool_pairs=(1 << 22) if args.paced else None)
    wall = max_over_ranks(pg, res["wall"], dev)
    total_all = sum_over_ranks(pg, float(res["pairs_timed"]), dev)  # each rank serves its own request stream
    if pg is not None:
        pg.destroy_process_group()
    if rank != 0:
        return
    n, lat = res["timed_requests"], res["latencies"]
    print(json.dumps({
        "metric": "Gpackets/s served (32 routers, Poisson batches) and slice-close-to-report p50/p99 ms",
        "value": round(total_all / wall / 1e9, 4), "unit": UNIT, "n_gpus": world,
        "steps": n, "warmup": res["warm_requests"], "ms_per_step": round(wall / max(1, n) * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"serving: {SERVE_ROUTERS} routers, batches 64K-4M pairs log-uniform, Poisson arrivals "
                               f"offering {SERVE_OFFERED:.0e} pairs/s, slice every 2^26 offered pairs "
                               f"({res['slice_s']*1e3:.1f} ms virtual), k=16, q=22, SLEA 5 x 2^16 x 4096, budget 40 GB, "
                               "16 staging slots of 2^22",
                   "virtual_seconds": args.serve_seconds, "requests": res["requests"], "pairs_timed": res["pairs_timed"],
                   "paced": args.paced, "step": "one admitted request"},
        "close_ms_p50": pctl(lat, 0.5), "close_ms_p99": pctl(lat, 0.99), "close_samples": len(lat),
        "offered_gpkts": SERVE_OFFERED / 1e9,
        "slices_reported": res["slices_reported"], "slot_waits": res["slot_waits"],
        "e2e": {"value": round(total_all / wall / 1e9, 4), "unit": UNIT,
                "h2d_bytes_per_step": int(res["pairs_timed"] * PAIR_BYTES / max(1, n)),
                "d2h_bytes_per_step": 0},
        "clocks": res["clocks"],
    }), flush=True)


def main_learned(args, rank, world, local):
    """Learned correction, MLP 18->64->64->1 (BF16 weights, FP32 sums): 1e6 training hosts
    from GPU episodes (k = 16, core-link estimator shapes, exact window cardinality
    log-uniform in [1e2, 1e6]), trained with the library's forward/backward/Adam kernels;
    1e5 held-out hosts scored through sse_query_learned against linear counting. One step =
    one training epoch over the hosts whose union SLE is at least 90% full; the warm-up
    epochs are the first epochs of the same training run."""
    import torch
    from paper_1805_09246_b300 import learn, sse
    from paper_1805_09246_b300.synth import episodes as ep

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = init_ranks(world)
    cfg = ep.EpisodeConfig()
    params = learn.learned_params(cfg.k, seed=rank)
    t0 = time.perf_counter()
    tr = learn.episodes(params, cfg, args.learn_train, routers=64, seed=rank)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    tt = learn.targets(tr)
    act = learn.active_cells(tr.x, params.k)
    rows = np.nonzero(act >= 0.9 * params.eta2)[0]
    mlp = sse.MLP(params.k + 2, hidden=64, max_batch=1 << 16, seed=rank + 1)
    rng = np.random.default_rng(rank + 2)
    batch, lr = 512, 1e-3
    learn.train(mlp, tr.x, tt, epochs=args.warmup, batch=batch, lr=lr, rows=rows, rng=rng)
    launches0 = mlp.kernel_launches
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(pg)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    e0.record(stream)
    losses = learn.train(mlp, tr.x, tt, epochs=args.steps, batch=batch, lr=lr, rows=rows, rng=rng,
                         first_epoch=args.warmup)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    wall = max_over_ranks(pg, time.perf_counter() - w0, dev)
    clk = clocks.stop()
    launches = mlp.kernel_launches - launches0
    elapsed = max_over_ranks(pg, e0.elapsed_time(e1) / 1e3, dev)
    samples_all = sum_over_ranks(pg, float(len(rows) * args.steps), dev)  # each rank trains its own network
    y = mlp.forward(tr.x).cpu().numpy()
    gate = learn.choose_gate(tr.lc.cpu().numpy(), y, tr.exact, act, params.eta2)
    mlp.set_gate(gate)
    mlp.set_feature_max(learn.feature_max(tr.x))
    te = learn.episodes(params, cfg, args.learn_test, routers=64, seed=rank + 1000, mlp=mlp)
    lc = te.lc.cpu().numpy().astype(np.float64)
    le = te.learned.cpu().numpy().astype(np.float64)
    ex = te.exact
    gated = learn.active_cells(te.x, params.k) >= gate
    rel = lambda e, m: float(np.median(np.abs(e[m] - ex[m]) / ex[m])) if m.any() else None
    every = np.ones(len(ex), bool)
    if pg is not None:
        pg.destroy_process_group()
    if rank != 0:
        return
    samples = len(rows) * args.steps
    flops_per_sample = 3 * 2 * (18 * 64 + 64 * 64 + 64)  # forward, input-side backward, weight gradients
    print(json.dumps({
        "metric": "learned correction: training samples/s (own forward/backward/Adam kernels); median relative "
                  "error learned vs linear counting on held-out hosts",
        "value": round(samples_all / elapsed, 1), "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights, f32 accumulate", "data": "synthetic",
        "config": {"workload": f"learned: MLP 18->64->64->1, {args.learn_train} training hosts from GPU episodes "
                               f"({cfg.hosts} hosts + {cfg.noise_pairs} noise pairs/slice per episode, 64 episodes per "
                               f"batch, slices 0..{cfg.query_slice}, k={cfg.k}), q=20, SLEA 5 x 2^16 x 4096; "
                               f"{args.learn_test} held-out hosts", "train_rows": int(len(rows)),
                   "minibatch": batch, "step": "one training epoch", "gate_min_active": int(gate)},
        "median_rel_err_learned": round(rel(le, every), 5), "median_rel_err_lc": round(rel(lc, every), 5),
        "median_rel_err_learned_above_gate": rel(le, gated), "median_rel_err_lc_above_gate": rel(lc, gated),
        "hosts_above_gate": round(float(gated.mean()), 4),
        "p90_rel_err_learned": round(float(np.quantile(np.abs(le - ex) / ex, 0.9)), 4),
        "p90_rel_err_lc": round(float(np.quantile(np.abs(lc - ex) / ex, 0.9)), 4),
        "final_loss": round(losses[-1], 5),
        "episodes": {"train_s": round(gen_s, 2), "scan_s": round(tr.seconds["scan"], 2),
                     "query_s": round(tr.seconds["query"], 3),
                     "learned_query_hosts_per_s": round(args.learn_test / te.seconds["query"], 1)},
        "roofline": {"bound": "alu", "kernel": "MLP training (backward + weight gradients)",
                     "achieved": round(samples * flops_per_sample / elapsed / 1e12, 4),
                     "peak": round(148 * 128 * 2 * 2.032e9 / 1e12, 1), "unit": "TFLOP/s",
                     "frac": round(samples * flops_per_sample / elapsed / (148 * 128 * 2 * 2.032e9), 6),
                     "traffic": None, "peak_source": "FP32 FMA: 148 SMs x 128 lanes x 2 x 2.032 GHz (nominal)"},
        "e2e": {"value": round(samples_all / wall, 1), "unit": "samples/s",
                "h2d_bytes_per_step": int(4 * len(rows)), "d2h_bytes_per_step": 4},
        "gpu_launches": int(launches), "clocks": clk,
    }), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "edge_routers":
        main_edge_routers(args, rank, world, local)
        return
    if args.workload == "serving":
        main_serving(args, rank, world, local)
        return
    if args.workload == "learned":
        main_learned(args, rank, world, local)
        return
    import torch
    from paper_1805_09246_b300 import sse

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = init_ranks(world)

    tr = make_traffic(rank)
    # paper_params: the same core-link traffic through the estimator of the paper's
    # experiments (q = q' = 17, eta' = 2^14, 16-bit stamps, window k = 300 slices)
    paper = args.workload == "paper_params"
    params = sse.paper_params(k=300) if paper else sse.core_link_params(k=8, seed=0)
    # the paper's estimator is sized for its trace (1-second slices of an OC192 link, about
    # 2^21 pairs): its slices are the first 2^21 pairs of each core-link slice
    n_slice = (1 << 21) if paper else PAIRS_PER_SLICE
    stream = torch.cuda.Stream()  # the estimator's own (non-blocking) stream
    est = sse.Estimator(params, stream=stream)
    if args.mode:
        est.set_update_mode(args.mode)
    if args.no_graph:  # the close's kernels launched one by one (per-kernel profiles)
        est.close_use_graph(False)

    # inputs: up to PREFILL generated slices for the window, then DISTINCT slices the steps
    # cycle through; a longer prefill (--prefill, e.g. to fill the paper's 300-slice window
    # for a profile) repeats the step slices after the first PREFILL, as the timed steps do
    distinct = max(1, args.distinct)
    prefill = min(args.prefill, PREFILL)
    host = [np.ascontiguousarray(tr.slice(0, t)[:n_slice]) for t in range(prefill + distinct)]
    dev_slices = [torch.from_numpy(h.view(np.int32)).to(dev) for h in host]
    torch.cuda.synchronize()

    def step_input(s):
        return dev_slices[prefill + s % distinct]

    for t in range(args.prefill):
        est.update(dev_slices[t] if t < prefill else step_input(t))
        est.close_slice()

    # autotune the update on the next slice's pairs (idempotent within the slice), untimed;
    # --update-variant fixes the variant instead (profiler runs, where event timing of the
    # candidates is distorted)
    if args.update_variant is None:
        tuned, tune_ms = est.autotune_update(step_input(0), reps=3)
    else:
        tuned, tune_ms = args.update_variant, []
        est.set_update_variant(tuned)

    for w in range(args.warmup):
        est.update(step_input(w))
        est.close_slice()

    # ---- timed region: K steps, inputs resident in HBM. Each step scans one slice and closes
    # it; the next slice's update is enqueued behind the close before its report is awaited,
    # so the device runs update, close, update, ... back to back.
    ev_start, ev_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    upd_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in [(ev_start, ev_end)] + upd_ev:  # created at their first record: outside the timed region
        a.record(stream)
        b.record(stream)
    launches0 = est.kernel_launches
    n_super = n_cand = 0
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(pg)
    torch.cuda.synchronize()
    ev_start.record(stream)
    upd_ev[0][0].record(stream)
    est.update(step_input(args.warmup))
    upd_ev[0][1].record(stream)
    for s in range(args.steps):
        if args.no_graph:  # kernels launched one by one: the close is synchronous
            rep = est.close_slice()
        else:
            est.close_slice_async()
        if s + 1 < args.steps:
            a, b = upd_ev[s + 1]
            a.record(stream)
            est.update(step_input(args.warmup + s + 1))
            b.record(stream)
        if not args.no_graph:
            rep = est.close_slice_wait()
        n_super += rep.n_super
        n_cand += rep.n_candidates
    ev_end.record(stream)
    last_rep = rep
    torch.cuda.synchronize()
    barrier(pg)
    clk = clocks.stop()
    launches = est.kernel_launches - launches0
    slice_stats = est.stats()
    elapsed_s = max_over_ranks(pg, ev_start.elapsed_time(ev_end) / 1e3, dev)
    upd_ms = sum(a.elapsed_time(b) for a, b in upd_ev) / args.steps

    # ---- slice-close latency (after the timed region): the slice boundary is a synchronised
    # stream; latency = sse_close_slice until the report is in host memory. It falls over the
    # first few hundred such closes after the pipelined run (measured: p50 from ~0.1 ms to
    # ~0.06 ms), so --latency-warmup closes of the same form come first, untimed.
    # The device time of a close (its graph alone: an event before the asynchronous launch
    # and one right behind it) is sampled on the same closes' form separately.
    n_lat = args.latency_samples
    n_dev = min(n_lat, 100)
    # the events are created (and first recorded) before the samples: a CUDA event is created
    # lazily at its first record, which would otherwise fall inside the measured interval
    lat_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_dev)]
    for a, b in lat_ev:
        a.record(stream)
        b.record(stream)
    s_in = args.warmup + args.steps
    for s in range(args.latency_warmup):
        est.update(step_input(s_in))
        s_in += 1
        stream.synchronize()
        est.close_slice()
    close_ms, close_cand = [], []
    for s in range(n_lat):
        est.update(step_input(s_in))
        s_in += 1
        stream.synchronize()
        t0 = time.perf_counter()
        r = est.close_slice()
        close_ms.append((time.perf_counter() - t0) * 1e3)
        close_cand.append(r.n_candidates)
    for s in range(n_dev):
        est.update(step_input(s_in))
        s_in += 1
        stream.synchronize()
        a, b = lat_ev[s]
        a.record(stream)
        if args.no_graph:  # kernels launched one by one: the close is synchronous
            est.close_slice()
            b.record(stream)
        else:
            est.close_slice_async()
            b.record(stream)
            est.close_slice_wait()
    torch.cuda.synchronize()
    close_dev = lat_ev
    total_pairs = args.steps * n_slice * world
    value = total_pairs / elapsed_s / 1e9

    # ---- end to end through the public API: pinned host slices -> report on the host
    e2e = None
    if not args.no_e2e:
        k_e2e = min(args.steps, 40)
        pinned = [torch.from_numpy(host[prefill + s % distinct].view(np.int32)).pin_memory()
                  for s in range(min(k_e2e, distinct))]
        e2e_est = sse.Estimator(params)
        if args.mode:
            e2e_est.set_update_mode(args.mode)
        e2e_est.set_update_variant(tuned)
        for t in range(prefill):
            e2e_est.update(dev_slices[t])
            e2e_est.close_slice()
        e2e_est.update_host(pinned[0])
        e2e_est.close_slice()
        d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # each slice's host-to-device copies run while the previous slice's close is on the GPU
        e2e_est.update_host(pinned[0])
        for s in range(k_e2e):
            e2e_est.close_slice_async()
            if s + 1 < k_e2e:
                e2e_est.update_host(pinned[(s + 1) % len(pinned)])
            r = e2e_est.close_slice_wait()
            d2h += 64 + r.n_candidates * 9  # report header + hosts/est/flags
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": round(k_e2e * n_slice * world / dt / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": n_slice * PAIR_BYTES, "d2h_bytes_per_step": int(d2h / k_e2e),
               "steps": k_e2e}
        del e2e_est, pinned

    # ---- roofs of the update's other units, measured on this device (sse_microbench)
    mb = sse.microbench(stream)
    torch.cuda.synchronize()
    upd_pps = n_slice / (upd_ms / 1e3)
    stamps_per_pair = params.r2 + params.r * 2.0 ** -est.derived["tau"]  # r' + r 2^-tau cells per pair
    l2_roof_pps = mb["l2_random_byte_stores_per_s"] / stamps_per_pair
    # the tiled design per pair: one shared-memory atomic per SLEA row, and every row's CTA
    # reads the 8-byte pair through the SM's load pipe (from L2 after the first)
    lsu_s_per_pair = params.r2 / mb["smem_random_atomics_per_s"] + params.r2 * PAIR_BYTES / mb["l2_stream_load_bytes_per_s"]

    hbm_peak, peak_kind = peaks()
    achieved = n_slice * PAIR_BYTES / (upd_ms / 1e3) / 1e9
    # DRAM bytes (read + write) of one k_update_tiled<8, 0, 1, 0> launch on this slice, from an ncu
    # capture of this kernel version (dram__bytes_read.sum + dram__bytes_write.sum); only
    # reported when that variant is the one timed
    traffic = TILED8_DRAM_BYTES if tuned == 3 and not paper else None
    roofline = {"bound": "hbm", "kernel": "sse update (k_update_tiled + k_apply_bits)", "achieved": round(achieved, 2),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": n_slice * PAIR_BYTES,
                "binding_unit": "SM L1/shared-memory pipe (ncu l1tex throughput on k_update_tiled)",
                "l2_stamp_roof_gpkts": round(l2_roof_pps / 1e9, 3),
                "l2_sector_frac": round(upd_pps / l2_roof_pps, 4),
                "l2_sector_note": (f"update rate / (measured random one-byte L2 stores/s / {stamps_per_pair:.3f} stamps "
                                   "per pair): the roof of stamping every cell in L2; above 1 the tiled design beats it"),
                "l1tex_roof_gpkts": round(1.0 / lsu_s_per_pair / 1e9, 3),
                "l1tex_frac": round(upd_pps * lsu_s_per_pair, 4),
                "l1tex_note": (f"update rate x ({params.r2} / measured random shared-memory atomics/s + "
                               f"{params.r2} x 8 B / measured L2 streaming-load B/s): share of the SM load pipe's "
                               "time the tiled design's algorithmic work takes"),
                "update_vs_skeleton": round(upd_pps / mb["tiled_skeleton_pairs_per_s"], 4),
                "skeleton_note": ("update rate / the rate of the tiled update's skeleton (same grid, loads and "
                                  "one shared atomic per pair and row, no hashing or sampling): the share of "
                                  "this design's measured floor that the update reaches"),
                "microbench": {k: (round(v / 1e9, 2) if isinstance(v, float) else v) for k, v in mb.items()},
                "microbench_unit": "G per second (stores, atomics) and GB/s (loads)"}

    # ---- paced serving leg: the serving configuration at its offered load, for the
    # slice-close-to-report latency of config E (each rank serves its own request stream)
    serving = None
    if args.serve_slices > 0 and not paper:
        del dev_slices
        torch.cuda.empty_cache()
        secs = (args.serve_slices + 2) * SERVE_SLICE_PAIRS / SERVE_OFFERED
        res = serve(rank, secs, paced=True, pool_pairs=1 << 22, warm=50)
        lat = res["latencies"]
        serving = {"serving_close_ms_p50": pctl(lat, 0.5), "serving_close_ms_p99": pctl(lat, 0.99),
                   "serving_close_samples": len(lat),
                   "serving_served_gpkts": round(res["pairs_timed"] / res["wall"] / 1e9, 4),
                   "serving_offered_gpkts": SERVE_OFFERED / 1e9,
                   "serving_config": {"routers": SERVE_ROUTERS, "paced": True, "virtual_s": round(res["virtual"], 3),
                                      "wall_s": round(res["wall"], 3), "requests": res["timed_requests"],
                                      "slot_waits": res["slot_waits"], "clocks": res["clocks"],
                                      "workload": "serving: 32 routers, batches 64K-4M pairs, Poisson arrivals paced at "
                                                  "2e9 pairs/s, slice every 2^26 offered pairs, k=16, q=22, "
                                                  "SLEA 5 x 2^16 x 4096; latency = slice boundary to report on the host"}}

    if rank != 0:
        return
    # ---- the other workloads of the configuration, each in a child process on this GPU once
    # the timed work above is done: 16 batched edge routers, and the learned correction
    legs = {}
    if not args.no_legs and not paper:
        torch.cuda.synchronize()
        e = run_leg(["--workload", "edge_routers", "--steps", "30", "--warmup", "3"])
        legs["edge_routers"] = e if "error" in e else {
            "value": e["value"], "unit": e["unit"], "ms_per_step": e["ms_per_step"], "step_ms_p50": e["step_ms_p50"],
            "step_ms_p99": e["step_ms_p99"], "gpu_launches": e["gpu_launches"], "clocks": e["clocks"],
            "workload": e["config"]["workload"], "pairs_per_step_mean": e["config"]["pairs_per_step_mean"]}
        l = run_leg(["--workload", "learned", "--steps", "27", "--warmup", "3"])
        legs["learned"] = l if "error" in l else {
            "train_samples_per_s": l["value"], "median_rel_err_learned": l["median_rel_err_learned"],
            "median_rel_err_lc": l["median_rel_err_lc"],
            "median_rel_err_learned_above_gate": l["median_rel_err_learned_above_gate"],
            "median_rel_err_lc_above_gate": l["median_rel_err_lc_above_gate"],
            "hosts_above_gate": l["hosts_above_gate"], "p90_rel_err_learned": l["p90_rel_err_learned"],
            "p90_rel_err_lc": l["p90_rel_err_lc"], "gpu_launches": l["gpu_launches"], "clocks": l["clocks"],
            "workload": l["config"]["workload"]}
    # the oracle on the host's cores: at one rank only (with more ranks the host runs their work)
    cpu = None if args.no_cpu or paper or world > 1 else cpu_baseline(host)
    close_sorted = sorted(close_ms)
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed_s / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16" if paper else "u8", "data": "synthetic",
        "config": {"workload": ("paper_params: core-link traffic cut to 2^21 pairs/slice (16M-host Zipf(1.05)); the paper's "
                                "estimator q=17, r=5, delta=5, SLEA r'=5 x (2^17 SLEs, eta'=2^14, delta'=16), "
                                "16-bit stamps, k=300, theta=1024")
                               if paper else CORE_LINK_WORKLOAD,
                   "pairs_per_step": n_slice,
                   "l2": ("16 distinct 16 MiB slices cycled (256 MiB): a step's input was evicted since its last use"
                          if paper else "inputs larger than L2 (256 MiB per step)"),
                   "prefill_slices": args.prefill,
                   "update_mode": args.mode, "update_variant": tuned,
                   "variant_ms": [round(t, 4) for t in tune_ms]},
        "update_gpkts": round(n_slice / (upd_ms / 1e3) / 1e9, 3),
        "update_ms": round(upd_ms, 4),
        "close_ms_p50": round(close_sorted[len(close_sorted) // 2], 4),
        "close_ms_p99": round(close_sorted[min(len(close_sorted) - 1, int(0.99 * len(close_sorted)))], 4),
        "close_event_ms_p50": round(sorted(a.elapsed_time(b) for a, b in close_dev)[len(close_dev) // 2], 4),
        "close_samples": len(close_ms), "close_warmup_samples": args.latency_warmup,
        "close_event_samples": len(close_dev),
        "close_candidates_mean": round(float(np.mean(close_cand)), 1) if close_cand else None,
        "candidates_per_slice": round(n_cand / args.steps, 1), "super_per_slice": round(n_super / args.steps, 1),
        "last_slice": {"hot_sre_per_row": slice_stats["hot"], "join_pairs": slice_stats["join_pairs"],
                       "sf": [round(c / est.derived["row_len2"], 4) for c in slice_stats["active2"]],
                       # candidates whose corrected weight hit Eq. 12's saturation clamp
                       "saturated": int(np.count_nonzero(last_rep.flags & sse.FLAG_SATURATED)),
                       "candidates": int(last_rep.n_candidates)},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk,
    }
    if serving:
        out.update(serving)
    out.update(legs)
    print(json.dumps(out), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
