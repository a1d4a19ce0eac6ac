"""The multi-rank plumbing of bench.py on the CPU: two gloo ranks (127.0.0.1) meet at the
barrier, the job's time is the slowest rank's (MAX) and its work the sum over ranks; each
rank scans its own router's trace; under a multi-rank launch only rank 0 runs and prints
the reference arm. No GPU is used."""
import contextlib
import io
import os
import socket
import sys

import pytest

from tests.conftest import ROOT

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, _ = bench.dist_env()
    pg = bench.init_ranks(w)
    bench.barrier(pg)
    slowest = bench.max_over_ranks(pg, 1.5 + r, "cpu")
    work = bench.sum_over_ranks(pg, 10.0 * (r + 1), "cpu")
    first_pair = bench.make_traffic(r).slice(0, 0)[:4].tolist()
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    if r != 0:  # rank 0's oracle run is the single-rank path, timed elsewhere
        with contextlib.redirect_stdout(buf):
            bench.run_reference(args, r, w)
    bench.barrier(pg)
    pg.destroy_process_group()
    out.put((r, w, slowest, work, first_pair, buf.getvalue()))


def test_two_gloo_ranks_max_time_summed_work_and_rank_traces():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    for r, w, slowest, work, _, printed in results:
        assert w == world
        assert slowest == 2.5  # the larger of 1.5 and 2.5
        assert work == 30.0    # 10 + 20
    assert results[0][4] != results[1][4]  # each rank scans its own trace
    assert results[1][5] == ""             # rank 1 of the reference arm prints nothing


def test_cpu_baseline_runs_until_its_time_and_slice_minimums():
    """The CPU baseline's threads scan slices in turn (from the first again when the given
    ones run out) until both the minimum time and the minimum slice count (over all
    threads) are reached; `cores` is the number of threads that ran."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    slices = [rng.integers(0, 2**32, (4096, 2), dtype=np.uint64).astype(np.uint32) for _ in range(2)]
    r = bench.cpu_baseline(slices, min_seconds=0.0, min_slices=5, max_slices=64, threads=1)
    assert "over 5 full core-link slices in all" in r["sample"] and r["cores"] == 1 and r["value"] > 0
    r = bench.cpu_baseline(slices, min_seconds=0.3, min_slices=1, max_slices=64, threads=2)
    assert r["cores"] == 2 and r["sample"].startswith("2 oracle estimators")
    n = int(r["sample"].split(" over ")[1].split()[0])
    assert n >= 1 and float(r["sample"].split("pairs, ")[1].split(" s)")[0]) >= 0.3 or n == 2 * 64
    r = bench.cpu_baseline(slices, min_seconds=0.0, min_slices=7, max_slices=2, threads=3)
    assert r["cores"] == 3 and int(r["sample"].split(" over ")[1].split()[0]) == 6  # 3 threads x at most 2


def test_oracle_threads_bounded_by_host_cores_and_cap():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.oracle_threads(None) == min(bench.host_cores(), bench.CPU_THREADS_MAX)
    assert bench.oracle_threads(3) == 3 and bench.oracle_threads(10**6) == bench.CPU_THREADS_MAX


def test_reference_arm_line_carries_the_contract_keys(monkeypatch, capsys):
    """The reference arm (the oracle on host threads) prints one JSON line with the keys the
    benchmark contract asks of it; a small trace stands in for the core-link slices."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    from paper_1805_09246_b300 import synth
    monkeypatch.setattr(bench, "make_traffic",
                        lambda rank: synth.Traffic(synth.TrafficConfig(seed=rank, n_slices=16)))
    args = bench.parse(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    bench.run_reference(args, 0, 1, threads=2)
    lines = [x for x in capsys.readouterr().out.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 2
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.CORE_LINK_WORKLOAD
