"""The serving loop: concurrent routers with staged admission produce, slice by slice,
exactly the reports of a sequential run of the same requests through the single-router
API and of the CPU oracle's routers merged per slice; a router's results are the same
alone and in the mix; a router that stops sending mid-run leaves the others' reports equal
to the oracle's without its late pairs."""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300.requests import poisson_requests
from tests import helpers
from tests.test_gpu_parity import compare_report, compare_state, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sse():
    from paper_1805_09246_b300 import sse as mod
    return mod


def stream(seed=41, routers=6):
    return poisson_requests(routers, duration_s=0.06, offered_pps=2e7, batch_min=500, batch_max=40000,
                            pool_pairs=1 << 17, seed=seed)


SLICE_S = 0.008


def sequential_reports(p, rs, n_routers):
    """Same requests, same slices, one call at a time through sse_update / sse_merge /
    sse_close_slice / sse_advance."""
    S = sse()
    routers = [S.Estimator(p) for _ in range(n_routers)]
    glob = S.Estimator(p)
    reports, cur = [], 0

    def close():
        glob.merge(routers)
        reports.append(glob.close_slice())
        for e in routers:
            e.advance()

    for t, r, start, size in rs.requests:
        while int(t / SLICE_S) > cur:
            close()
            cur += 1
        routers[r].update(helpers.to_device(rs.pairs(r, start, size)))
    close()
    return reports, routers


def oracle_reports(p, rs, n_routers, keep=lambda t, r: True):
    """The oracle's view of the same requests: each admitted batch is scanned into its
    router's oracle in the slice floor(t / SLICE_S) of its arrival time; at each slice
    boundary the global oracle merges the routers (Algorithms 2 and 7: the smallest distance
    per cell) and detects (Algorithms 4, 5 and 8), then every oracle advances."""
    routers = [oracle.Oracle(oracle_params(p)) for _ in range(n_routers)]
    og = oracle.Oracle(oracle_params(p))
    dets, cur = [], 0

    def close():
        og.merge(routers)
        dets.append(og.detect())
        for o in routers:
            o.advance()
        og.advance()

    for t, r, start, size in rs.requests:
        while int(t / SLICE_S) > cur:
            close()
            cur += 1
        if keep(t, r):
            routers[r].scan(rs.pairs(r, start, size))
    close()
    return dets, routers


@pytest.mark.parametrize("q", [14, 17])  # q = 17, delta = 5: the global close joins from the top row down
def test_server_reports_match_oracle(q):
    """Every report of the serving loop (hosts and flags exact, estimates within 1e-6
    relative) against the merged oracle routers fed the same admitted batches."""
    S = sse()
    p = S.Params(q=q, seed=44)
    rs = stream(seed=44)
    srv = S.Server(p, n_routers=6, slots=3, slot_pairs=8192, memory_budget=1 << 32, slice_seconds=SLICE_S)
    for t, r, start, size in rs.requests:
        srv.submit(r, t, rs.pairs(r, start, size))
    srv.flush()
    got = srv.poll()
    dets, orcs = oracle_reports(p, rs, 6)
    assert len(got) == len(dets) >= 5
    for (rep, _), det in zip(got, dets):
        compare_report(rep, det)
    assert sum(rep.n_super for rep, _ in got) > 0
    for r in range(6):
        compare_state(srv.router(r), orcs[r], p, srv.router(r).slice)


def test_router_drop_out_mid_run():
    """Router 2 stops sending at 40 % of the run (a host-side drop-out: its requests are
    never submitted). The server keeps closing slices; its reports equal the oracle's
    without router 2's late pairs, and router 2's cells expire out of the window, so its
    state ends equal to an oracle router that saw only its early pairs."""
    S = sse()
    p = S.Params(seed=45)
    rs = stream(seed=45)
    t_stop = 0.4 * rs.requests[-1][0]
    keep = lambda t, r: not (r == 2 and t >= t_stop)  # noqa: E731
    srv = S.Server(p, n_routers=6, slots=3, slot_pairs=8192, memory_budget=1 << 32, slice_seconds=SLICE_S)
    dropped = 0
    for t, r, start, size in rs.requests:
        if keep(t, r):
            srv.submit(r, t, rs.pairs(r, start, size))
        else:
            dropped += 1
    assert dropped > 0
    srv.flush()
    got = srv.poll()
    dets, orcs = oracle_reports(p, rs, 6, keep)
    assert len(got) == len(dets) >= 5
    for (rep, _), det in zip(got, dets):
        compare_report(rep, det)
    for r in range(6):
        compare_state(srv.router(r), orcs[r], p, srv.router(r).slice)
    # k slices after router 2's last pairs, the merges have reset every one of its cells
    last = max(int(t / SLICE_S) for t, r, _, _ in rs.requests if r == 2 and keep(t, r))
    assert len(got) - 1 - last >= p.k
    sre, sle = srv.router(2).read_stamps()
    assert not sre.any() and not sle.any()


def test_server_matches_sequential_api():
    S = sse()
    p = S.Params(seed=41)
    rs = stream()
    srv = S.Server(p, n_routers=6, slots=3, slot_pairs=8192, memory_budget=1 << 32, slice_seconds=SLICE_S)
    for t, r, start, size in rs.requests:
        srv.submit(r, t, rs.pairs(r, start, size))
    srv.flush()
    got = srv.poll()
    want, routers = sequential_reports(p, rs, 6)
    assert len(got) == len(want) >= 5
    assert [rep.slice for rep, _ in got] == list(range(len(want)))
    for (rep, lat), ref in zip(got, want):
        assert np.array_equal(rep.hosts, ref.hosts) and np.array_equal(rep.flags, ref.flags)
        assert np.array_equal(rep.est, ref.est)
        assert lat > 0
    assert sum(rep.n_super for rep, _ in got) > 0
    st = srv.stats()
    assert st["requests"] == len(rs.requests) and st["slices_closed"] == len(want)
    assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
    for r in range(6):
        for x, y in zip(srv.router(r).read_stamps(), routers[r].read_stamps()):
            assert np.array_equal(x, y)


def test_router_results_same_alone_and_in_the_mix():
    S = sse()
    p = S.Params(seed=42)
    rs = stream(seed=42)
    mix = S.Server(p, n_routers=6, slots=4, slot_pairs=8192, memory_budget=1 << 32, slice_seconds=SLICE_S)
    alone = S.Server(p, n_routers=6, slots=4, slot_pairs=8192, memory_budget=1 << 32, slice_seconds=SLICE_S)
    for t, r, start, size in rs.requests:
        mix.submit(r, t, rs.pairs(r, start, size))
        if r == 0:
            alone.submit(0, t, rs.pairs(0, start, size))
    alone.submit(0, rs.requests[-1][0], np.zeros((0, 2), np.uint32))  # same final slice
    mix.flush()
    alone.flush()
    for x, y in zip(mix.router(0).read_stamps(), alone.router(0).read_stamps()):
        assert np.array_equal(x, y)
    hosts = np.unique(rs.pools[0][:2000, 0])
    e_mix, f_mix = mix.router(0).query(helpers.to_device(hosts))
    e_alone, f_alone = alone.router(0).query(helpers.to_device(hosts))
    assert torch.equal(e_mix, e_alone) and torch.equal(f_mix, f_alone)


def test_admission_budget_and_late_requests():
    S = sse()
    p = S.Params(seed=43)
    with pytest.raises(S.SSEError):
        S.Server(p, n_routers=8, slots=2, slot_pairs=1 << 20, memory_budget=1 << 20)
    srv = S.Server(p, n_routers=2, slots=2, slot_pairs=4096, memory_budget=1 << 32, slice_seconds=0.01)
    srv.submit(0, 0.025, np.zeros((10, 2), np.uint32))
    with pytest.raises(S.SSEError):
        srv.submit(1, 0.005, np.zeros((10, 2), np.uint32))  # slice 0 is already closed
    srv.flush()
    assert [rep.slice for rep, _ in srv.poll()] == [0, 1, 2]
