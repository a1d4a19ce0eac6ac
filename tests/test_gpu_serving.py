"""The serving loop: concurrent routers with staged admission produce, slice by slice,
exactly the reports of a sequential run of the same requests through the single-router
API; a router's results are the same alone and in the mix."""
import numpy as np
import pytest

from paper_1805_09246_b300.requests import poisson_requests
from tests import helpers

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
