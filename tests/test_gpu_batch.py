"""Multi-router batches: one persistent update launch per slice, merge into the global
estimator, detection, CUDA-graph replay — checked against separate estimators driven
through the single-router API and against the oracle's routers and merge."""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers
from tests.test_gpu_parity import compare_report, compare_state, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sse():
    from paper_1805_09246_b300 import sse as mod
    return mod


def router_traffic(n_routers, n_slices, seed, load_min=1 << 12, load_max=1 << 17):
    cfg = synth.TrafficConfig(seed=seed, n_slices=n_slices, n_routers=n_routers, load_min=load_min,
                              load_max=load_max, n_sources=20_000, n_planted=12, planted_min=1500,
                              planted_max=6000, group_min=1, group_max=min(3, n_routers))
    tr = synth.Traffic(cfg)
    return [[tr.slice(r, t) for r in range(n_routers)] for t in range(n_slices)]


def run_reference(p, slices):
    """The same work through the single-router API: routers, global merge, global close."""
    S = sse()
    routers = [S.Estimator(p) for _ in slices[0]]
    glob = S.Estimator(p)
    reports = []
    for t, per_router in enumerate(slices):
        for e, pairs in zip(routers, per_router):
            if len(pairs):
                e.update(helpers.to_device(pairs))
        glob.merge(routers)
        reports.append(glob.close_slice())
        for e in routers:
            e.advance()
    return routers, glob, reports


@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("q", [14, 17])  # q = 17, delta = 5: the global close joins from the top row down
def test_batch_matches_single_router_api_and_oracle(graph, q):
    S = sse()
    p = S.Params(q=q, seed=31)
    R, T = 5, 6
    slices = router_traffic(R, T, seed=31)
    cap = max(len(x) for s in slices for x in s)
    batch = S.Batch(p, R, cap, use_graph=graph)
    _, ref_glob, ref_reports = run_reference(p, slices)
    orcs = [oracle.Oracle(oracle_params(p)) for _ in range(R)]
    og = oracle.Oracle(oracle_params(p))
    for t, per_router in enumerate(slices):
        for r, pairs in enumerate(per_router):
            batch.load(r, helpers.to_device(pairs) if len(pairs) else pairs)
        rep = batch.step([len(x) for x in per_router])
        ref = ref_reports[t]
        assert np.array_equal(rep.hosts, ref.hosts) and np.array_equal(rep.flags, ref.flags)
        assert np.array_equal(rep.est, ref.est)
        # oracle: routers scan, the global estimator merges them and detects
        for o, pairs in zip(orcs, per_router):
            if t:
                o.advance()
            o.scan(pairs)
        if t:
            og.advance()
        og.merge(orcs)
        compare_report(rep, og.detect())
    compare_state(batch.global_estimator(), og, p, T - 1)
    for r in range(R):
        compare_state(batch.router(r), orcs[r], p, T - 1)
    assert batch.router(0).slice == T and batch.global_estimator().slice == T
    assert batch.kernel_launches > 0


def batch_against_oracle(batch, p, slices):
    """Steps `batch` through `slices`; after every step the report equals the detection of
    the oracle's routers merged into a global oracle (Algorithms 2 and 7, then 4, 5 and 8);
    at the end the global and every router state equal the oracle's."""
    R, T = len(slices[0]), len(slices)
    orcs = [oracle.Oracle(oracle_params(p)) for _ in range(R)]
    og = oracle.Oracle(oracle_params(p))
    found = 0
    for t, per_router in enumerate(slices):
        rep = batch.step(inputs=[helpers.to_device(x) for x in per_router])
        for o, pairs in zip(orcs, per_router):
            if t:
                o.advance()
            o.scan(pairs)
        if t:
            og.advance()
        og.merge(orcs)
        compare_report(rep, og.detect())
        found += rep.n_super
    compare_state(batch.global_estimator(), og, p, T - 1)
    for r in range(R):
        compare_state(batch.router(r), orcs[r], p, T - 1)
    return found


@pytest.mark.parametrize("item_pairs,unroll", [(1024, 2), (1024, 4), (1024, 8), (1025, 2)])
def test_batch_chunked_items_match_oracle(item_pairs, unroll):
    """Every router's slice spans 3-40 work items of the persistent update: items resume in
    the middle of a router's pairs (with item_pairs = 1025, at odd pairs, so the 16-byte peel
    runs), the last item of a router is partial, the RSRA owner of an item is chunk mod
    tiles, and a CTA flushes its bitmap whenever its next item belongs to another router.
    Reports and states against oracle routers and their merge."""
    S = sse()
    p = S.Params(seed=36)
    R, T = 5, 4
    slices = router_traffic(R, T, seed=36 + item_pairs + unroll, load_min=3 * item_pairs + 1,
                            load_max=40 * item_pairs)
    counts = [len(x) for s in slices for x in s]
    assert min(counts) > 2 * item_pairs and any(c % item_pairs for c in counts)
    batch = S.Batch(p, R, max(counts))
    batch.configure(item_pairs, unroll)
    assert batch_against_oracle(batch, p, slices) > 0


def test_batch_tuner_item_size_with_routers_over_several_items():
    """The tuner's smallest item size, 2^18 pairs, with every router above it (loads up to
    three items, none a multiple of the item): state and reports against the oracle."""
    S = sse()
    p = S.Params(seed=37)
    R, T = 3, 3
    slices = router_traffic(R, T, seed=37, load_min=(1 << 18) + 3, load_max=3 << 18)
    counts = [len(x) for s in slices for x in s]
    assert min(counts) > 1 << 18 and all(c % (1 << 18) for c in counts)
    batch = S.Batch(p, R, max(counts), use_graph=False)
    batch.configure(1 << 18, 4)
    batch_against_oracle(batch, p, slices)


def test_batch_graph_replay_equals_direct_launches_and_tuning_keeps_results():
    S = sse()
    p = S.Params(seed=32)
    R, T = 4, 5
    slices = router_traffic(R, T, seed=32)
    cap = max(len(x) for s in slices for x in s)
    a = S.Batch(p, R, cap, use_graph=True)
    b = S.Batch(p, R, cap, use_graph=False)
    for t, per_router in enumerate(slices):
        counts = [len(x) for x in per_router]
        dev = [helpers.to_device(x) for x in per_router]
        torch.cuda.synchronize()
        for r, pairs in enumerate(per_router):
            b.load(r, pairs)
        if t == 1:
            chosen, times = b.tune(counts)
            assert 0 <= chosen < 9 and all(x > 0 for x in times)
            chosen, times = a.tune(counts, inputs=dev)
        ra, rb = a.step(inputs=dev), b.step(counts)  # caller buffers in place vs loaded inputs
        assert np.array_equal(ra.hosts, rb.hosts) and np.array_equal(ra.est, rb.est)
        assert np.array_equal(ra.flags, rb.flags)
    for x, y in zip(a.global_estimator().read_stamps(), b.global_estimator().read_stamps()):
        assert np.array_equal(x, y)


def test_batch_rejects_counts_above_capacity_and_handles_empty_routers():
    S = sse()
    p = S.Params(seed=33)
    batch = S.Batch(p, 3, 1000)
    with pytest.raises(S.SSEError):
        batch.load(0, np.zeros((1001, 2), np.uint32))
    assert batch.step([0, 0, 0]).n_candidates == 0
    from paper_1805_09246_b300.sse import lib
    import ctypes
    counts = np.array([5, 2000, 0], np.uint64)
    assert lib().sse_batch_step(batch._b, ctypes.c_void_p(counts.ctypes.data), None) == S.ERR_CAPACITY


def test_batch_router_expiry_across_stamp_cycle():
    """Over 300 slices (more than one 8-bit stamp cycle) with k = 3: routers expire their old
    cells every 251 slices, the global estimator receives the routers' writes directly; both
    keep the oracle's state and reports (routers scanned alone, global = their merge)."""
    S = sse()
    p = S.Params(q=10, delta=8, q2=6, eta2=64, delta2=8, k=3, theta=8, seed=34)
    rng = np.random.default_rng(34)
    R = 2
    batch = S.Batch(p, R, 1024)
    orcs = [oracle.Oracle(oracle_params(p)) for _ in range(R)]
    og = oracle.Oracle(oracle_params(p))
    for t in range(300):
        per_router = []
        for r in range(R):
            pairs = rng.integers(0, 2**32, (150, 2), dtype=np.uint64).astype(np.uint32)
            pairs[:, 0] %= 11
            per_router.append(pairs)
        rep = batch.step(inputs=[helpers.to_device(x) for x in per_router])
        for o, pairs in zip(orcs, per_router):
            if t:
                o.advance()
            o.scan(pairs)
        if t:
            og.advance()
        og.scan(np.concatenate(per_router))
        if t % 50 == 0 or t >= 295:
            compare_report(rep, og.detect())
            compare_state(batch.global_estimator(), og, p, t)
            for r in range(R):
                compare_state(batch.router(r), orcs[r], p, t)


@pytest.mark.parametrize("graph", [True, False])
def test_batch_async_steps_equal_synchronous_steps(graph):
    """Steps enqueued two ahead of their reports (sse_batch_step_async / _wait) give the
    reports, slices and state of synchronous steps; calls that would race a pending step
    are refused with STATE."""
    S = sse()
    p = S.Params(seed=35)
    R, T = 4, 7
    slices = router_traffic(R, T, seed=35)
    dev = [[helpers.to_device(x) for x in per_router] for per_router in slices]
    torch.cuda.synchronize()
    cap = max(len(x) for s in slices for x in s)
    a = S.Batch(p, R, cap, use_graph=graph)
    b = S.Batch(p, R, cap, use_graph=graph)
    sync = [a.step(inputs=dev[t]) for t in range(T)]
    got = []
    b.step_async(inputs=dev[0])
    for t in range(1, T):
        b.step_async(inputs=dev[t])
        assert b.pending == 2
        with pytest.raises(S.SSEError):
            b.step_async(inputs=dev[t])  # a third pending step
        with pytest.raises(S.SSEError):
            b.set_mode(S.BATCH_ROUTERS)
        got.append(b.step_wait())
    got.append(b.step_wait())
    assert b.pending == 0
    with pytest.raises(S.SSEError):
        b.step_wait()  # nothing pending
    for x, y in zip(sync, got):
        assert x.slice == y.slice and x.n_candidates == y.n_candidates and x.n_super == y.n_super
        assert np.array_equal(x.hosts, y.hosts) and np.array_equal(x.est, y.est)
        assert np.array_equal(x.flags, y.flags)
    assert a.global_estimator().slice == b.global_estimator().slice == T
    for x, y in zip(a.global_estimator().read_stamps(), b.global_estimator().read_stamps()):
        assert np.array_equal(x, y)
    for r in range(R):
        for x, y in zip(a.router(r).read_stamps(), b.router(r).read_stamps()):
            assert np.array_equal(x, y)
