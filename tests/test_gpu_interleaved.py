"""Calls interleaved with a slice's updates, through the C ABI.

The tiled update collects a slice's SLEA cells as bits and stamps them afterwards. Whatever
the calls between updates (query, features, read_stamps, export, merge of estimators on
other streams, advance, an asynchronous close with the next slice's update behind it), each
observation must equal that of the direct update, which stamps every cell at once, and the
oracle's (Algorithms 3 and 6, then 8 at the close).
"""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers
from tests.test_gpu_parity import DIRECT, TILED, close_enough, compare_report, compare_state, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sse():
    from paper_1805_09246_b300 import sse as mod
    return mod


def same_report(a, b):
    assert np.array_equal(a.hosts, b.hosts) and np.array_equal(a.flags, b.flags)
    assert np.array_equal(a.est, b.est) and a.n_super == b.n_super


@pytest.mark.parametrize("stamp_bits", [8, 16])
def test_calls_between_updates_see_the_tiled_cells(stamp_bits):
    """Each slice is scanned in two halves, with a query between them; after the second
    half a reading call of one kind (stamps, export, features, advance of a copy) and then
    the close, alternately from the captured graph and kernel by kernel."""
    S = sse()
    p = S.Params(seed=5, stamp_bits=stamp_bits, k=4)
    tr = synth.Traffic(synth.small_trace(seed=5))
    tiled, direct = S.Estimator(p), S.Estimator(p)
    tiled.set_update_mode(TILED)
    direct.set_update_mode(DIRECT)
    orc = oracle.Oracle(oracle_params(p))
    ip, _ = tr.planted()
    hosts = np.concatenate([ip, tr.slice(0, 0)[:200, 0]]).astype(np.uint32)
    d_hosts = helpers.to_device(hosts)
    for t in range(6):
        if t:
            orc.advance()
        pairs = tr.slice(0, t)
        half = len(pairs) // 2
        for e in (tiled, direct):
            e.update(helpers.to_device(pairs[:half]))
        orc.scan(pairs[:half])
        (et, ft), (ed, fd) = tiled.query(d_hosts), direct.query(d_hosts)
        want = orc.estimate(hosts)
        assert np.array_equal(et.cpu().numpy(), ed.cpu().numpy())
        assert np.array_equal(ft.cpu().numpy(), fd.cpu().numpy())
        assert np.array_equal(ft.cpu().numpy(), want["flags"])
        assert close_enough(et.cpu().numpy(), want["est"])
        for e in (tiled, direct):
            e.update(helpers.to_device(pairs[half:]))
        orc.scan(pairs[half:])
        if t % 3 == 0:
            compare_state(tiled, orc, p, t)
            st, sd = tiled.read_stamps(), direct.read_stamps()
            assert np.array_equal(st[0], sd[0]) and np.array_equal(st[1], sd[1])
        elif t % 3 == 1:
            assert tiled.export_state() == direct.export_state()
        elif stamp_bits == 8:  # features are defined on 8-bit cells
            assert torch.equal(tiled.features(d_hosts), direct.features(d_hosts))
        graph = t % 2 == 0
        tiled.close_use_graph(graph)
        direct.close_use_graph(graph)
        rt, rd = tiled.close_slice(), direct.close_slice()
        compare_report(rt, orc.detect())
        same_report(rt, rd)
        compare_state(tiled, orc, p, t)


def test_merge_of_tiled_sources_on_other_streams():
    """Two routers on streams of their own, each updated by the tiled kernel, merged into a
    third estimator updated the same way: the merged state and the next close equal the
    oracle's merge."""
    S = sse()
    p = S.Params(seed=9)
    tr = synth.Traffic(synth.TrafficConfig(seed=9, n_routers=3, n_slices=4))
    ests = [S.Estimator(p, stream=torch.cuda.Stream()) for _ in range(3)]
    orcs = [oracle.Oracle(oracle_params(p)) for _ in range(3)]
    for e in ests:
        e.set_update_mode(TILED)
    for t in range(4):
        for r in range(3):
            if t:
                orcs[r].advance()
            pairs = tr.slice(r, t)
            ests[r].update(helpers.to_device(pairs))
            orcs[r].scan(pairs)
        for r in (1, 2):  # the sources' streams must be done before the merge reads them
            ests[r].sync()
        ests[0].merge([ests[1], ests[2]])
        orcs[0].merge([orcs[1], orcs[2]])
        compare_state(ests[0], orcs[0], p, t)
        for r in range(3):
            rep = ests[r].close_slice()
            compare_report(rep, orcs[r].detect())


def test_pipelined_closes_and_advance():
    """The benchmark's order (the next slice's update enqueued behind an asynchronous
    close, before its report is read) and sse_advance (a close pass without detection):
    every tiled cell carries the stamp of its own slice."""
    S = sse()
    p = S.Params(seed=13, k=3)
    tr = synth.Traffic(synth.small_trace(seed=13))
    tiled, direct = S.Estimator(p), S.Estimator(p)
    tiled.set_update_mode(TILED)
    direct.set_update_mode(DIRECT)
    orc = oracle.Oracle(oracle_params(p))
    slices = [tr.slice(0, t) for t in range(8)]
    for e in (tiled, direct):
        e.update(helpers.to_device(slices[0]))
    orc.scan(slices[0])
    for t in range(7):
        if t == 3:  # a slice ended without detection
            for e in (tiled, direct):
                e.advance()
        else:
            for e in (tiled, direct):
                e.close_slice_async()
        orc.advance()
        for e in (tiled, direct):
            e.update(helpers.to_device(slices[t + 1]))
        orc.scan(slices[t + 1])
        if t != 3:
            rt, rd = tiled.close_slice_wait(), direct.close_slice_wait()
            same_report(rt, rd)
        compare_state(tiled, orc, p, t + 1)
    rep = tiled.close_slice()
    compare_report(rep, orc.detect())
