"""16-bit stamps: the paper's cell width (Section 3.2 keeps 16-bit distances) and its
sliding-window length k = 300 (Section 5). The GPU state, reports and merges are checked
against the oracle as for 8-bit stamps, including windows longer than 255 slices and the
wrap of the 65535-slice stamp cycle."""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers
from tests.test_gpu_parity import compare_report, compare_state, oracle_params, run_both, close_enough

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIRECT, TILED = 1, 2


def S():
    from paper_1805_09246_b300 import sse
    return sse


@pytest.mark.parametrize("mode", [DIRECT, TILED])
def test_small_trace_16bit_matches_oracle(mode):
    sse = S()
    p = sse.Params(stamp_bits=16, seed=21)
    tr = synth.Traffic(synth.small_trace(seed=21))
    _, _, reports = run_both(p, [tr.slice(0, t) for t in range(6)], mode=mode)
    assert sum(r.n_super for r in reports) > 50


@pytest.mark.parametrize("mode", [DIRECT, TILED])
def test_window_of_300_slices(mode):
    """k = 300: hosts keep contributing for 300 slices (longer than an 8-bit cycle); states
    and reports equal the oracle's at slices inside, at the edge of and past the window."""
    sse = S()
    p = sse.Params(q=12, q2=10, eta2=256, k=300, theta=200, stamp_bits=16, seed=22)
    rng = np.random.default_rng(22)
    est = sse.Estimator(p)
    est.set_update_mode(mode)
    orc = oracle.Oracle(oracle_params(p))
    heavy = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
    checks = {0, 150, 299, 300, 301, 330}
    for t in range(331):
        if t:
            orc.advance()
        bg = rng.integers(0, 2**32, (256, 2), dtype=np.uint64).astype(np.uint32)
        if t < 40:  # four hosts reach 600+ destinations early, then stop
            hv = np.stack([np.repeat(heavy, 16), rng.integers(0, 2**32, 64, dtype=np.uint64).astype(np.uint32)], 1)
            bg = np.concatenate([bg, hv])
        est.update(helpers.to_device(bg))
        orc.scan(bg)
        if t in checks:
            rep = est.close_slice()
            compare_state(est, orc, p, t)
            det = orc.detect()
            compare_report(rep, det)
            if t == 299:
                assert len(np.intersect1d(heavy, rep.hosts)) == 4  # still inside the window
        else:
            est.advance()
    orc.advance()
    # slice 331: the window 32..331 still holds the heavy hosts' last slices
    est_q, flags = est.query(torch.from_numpy(heavy.view(np.int32)).cuda())
    ref = orc.estimate(heavy)
    assert close_enough(est_q.cpu().numpy(), ref["est"])


def _paper_close_checks(est, orc, p, t, brute=False, extra_hosts=None):
    """State, hot SREs, row counts and report at slice t; with `brute`, the candidate set
    also against every 32-bit address whose r SREs are hot, and a query of the candidates
    (plus `extra_hosts`) with per-distance counts against the oracle's Algorithm 8."""
    det = orc.detect()
    if brute:  # the query evaluates the window ending at the current slice: before the close
        hosts = det["hosts"] if extra_hosts is None else np.union1d(det["hosts"], extra_hosts)
        e, f, h = est.query(helpers.to_device(hosts), hist=True)
        ref = orc.estimate(hosts, hist=True)
        assert close_enough(e.cpu().numpy(), ref["est"])
        assert np.array_equal(f.cpu().numpy(), ref["flags"])
        assert np.array_equal(h.cpu().numpy().view(np.uint32), ref["hist"])
        assert ref["hist"][:, 256:].any()  # distances above 255 occur
    rep = est.close_slice()
    compare_state(est, orc, p, t)
    assert np.array_equal(est.hot_bitmap(), orc.hot())
    assert est.stats()["active2"] == orc.row_counts().tolist()
    compare_report(rep, det)
    if brute:
        assert np.array_equal(rep.hosts, orc.candidates_brute())
    return rep


@pytest.mark.parametrize("mode", [DIRECT, TILED])
def test_paper_parameters_match_oracle(mode):
    """The paper's own estimator (Section 5): r = r' = 5, q = q' = 17, delta = 5, delta' = 16,
    eta' = 2^14, 16-bit cells, sliding window k = 300. Traffic: 20 slices of 2^17 pairs, 260
    slices without traffic, 20 more slices of 2^17 pairs, then 6 empty slices (20 planted
    hosts of 2k-20k destinations over a Zipf(1.1) background). A row of 2.1 M cells takes two
    bitmap pieces in the tiled update; the estimate gathers 16-bit cells of 2^14-cell SLEs,
    looks U up in the 16,385-entry table of the close, and the query's per-distance counts
    (k > 256) hold distances above 255. Every check of the close against the oracle at
    slices 0, 19, 290, 299 and 305; at 299 the candidates also against brute force over all
    2^32 addresses and the query with histograms against Algorithm 8."""
    sse = S()
    p = sse.paper_params()
    assert (p.q, p.q2, p.delta, p.eta2, p.k, p.stamp_bits) == (17, 17, 5, 1 << 14, 300, 16)
    tr = synth.Traffic(synth.TrafficConfig(seed=25, n_slices=40))
    est = sse.Estimator(p)
    est.set_update_mode(mode)
    orc = oracle.Oracle(oracle_params(p))
    rng = np.random.default_rng(25)
    t = 0
    reports = []
    for phase in range(2):
        for j in range(20):
            if t:
                orc.advance()
            pairs = tr.slice(0, 20 * phase + j)
            est.update(helpers.to_device(pairs))
            orc.scan(pairs)
            if t in (0, 19, 290):
                reports.append(_paper_close_checks(est, orc, p, t))
            elif t == 299:
                extra = rng.integers(0, 2**32, 200, dtype=np.uint64).astype(np.uint32)
                reports.append(_paper_close_checks(est, orc, p, t, brute=True, extra_hosts=extra))
            else:
                est.advance()
            t += 1
        if phase == 0:
            for _ in range(260):  # slices 20..279 carry no traffic
                orc.advance()
                est.advance()
                t += 1
    for _ in range(6):  # slices 300..305: the first slices leave the window
        orc.advance()
        if t < 305:
            est.advance()
        t += 1
    reports.append(_paper_close_checks(est, orc, p, 305))
    assert reports[3].n_super >= 10  # planted hosts of both phases are inside the window at 299
    assert reports[3].n_super >= reports[1].n_super


def test_16bit_stamp_cycle_wraps():
    """65,540 slice advances wrap the 16-bit stamp cycle: every old cell has expired, and the
    slices after the wrap give the state of a fresh oracle that saw only them."""
    sse = S()
    p = sse.Params(q=10, delta=8, q2=6, eta2=64, delta2=8, k=5, theta=8, stamp_bits=16, seed=23)
    rng = np.random.default_rng(23)
    est = sse.Estimator(p)
    for t in range(4):
        pairs = rng.integers(0, 2**32, (300, 2), dtype=np.uint64).astype(np.uint32)
        pairs[:, 0] %= 9
        est.update(helpers.to_device(pairs))
        est.advance()
    for _ in range(65540 - 4):
        est.advance()
    fresh = oracle.Oracle(oracle_params(p))
    for t in range(6):
        if t:
            fresh.advance()
        pairs = rng.integers(0, 2**32, (300, 2), dtype=np.uint64).astype(np.uint32)
        pairs[:, 0] %= 9
        est.update(helpers.to_device(pairs))
        fresh.scan(pairs)
        rep = est.close_slice()
        compare_state(est, fresh, p, 65540 + t)
        compare_report(rep, fresh.detect())


def test_merge_and_checkpoint_16bit():
    sse = S()
    p = sse.Params(stamp_bits=16, k=6, seed=24)
    tr = synth.Traffic(synth.small_trace(seed=24))
    rng = np.random.default_rng(24)
    routers = [sse.Estimator(p) for _ in range(2)]
    orcs = [oracle.Oracle(oracle_params(p)) for _ in range(2)]
    for t in range(3):
        pairs = tr.slice(0, t)
        owner = rng.integers(0, 2, len(pairs))
        for j in range(2):
            if t:
                orcs[j].advance()
                routers[j].advance()
            routers[j].update(helpers.to_device(pairs[owner == j]))
            orcs[j].scan(pairs[owner == j])
    glob = sse.Estimator(p)
    for _ in range(2):
        glob.advance()
    glob.merge(routers)
    og = oracle.Oracle(oracle_params(p))
    for _ in range(2):
        og.advance()
    og.merge(orcs)
    compare_state(glob, og, p, 2)
    blob = glob.export_state()
    clone = sse.Estimator(p)
    clone.import_state(blob)
    compare_report(clone.close_slice(), og.detect())
    compare_state(clone, og, p, 2)


def test_batches_and_features_need_8bit_stamps():
    sse = S()
    p = sse.Params(stamp_bits=16)
    with pytest.raises(sse.SSEError):
        sse.Batch(p, 2, 1024)
    e = sse.Estimator(p)
    with pytest.raises(sse.SSEError):
        e.features(torch.zeros(4, dtype=torch.int32, device="cuda"))
