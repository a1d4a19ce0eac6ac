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
