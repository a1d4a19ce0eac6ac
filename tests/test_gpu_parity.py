"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same inputs.

Bar: bit-exact estimator state (canonical ages), hot SREs, active-cell counts, candidate
and super point sets and flags; estimates (float32) within 1e-6 relative of the oracle's
FP64 values.
"""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EST_RTOL = 1e-6


def sse():
    from paper_1805_09246_b300 import sse as mod
    return mod


def oracle_params(p):
    return oracle.Params(r=p.r, q=p.q, delta=p.delta, eta=p.eta, r2=p.r2, q2=p.q2, delta2=p.delta2,
                         eta2=p.eta2, k=p.k, theta=p.theta, seed=p.seed, rhfg_hash=p.rhfg_hash)


def compare_state(est, orc, p, slice_index):
    sre_s, sle_s = est.read_stamps()
    o_sre, o_sle = helpers.oracle_canonical(orc, p.k)
    g_sre = helpers.canonical_from_stamps(sre_s, slice_index, p.k, p.stamp_bits)
    g_sle = helpers.canonical_from_stamps(sle_s, slice_index, p.k, p.stamp_bits)
    assert np.array_equal(g_sre, o_sre), "RSRA state differs"
    assert np.array_equal(g_sle, o_sle), "SLEA state differs"


def close_enough(got, ref):
    got = np.asarray(got, np.float64)
    return np.all(np.abs(got - ref) <= EST_RTOL * np.maximum(np.abs(ref), 1e-30))


def compare_report(rep, det):
    assert np.array_equal(rep.hosts, det["hosts"]), "candidate sets differ"
    assert np.array_equal(rep.flags, det["flags"]), "flags differ"
    assert close_enough(rep.est, det["est"])
    assert rep.n_super == int((det["flags"] & oracle.SUPER).astype(bool).sum())


def run_both(p, slices, mode=None, check_state=True):
    S = sse()
    est = S.Estimator(p)
    if mode is not None:
        est.set_update_mode(mode)
    orc = oracle.Oracle(oracle_params(p))
    reports = []
    for t, pairs in enumerate(slices):
        if t:
            orc.advance()
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        rep = est.close_slice()
        det = orc.detect()
        if check_state:
            compare_state(est, orc, p, t)
            assert np.array_equal(est.hot_bitmap(), orc.hot())
            st = est.stats()
            assert st["active2"] == orc.row_counts().tolist()
        compare_report(rep, det)
        reports.append(rep)
    return est, orc, reports


DIRECT, TILED = 1, 2


@pytest.mark.parametrize("mode", [DIRECT, TILED])
def test_small_trace_end_to_end(mode):
    """The 8-slice, 2^17-pair trace: every slice's state, hot SREs, counts and report."""
    S = sse()
    p = S.Params()
    tr = synth.Traffic(synth.small_trace())
    _, _, reports = run_both(p, [tr.slice(0, t) for t in range(8)], mode=mode)
    assert sum(r.n_super for r in reports) > 100  # the planted super points are found


def test_close_pass_with_a_ragged_last_warp_step():
    """r * 2^q = 288 SREs (r=9, q=5): the close pass covers 64 SREs per warp step, so its
    last step holds only 32. State (expiry), hot bitmap, counts and reports."""
    S = sse()
    p = S.Params(r=9, q=5, delta=4, q2=6, eta2=64, delta2=8, k=3, theta=8, seed=31)
    rng = np.random.default_rng(31)
    slices = []
    for _ in range(5):
        pairs = rng.integers(0, 2**32, (3000, 2), dtype=np.uint64).astype(np.uint32)
        pairs[:, 0] %= 5
        slices.append(pairs)
    run_both(p, slices)


def test_join_probes_global_any_hot_bitmaps():
    """q - delta = 19: the "any hot" bitmaps of rows 2 and 3 (64 KiB each) are too large to
    stage in shared memory, so the join from row 0 up probes them in global memory. Hot SREs,
    counts and reports against the oracle."""
    S = sse()
    p = S.Params(r=5, q=23, delta=4, seed=23)
    tr = synth.Traffic(synth.small_trace(seed=23))
    est = S.Estimator(p)
    est.set_join(S.JOIN_FORWARD)
    orc = oracle.Oracle(oracle_params(p))
    found = 0
    for t in range(3):
        if t:
            orc.advance()
        pairs = tr.slice(0, t)
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        rep = est.close_slice()
        assert np.array_equal(est.hot_bitmap(), orc.hot())
        assert est.stats()["active2"] == orc.row_counts().tolist()
        compare_report(rep, orc.detect())
        found += rep.n_candidates
    assert found > 0


@pytest.mark.parametrize("mode", [DIRECT, TILED])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 1000, 65537, 300001])
def test_ragged_sizes_and_tiles(n, mode):
    S = sse()
    p = S.Params(q=12, delta=7, q2=8, eta2=256, k=2, theta=16, seed=n)
    rng = np.random.default_rng(n)
    src = rng.integers(0, 2**32, 97, dtype=np.uint64).astype(np.uint32)
    pairs = np.stack([src[rng.integers(0, 97, n)], rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)], 1)
    run_both(p, [pairs, pairs[: n // 2 + 1], pairs[::-1].copy()], mode=mode)


def test_every_update_variant_matches_oracle():
    """Each autotuner variant (direct and every tiled form) gives the oracle's state."""
    S = sse()
    p = S.Params(seed=19)
    tr = synth.Traffic(synth.small_trace(seed=19))
    slices = [tr.slice(0, t) for t in range(2)]
    for v in range(S.update_variant_count()):
        est = S.Estimator(p)
        est.set_update_mode(TILED if v else DIRECT)
        est.set_update_variant(v)
        orc = oracle.Oracle(oracle_params(p))
        for t, pairs in enumerate(slices):
            if t:
                orc.advance()
                est.advance()
            est.update(helpers.to_device(pairs))
            orc.scan(pairs)
        compare_state(est, orc, p, 1)


def test_autotune_keeps_state_and_picks_a_variant():
    S = sse()
    p = S.Params(seed=20)
    tr = synth.Traffic(synth.small_trace(seed=20))
    pairs = helpers.to_device(tr.slice(0, 0))
    a, b = S.Estimator(p), S.Estimator(p)
    a.update(pairs)
    chosen, times = b.autotune_update(pairs, reps=2)
    assert 0 <= chosen < S.update_variant_count() and len(times) == S.update_variant_count()
    assert all(t > 0 for t in times) and times[chosen] == min(times)
    for x, y in zip(a.read_stamps(), b.read_stamps()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("params", ["paper", "core_link", "many_rows", "ragged_pieces"])
def test_update_strategies_agree(params):
    """Direct and every tiled variant leave bit-identical stamps, including rows split into
    several shared-memory pieces (the paper's q'=17 rows; three pieces whose last one, rounded
    up to 1024 cells, reaches 1024 cells past the row pitch) and misaligned group starts."""
    S = sse()
    p = {"paper": S.paper_params(k=8), "core_link": S.core_link_params(),
         "many_rows": S.Params(r2=16, q2=14, eta2=2048, seed=4),
         "ragged_pieces": S.Params(q2=17, delta2=32, eta2=4096, seed=6)}[params]
    rng = np.random.default_rng(7)
    n = (1 << 22) + 3
    src = rng.integers(0, 2**32, 1 << 20, dtype=np.uint64).astype(np.uint32)
    pairs = np.stack([src[rng.integers(0, 1 << 20, n)], rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)], 1)
    a = S.Estimator(p)
    a.set_update_mode(DIRECT)
    tiled = []  # every tiled form the autotuner may pick
    for v in range(1, S.update_variant_count()):
        b = S.Estimator(p)
        b.set_update_mode(TILED)
        b.set_update_variant(v)
        tiled.append(b)
    for t in range(2):
        buf = helpers.to_device(np.concatenate([np.zeros((1, 2), np.uint32), pairs]))
        a.update(buf[1:])
        want = a.read_stamps()
        for b in tiled:
            b.update(buf[1:])
            for x, y in zip(want, b.read_stamps()):
                assert np.array_equal(x, y)
            b.advance()
        a.advance()
        pairs = pairs[::-1].copy()


@pytest.mark.parametrize("mode", [DIRECT, TILED])
@pytest.mark.parametrize("offset,n", [(1, 10001), (5, 70001), (15, 70000), (16, 70001), (9, 3), (3, 12)])
def test_misaligned_device_pointer(offset, n, mode):
    """Pairs starting `offset` pairs past a 128-byte boundary: the tiled update's head (the
    pairs before the first 128-byte line, up to 15, all of them when n is smaller) and the
    direct update's 16-byte peel, against the oracle."""
    S = sse()
    p = S.Params(seed=3 + offset)
    rng = np.random.default_rng(3 + offset)
    pairs = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    pairs[:, 0] = pairs[:, 0] % 50
    buf = helpers.to_device(np.concatenate([np.zeros((offset, 2), np.uint32), pairs]))
    assert buf.data_ptr() % 128 == 0
    est = S.Estimator(p)
    est.set_update_mode(mode)
    est.update(buf[offset:])
    orc = oracle.Oracle(oracle_params(p))
    orc.scan(pairs)
    compare_state(est, orc, p, 0)


def test_window_wraps_stamp_cycle():
    """More than 255 slices: stamps reuse values, expiry keeps the window exact."""
    S = sse()
    p = S.Params(q=10, delta=8, q2=6, eta2=64, delta2=8, k=3, theta=8, seed=9)
    rng = np.random.default_rng(9)
    est = S.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    for t in range(300):
        if t:
            orc.advance()
        pairs = rng.integers(0, 2**32, (200, 2), dtype=np.uint64).astype(np.uint32)
        pairs[:, 0] %= 7
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        if t % 37 == 0 or t >= 297:
            rep = est.close_slice()
            compare_state(est, orc, p, t)
            compare_report(rep, orc.detect())
        else:
            est.advance()
    assert est.slice == 300


@pytest.mark.parametrize("sle_rows", ["core_link", "sixteen_times_longer"])
def test_core_link_full_size_parity(sle_rows):
    """Three 2^25-pair slices of the core-link trace in the benchmark's configuration
    (automatic update strategy): state, hot SREs, row counts, candidates (against the
    definitional brute force over all 2^32 addresses) and estimates. The benchmark's SLEA
    rows (2^16 SLEs) are saturated at this load, so most estimates take Eq. 12's clamp; with
    rows of 2^20 SLEs (q' = 20, ten bitmap pieces per row in the tiled update) they are not,
    and the estimates are compared in the regime where Eq. 12 corrects a partly filled union
    SLE."""
    S = sse()
    p = S.core_link_params()
    if sle_rows == "sixteen_times_longer":
        p = S.Params(q=20, q2=20, eta2=4096, k=8, seed=0)
    tr = synth.Traffic(synth.core_link())
    est = S.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    for t in range(3):
        pairs = tr.slice(0, t)
        if t:
            orc.advance()
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        rep = est.close_slice()
    compare_state(est, orc, p, 2)
    assert np.array_equal(est.hot_bitmap(), orc.hot())
    assert est.stats()["active2"] == orc.row_counts().tolist()
    want = orc.candidates_brute()
    assert np.array_equal(rep.hosts, want)
    ref = orc.estimate(want)
    assert np.array_equal(rep.flags, ref["flags"])
    assert close_enough(rep.est, ref["est"])
    ip, _ = tr.planted()
    assert len(np.intersect1d(ip, rep.super_points)) > 20
    if sle_rows == "sixteen_times_longer":
        sf = np.array(orc.row_counts()) / orc.row_len2
        assert sf.max() < 0.9  # rows far from full
        assert np.count_nonzero((ref["flags"] & oracle.SATURATED) == 0) > len(want) // 4


def test_k1_discrete_window():
    S = sse()
    p = S.Params(k=1, theta=256, seed=11)
    tr = synth.Traffic(synth.small_trace(seed=11))
    run_both(p, [tr.slice(0, t) for t in range(3)])


def test_estimates_across_the_whole_range_of_U():
    """Hosts with 1 .. 2000 distinct destinations on 64-cell SLEs (eta' = 64): union counts
    from a few cells to every cell, so w / eta' falls in both halves of [0, 1) and at the
    saturation clamp. The per-host query path (Eq. 12 and Eq. 8 for each host) and the close's
    table over U (its reported candidates) against the oracle: flags exact, estimates within
    the FP32 tolerance."""
    S = sse()
    p = S.Params(q2=6, eta2=64, delta2=8, k=2, theta=16, seed=41)
    rng = np.random.default_rng(41)
    counts = [1, 2, 4, 8, 12, 16, 24, 32, 40, 48, 56, 64, 96, 128, 256, 512, 2000]
    hosts = np.unique(rng.integers(0, 2**32, 4 * len(counts), dtype=np.uint64).astype(np.uint32))
    hosts = rng.permutation(hosts)[: len(counts)]
    pairs = np.concatenate([np.stack([np.full(c, h, np.uint32),
                                      rng.integers(0, 2**32, c, dtype=np.uint64).astype(np.uint32)], 1)
                            for h, c in zip(hosts, counts)])
    pairs = pairs[rng.permutation(len(pairs))]
    est = S.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    est.update(helpers.to_device(pairs))
    orc.scan(pairs)
    e, f = est.query(helpers.to_device(hosts))
    ref = orc.estimate(hosts)
    assert close_enough(e.cpu().numpy(), ref["est"])
    assert np.array_equal(f.cpu().numpy(), ref["flags"])
    x = ref["w"] / p.eta2
    assert (x > 0).any() and (x < 0.5).any() and (x >= 0.5).any()
    assert (ref["flags"] & oracle.SATURATED).any()
    rep = est.close_slice()
    det = orc.detect()
    compare_report(rep, det)
    assert rep.n_candidates >= 8
    big = det["est"] >= p.eta2 * np.log(2.0)  # est >= eta' ln 2 exactly when w / eta' >= 1/2
    assert big.any() and (~big).any()  # the table path sees both halves too


def test_query_matches_oracle_estimates():
    S = sse()
    p = S.Params(k=4, seed=12)
    tr = synth.Traffic(synth.small_trace(seed=12))
    est = S.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    for t in range(3):
        if t:
            orc.advance()
        pairs = tr.slice(0, t)
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        if t < 2:
            est.advance()
    ip, _ = tr.planted()
    rng = np.random.default_rng(1)
    hosts = np.concatenate([ip, tr.slice(0, 0)[:500, 0],
                            rng.integers(0, 2**32, 300, dtype=np.uint64).astype(np.uint32)])
    e, f, h = est.query(helpers.to_device(hosts), hist=True)
    ref = orc.estimate(hosts, hist=True)
    assert close_enough(e.cpu().numpy(), ref["est"])
    assert np.array_equal(f.cpu().numpy(), ref["flags"])
    assert np.array_equal(h.cpu().numpy().view(np.uint32), ref["hist"])
    compare_state(est, orc, p, 2)  # the query changed nothing


def test_merge_of_routers_equals_union():
    """Three routers' estimators merged on the device equal one estimator of all pairs,
    and both equal the oracle's merge."""
    S = sse()
    p = S.Params(seed=13)
    tr = synth.Traffic(synth.small_trace(seed=13))
    rng = np.random.default_rng(13)
    routers = [S.Estimator(p) for _ in range(3)]
    whole = S.Estimator(p)
    orcs = [oracle.Oracle(oracle_params(p)) for _ in range(3)]
    for t in range(5):
        pairs = tr.slice(0, t)
        owner = rng.integers(0, 3, len(pairs))
        for j in range(3):
            if t:
                orcs[j].advance()
            routers[j].update(helpers.to_device(pairs[owner == j]))
            orcs[j].scan(pairs[owner == j])
        whole.update(helpers.to_device(pairs))
        if t < 4:
            for e in routers + [whole]:
                e.advance()
    glob = S.Estimator(p)
    for _ in range(4):
        glob.advance()
    glob.merge(routers)
    og = oracle.Oracle(oracle_params(p))
    for _ in range(4):
        og.advance()
    og.merge(orcs)
    compare_state(glob, og, p, 4)
    for x, y in zip(glob.read_stamps(), whole.read_stamps()):
        assert np.array_equal(helpers.canonical_from_stamps(x, 4, p.k), helpers.canonical_from_stamps(y, 4, p.k))
    compare_report(glob.close_slice(), og.detect())
    with pytest.raises(S.SSEError):
        routers[0].merge([glob])  # glob moved past the routers' slice


def test_update_host_paths_match_device_path():
    S = sse()
    p = S.Params(seed=14)
    tr = synth.Traffic(synth.small_trace(seed=14))
    pairs = np.concatenate([tr.slice(0, 0), tr.slice(0, 1)])
    a, b, c = S.Estimator(p), S.Estimator(p), S.Estimator(p)
    a.update(helpers.to_device(pairs))
    b.update_host(pairs)  # pageable
    pinned = torch.from_numpy(pairs.view(np.int32)).pin_memory()
    c.update_host(pinned)
    for x, y, z in zip(a.read_stamps(), b.read_stamps(), c.read_stamps()):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_checkpoint_roundtrip():
    S = sse()
    p = S.Params(seed=15)
    tr = synth.Traffic(synth.small_trace(seed=15))
    a = S.Estimator(p)
    for t in range(3):
        a.update(helpers.to_device(tr.slice(0, t)))
        if t < 2:
            a.advance()
    blob = a.export_state()
    b = S.Estimator(p)
    b.import_state(blob)
    assert b.slice == a.slice == 2
    for x, y in zip(a.read_stamps(), b.read_stamps()):
        assert np.array_equal(x, y)
    ra, rb = a.close_slice(), b.close_slice()
    assert np.array_equal(ra.hosts, rb.hosts) and np.array_equal(ra.est, rb.est)
    with pytest.raises(S.SSEError):
        S.Estimator(S.Params(seed=16)).import_state(blob)


def _planted_state(p, orc, hosts, rng, noise_cells=20000):
    sre = np.full((p.r, 1 << p.q, p.eta), helpers.INF, np.uint16)
    for aip in hosts.tolist():
        for i in range(p.r):
            sre[i, orc.rhfg(i, aip), :3] = rng.integers(0, p.k, 3)
    _, sle = orc.raw()
    sle[:, rng.integers(0, orc.row_len2, noise_cells)] = 0
    orc.set_raw(sre, sle)
    return sre, sle


def test_many_candidates_sorted_and_capacity():
    """Planted hot SREs for thousands of hosts: candidate set = oracle's (brute force),
    ascending across several sort chunks; a small capacity reports a truncated prefix."""
    S = sse()
    p = S.Params(q=20, k=2, theta=64, max_candidates=1 << 14, seed=17)
    orc = oracle.Oracle(oracle_params(p))
    rng = np.random.default_rng(17)
    hosts = np.unique(rng.integers(0, 2**32, 9000, dtype=np.uint64).astype(np.uint32))
    sre, sle = _planted_state(p, orc, hosts, rng)
    want = orc.candidates_brute()
    assert len(want) > 2 * 4096
    est = S.Estimator(p)
    blob = helpers.state_blob(est.export_state(), helpers.stamps_from_distances(sre, 0, p.k),
                              helpers.stamps_from_distances(sle, 0, p.k), est.derived["row_pitch2"])
    est.import_state(blob)
    clone = S.Estimator(p)
    clone.import_state(blob)
    rep = est.close_slice()
    assert np.array_equal(rep.hosts, want)
    ref = orc.estimate(want)
    assert np.array_equal(rep.flags, ref["flags"])
    assert close_enough(rep.est, ref["est"])
    small = clone.close_slice(cap=1000, raise_on_capacity=False)
    assert small.status == S.ERR_CAPACITY and small.truncated
    assert small.n_candidates == len(want)
    assert np.array_equal(small.hosts, want[:1000])


def test_sort_paths_alternate_in_the_close_graph():
    """The one-launch candidate sort ranks up to 4096 candidates and chunk-sorts and merges
    more (grid barriers between the merge passes): slices alternating between thousands of
    candidates (planted) and a handful, closed from the CUDA graph, give the reports of the
    kernels launched one by one, and the planted slice's candidates are the oracle's (brute
    force)."""
    S = sse()
    p = S.Params(q=20, k=2, theta=64, max_candidates=1 << 14, seed=23)
    orc = oracle.Oracle(oracle_params(p))
    rng = np.random.default_rng(23)
    hosts = np.unique(rng.integers(0, 2**32, 6000, dtype=np.uint64).astype(np.uint32))
    sre, sle = _planted_state(p, orc, hosts, rng)
    want = orc.candidates_brute()
    assert len(want) > 4096
    g, d = S.Estimator(p), S.Estimator(p)
    d.close_use_graph(False)
    blob = helpers.state_blob(g.export_state(), helpers.stamps_from_distances(sre, 0, p.k),
                              helpers.stamps_from_distances(sle, 0, p.k), g.derived["row_pitch2"])
    tr = synth.Traffic(synth.small_trace(seed=23))
    counts = []
    for t in range(6):
        if t % 3 == 0:  # replant (a fresh slice-0 state)
            g.import_state(blob)
            d.import_state(blob)
        else:
            pairs = helpers.to_device(tr.slice(0, t))
            g.update(pairs)
            d.update(pairs)
        rg, rd = g.close_slice(), d.close_slice()
        assert np.array_equal(rg.hosts, rd.hosts) and np.array_equal(rg.flags, rd.flags)
        assert np.array_equal(rg.est, rd.est) and rg.n_super == rd.n_super
        if t % 3 == 0:
            assert np.array_equal(rg.hosts, want)
        counts.append(rg.n_candidates)
    assert max(counts) > 4096 and min(counts) <= 4096


def test_few_low_bits_per_row_without_any_hot_filter():
    """q - delta < 5 (r = 8, q = 8, delta = 4): the join runs without row 3's any-hot bitmap;
    state, hot SREs and reports still match the oracle."""
    S = sse()
    p = S.Params(r=8, q=8, delta=4, r2=5, q2=12, eta2=1024, delta2=16, k=3, theta=1024, seed=29)
    rng = np.random.default_rng(29)
    slices = []
    for t in range(4):
        src = rng.integers(0, 2**32, 6, dtype=np.uint64).astype(np.uint32)
        heavy = np.stack([np.repeat(src, 3000), rng.integers(0, 2**32, 6 * 3000, dtype=np.uint64).astype(np.uint32)], 1)
        noise = rng.integers(0, 2**32, (500, 2), dtype=np.uint64).astype(np.uint32)
        slices.append(np.ascontiguousarray(np.concatenate([heavy, noise])[rng.permutation(6 * 3000 + 500)]))
    run_both(p, slices)


def test_candidate_overflow_is_reported():
    S = sse()
    p = S.Params(q=14, k=2, theta=64, max_candidates=64, seed=18)
    orc = oracle.Oracle(oracle_params(p))
    rng = np.random.default_rng(18)
    hosts = rng.integers(0, 2**32, 200, dtype=np.uint64).astype(np.uint32)
    sre, sle = _planted_state(p, orc, hosts, rng, noise_cells=10)
    est = S.Estimator(p)
    blob = helpers.state_blob(est.export_state(), helpers.stamps_from_distances(sre, 0, p.k),
                              helpers.stamps_from_distances(sle, 0, p.k), est.derived["row_pitch2"])
    est.import_state(blob)
    rep = est.close_slice(raise_on_capacity=False)
    assert rep.status == S.ERR_CAPACITY and rep.truncated and rep.n_candidates >= 200
    assert len(rep.hosts) == 64 and np.all(np.diff(rep.hosts.astype(np.int64)) > 0)
    est.update(helpers.to_device(np.zeros((4, 2), np.uint32)))  # the handle is still usable
    est.sync()


def test_invalid_arguments():
    S = sse()
    with pytest.raises(S.SSEError):
        S.Estimator(S.Params(k=0))
    est = S.Estimator(S.Params())
    est.update(helpers.to_device(np.zeros((0, 2), np.uint32)))  # empty batch is a no-op
    with pytest.raises(S.SSEError):
        est.merge([est])
    lib = S.lib()
    assert lib.sse_update(est.handle, None, 5) < 0
    assert lib.sse_query(est.handle, None, 3, None, None, None) < 0
    assert lib.sse_set_update_mode(est.handle, 7) < 0
    est.sync()


def test_close_graph_equals_direct_launches():
    """sse_close_slice replayed from its CUDA graph gives the same reports, statistics and
    state as the kernels launched one by one, also when a handle switches between them."""
    S = sse()
    p = S.Params(seed=41)
    tr = synth.Traffic(synth.small_trace(seed=41))
    a, b = S.Estimator(p), S.Estimator(p)
    b.close_use_graph(False)
    for t in range(6):
        pairs = helpers.to_device(tr.slice(0, t))
        a.update(pairs)
        b.update(pairs)
        if t == 3:
            a.close_use_graph(False)
            b.close_use_graph(True)
        ra, rb = a.close_slice(), b.close_slice()
        assert np.array_equal(ra.hosts, rb.hosts) and np.array_equal(ra.est, rb.est)
        assert np.array_equal(ra.flags, rb.flags) and ra.n_super == rb.n_super and ra.slice == rb.slice == t
        assert a.stats() == b.stats()
    for x, y in zip(a.read_stamps(), b.read_stamps()):
        assert np.array_equal(x, y)
    assert a.slice == b.slice == 6


def test_async_close_pipelined_with_next_update():
    """close_slice_async + the next slice's update + close_slice_wait gives the reports and
    state of the synchronous close; misuse is refused with STATE."""
    S = sse()
    p = S.Params(seed=42)
    tr = synth.Traffic(synth.small_trace(seed=42))
    slices = [helpers.to_device(tr.slice(0, t)) for t in range(6)]
    a, b = S.Estimator(p), S.Estimator(p)
    ref = []
    for x in slices:
        a.update(x)
        ref.append(a.close_slice())
    got = []
    b.update(slices[0])
    for t in range(6):
        b.close_slice_async()
        with pytest.raises(S.SSEError):
            b.close_slice_async()  # one close at a time
        with pytest.raises(S.SSEError):
            b.close_slice()
        if t + 1 < 6:
            b.update(slices[t + 1])  # scanned into the next slice while the report is produced
        got.append(b.close_slice_wait())
    with pytest.raises(S.SSEError):
        b.close_slice_wait()  # nothing pending
    for ra, rb in zip(ref, got):
        assert ra.slice == rb.slice
        assert np.array_equal(ra.hosts, rb.hosts) and np.array_equal(ra.est, rb.est)
        assert np.array_equal(ra.flags, rb.flags)
    for x, y in zip(a.read_stamps(), b.read_stamps()):
        assert np.array_equal(x, y)


def test_async_reports_interleaved_with_other_closes():
    """An asynchronous close writes its report on a second stream while the next work runs;
    synchronous closes (report inside the close graph), closes launched kernel by kernel,
    slice advances and a reset that follow it must wait for that report. Every report, and
    the state, equal those of a handle that only closes synchronously; the last reports
    against the oracle."""
    S = sse()
    p = S.Params(q=17, seed=43)
    tr = synth.Traffic(synth.small_trace(seed=43))
    pairs = [tr.slice(0, t) for t in range(8)]
    slices = [helpers.to_device(x) for x in pairs]
    plan = ["async", "sync", "async", "advance", "async", "direct", "async", "sync"]
    a, b = S.Estimator(p), S.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    for t, (x, how) in enumerate(zip(slices, plan)):
        if t:
            orc.advance()
        orc.scan(pairs[t])
        a.update(x)
        b.update(x)
        if how == "advance":
            a.advance()
            b.advance()
            continue
        ra = a.close_slice()
        if how == "async":
            b.close_slice_async()
            rb = b.close_slice_wait()
        elif how == "direct":
            b.close_use_graph(False)
            rb = b.close_slice()
            b.close_use_graph(True)
        else:
            rb = b.close_slice()
        assert ra.slice == rb.slice == t
        assert np.array_equal(ra.hosts, rb.hosts) and np.array_equal(ra.est, rb.est)
        assert np.array_equal(ra.flags, rb.flags) and ra.n_super == rb.n_super
        compare_report(rb, orc.detect())
    for x, y in zip(a.read_stamps(), b.read_stamps()):
        assert np.array_equal(x, y)
    b.update(slices[0])
    b.close_slice_async()
    b.close_slice_wait()
    b.reset()  # after an asynchronous report
    b.update(slices[0])
    fresh = S.Estimator(p)
    fresh.update(slices[0])
    rf, rb = fresh.close_slice(), b.close_slice()
    assert np.array_equal(rf.hosts, rb.hosts) and np.array_equal(rf.est, rb.est)


@pytest.mark.parametrize("rhfg_hash", [0, 1])
def test_directions_and_tabulation_rhfg0(rhfg_hash):
    """Definition 1 either way: SSE_DIR_DST equals scanning the exchanged pairs, SSE_DIR_BOTH
    equals scanning both; with RHFG[0] by simple tabulation as well (states and reports
    against the oracle, candidates against the definitional brute force)."""
    S = sse()
    p = S.Params(seed=61, rhfg_hash=rhfg_hash)
    tr = synth.Traffic(synth.small_trace(seed=61))
    slices = [tr.slice(0, t) for t in range(3)]
    swapped = [x[:, ::-1].copy() for x in slices]
    both = [np.concatenate([x, y]) for x, y in zip(slices, swapped)]
    ref_dst = S.Estimator(p)
    dst = S.Estimator(p)
    dst.set_direction(S.DIR_DST)
    two = S.Estimator(p)
    two.set_direction(S.DIR_BOTH)
    orc = oracle.Oracle(oracle_params(p))
    for t in range(3):
        if t:
            orc.advance()
        ref_dst.update(helpers.to_device(swapped[t]))
        dst.update(helpers.to_device(slices[t]))
        two.update(helpers.to_device(slices[t]))
        orc.scan(both[t])
        ra, rb, rc = ref_dst.close_slice(), dst.close_slice(), two.close_slice()
        assert np.array_equal(ra.hosts, rb.hosts) and np.array_equal(ra.est, rb.est)
        compare_report(rc, orc.detect())
        compare_state(two, orc, p, t)
    for x, y in zip(ref_dst.read_stamps(), dst.read_stamps()):
        assert np.array_equal(x, y)
    if rhfg_hash:
        assert np.array_equal(rc.hosts, orc.candidates_brute())
