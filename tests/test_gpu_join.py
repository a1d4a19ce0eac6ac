"""The close's two joins (sse_set_join) against each other and against the oracle.

The join from rows 0, 1, 2 up (Algorithms 4-5 in the paper's order) and the join from rows
0 and r-1 down (B(r-1) keeps only s = 32 - (r-1)*delta address bits, so row r-1's hot SREs
pair with he_0 inside one column block of 2^s) list the same chains. Every shape below has
delta <= 5 and 4 <= r <= 6, where the join from the top row down applies; candidates are
compared with the definitional brute force over all 2^32 addresses, flags exactly and
estimates within the FP32 tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers
from tests.test_gpu_parity import close_enough, compare_report, oracle_params, sse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def planted_state(p, orc, rng, n_hosts, noise_share):
    """Hot SREs of n_hosts random hosts in every row, plus a noise_share of each row's SREs
    made hot at random (chains that end before row r-1, or complete by chance)."""
    sre = np.full((p.r, 1 << p.q, p.eta), helpers.INF, np.uint16)
    hosts = np.unique(rng.integers(0, 2**32, n_hosts, dtype=np.uint64).astype(np.uint32))
    for aip in hosts.tolist():
        for i in range(p.r):
            sre[i, orc.rhfg(i, aip), :3] = rng.integers(0, p.k, 3)
    for i in range(p.r):
        cols = rng.integers(0, 1 << p.q, int(noise_share * (1 << p.q)))
        sre[i, cols, :3] = rng.integers(0, p.k, (len(cols), 3))
    _, sle = orc.raw()
    sle[:, rng.integers(0, orc.row_len2, 20000)] = 0
    orc.set_raw(sre, sle)
    return sre, sle


def estimators(p, sre, sle, modes):
    S = sse()
    out = []
    for mode in modes:
        est = S.Estimator(p)
        est.set_join(mode)
        blob = helpers.state_blob(est.export_state(), helpers.stamps_from_distances(sre, 0, p.k),
                                  helpers.stamps_from_distances(sle, 0, p.k), est.derived["row_pitch2"])
        est.import_state(blob)
        out.append(est)
    return out


# (r, q, delta, planted hosts, noise share): s = 32 - (r-1)*delta, 2^(q-s) column blocks
PLANTED = [
    (5, 17, 5, 1500, 0.015),  # the paper's estimator: s = 12, 32 blocks; ~2.6 % hot per row
    (5, 20, 4, 5000, 0.004),  # the core link's: s = 16, 16 blocks
    (6, 12, 5, 150, 0.05),    # s = 7, 32 blocks of 128 columns; groups of 32 often hot
    (6, 16, 4, 1000, 0.03),   # s = 12, 16 blocks
    (6, 19, 5, 800, 0.012),   # s = 7: 4096 blocks, more than the 1024 block-list CTAs (4 each)
]


@pytest.mark.parametrize("r,q,delta,n_hosts,noise", PLANTED)
def test_joins_match_brute_force_on_dense_hot_rows(r, q, delta, n_hosts, noise):
    S = sse()
    p = S.Params(r=r, q=q, delta=delta, k=2, theta=64, seed=q * 10 + r)
    orc = oracle.Oracle(oracle_params(p))
    rng = np.random.default_rng(q * 10 + r)
    sre, sle = planted_state(p, orc, rng, n_hosts, noise)
    want = orc.candidates_brute()
    fwd, bwd = estimators(p, sre, sle, [S.JOIN_FORWARD, S.JOIN_BACKWARD])
    rf, rb = fwd.close_slice(), bwd.close_slice()
    assert len(want) >= n_hosts * 0.9
    assert np.array_equal(rb.hosts, want), "join from the top row down"
    assert np.array_equal(rf.hosts, want), "join from row 0 up"
    ref = orc.estimate(want)
    for rep in (rf, rb):
        assert np.array_equal(rep.flags, ref["flags"])
        assert close_enough(rep.est, ref["est"])
    # the pairs each join started from: HSE(0) x HSE(1), or HSE(0) x HSE(r-1) by column block
    hot = orc.hot()
    h0, h1, hl = (np.flatnonzero(hot[i]) for i in (0, 1, r - 1))
    s, nb = 32 - (r - 1) * delta, 1 << (q - (32 - (r - 1) * delta))
    by_block = np.dot(np.bincount(h0 >> s, minlength=nb), np.bincount(hl >> s, minlength=nb))
    assert fwd.stats()["join_pairs"] == len(h0) * len(h1)
    assert bwd.stats()["join_pairs"] == by_block < len(h0) * len(h1)


def test_join_overflow_reports_the_same_count():
    """More candidates than max_candidates: both joins count every candidate, report the
    same truncated prefix and flag CAPACITY."""
    S = sse()
    p = S.Params(r=6, q=12, delta=5, k=2, theta=64, max_candidates=100, seed=61)
    orc = oracle.Oracle(oracle_params(p))
    rng = np.random.default_rng(61)
    sre, sle = planted_state(p, orc, rng, 400, 0.05)
    want = orc.candidates_brute()
    assert len(want) > 300
    fwd, bwd = estimators(p, sre, sle, [S.JOIN_FORWARD, S.JOIN_BACKWARD])
    for est in (fwd, bwd):
        rep = est.close_slice(raise_on_capacity=False)
        assert rep.status == S.ERR_CAPACITY and rep.truncated
        assert rep.n_candidates == len(want)
        assert len(rep.hosts) == 100 and np.all(np.diff(rep.hosts.astype(np.int64)) > 0)
        assert np.all(np.isin(rep.hosts, want))


# (r, q, delta): traffic through both joins, every slice against the oracle's tuple growth
TRAFFIC = [(4, 22, 5), (5, 23, 3), (5, 17, 5), (6, 16, 4)]


@pytest.mark.parametrize("r,q,delta", TRAFFIC)
def test_joins_match_oracle_on_traffic(r, q, delta):
    S = sse()
    p = S.Params(r=r, q=q, delta=delta, q2=12, eta2=1024, k=3, theta=256, seed=r + q)
    cfg = synth.TrafficConfig(seed=r + q, n_slices=4, load_min=1 << 17, load_max=1 << 17, n_planted=400,
                              planted_min=600, planted_max=3000)
    tr = synth.Traffic(cfg)
    fwd, bwd = S.Estimator(p), S.Estimator(p)
    fwd.set_join(S.JOIN_FORWARD)
    bwd.set_join(S.JOIN_BACKWARD)
    orc = oracle.Oracle(oracle_params(p))
    found = 0
    for t in range(4):
        if t:
            orc.advance()
        pairs = tr.slice(0, t)
        orc.scan(pairs)
        d = helpers.to_device(pairs)
        fwd.update(d)
        bwd.update(d)
        det = orc.detect()
        compare_report(fwd.close_slice(), det)
        rep = bwd.close_slice()
        compare_report(rep, det)
        found += rep.n_candidates
    assert found > 400


def test_set_join_switches_between_closes():
    """The join can change between closes of one handle (the close graph is captured again);
    a mode the parameters do not admit, or an unknown one, is refused."""
    S = sse()
    p = S.Params(q=17, seed=71)  # the paper's q: delta = 5, s = 12
    tr = synth.Traffic(synth.small_trace(seed=71))
    est = S.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    for t, mode in enumerate([S.JOIN_AUTO, S.JOIN_FORWARD, S.JOIN_BACKWARD, S.JOIN_FORWARD, S.JOIN_AUTO]):
        if t:
            orc.advance()
        est.set_join(mode)
        pairs = tr.slice(0, t)
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        compare_report(est.close_slice(), orc.detect())
    with pytest.raises(S.SSEError):
        est.set_join(7)
    small = S.Estimator(S.Params(q=14))  # delta = 6: only the join from row 0 up
    small.set_join(S.JOIN_FORWARD)
    with pytest.raises(S.SSEError):
        small.set_join(S.JOIN_BACKWARD)


def test_join_edge_cases():
    """No hot SRE at all; hot SREs in every row but the top one (no pair to start from, and no
    chain from row 0 up either); a single planted host. Both joins against the brute force."""
    S = sse()
    p = S.Params(r=5, q=17, delta=5, k=2, theta=64, seed=81)
    rng = np.random.default_rng(81)
    cases = []
    orc = oracle.Oracle(oracle_params(p))
    cases.append(("empty", orc, *orc.raw()))
    orc = oracle.Oracle(oracle_params(p))
    sre, sle = planted_state(p, orc, rng, 0, 0.03)
    sre[p.r - 1] = helpers.INF  # the top row holds no hot SRE
    orc.set_raw(sre, sle)
    cases.append(("no top row", orc, sre, sle))
    orc = oracle.Oracle(oracle_params(p))
    cases.append(("one host", orc, *planted_state(p, orc, rng, 1, 0.0)))
    for name, orc, sre, sle in cases:
        want = orc.candidates_brute()
        assert len(want) == {"empty": 0, "no top row": 0, "one host": 1}[name], name
        fwd, bwd = estimators(p, sre, sle, [S.JOIN_FORWARD, S.JOIN_BACKWARD])
        rf, rb = fwd.close_slice(), bwd.close_slice()
        assert np.array_equal(rf.hosts, want) and np.array_equal(rb.hosts, want), name
        if name != "one host":
            assert bwd.stats()["join_pairs"] == 0, name
