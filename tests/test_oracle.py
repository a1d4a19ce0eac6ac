"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against the paper's
worked examples (golden fixtures), a published known answer, a closed form, an
invariant the method must have, or brute force on small inputs.
"""
import numpy as np
import pytest

import oracle
from oracle import Oracle, Params
from paper_1805_09246_b300 import synth
from tests.conftest import read_golden

INF = 65535


def small_params(**kw):
    base = dict(r=5, q=14, delta=0, eta=8, r2=5, q2=10, delta2=16, eta2=256, k=3, theta=64, seed=7)
    base.update(kw)
    return Params(**base)


def random_pairs(rng, n, n_src=200, n_dst=5000):
    src = rng.integers(0, 2**32, n_src, dtype=np.uint64).astype(np.uint32)
    dst = rng.integers(0, 2**32, n_dst, dtype=np.uint64).astype(np.uint32)
    return np.stack([src[rng.integers(0, n_src, n)], dst[rng.integers(0, n_dst, n)]], axis=1)


# ---------------------------------------------------------------- paper examples

def test_lsb_paper_examples():
    for x, want in read_golden("lsb_examples.txt"):
        assert oracle.lsb(int(x)) == int(want)


def test_lsb_brute_force():
    rng = np.random.default_rng(1)
    for x in rng.integers(1, 2**32, 2000, dtype=np.uint64).tolist():
        low = x & -x
        assert oracle.lsb(x) == low.bit_length() - 1
    assert oracle.lsb(0) == 32  # reading: LSB(0) passes every tau <= 32


def test_paper_parameter_derivation():
    g = {k: int(v) for k, v in read_golden("paper_parameters.txt")}
    p = Params(r=g["r"], q=g["q"], delta=0, eta=g["eta"], r2=g["r2"], q2=g["q2"],
               delta2=g["delta2"], eta2=g["eta2"], k=8, theta=g["theta"])
    d = oracle.derive(p)
    assert d["delta"] == g["delta"]
    assert d["tau"] == g["tau"]
    assert d["hot_min"] == g["hot_min"]
    assert d["row_len2"] == g["row_len2"]


def test_parameter_constraints_enforced():
    # Eq. 6 needs delta < q and (r-2)*delta + q >= 32.
    with pytest.raises(ValueError):
        oracle.derive(Params(r=5, q=14, delta=5))  # 3*5 + 14 = 29 < 32
    with pytest.raises(ValueError):
        oracle.derive(Params(r=3, q=14, delta=14))  # delta == q
    assert oracle.derive(Params(r=5, q=14, delta=6))["delta"] == 6


def test_splitmix64_known_answers():
    want = [int(row[0], 16) for row in read_golden("splitmix64_seed0.txt")]
    assert oracle.splitmix64(0, len(want)) == want


def test_tau_is_ceil_log2():
    # Eq. 1 against the real-valued formula away from exact powers of two.
    for eta in (8, 16):
        for theta in (1, 3, 8, 9, 100, 1000, 1024, 1025, 5000, 123457):
            want = max(0, int(np.ceil(np.log2(theta / eta) - 1e-12)))
            assert oracle.derive(Params(eta=eta, theta=theta))["tau"] == want


# ---------------------------------------------------------------- hash functions

def test_hash_keys_follow_splitmix64_order():
    o = Oracle(small_params(seed=12345))
    stream = oracle.splitmix64(12345, 2 * (4 + 5))
    keys = o.keys().astype(np.uint64)
    assert keys[0::2].tolist() == [v | 1 for v in stream[0::2]]
    assert keys[1::2].tolist() == stream[1::2]


def test_hash_definition_and_ranges():
    p = small_params(seed=99)
    o = Oracle(p)
    keys = [int(v) for v in o.keys()]
    M = (1 << 64) - 1

    def mas(key_index, x, m):
        a, b = keys[2 * key_index], keys[2 * key_index + 1]
        return ((a * x + b) & M) >> (64 - m) if m else 0

    rng = np.random.default_rng(3)
    for x in rng.integers(0, 2**32, 300, dtype=np.uint64).tolist():
        assert o.h1(x) == mas(0, x, 32)
        assert o.h2(x) == mas(1, x, 3)
        assert o.h3(x) == mas(2, x, 8)
        assert o.rhfg0(x) == mas(3, x, p.q)
        for i in range(p.r2):
            assert o.lh(i, x) == mas(4 + i, x, p.q2)


def test_h3_uniform():
    o = Oracle(small_params(seed=5))
    xs = np.arange(1 << 15, dtype=np.uint32) * np.uint32(2654435761)
    counts = np.bincount([o.h3(int(x)) for x in xs], minlength=256)
    expected = len(xs) / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 400  # 255 dof; p ~ 1e-8 above this


def test_rhfg_eq7_recovers_address_bits():
    p = small_params(seed=17)
    o = Oracle(p)
    d = o.delta
    rng = np.random.default_rng(4)
    for aip in rng.integers(0, 2**32, 2000, dtype=np.uint64).tolist():
        h0 = o.rhfg0(aip)
        assert o.rhfg(0, aip) == h0
        for i in range(1, p.r):
            assert o.rhfg(i, aip) ^ h0 == (aip >> (i * d)) % (1 << p.q)


# ---------------------------------------------------------------- update (Alg. 3, Alg. 6)

def test_single_pair_touches_exactly_its_cells():
    p = small_params(seed=21, theta=1)  # tau = 0: every pair updates RSRA
    o = Oracle(p)
    aip, bip = 0x0A000001, 0xC0A80101
    o.scan(np.array([[aip, bip]], dtype=np.uint32))
    sre, sle = o.raw()
    want_sre = np.full_like(sre, INF)
    for i in range(p.r):
        want_sre[i, o.rhfg(i, aip), o.h2(bip)] = 0
    want_sle = np.full_like(sle, INF)
    for i in range(p.r2):
        want_sle[i, o.lh(i, aip) * p.delta2 + o.h3(bip)] = 0
    assert np.array_equal(sre, want_sre)
    assert np.array_equal(sle, want_sle)


def test_rsra_sampling_follows_lsb_threshold():
    p = small_params(seed=22, theta=1024)  # tau = 7
    o = Oracle(p)
    assert o.d["tau"] == 7
    rng = np.random.default_rng(5)
    bips = rng.integers(0, 2**32, 4000, dtype=np.uint64).astype(np.uint32)
    pairs = np.stack([np.full_like(bips, 0x01020304), bips], axis=1)
    o.scan(pairs)
    sre, _ = o.raw()
    touched = (sre == 0).any(axis=(0, 2)).sum()
    sampled = [b for b in bips.tolist() if oracle.lsb(o.h1(b)) >= 7]
    assert 0 < len(sampled) < 80
    # every sampled bip set its cell in all r rows
    for b in sampled:
        for i in range(p.r):
            assert sre[i, o.rhfg(i, 0x01020304), o.h2(b)] == 0
    assert touched <= p.r


def test_slice_update_increments_and_saturates():
    p = small_params(seed=23, k=2)
    o = Oracle(p)
    o.scan(np.array([[1, 2]], dtype=np.uint32))
    _, sle0 = o.raw()
    o.advance()
    o.advance()
    _, sle2 = o.raw()
    assert np.array_equal(sle2[sle0 == 0], np.full((sle0 == 0).sum(), 2, np.uint16))
    assert (sle2[sle0 == INF] == INF).all()


def test_scan_order_invariance():
    p = small_params(seed=24)
    rng = np.random.default_rng(6)
    pairs = random_pairs(rng, 20000)
    a, b = Oracle(p), Oracle(p)
    a.scan(pairs)
    b.scan(pairs[rng.permutation(len(pairs))])
    for x, y in zip(a.raw(), b.raw()):
        assert np.array_equal(x, y)


def test_window_invariant():
    """After slices 0..t the active state equals a fresh estimator fed slices t-k+1..t."""
    p = small_params(seed=25, k=3)
    rng = np.random.default_rng(7)
    slices = [random_pairs(rng, 5000, n_src=150) for _ in range(7)]
    full = Oracle(p)
    for t, s in enumerate(slices):
        if t:
            full.advance()
        full.scan(s)
        fresh = Oracle(p)
        lo = max(0, t - p.k + 1)
        for u in range(lo, t + 1):
            if u > lo:
                fresh.advance()
            fresh.scan(slices[u])
        for x, y in zip(full.canonical(), fresh.canonical()):
            assert np.array_equal(x, y)


def test_k1_is_the_discrete_window():
    """k = 1: active cells are exactly the ones set in the current slice (RE / LE)."""
    p = small_params(seed=26, k=1)
    rng = np.random.default_rng(8)
    o = Oracle(p)
    for t in range(3):
        if t:
            o.advance()
        s = random_pairs(rng, 4000)
        o.scan(s)
        only = Oracle(p)
        only.scan(s)
        _, sle_only = only.raw()
        _, can = o.canonical()
        assert np.array_equal(can == 0, sle_only == 0)
        assert ((can == 0) | (can == 255)).all()


def test_row_counts_are_active_cells():
    p = small_params(seed=27)
    o = Oracle(p)
    o.scan(random_pairs(np.random.default_rng(9), 30000))
    o.advance()
    o.scan(random_pairs(np.random.default_rng(10), 30000))
    _, sle = o.raw()
    assert np.array_equal(o.row_counts(), (sle < p.k).sum(axis=1).astype(np.uint64))


# ---------------------------------------------------------------- merge (Alg. 2, Alg. 7)

def _split_run(p, slices, parts, rng):
    ors = [Oracle(p) for _ in range(parts)]
    for t, s in enumerate(slices):
        owner = rng.integers(0, parts, len(s))
        for j, o in enumerate(ors):
            if t:
                o.advance()
            o.scan(s[owner == j])
    return ors


def test_merge_equals_estimator_of_union():
    p = small_params(seed=28)
    rng = np.random.default_rng(11)
    slices = [random_pairs(rng, 8000) for _ in range(4)]
    whole = Oracle(p)
    for t, s in enumerate(slices):
        if t:
            whole.advance()
        whole.scan(s)
    parts = _split_run(p, slices, 3, rng)
    merged = Oracle(p)
    for _ in range(len(slices) - 1):
        merged.advance()
    merged.merge(parts)
    for x, y in zip(merged.raw(), whole.raw()):
        assert np.array_equal(x, y)


def test_merge_commutative_associative_idempotent():
    p = small_params(seed=29)
    rng = np.random.default_rng(12)
    slices = [random_pairs(rng, 6000) for _ in range(3)]
    a, b, c = _split_run(p, slices, 3, rng)

    def fresh_like():
        o = Oracle(p)
        for _ in range(len(slices) - 1):
            o.advance()
        return o

    ab_c = fresh_like(); ab_c.merge([a, b]); ab_c.merge([c])
    c_ba = fresh_like(); c_ba.merge([c]); c_ba.merge([b, a])
    aa = fresh_like(); aa.merge([a, a])
    a_only = fresh_like(); a_only.merge([a])
    for x, y in zip(ab_c.raw(), c_ba.raw()):
        assert np.array_equal(x, y)
    for x, y in zip(aa.raw(), a_only.raw()):
        assert np.array_equal(x, y)
    for x, y in zip(a_only.raw(), a.raw()):
        assert np.array_equal(x, y)


def test_literal_max_merge_is_not_the_union():
    """Documents the merge reading: keeping the larger distance (Alg. 7 taken literally)
    loses cells active at only one router, so it cannot be the global estimator."""
    p = small_params(seed=30)
    rng = np.random.default_rng(13)
    slices = [random_pairs(rng, 6000) for _ in range(2)]
    a, b = _split_run(p, slices, 2, rng)
    whole = Oracle(p)
    whole.scan(slices[0]); whole.advance(); whole.scan(slices[1])
    _, la = a.raw(); _, lb = b.raw(); _, lw = whole.raw()
    assert not np.array_equal(np.maximum(la, lb), lw)
    assert np.array_equal(np.minimum(la, lb), lw)


def test_merge_rejects_mismatch():
    a = Oracle(small_params(seed=31))
    b = Oracle(small_params(seed=32))
    with pytest.raises(ValueError):
        a.merge([b])
    c = Oracle(small_params(seed=31))
    c.advance()
    with pytest.raises(ValueError):
        a.merge([c])


# ---------------------------------------------------------------- candidates (Alg. 4, Alg. 5)

def _plant_hot_state(p, o, hosts, noise_frac, rng):
    """RSRA where every SRE of the given hosts is hot, plus random hot SREs as noise."""
    sre = np.full((p.r, 1 << p.q, p.eta), INF, dtype=np.uint16)
    hot_min = o.d["hot_min"]
    for aip in hosts:
        for i in range(p.r):
            sre[i, o.rhfg(i, int(aip)), :hot_min] = 0
    n_noise = int(noise_frac * (1 << p.q))
    for i in range(p.r):
        cols = rng.choice(1 << p.q, n_noise, replace=False)
        sre[i, cols, :hot_min] = rng.integers(0, p.k, size=(n_noise, hot_min))
    # lukewarm SREs (one cell short of hot) must not count
    for i in range(p.r):
        cols = rng.choice(1 << p.q, n_noise, replace=False)
        sre[i, cols, : hot_min - 1] = np.minimum(sre[i, cols, : hot_min - 1], 1)
    o.set_raw(sre, None)


@pytest.mark.parametrize("q,delta", [(14, 6), (12, 7), (17, 5)])
def test_candidates_match_brute_force(q, delta):
    p = small_params(q=q, delta=delta, seed=33 + q)
    o = Oracle(p)
    rng = np.random.default_rng(q)
    hosts = rng.integers(0, 2**32, 40, dtype=np.uint64).astype(np.uint32)
    _plant_hot_state(p, o, hosts, 0.02, rng)
    tuples = o.candidates()
    brute = o.candidates_brute()
    assert np.array_equal(tuples, brute)
    assert set(hosts.tolist()) <= set(brute.tolist())
    # every candidate's r estimators are hot (definition)
    hot = o.hot()
    for aip in brute.tolist():
        assert all(hot[i, o.rhfg(i, aip)] for i in range(p.r))


def test_candidates_on_traffic_match_brute_force():
    p = Params(seed=0)  # q=14, delta=6
    o = Oracle(p)
    tr = synth.Traffic(synth.small_trace())
    for t in range(4):
        if t:
            o.advance()
        o.scan(tr.slice(0, t))
    assert np.array_equal(o.candidates(), o.candidates_brute())


def test_address_bits_beyond_32_are_rejected():
    # (r-1)*delta + q > 32: tuples whose top B(r-1) bits are not zero regain no host.
    p = small_params(q=12, delta=7, seed=40)
    o = Oracle(p)
    sre = np.full((p.r, 1 << p.q, p.eta), INF, dtype=np.uint16)
    he0 = 5
    # a consistent tuple for aip = 0xFFFFFFFF except row 4 claims bits above 32
    aip = 0xFFFFFFFF
    cols = [o.rhfg(i, aip) for i in range(p.r)]
    for i, c in enumerate(cols):
        sre[i, c, :3] = 0
    o.set_raw(sre, None)
    assert aip in o.candidates().tolist()
    bad_b4 = (cols[0] ^ cols[4]) | (1 << (p.q - 1))  # top bit lies above address bit 31
    sre[4, cols[4], :3] = INF
    sre[4, cols[0] ^ bad_b4, :3] = 0
    o.set_raw(sre, None)
    assert len(o.candidates()) == 0 == len(o.candidates_brute())
    del he0


# ---------------------------------------------------------------- estimation (Alg. 8, Eq. 8-12)

def test_union_sle_is_per_cell_intersection_with_max_distance():
    p = small_params(r2=3, q2=6, delta2=4, eta2=64, k=4, seed=41)
    o = Oracle(p)
    aip = 0x11223344
    sle = np.full((p.r2, o.row_len2), INF, dtype=np.uint16)
    # row i: cell z active with distance i iff z % (i + 2) == 0
    for i in range(p.r2):
        base = o.lh(i, aip) * p.delta2
        for z in range(p.eta2):
            if z % (i + 2) == 0:
                sle[i, base + z] = i
    o.set_raw(None, sle)
    e = o.estimate([aip], hist=True)
    both = [z for z in range(p.eta2) if z % 2 == 0 and z % 3 == 0 and z % 4 == 0]
    assert e["U"][0] == len(both)
    # the union SLE keeps the largest distance over rows: 2
    assert e["hist"][0].tolist() == [0, 0, len(both), 0]


def test_lone_host_counts_distinct_cell_hashes():
    """One host alone: |USLE|^k is the number of distinct H3 values of its opposite hosts,
    and every SLEA row holds exactly those cells."""
    p = small_params(q2=12, eta2=1024, k=2, seed=42)
    o = Oracle(p)
    rng = np.random.default_rng(14)
    bips = rng.integers(0, 2**32, 700, dtype=np.uint64).astype(np.uint32)
    aip = 0xDEADBEEF
    o.scan(np.stack([np.full_like(bips, aip), bips], axis=1))
    D = len({o.h3(int(b)) for b in bips})
    e = o.estimate([aip])
    assert e["U"][0] == D
    assert o.row_counts().tolist() == [D] * p.r2
    assert 0 <= e["w"][0] <= D


def test_estimate_unbiased_under_noise():
    """Eq. 11-12: with other hosts' cells spread at random over the rows, the corrected
    weight w^ is, on average, the weight of the host's own SLE; Eq. 8 on it gives back n.
    Dropping the noise term, the denominator or flipping a sign moves the mean by >100 cells."""
    # q' = 12 keeps the row-end effect small: SF averages over the whole row, whose ends
    # are covered by fewer SLEs, so an interior host sees (eta'-delta')/(2^q' delta') more noise.
    p = small_params(q2=12, eta2=1024, k=1, seed=43)
    n = 800
    rng = np.random.default_rng(15)
    ws, ests, own = [], [], []
    for trial in range(24):
        o = Oracle(Params(**{**p.__dict__, "seed": 1000 + trial}))
        aip = int(rng.integers(0, 2**32))
        bips = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
        noise = random_pairs(rng, 112000, n_src=20000, n_dst=4_000_000)
        o.scan(noise)
        o.scan(np.stack([np.full_like(bips, aip), bips], axis=1))
        e = o.estimate([aip])
        assert not (e["flags"][0] & oracle.SATURATED)
        ws.append(e["w"][0])
        ests.append(e["est"][0])
        own.append(len({o.h3(int(b)) for b in bips}))
    sf = o.row_counts() / o.row_len2
    assert 0.7 < sf.min() < sf.max() < 0.9  # noise cells are a third of the union SLE
    diff = np.array(ws) - np.array(own)
    assert abs(diff.mean()) < 20
    assert abs(np.mean(ests) / n - 1) < 0.08


def test_decision_in_weight_domain_matches_estimate_threshold():
    """Reading of Eq. 8 + threshold: est >= theta iff w^ >= w_theta, away from rounding."""
    for eta2, theta in [(1024, 1024), (4096, 1024), (16384, 1024), (256, 64)]:
        w_theta = oracle.derive(Params(eta2=eta2, q2=8, theta=theta))["w_theta"]
        w = np.linspace(0, eta2 - 1, 200001)
        est = -eta2 * np.log((eta2 - w) / eta2)
        far = np.abs(w - w_theta) > 1e-9 * eta2
        assert np.array_equal((est >= theta)[far], (w >= w_theta)[far])


@pytest.mark.parametrize("counts,U,case", [((60, 80, 100), 30, "P < 1/2"),
                                           ((170, 180, 185), 60, "P > 1/2"),
                                           ((150, 150, 150), 20, "w < 0")])
def test_corrected_weight_and_estimate_closed_form(counts, U, case):
    """Eq. 11-12 and Eq. 8 worked by hand on a hand-set SLEA: r' = 3 rows of
    L' = 2^q' * delta' + eta' - delta' = 188 cells; row i holds exactly counts[i] active cells
    (distance < k), U of the host's eta' = 64 union cells are active in all three rows and a
    few more in one row only, inactive cells hold distances >= k. Then
    P = (c_0/L') (c_1/L') (c_2/L'), multiplied in row order; w = (U - eta' P) / (1 - P),
    clamped at 0; est = -eta' ln(1 - w/eta'); super iff w >= eta'(1 - e^(-theta/eta')).
    The oracle's w must be the same double, so a wrong L', a wrong product, a dropped
    term or a sign error fails."""
    import math
    p = small_params(r2=3, q2=5, delta2=4, eta2=64, k=4, theta=32, seed=46)
    o = Oracle(p)
    L = o.row_len2
    assert L == 32 * 4 + 64 - 4 == 188
    aip = 0x5EED1234
    rng = np.random.default_rng(46)
    sle = np.full((p.r2, L), INF, dtype=np.uint16)
    sle[:, ::7] = p.k  # inactive: distance exactly k
    sle[:, 3::11] = p.k + 3
    zs = rng.permutation(p.eta2)
    common, extra = zs[:U], np.array_split(zs[U:], p.r2)  # extra[i]: active in row i only
    for i in range(p.r2):
        base = o.lh(i, aip) * p.delta2
        inside = np.concatenate([common, extra[i]]) + base
        outside = np.setdiff1d(np.arange(L), np.arange(base, base + p.eta2))
        m = counts[i] - len(inside)
        assert 0 <= m <= len(outside)
        active = np.concatenate([inside, rng.choice(outside, m, replace=False)])
        sle[i, active] = rng.integers(0, p.k, len(active))
    o.set_raw(None, sle)
    assert o.row_counts().tolist() == list(counts)
    e = o.estimate([aip])
    assert e["U"][0] == U
    eta2 = float(p.eta2)
    P = 1.0
    for c in counts:
        P = P * (c / L)
    w = (U - eta2 * P) / (1.0 - P)
    if case == "w < 0":
        assert w < 0
        w = 0.0
    else:
        assert 0 < w < eta2 - 1 and (P < 0.5) == (case == "P < 1/2")
    est = -eta2 * math.log((eta2 - w) / eta2)
    assert e["w"][0] == w
    assert abs(e["est"][0] - est) <= 1e-12 * max(est, 1e-300)
    w_theta = eta2 * (1.0 - math.exp(-p.theta / eta2))
    assert bool(e["flags"][0] & oracle.SUPER) == (w >= w_theta)
    assert not e["flags"][0] & oracle.SATURATED
    if case != "w < 0":
        assert e["flags"][0] & oracle.SUPER  # both positive cases are above theta = 32


def test_saturation_and_clamping():
    p = small_params(q2=4, delta2=4, eta2=64, k=2, seed=44)
    o = Oracle(p)
    sle = np.zeros((p.r2, o.row_len2), dtype=np.uint16)  # every cell active: SF = 1
    o.set_raw(None, sle)
    e = o.estimate([123])
    assert e["flags"][0] & oracle.SATURATED
    assert e["w"][0] == p.eta2 - 1
    assert np.isclose(e["est"][0], p.eta2 * np.log(p.eta2))
    sle[:] = INF
    o.set_raw(None, sle)
    e = o.estimate([123])
    assert e["w"][0] == 0 and e["est"][0] == 0 and e["flags"][0] == 0


# ---------------------------------------------------------------- ground truth (Def. 1, 2)

def test_exact_counts_match_naive_recount():
    p = small_params(k=3, seed=45)
    rng = np.random.default_rng(16)
    o = Oracle(p, track_exact=True)
    slices = [random_pairs(rng, 3000, n_src=40, n_dst=400) for _ in range(6)]
    for t, s in enumerate(slices):
        if t:
            o.advance()
        o.scan(s)
        window = np.concatenate(slices[max(0, t - p.k + 1): t + 1])
        naive = {}
        for a, b in window.tolist():
            naive.setdefault(a, set()).add(b)
        hosts = np.array(sorted(naive), dtype=np.uint32)
        assert o.exact_counts(hosts).tolist() == [len(naive[h]) for h in hosts.tolist()]
        theta = 60
        sup, card = o.exact_super(theta)
        want = sorted(h for h in naive if len(naive[h]) >= theta)
        assert sup.tolist() == want
        assert card.tolist() == [len(naive[h]) for h in want]


def test_detection_on_small_trace():
    """End to end on the 8-slice trace: detected sliding super points agree with the exact
    ones (Def. 2) up to the estimator's error near theta."""
    p = Params(seed=0)
    o = Oracle(p, track_exact=True)
    tr = synth.Traffic(synth.small_trace())
    tp = fp = fn = 0
    for t in range(8):
        if t:
            o.advance()
        o.scan(tr.slice(0, t))
        det = o.detect()
        found = set(det["hosts"][(det["flags"] & oracle.SUPER) > 0].tolist())
        exact, card = o.exact_super()
        truth = set(exact.tolist())
        tp += len(found & truth)
        fp += len(found - truth)
        fn += len(truth - found)
        # every exact super point well above theta is found
        assert set(exact[card >= 2 * p.theta].tolist()) <= found
    assert tp >= 120 and fp <= 5 and fn <= 10


# ---------------------------------------------------------------- learned correction (FP64 reference)

def test_mlp_gradient_matches_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(50)
    D, H, n = 6, 8, 13
    theta = rng.normal(0, 0.5, mlp.param_count(D, H))
    x = rng.normal(0, 1, (n, D))
    t = rng.normal(0, 1, n)
    _, g = mlp.gradient(theta, x, t, D, H)
    eps = 1e-6
    num = np.zeros_like(theta)
    for k in range(theta.size):
        e = np.zeros_like(theta)
        e[k] = eps
        num[k] = (mlp.loss(theta + e, x, t, D, H) - mlp.loss(theta - e, x, t, D, H)) / (2 * eps)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_mlp_forward_closed_form():
    """With identity-like weights the network is a hand-computable function."""
    from oracle import mlp
    D, H = 2, 2
    W1 = np.array([[1.0, 0.0], [0.0, -1.0]])
    b1 = np.array([0.5, 0.0])
    W2 = np.eye(2)
    b2 = np.zeros(2)
    W3 = np.array([2.0, 3.0])
    b3 = 1.0
    theta = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])
    x = np.array([[1.0, -2.0], [-3.0, 4.0]])
    # sample 0: h1 = relu([1.5, 2]) = [1.5, 2] -> y = 1 + 2*1.5 + 3*2 = 10
    # sample 1: h1 = relu([-2.5, -4]) = [0, 0] -> y = 1
    assert np.allclose(mlp.forward(theta, x, D, H), [10.0, 1.0])


def test_bf16_rounding():
    from oracle import mlp
    vals = np.array([1.0, 1.0 + 2**-8, 1.0 + 2**-7, 1.0 + 3 * 2**-8, -2.5, 3.1415927], np.float32)
    got = mlp.bf16(vals)
    # 1+2^-8 is the tie between 1 and 1+2^-7: rounds to even (1); 1+3*2^-8 rounds up to 1+2^-6
    assert got.tolist()[:5] == [1.0, 1.0, 1.0 + 2**-7, 1.0 + 2**-6, -2.5]
    assert abs(got[5] - 3.140625) < 1e-12


def test_sre_weights_and_features():
    p = small_params(seed=51, k=3)
    o = Oracle(p)
    rng = np.random.default_rng(51)
    o.scan(random_pairs(rng, 20000, n_src=50))
    hosts = np.unique(random_pairs(rng, 200, n_src=50)[:, 0])
    sre, _ = o.raw()
    w = o.sre_weights(hosts)
    for j, aip in enumerate(hosts.tolist()):
        for i in range(p.r):
            assert w[j, i] == (sre[i, o.rhfg(i, aip)] < p.k).sum()
    f = o.features(hosts)
    e = o.estimate(hosts, hist=True)
    assert f.shape == (len(hosts), p.k + 2)
    assert np.allclose(np.expm1(f[:, : p.k]).round(), e["hist"])
    assert np.allclose(np.expm1(f[:, p.k]).round(), w.sum(1))


def test_tabulation_rhfg0_structure_and_tables():
    """RHFG[0] by simple tabulation (the family Section 3.3 cites): the value is the XOR of
    four byte-indexed table entries drawn from SplitMix64 after the keys, so (i) changing
    one byte of the address changes the hash by an amount that does not depend on the other
    bytes, and (ii) RHFG[0](0) is the XOR of the first entry of each table."""
    p = oracle.Params(q=14, r2=5, seed=77, rhfg_hash=1)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(77)
    for j in range(4):
        a, b = rng.integers(0, 256, 2)
        diffs = set()
        for x in rng.integers(0, 2**32, 20, dtype=np.uint64).astype(np.uint32):
            x = int(x) & ~(0xFF << (8 * j))
            diffs.add(o.rhfg0(x | (int(a) << (8 * j))) ^ o.rhfg0(x | (int(b) << (8 * j))))
        assert len(diffs) == 1
    draws = oracle.splitmix64(77, 2 * (4 + p.r2) + 1024)[2 * (4 + p.r2):]
    tab = [[d >> 32 for d in draws[256 * j:256 * (j + 1)]] for j in range(4)]
    assert o.rhfg0(0) == (tab[0][0] ^ tab[1][0] ^ tab[2][0] ^ tab[3][0]) >> (32 - p.q)
    x = 0x12345678
    want = tab[0][0x78] ^ tab[1][0x56] ^ tab[2][0x34] ^ tab[3][0x12]
    assert o.rhfg0(x) == want >> (32 - p.q)
    # the RHFG chain of Eq. 6 and its inversion (Eq. 7) hold for any RHFG[0]
    for x in rng.integers(0, 2**32, 200, dtype=np.uint64).astype(np.uint32):
        he0 = o.rhfg0(int(x))
        for i in range(1, p.r):
            assert o.rhfg(i, int(x)) ^ he0 == (int(x) >> (i * o.delta)) & ((1 << p.q) - 1)


# ---------------------------------------------------------------- sanitizer build

SANITIZED_RUN = r"""
import numpy as np
import oracle
from paper_1805_09246_b300 import synth
tr = synth.Traffic(synth.small_trace(seed=3))
p = oracle.Params(k=3, seed=3)
a, b = oracle.Oracle(p, track_exact=True), oracle.Oracle(p)
for t in range(4):
    if t:
        a.advance(); b.advance()
    s = tr.slice(0, t)
    a.scan(s[::2]); b.scan(s[1::2])
a.merge([b])
det = a.detect()
assert len(det["hosts"]) > 0
e = a.estimate(det["hosts"], hist=True)
a.features(det["hosts"][:8]); a.sre_weights(det["hosts"][:8])
a.exact_counts(det["hosts"]); a.exact_super()
sre, sle = a.raw(); a.set_raw(sre, sle); a.canonical(); a.hot(); a.row_counts()
t = oracle.Oracle(oracle.Params(q=10, delta=8, q2=6, eta2=64, delta2=8, k=2, theta=8, seed=4, rhfg_hash=1))
few = tr.slice(0, 0)[:600].copy()
few[:, 0] %= 11  # eleven hosts: a handful of hot SREs per row
t.scan(few)
assert len(t.detect()["hosts"]) > 0
print("sanitized oracle ok", len(det["hosts"]))
"""


@pytest.mark.slow
def test_oracle_under_address_and_undefined_behavior_sanitizers(tmp_path):
    """The oracle built with -fsanitize=address,undefined (every report aborts) runs scan,
    advance, merge, detection, estimation with histograms, exact counts, raw state and the
    tabulation hash on a small trace in a child process."""
    import os
    import subprocess
    import sys
    lib = oracle.build(sanitize=True, out=str(tmp_path / "liborc_asan.so"))
    asan = subprocess.run(["g++", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run(["g++", "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    env = dict(os.environ, SSE_ORACLE_LIB=lib, LD_PRELOAD=f"{asan}:{ubsan}",
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", SANITIZED_RUN], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "sanitized oracle ok" in r.stdout
