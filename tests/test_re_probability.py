"""The rough estimator's detection probability (Section 3.2, Eq. 2-5): the oracle's closed
form pinned to brute force, textbook identities and normalisation, then compared with
Monte-Carlo runs of the oracle's own estimator (its hashes, sampling and cells)."""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import re_probability as rp


@pytest.mark.parametrize("eta", [1, 2, 3, 4])
def test_surjections_equal_brute_force(eta):
    for alpha in range(0, 8):
        brute = sum(1 for f in itertools.product(range(eta), repeat=alpha) if len(set(f)) == eta)
        assert rp.surjections(alpha, eta) == brute


def test_surjections_equal_inclusion_exclusion():
    for eta in range(1, 9):
        for alpha in range(eta, 41):
            closed = sum((-1) ** j * math.comb(eta, j) * (eta - j) ** alpha for j in range(eta + 1))
            assert rp.surjections(alpha, eta) == closed


def test_cells_set_distribution():
    """Eq. 2 is a distribution over eta1 whose mean is eta (1 - (1 - 1/eta)^alpha)."""
    eta = 8
    for alpha in [1, 2, 5, 8, 20, 60]:
        probs = [rp.pr_cells_set(alpha, eta, e) for e in range(eta + 1)]
        assert abs(sum(probs) - 1.0) < 1e-12
        mean = sum(e * q for e, q in enumerate(probs))
        assert abs(mean - eta * (1 - (1 - 1 / eta) ** alpha)) < 1e-12
    assert rp.pr_cells_set(3, 8, 4) == 0.0 and rp.pr_cells_set(0, 8, 0) == 1.0


def test_scan_distribution_is_normalised_and_monotone():
    eta, tau = 8, 7
    for n in [0, 50, 400, 1024, 4096]:
        probs = [rp.pr_cells_after_scan(n, eta, tau, e, alpha_max=400) for e in range(eta + 1)]
        assert abs(sum(probs) - 1.0) < 1e-9
    # more destinations -> more likely reported
    reported = [rp.pr_reported(n, eta, tau, 3, alpha_max=400) for n in [100, 400, 1024, 2048, 4096]]
    assert all(a < b for a, b in zip(reported, reported[1:]))
    assert reported[2] > 0.6 and reported[-1] > 0.999  # theta = 1024 hosts are reported with high probability


def _lone_hosts(n_hosts, n_dst, seed):
    rng = np.random.default_rng(seed)
    hosts = np.unique(rng.integers(0, 2**32, n_hosts, dtype=np.uint64).astype(np.uint32))
    pairs = np.stack([np.repeat(hosts, n_dst),
                      rng.integers(0, 2**32, len(hosts) * n_dst, dtype=np.uint64).astype(np.uint32)], 1)
    return hosts, pairs


def _unshared(orc, hosts):
    """Hosts whose row-0 SRE no other host of the set uses (no collisions)."""
    cols = np.array([orc.rhfg(0, int(h)) for h in hosts])
    _, inv, counts = np.unique(cols, return_inverse=True, return_counts=True)
    return counts[inv] == 1


@pytest.mark.parametrize("n_dst", [400, 1024, 2048])
def test_oracle_estimator_matches_eq5(n_dst):
    """Monte Carlo: lone hosts with n distinct destinations in one slice (k = 1); the
    distribution of their SRE weights (set cells of 8) follows Eq. 4, and the share
    reported hot (>= 3 cells) Eq. 5, within 4.5 standard errors."""
    p = oracle.Params(q=17, k=1, theta=1024, seed=31 + n_dst)
    orc = oracle.Oracle(p)
    hosts, pairs = _lone_hosts(600, n_dst, seed=n_dst)
    orc.scan(pairs)
    keep = _unshared(orc, hosts)
    w = orc.sre_weights(hosts[keep])[:, 0]
    m = len(w)
    tau = oracle.derive(p)["tau"]
    for e in range(9):
        q = rp.pr_cells_after_scan(n_dst, 8, tau, e, alpha_max=400)
        got = np.mean(w == e)
        assert abs(got - q) <= 4.5 * math.sqrt(max(q * (1 - q), 1e-4) / m), (e, got, q)
    q = rp.pr_reported(n_dst, 8, tau, 3, alpha_max=400)
    got = np.mean(w >= 3)
    assert abs(got - q) <= 4.5 * math.sqrt(q * (1 - q) / m + 1e-6), (got, q)
