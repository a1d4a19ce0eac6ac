"""Learned-correction episodes: the host generator's streams and the exact window
cardinalities that serve as training targets, checked against the oracle's exact sliding
distinct counts (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300.synth import episodes as ep


def small_cfg(**kw):
    base = dict(hosts=6, k=16, query_slice=23, card_min=50, card_max=3000, active_max=24, noise_pairs=700)
    base.update(kw)
    return ep.EpisodeConfig(**base)


def test_layout_and_streams():
    cfg = small_cfg()
    t = ep.sample_hosts(cfg, 3, np.random.default_rng(5))
    assert (t.ip >> 31 == 1).all()
    for r in range(3):
        assert len(np.unique(t.ip[r * 6:(r + 1) * 6])) == 6
    total = np.zeros(t.ip.size, np.uint64)
    for s in range(cfg.query_slice + 1):
        pairs, per_router = ep.fill_cpu(t, s, cfg.noise_pairs, seed=9)
        counts = ep.slice_counts(t, s)
        total += counts
        host_off, noise_off, _ = ep.layout(t, s, cfg.noise_pairs)
        assert len(pairs) == per_router.sum() == counts.sum() + 3 * cfg.noise_pairs
        for h in range(t.ip.size):
            seg = pairs[int(host_off[h]):int(host_off[h] + counts[h])]
            assert (seg[:, 0] == t.ip[h]).all()
            assert len(np.unique(seg[:, 1])) == len(seg)
        for r in range(3):
            noise = pairs[int(noise_off[r]):int(noise_off[r]) + cfg.noise_pairs]
            assert (noise[:, 0] >> 31 == 0).all()
    assert np.array_equal(total, t.card.astype(np.uint64))  # every destination sent exactly once


def test_streams_depend_on_seed_slice_and_router():
    cfg = small_cfg(noise_pairs=64)
    t = ep.sample_hosts(cfg, 2, np.random.default_rng(6))
    a, _ = ep.fill_cpu(t, 20, 64, seed=1)
    b, _ = ep.fill_cpu(t, 20, 64, seed=2)
    c, _ = ep.fill_cpu(t, 21, 64, seed=1)
    _, noise_off, _ = ep.layout(t, 20, 64)
    n0 = a[int(noise_off[0]):int(noise_off[0]) + 64]
    n1 = a[int(noise_off[1]):int(noise_off[1]) + 64]
    assert not np.array_equal(n0, n1)
    assert not np.array_equal(a, b)
    assert not np.array_equal(a[-64:], c[-64:])


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_window_equals_oracle_exact_counts(seed):
    """The training targets are the oracle's exact sliding distinct counts of the same
    traffic: the episode's slices scanned by an exact-tracking oracle, queried at slice Q."""
    cfg = small_cfg()
    t = ep.sample_hosts(cfg, 2, np.random.default_rng(seed))
    o = [oracle.Oracle(oracle.Params(k=cfg.k, seed=seed), track_exact=True) for _ in range(2)]
    for s in range(cfg.query_slice + 1):
        pairs, per_router = ep.fill_cpu(t, s, cfg.noise_pairs, seed=100 + seed)
        start = 0
        for r in range(2):
            if s:
                o[r].advance()
            o[r].scan(pairs[start:start + int(per_router[r])])
            start += int(per_router[r])
    exact = ep.exact_window(t, cfg.query_slice - cfg.k + 1, cfg.query_slice)
    got = np.concatenate([o[r].exact_counts(t.ip[r * 6:(r + 1) * 6]) for r in range(2)])
    assert np.array_equal(got.astype(np.uint64), exact)
    assert (exact > 0).all()
    # and the window shares of the scaled cardinalities stay within a destination of the drawn target
    w = exact.astype(np.float64)
    assert (w >= cfg.card_min - 1).all() and (w <= cfg.card_max + 1).all()
