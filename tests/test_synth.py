"""The seeded traffic generator: published Philox answers, determinism, recipe shape."""
import numpy as np

from paper_1805_09246_b300 import synth
from tests.conftest import read_golden


def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        out = synth.philox4x32_10(vals[0:4], vals[4:6])
        assert out.tolist() == vals[6:10]


def test_deterministic_across_thread_counts():
    cfg = synth.small_trace(seed=3)
    a = synth.Traffic(cfg, threads=1).slice(0, 2)
    b = synth.Traffic(cfg, threads=7).slice(0, 2)
    assert np.array_equal(a, b)


def test_small_trace_shape():
    tr = synth.Traffic(synth.small_trace())
    ip, card = tr.planted()
    assert len(ip) == 20 and len(set(ip.tolist())) == 20
    assert card.min() >= 2000 and card.max() <= 20000
    total_planted = 0
    for t in range(8):
        s = tr.slice(0, t)
        assert s.shape == (1 << 17, 2)
        total_planted += tr.planted_in(0, t)
        # planted pairs are present with their own source addresses
        assert np.isin(s[:, 0], ip).sum() == tr.planted_in(0, t)
    assert total_planted == card.sum()
    # background sources come from a 50k population, popular ones repeat (Zipf)
    bg = np.concatenate([tr.slice(0, t) for t in range(2)])
    bg = bg[~np.isin(bg[:, 0], ip)]
    srcs, counts = np.unique(bg[:, 0], return_counts=True)
    assert len(srcs) < 50_000 and counts.max() > 1000
    # every background source has at most 50 distinct destinations
    per_src = np.unique(np.unique(bg, axis=0)[:, 0], return_counts=True)[1]
    assert per_src.max() <= 50


def test_planted_destinations_are_distinct_and_sent_once():
    tr = synth.Traffic(synth.small_trace(seed=1))
    ip, card = tr.planted()
    allp = np.concatenate([tr.slice(0, t) for t in range(8)])
    for h, c in zip(ip.tolist()[:5], card.tolist()[:5]):
        d = allp[allp[:, 0] == h, 1]
        assert len(d) == c
        assert len(np.unique(d)) >= c - 2  # 32-bit random destinations; collisions are rare


def test_uneven_router_loads():
    cfg = synth.TrafficConfig(seed=2, n_slices=3, n_routers=4, load_min=1 << 12, load_max=1 << 16,
                              n_sources=10_000, n_planted=5, planted_min=100, planted_max=300,
                              group_min=1, group_max=3)
    tr = synth.Traffic(cfg)
    lens = [tr.slice_len(r, t) for r in range(4) for t in range(3)]
    assert min(lens) >= 1 << 12 and max(lens) <= 1 << 16 and len(set(lens)) > 3
    ip, card = tr.planted()
    seen = sum(np.isin(tr.slice(r, t)[:, 0], ip).sum() for r in range(4) for t in range(3))
    assert seen == card.sum()
