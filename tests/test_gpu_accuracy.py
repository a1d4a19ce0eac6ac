"""Sliding-window accuracy (Section 5: FPR, FNR, TFR against exact window cardinalities) of
the GPU estimator on synthetic traffic, at a 16-slice window with 8-bit stamps and at the
paper's parameters (k = 300, 16-bit stamps). The bounds are loose regression guards; the
measured values are printed (run with -s)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(params, cfg):
    from paper_1805_09246_b300 import accuracy
    res = accuracy.sliding_accuracy(params, cfg)
    s = accuracy.summary(res)
    print(f"\n{params.k}-slice window, {params.stamp_bits}-bit stamps: {s}")
    return res, s


def test_accuracy_16_slice_window():
    from paper_1805_09246_b300 import accuracy, sse
    p = sse.core_link_params(k=16, seed=51)
    res, s = run(p, accuracy.AccuracyConfig(slices=64, seed=51))
    assert s["windows"] == 64 - 15 and s["mean_true_super"] > 10
    assert s["fnr"] < 0.1 and s["tfr"] < 0.3


def test_accuracy_paper_parameters_k300():
    from paper_1805_09246_b300 import accuracy, sse
    p = sse.paper_params(k=300)
    p.seed = 52
    cfg = accuracy.AccuracyConfig(slices=320, hosts=150, active_max=200, noise_pairs=1 << 11, seed=52)
    res, s = run(p, cfg)
    assert s["windows"] == 21 and s["mean_true_super"] > 10
    assert s["fnr"] < 0.1 and s["tfr"] < 0.3
