"""Sliding-window detection accuracy (FPR, FNR and TFR, the paper's Section 5 definitions)
of the GPU estimator against exact sliding cardinalities.

Traffic: planted hosts whose destinations are distinct by construction and spread evenly
over an activity interval (``synth.episodes``), so the exact number a host contacts in
any window is a closed form, plus background noise whose sources never reach the
threshold. Each slice is scanned and closed; the reported super points of the window
ending there are compared with the hosts whose exact window cardinality reaches theta:
FPR = false positives / true super points, FNR = missed / true super points, TFR = FPR +
FNR. Every step runs in the library's kernels; this module only marshals.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import sse
from .synth import episodes as ep


@dataclass
class AccuracyConfig:
    """Recipe of the sliding-accuracy traffic."""
    slices: int = 64              # slices scanned (windows end at every slice)
    hosts: int = 150              # planted hosts
    card_min: float = 256.0       # total destinations per host, log-uniform (theta / 4 .. 16 theta)
    card_max: float = 16384.0
    active_max: int = 24          # activity interval length, 1..active_max slices
    noise_pairs: int = 1 << 14    # background pairs per slice (sources of one destination)
    seed: int = 0


def sample_hosts(cfg: AccuracyConfig, rng: np.random.Generator) -> ep.HostTable:
    """Hosts with distinct addresses (top bit set), activity intervals starting anywhere in
    the run and total cardinalities log-uniform in [card_min, card_max]."""
    n = cfg.hosts
    first = rng.integers(0, cfg.slices, n)
    length = rng.integers(1, cfg.active_max + 1, n)
    last = np.minimum(first + length - 1, cfg.slices - 1)
    card = np.rint(np.exp(rng.uniform(np.log(cfg.card_min), np.log(cfg.card_max), n))).astype(np.uint32)
    while True:
        ip = rng.integers(0, 1 << 31, n, dtype=np.uint64).astype(np.uint32) | np.uint32(0x80000000)
        if len(np.unique(ip)) == n:
            break
    return ep.HostTable(ip=ip, card=np.maximum(card, 1), first=first.astype(np.uint32), last=last.astype(np.uint32),
                        routers=1, hosts=n)


@dataclass
class WindowResult:
    slice: int
    true_super: int
    reported: int
    false_pos: int
    false_neg: int

    @property
    def fpr(self) -> float:
        return self.false_pos / self.true_super if self.true_super else 0.0

    @property
    def fnr(self) -> float:
        return self.false_neg / self.true_super if self.true_super else 0.0

    @property
    def tfr(self) -> float:
        return self.fpr + self.fnr


def sliding_accuracy(params: sse.Params, cfg: AccuracyConfig, warm: int | None = None) -> list[WindowResult]:
    """Scans cfg.slices slices and returns the accuracy of every window that ends at slice
    >= warm (default: once the window is full, k - 1)."""
    import torch
    rng = np.random.default_rng(cfg.seed)
    table = sample_hosts(cfg, rng)
    dev = ep.DeviceTable(table)
    est = sse.Estimator(params)
    k = params.k
    warm = k - 1 if warm is None else warm
    planted = table.ip
    out = []
    for s in range(cfg.slices):
        (pairs,) = dev.fill(s, cfg.noise_pairs, cfg.seed + 1)
        torch.cuda.current_stream().synchronize()
        est.update(pairs)
        rep = est.close_slice()
        if s < warm:
            continue
        exact = ep.exact_window(table, max(0, s - k + 1), s)
        truth = set(planted[exact >= params.theta].tolist())
        found = set(rep.hosts[(rep.flags & sse.FLAG_SUPER) != 0].tolist())
        out.append(WindowResult(slice=s, true_super=len(truth), reported=len(found),
                                false_pos=len(found - truth), false_neg=len(truth - found)))
    return out


def summary(results: list[WindowResult]) -> dict:
    return dict(windows=len(results),
                mean_true_super=float(np.mean([r.true_super for r in results])),
                fpr=float(np.mean([r.fpr for r in results])), fnr=float(np.mean([r.fnr for r in results])),
                tfr=float(np.mean([r.tfr for r in results])))
