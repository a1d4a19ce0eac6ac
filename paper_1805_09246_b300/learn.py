"""Learned cardinality correction: episodes on the GPU, training with the library's own MLP
kernels, and scoring against linear counting.

The pipeline, every step of which runs in libsse's kernels (this module only marshals):

1. ``episodes``: groups of independent episodes, one per router of an ``sse.Batch`` in
   routers-only mode, scan slices 0..Q of generated traffic (the last slice is left open,
   so the window is Q-k+1..Q); each planted host is then queried on its router for its
   features (``sse_features``) and linear-counting estimate (Algorithm 8, ``sse_query``).
   The exact window cardinality comes from the generator's construction.
2. ``train``: the network maps features to log(exact) - log(max(LC, 1)); minibatch Adam
   epochs (``sse_mlp_train_epoch``) over host-shuffled permutations.
3. ``evaluate``: fresh episodes queried with ``sse_query_learned`` (learned estimate with the
   linear-counting fallback) and the median relative error of both estimates.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import sse
from .synth import episodes as ep


def learned_params(k: int = 16, seed: int = 0) -> sse.Params:
    """Estimator shapes of the learned-correction runs: core-link sizes (SRE rows of 2^20,
    2^16 SLEs of 2^12 cells) with a 16-slice window."""
    return sse.core_link_params(k=k, seed=seed)


@dataclass
class Samples:
    """Per-host results of a set of episodes (device tensors unless noted)."""
    x: object            # float32 [n, k + 2] features
    lc: object           # float32 [n] linear-counting estimate
    flags: object        # uint8 [n]
    exact: np.ndarray    # float64 [n] exact window cardinality (host)
    learned: object = None  # float32 [n] learned estimate, when a network was given
    seconds: dict = field(default_factory=dict)


def draw_group(cfg: ep.EpisodeConfig, routers: int, rng: np.random.Generator) -> tuple[ep.HostTable, int]:
    """One group of episodes: its host table and the seed of its pair streams."""
    table = ep.sample_hosts(cfg, routers, rng)
    return table, int(rng.integers(0, 2**63))


def episodes(params: sse.Params, cfg: ep.EpisodeConfig, n_hosts: int, routers: int = 64, seed: int = 0,
             mlp: "sse.MLP | None" = None) -> Samples:
    """Runs ceil(n_hosts / (routers * cfg.hosts)) groups of episodes and returns the first
    n_hosts hosts' samples."""
    import torch
    assert params.k == cfg.k
    rng = np.random.default_rng(seed)
    batch = sse.Batch(params, routers, 1)
    H = cfg.hosts
    per_group = routers * H
    groups = -(-n_hosts // per_group)
    xs, lcs, fls, exs, les = [], [], [], [], []
    t_scan = t_query = 0.0
    Q = cfg.query_slice
    for g in range(groups):
        table, gseed = draw_group(cfg, routers, rng)
        dev = ep.DeviceTable(table)
        t0 = time.perf_counter()
        batch.reset()
        for s in range(Q + 1):
            views = dev.fill(s, cfg.noise_pairs, gseed)
            batch.set_mode(sse.BATCH_SCAN if s == Q else sse.BATCH_ROUTERS)
            batch.step(inputs=views)
        t1 = time.perf_counter()
        x = torch.empty((per_group, params.k + 2), dtype=torch.float32, device="cuda")
        outs = []
        for r in range(routers):  # the routers share the batch's stream
            e = batch.router(r)
            h = dev.ip[r * H:(r + 1) * H]
            e.features(h, out=x[r * H:(r + 1) * H])
            outs.append(e.query_learned(mlp, h) if mlp is not None else e.query(h))
        batch.router(0).sync()
        if mlp is not None:
            le = torch.cat([o[0] for o in outs])
            lc = torch.cat([o[1] for o in outs])
            fl = torch.cat([o[2] for o in outs])
        else:
            le = None
            lc = torch.cat([o[0] for o in outs])
            fl = torch.cat([o[1] for o in outs])
        torch.cuda.synchronize()
        t_query += time.perf_counter() - t1
        t_scan += t1 - t0
        xs.append(x)
        lcs.append(lc)
        fls.append(fl)
        exs.append(ep.exact_window(table, Q - cfg.k + 1, Q).astype(np.float64))
        if le is not None:
            les.append(le)
    batch.close()
    cat = lambda a: torch.cat(a)[:n_hosts]
    return Samples(x=cat(xs), lc=cat(lcs), flags=cat(fls), exact=np.concatenate(exs)[:n_hosts],
                   learned=cat(les) if les else None, seconds={"scan": t_scan, "query": t_query})


def targets(s: Samples):
    """Training target: log(exact) - log(max(LC, 1)) (float32 device tensor)."""
    import torch
    exact = torch.from_numpy(s.exact).to(s.lc.device)
    return (torch.log(exact) - torch.log(torch.clamp(s.lc.double(), min=1.0))).float().contiguous()


def train(mlp: "sse.MLP", x, t, epochs: int = 30, batch: int = 512, lr: float = 1e-3, seed: int = 0,
          decay: float = 0.9, rows: np.ndarray | None = None, first_epoch: int = 0,
          rng: np.random.Generator | None = None) -> list[float]:
    """Minibatch Adam epochs first_epoch .. first_epoch+epochs-1 (learning rate lr * decay^e)
    on the GPU over `rows` (default: all samples); the order of each epoch is drawn on the
    host."""
    import torch
    rng = np.random.default_rng(seed) if rng is None else rng
    rows = np.arange(x.shape[0]) if rows is None else np.asarray(rows)
    losses = []
    for e in range(first_epoch, first_epoch + epochs):
        perm = torch.from_numpy(rng.permutation(rows).astype(np.int32)).to(x.device)
        losses.append(mlp.train_epoch(x, t, perm, batch, lr * decay**e))
    return losses


def active_cells(x, k: int) -> np.ndarray:
    """Active union-SLE cells of each sample, recovered from its features (as the gate does)."""
    xs = x[:, :k].double().cpu().numpy() if hasattr(x, "cpu") else np.asarray(x, np.float64)[:, :k]
    return np.rint(np.expm1(xs)).sum(axis=1)


def choose_gate(lc: np.ndarray, y: np.ndarray, exact: np.ndarray, active: np.ndarray, eta2: int,
                fills=(0.0, 0.5, 0.8, 0.9, 0.95, 0.97, 0.98, 0.99, 0.995, 0.998, 1.0)) -> int:
    """The gate (minimum active cells) that minimises the median relative error of the
    combined estimate on the given (training) samples."""
    lc = np.asarray(lc, np.float64)
    net = np.maximum(lc, 1.0) * np.exp(np.asarray(y, np.float64))
    best, best_err = eta2 + 1, np.inf
    for f in fills:
        gate = int(np.ceil(f * eta2))
        est = np.where(active >= gate, net, lc)
        err = float(np.median(np.abs(est - exact) / exact))
        if err < best_err:
            best, best_err = gate, err
    return best


def feature_max(x) -> np.ndarray:
    """Per-feature maxima of the training features (the range outside which the learned
    estimate falls back to linear counting)."""
    return x.max(dim=0).values.cpu().numpy()


def median_rel_error(est, exact: np.ndarray) -> float:
    e = est.double().cpu().numpy() if hasattr(est, "cpu") else np.asarray(est, np.float64)
    return float(np.median(np.abs(e - exact) / exact))


def run(n_train: int = 1_000_000, n_test: int = 100_000, routers: int = 64, epochs: int = 30,
        cfg: ep.EpisodeConfig | None = None, seed: int = 0, hidden: int = 64, train_min_fill: float = 0.9,
        batch: int = 512, lr: float = 1e-3) -> dict:
    """End to end: training episodes, training (on the samples whose union SLE is at least
    train_min_fill full, where linear counting degrades), the gate chosen on the training
    samples, held-out episodes, median relative errors."""
    import torch
    cfg = cfg or ep.EpisodeConfig()
    params = learned_params(cfg.k, seed=seed)
    t0 = time.perf_counter()
    tr = episodes(params, cfg, n_train, routers=routers, seed=seed)
    t1 = time.perf_counter()
    mlp = sse.MLP(params.k + 2, hidden=hidden, max_batch=1 << 16, seed=seed + 1)
    tt = targets(tr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    act = active_cells(tr.x, params.k)
    rows = np.nonzero(act >= train_min_fill * params.eta2)[0]
    losses = train(mlp, tr.x, tt, epochs=epochs, seed=seed + 2, rows=rows, batch=batch, lr=lr)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    mlp.set_feature_max(feature_max(tr.x))
    y = mlp.forward(tr.x).cpu().numpy()
    gate = choose_gate(tr.lc.cpu().numpy(), y, tr.exact, act, params.eta2)
    mlp.set_gate(gate)
    te = episodes(params, cfg, n_test, routers=routers, seed=seed + 1000, mlp=mlp)
    t4 = time.perf_counter()
    return dict(mlp=mlp, train=tr, test=te, losses=losses, gate=gate, trained_on=len(rows),
                err_lc=median_rel_error(te.lc, te.exact), err_learned=median_rel_error(te.learned, te.exact),
                seconds=dict(train_episodes=t1 - t0, training=t3 - t2, test_episodes=t4 - t3),
                samples_per_s=len(rows) * epochs / max(t3 - t2, 1e-9))
