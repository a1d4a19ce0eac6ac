"""Seeded request streams for the serving loop (inputs only).

Each router's pairs come from the synthetic trace generator; they are cut into batches of
log-uniform size and given Poisson arrival times so that the routers together offer a
fixed aggregate packet rate. A request is (time, router, start, size): the batch is pairs
start .. start+size-1 of the router's pool, wrapping around.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth


@dataclass
class RequestStream:
    pools: list  # per router: uint32 array (pool_pairs, 2)
    requests: list  # (time, router, start, size), by time

    def pairs(self, router: int, start: int, size: int) -> np.ndarray:
        pool = self.pools[router]
        if start + size <= len(pool):
            return pool[start:start + size]
        return np.take(pool, np.arange(start, start + size), axis=0, mode="wrap")


def poisson_requests(n_routers: int, duration_s: float, offered_pps: float, batch_min: int, batch_max: int,
                     pool_pairs: int | None = None, seed: int = 0, wrap: bool = True) -> RequestStream:
    """pool_pairs=None sizes every router's pool to its whole request stream, so no batch
    wraps around and every batch is a contiguous view of the pool. With wrap=False a batch
    that would run past the end of its pool starts at the pool's beginning instead, so
    every batch is a contiguous view of the pool whatever its size (pool_pairs must be at
    least batch_max)."""
    rng = np.random.default_rng(seed)
    mean_batch = (batch_max - batch_min) / np.log(batch_max / batch_min)
    rate = offered_pps / n_routers / mean_batch  # batches per second per router
    plan = []
    for r in range(n_routers):
        t = 0.0
        while True:
            t += rng.exponential(1.0 / rate)
            if t >= duration_s:
                break
            plan.append((t, r, int(np.exp(rng.uniform(np.log(batch_min), np.log(batch_max))))))
    per_router = np.zeros(n_routers, np.int64)
    for _, r, size in plan:
        per_router[r] += size
    pool = int(pool_pairs or max(1, per_router.max()))
    cfg = synth.TrafficConfig(seed=seed, n_slices=1, n_routers=n_routers, load_min=pool, load_max=pool,
                              n_sources=200_000, zipf_s=1.05, n_planted=4 * n_routers, planted_min=2000,
                              planted_max=20000, group_min=1, group_max=min(8, n_routers))
    tr = synth.Traffic(cfg)
    pools = [tr.slice(r, 0) for r in range(n_routers)]
    if not wrap and pool < batch_max:
        raise ValueError("pool_pairs below batch_max with wrap=False")
    reqs, pos = [], np.zeros(n_routers, np.int64)
    for t, r, size in plan:
        if not wrap and pos[r] + size > pool:
            pos[r] = 0
        reqs.append((t, r, int(pos[r]), size))
        pos[r] = (pos[r] + size) % pool
    reqs.sort(key=lambda x: (x[0], x[1]))
    return RequestStream(pools, reqs)
