"""Training episodes for the learned cardinality correction (inputs only; no estimator
arithmetic).

An episode is one router's traffic over slices 0..Q: ``hosts`` planted hosts, each with an
address whose top bit is set, a total cardinality ``card`` and an activity interval
``first..last``, plus background noise (sources with the top bit clear). Host h sends
destinations j = 0..card-1, spread evenly over its active slices (in slice s the j with
floor(card*(s-first)/L) <= j < floor(card*(s-first+1)/L), L = last-first+1), and each j
maps to a distinct destination address, so the exact number of distinct destinations a
host contacts in any window of slices is known by construction (``exact_window``).

The host tables are drawn here with numpy; the pairs themselves are written by
``libsynth_gpu.so`` (``synth_gpu.cu``) on the device, or by its host twin for checks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth_gpu.cu")
_LIB = os.path.join(_HERE, "libsynth_gpu.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def build(force: bool = False) -> str:
    """Compile ``libsynth_gpu.so`` in place for sm_103a (nvcc cross-compiles without a GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = [NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
               "-shared", "-Xcompiler", "-fPIC", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.synth_gpu_hosts.argtypes = [vp, vp, vp, vp, vp, u32, u32, u64, vp, vp]
        lib.synth_gpu_hosts.restype = ctypes.c_int
        lib.synth_gpu_noise.argtypes = [vp, u32, u64, u32, u64, vp, vp]
        lib.synth_gpu_noise.restype = ctypes.c_int
        lib.synth_cpu_hosts.argtypes = [vp, vp, vp, vp, vp, u32, u32, u64, vp]
        lib.synth_cpu_hosts.restype = None
        lib.synth_cpu_noise.argtypes = [vp, u32, u64, u32, u64, vp]
        lib.synth_cpu_noise.restype = None
        _lib = lib
    return _lib


@dataclass
class EpisodeConfig:
    """Recipe of the learned correction's episodes (window k = 16, query at slice Q)."""
    hosts: int = 24               # planted hosts per episode
    k: int = 16                   # window length (slices)
    query_slice: int = 23         # Q: slices 0..Q are scanned, the window is Q-k+1..Q
    card_min: float = 1e2         # exact window cardinality, log-uniform in [card_min, card_max]
    card_max: float = 1e6
    active_max: int = 24          # longest activity interval (slices)
    p_until_query: float = 0.6    # share of hosts still active at the query slice
    noise_pairs: int = 1 << 14    # background pairs per slice (a fifth of an SLE row over the window)


@dataclass
class HostTable:
    """Planted hosts of a group of episodes (one episode per router), flat [routers*hosts]."""
    ip: np.ndarray      # uint32, top bit set, distinct within an episode
    card: np.ndarray    # uint32 total distinct destinations
    first: np.ndarray   # uint32 first active slice
    last: np.ndarray    # uint32 last active slice
    routers: int
    hosts: int


def sample_hosts(cfg: EpisodeConfig, routers: int, rng: np.random.Generator) -> HostTable:
    """Draws `routers` episodes' hosts: the window cardinality log-uniform, the activity
    interval ending inside the window (at Q with probability p_until_query) and of uniform
    length 1..active_max (so some hosts started before the window), and the total
    cardinality scaled from the window's share of the activity."""
    n = routers * cfg.hosts
    Q, k = cfg.query_slice, cfg.k
    lo_w = Q - k + 1
    w = np.exp(rng.uniform(np.log(cfg.card_min), np.log(cfg.card_max), n))
    last = np.where(rng.random(n) < cfg.p_until_query, Q, rng.integers(lo_w, Q + 1, n))
    length = rng.integers(1, cfg.active_max + 1, n)
    first = np.maximum(last - length + 1, 0)
    L = last - first + 1
    overlap = last - np.maximum(first, lo_w) + 1
    card = np.maximum(np.rint(w * L / overlap), 1).astype(np.uint64)
    card = np.minimum(card, np.uint64(2**31)).astype(np.uint32)
    ip = np.empty(n, np.uint32)
    for r in range(routers):  # distinct addresses within each episode
        sl = slice(r * cfg.hosts, (r + 1) * cfg.hosts)
        while True:
            cand = rng.integers(0, 1 << 31, cfg.hosts, dtype=np.uint64).astype(np.uint32) | np.uint32(0x80000000)
            if len(np.unique(cand)) == cfg.hosts:
                ip[sl] = cand
                break
    return HostTable(ip=ip, card=card, first=first.astype(np.uint32), last=last.astype(np.uint32),
                     routers=routers, hosts=cfg.hosts)


def slice_counts(t: HostTable, s: int) -> np.ndarray:
    """Pairs each host sends in slice s (uint64 [routers*hosts])."""
    c = t.card.astype(np.uint64)
    first = t.first.astype(np.int64)
    L = (t.last.astype(np.int64) - first + 1).astype(np.uint64)
    active = (s >= t.first) & (s <= t.last)
    rel = np.where(active, s - first, 0).astype(np.uint64)
    n = c * (rel + np.uint64(1)) // L - c * rel // L
    return np.where(active, n, 0).astype(np.uint64)


def exact_window(t: HostTable, lo: int, hi: int) -> np.ndarray:
    """Distinct destinations each host contacts in slices lo..hi (by construction)."""
    c = t.card.astype(np.uint64)
    first = t.first.astype(np.int64)
    L = (t.last.astype(np.int64) - first + 1).astype(np.uint64)
    a = np.maximum(first, lo)
    b = np.minimum(t.last.astype(np.int64), hi)
    ok = a <= b
    j_hi = c * np.where(ok, b - first + 1, 0).astype(np.uint64) // L
    j_lo = c * np.where(ok, a - first, 0).astype(np.uint64) // L
    return np.where(ok, j_hi - j_lo, 0).astype(np.uint64)


def layout(t: HostTable, s: int, noise_pairs: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Pair offsets of one slice in a buffer holding every router's pairs back to back
    (router r: its hosts' pairs, then its noise): (host offsets [routers*hosts], noise
    offsets [routers], pairs per router [routers])."""
    n = slice_counts(t, s).reshape(t.routers, t.hosts)
    per_router = n.sum(axis=1) + np.uint64(noise_pairs)
    start = np.concatenate([[0], np.cumsum(per_router)[:-1]]).astype(np.uint64)
    host_off = (start[:, None] + np.concatenate([np.zeros((t.routers, 1), np.uint64),
                                                 np.cumsum(n, axis=1)[:, :-1]], axis=1)).reshape(-1)
    noise_off = start + n.sum(axis=1)
    return host_off.astype(np.uint64), noise_off.astype(np.uint64), per_router.astype(np.uint64)


def fill_cpu(t: HostTable, s: int, noise_pairs: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Host twin of the device generator: (pairs [total, 2] uint32, pairs per router)."""
    lib = _load()
    host_off, noise_off, per_router = layout(t, s, noise_pairs)
    out = np.zeros((int(per_router.sum()), 2), np.uint32)
    arrs = [np.ascontiguousarray(a) for a in (t.ip, t.card, t.first, t.last, host_off, noise_off)]
    lib.synth_cpu_hosts(*[a.ctypes.data for a in arrs[:5]], t.routers * t.hosts, s, seed, out.ctypes.data)
    lib.synth_cpu_noise(arrs[5].ctypes.data, t.routers, noise_pairs, s, seed, out.ctypes.data)
    return out, per_router


class DeviceTable:
    """A HostTable resident on the device, with a pair buffer that grows as needed."""

    def __init__(self, t: HostTable, device="cuda"):
        import torch
        self.t = t
        self.torch = torch
        self.device = device
        as_t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(device)
        self.ip, self.card, self.first, self.last = (as_t(a) for a in (t.ip, t.card, t.first, t.last))
        self.buf = torch.empty(0, dtype=torch.int32, device=device)

    def fill(self, s: int, noise_pairs: int, seed: int):
        """Writes slice s's pairs on the current stream; returns one (n_r, 2) int32 view per router."""
        torch = self.torch
        lib = _load()
        host_off, noise_off, per_router = layout(self.t, s, noise_pairs)
        total = int(per_router.sum())
        if self.buf.numel() < 2 * total:
            self.buf = torch.empty(2 * total + (1 << 20), dtype=torch.int32, device=self.device)
        offs = torch.from_numpy(np.concatenate([host_off, noise_off]).view(np.int64)).to(self.device)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        n_hosts = self.t.routers * self.t.hosts
        rc = lib.synth_gpu_hosts(self.ip.data_ptr(), self.card.data_ptr(), self.first.data_ptr(),
                                 self.last.data_ptr(), offs.data_ptr(), n_hosts, s, seed, self.buf.data_ptr(), stream)
        rc |= lib.synth_gpu_noise(offs.data_ptr() + 8 * n_hosts, self.t.routers, noise_pairs, s, seed,
                                  self.buf.data_ptr(), stream)
        if rc:
            raise RuntimeError("synth_gpu launch failed")
        self._offs = offs  # kept alive until the kernels have run
        views, start = [], 0
        for n in per_router.tolist():
            views.append(self.buf[2 * start: 2 * (start + n)].view(n, 2))
            start += n
        return views
