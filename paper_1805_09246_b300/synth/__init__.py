"""Seeded synthetic IP-pair traffic (inputs only; no estimator arithmetic).

The generator is a small C++ library (``synth.cpp``) driven through ctypes. Both the
CUDA library's callers and the CPU oracle read its output as plain ``uint32`` arrays of
shape ``(n, 2)`` holding ``(src, dst)``; the source address plays the role of ``aip``
and the destination that of ``bip``.

Workload presets follow the sizes the method is evaluated at: ``small_trace`` (one
router, 8 slices of 2^17 pairs, the size the CPU oracle checks in seconds),
``core_link`` (one router, 64 slices of 2^25 pairs), ``edge_routers`` (16 routers with
uneven loads whose super points are split across router groups).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cpp")
_LIB = os.path.join(_HERE, "libsynth.so")


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` in place (g++, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", _LIB, _SRC]
        subprocess.run(cmd, check=True)
    return _LIB


class _Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_slices", ctypes.c_uint32),
        ("n_routers", ctypes.c_uint32),
        ("load_min", ctypes.c_uint64),
        ("load_max", ctypes.c_uint64),
        ("n_sources", ctypes.c_uint32),
        ("bg_dst_min", ctypes.c_uint32),
        ("bg_dst_max", ctypes.c_uint32),
        ("n_planted", ctypes.c_uint32),
        ("planted_min", ctypes.c_uint32),
        ("planted_max", ctypes.c_uint32),
        ("planted_log", ctypes.c_uint32),
        ("group_min", ctypes.c_uint32),
        ("group_max", ctypes.c_uint32),
        ("planted_slice_lo", ctypes.c_uint32),
        ("planted_slice_hi", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("zipf_s", ctypes.c_double),
    ]


@dataclass
class TrafficConfig:
    """Recipe of one synthetic trace (all counts are pairs or hosts)."""
    seed: int = 0
    n_slices: int = 8
    n_routers: int = 1
    load_min: int = 1 << 17
    load_max: int = 1 << 17
    n_sources: int = 50_000
    zipf_s: float = 1.1
    bg_dst_min: int = 1
    bg_dst_max: int = 50
    n_planted: int = 20
    planted_min: int = 2000
    planted_max: int = 20000
    planted_log: bool = False
    group_min: int = 1
    group_max: int = 1
    planted_slice_lo: int = 0
    planted_slice_hi: int | None = None

    def to_c(self) -> _Config:
        hi = self.n_slices if self.planted_slice_hi is None else self.planted_slice_hi
        return _Config(self.seed, self.n_slices, self.n_routers, self.load_min, self.load_max,
                       self.n_sources, self.bg_dst_min, self.bg_dst_max, self.n_planted,
                       self.planted_min, self.planted_max, int(self.planted_log), self.group_min,
                       self.group_max, self.planted_slice_lo, hi, 0, float(self.zipf_s))


def small_trace(seed: int = 0) -> TrafficConfig:
    """2^20 pairs in 8 slices of 2^17; 50k Zipf(1.1) sources with 1-50 destinations;
    20 planted super points of 2k-20k destinations spread over the slices."""
    return TrafficConfig(seed=seed)


def core_link(seed: int = 0, n_slices: int = 64) -> TrafficConfig:
    """64 slices of 2^25 pairs; 16M-host Zipf(1.05) population (about 3.9M distinct
    sources per slice); 200 planted super points, cardinality log-uniform in [1e3, 1e6]."""
    return TrafficConfig(seed=seed, n_slices=n_slices, load_min=1 << 25, load_max=1 << 25,
                         n_sources=16_000_000, zipf_s=1.05, n_planted=200, planted_min=1000,
                         planted_max=1_000_000, planted_log=True)


def edge_routers(seed: int = 0, n_slices: int = 16, n_routers: int = 16) -> TrafficConfig:
    """16 routers, per-slice loads log-uniform in [2^20, 2^25]; super points split across
    1-8 routers each."""
    return TrafficConfig(seed=seed, n_slices=n_slices, n_routers=n_routers, load_min=1 << 20,
                         load_max=1 << 25, n_sources=16_000_000, zipf_s=1.05, n_planted=200,
                         planted_min=1000, planted_max=1_000_000, planted_log=True, group_min=1,
                         group_max=min(8, n_routers))


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        lib.synth_create.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(vp)]
        lib.synth_create.restype = ctypes.c_int
        lib.synth_destroy.argtypes = [vp]
        lib.synth_slice_len.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
        lib.synth_slice_len.restype = ctypes.c_uint64
        lib.synth_planted_in.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
        lib.synth_planted_in.restype = ctypes.c_uint64
        lib.synth_planted.argtypes = [vp, vp, vp]
        lib.synth_source_ip.argtypes = [vp, ctypes.c_uint32]
        lib.synth_source_ip.restype = ctypes.c_uint32
        lib.synth_fill.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, vp, ctypes.c_uint64, ctypes.c_int]
        lib.synth_fill.restype = ctypes.c_int
        lib.synth_philox.argtypes = [vp, vp, vp]
        _lib = lib
    return _lib


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (for known-answer checks)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.synth_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


class Traffic:
    """A synthetic trace: ``slice(router, t)`` returns that stream's pairs."""

    def __init__(self, cfg: TrafficConfig, threads: int | None = None):
        self.cfg = cfg
        self._lib = _load()
        self._h = ctypes.c_void_p()
        c = cfg.to_c()
        rc = self._lib.synth_create(ctypes.byref(c), ctypes.byref(self._h))
        if rc != 0:
            raise ValueError(f"invalid traffic config: {cfg}")
        self.threads = threads or max(1, os.cpu_count() or 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.synth_destroy(h)
            self._h = None

    def slice_len(self, router: int, t: int) -> int:
        return int(self._lib.synth_slice_len(self._h, router, t))

    def planted_in(self, router: int, t: int) -> int:
        return int(self._lib.synth_planted_in(self._h, router, t))

    def slice(self, router: int, t: int, out: np.ndarray | None = None) -> np.ndarray:
        n = self.slice_len(router, t)
        if out is None:
            out = np.empty((n, 2), dtype=np.uint32)
        else:
            assert out.dtype == np.uint32 and out.flags.c_contiguous and out.size >= 2 * n
            out = out.reshape(-1)[: 2 * n].reshape(n, 2)
        rc = self._lib.synth_fill(self._h, router, t, out.ctypes.data, n, self.threads)
        if rc != 0:
            raise ValueError(f"synth_fill failed ({rc})")
        return out

    def planted(self) -> tuple[np.ndarray, np.ndarray]:
        """Planted super point addresses and their total cardinalities."""
        n = self.cfg.n_planted
        ip = np.zeros(n, dtype=np.uint32)
        card = np.zeros(n, dtype=np.uint32)
        if n:
            self._lib.synth_planted(self._h, ip.ctypes.data, card.ctypes.data)
        return ip, card

    def source_ip(self, rank: int) -> int:
        return int(self._lib.synth_source_ip(self._h, rank))
