"""CPU oracle of the sliding super point method — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-checkable restatement of what the paper computes
("Memory efficient distributed sliding super point cardinality estimation by GPU"):
the sliding rough estimator array RSRA (Algorithms 1-3), candidate tuple growth and
host regaining (Algorithms 4-5), the sliding linear estimator array SLEA
(Algorithm 6) and its merge (Algorithms 2 and 7), and cardinality estimation with
noise correction (Algorithm 8, Eq. 8-12), in the paper's encoding (16-bit distances).
It also computes the exact sliding cardinality |OH(aip,t,k)| (Definition 1) and the
exact super point set (Definition 2) as ground truth.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package. It shares no code with the CUDA library.

Every function is pinned by the ``-m "not gpu"`` tests against the paper's worked
examples, closed forms, invariants and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sse_oracle.cpp")
# SSE_ORACLE_LIB: load another build of the same source (the sanitizer build of the tests)
_LIB = os.environ.get("SSE_ORACLE_LIB") or os.path.join(_HERE, "liborc.so")

SUPER = 1
SATURATED = 2


def build(force: bool = False, sanitize: bool = False, out: str | None = None) -> str:
    """Compile ``liborc.so`` (plain C++17, no FMA contraction). ``sanitize`` builds with
    AddressSanitizer and UndefinedBehaviorSanitizer (any report aborts) into ``out``."""
    lib = out or _LIB
    if sanitize or force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off"]
        if sanitize:
            cmd += ["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]
        subprocess.run(cmd + ["-o", lib, _SRC], check=True)
    return lib


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("r", "q", "delta", "eta", "r2", "q2", "delta2", "eta2", "k", "theta", "rhfg_hash", "pad")] + \
               [("seed", ctypes.c_uint64)]


class _Derived(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_uint32), ("tau", ctypes.c_uint32), ("hot_min", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("row_len2", ctypes.c_uint64), ("rho", ctypes.c_double),
                ("w_theta", ctypes.c_double)]


@dataclass
class Params:
    """The paper's symbols: RSRA (r, q, delta, eta), SLEA (r', q', delta', eta'),
    window k, threshold theta. ``delta = 0`` derives ceil((32-q)/(r-2))."""
    r: int = 5
    q: int = 14
    delta: int = 0
    eta: int = 8
    r2: int = 5
    q2: int = 12
    delta2: int = 16
    eta2: int = 1024
    k: int = 4
    theta: int = 1024
    seed: int = 0
    rhfg_hash: int = 0  # RHFG[0]: 0 multiply-add-shift, 1 simple tabulation (Section 3.3)

    def to_c(self) -> _Params:
        return _Params(self.r, self.q, self.delta, self.eta, self.r2, self.q2, self.delta2,
                       self.eta2, self.k, self.theta, self.rhfg_hash, 0, self.seed)


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.orc_derive.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Params), ctypes.POINTER(_Derived)]
        lib.orc_derive.restype = ctypes.c_int
        lib.orc_splitmix64.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_splitmix64.restype = u64
        lib.orc_lsb.argtypes = [u32]
        lib.orc_lsb.restype = u32
        lib.orc_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.POINTER(vp)]
        lib.orc_create.restype = ctypes.c_int
        lib.orc_destroy.argtypes = [vp]
        lib.orc_hash.argtypes = [vp, ctypes.c_int, u32]
        lib.orc_hash.restype = u32
        lib.orc_rhfg.argtypes = [vp, u32, u32]
        lib.orc_rhfg.restype = u32
        lib.orc_keys.argtypes = [vp, vp]
        lib.orc_slice.argtypes = [vp]
        lib.orc_slice.restype = u64
        lib.orc_scan.argtypes = [vp, vp, u64]
        lib.orc_advance.argtypes = [vp]
        lib.orc_raw.argtypes = [vp, vp, vp]
        lib.orc_set_raw.argtypes = [vp, vp, vp]
        lib.orc_canonical.argtypes = [vp, vp, vp]
        lib.orc_hot.argtypes = [vp, vp]
        lib.orc_row_counts.argtypes = [vp, vp]
        lib.orc_candidates.argtypes = [vp, vp, u64]
        lib.orc_candidates.restype = ctypes.c_int64
        lib.orc_candidates_brute.argtypes = [vp, vp, u64, ctypes.c_int]
        lib.orc_candidates_brute.restype = ctypes.c_int64
        lib.orc_estimate.argtypes = [vp, vp, u64, vp, vp, vp, vp, vp]
        lib.orc_detect.argtypes = [vp, vp, vp, vp, vp, u64]
        lib.orc_detect.restype = ctypes.c_int64
        lib.orc_sre_weights.argtypes = [vp, vp, u64, vp]
        lib.orc_merge.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int]
        lib.orc_merge.restype = ctypes.c_int
        lib.orc_exact_counts.argtypes = [vp, vp, u64, vp]
        lib.orc_exact_counts.restype = ctypes.c_int
        lib.orc_exact_super.argtypes = [vp, u32, vp, vp, u64]
        lib.orc_exact_super.restype = ctypes.c_int64
        _lib = lib
    return _lib


def derive(p: Params) -> dict:
    """Validated parameters and derived constants (delta, tau, hot_min, row length, w_theta)."""
    lib = _load()
    out, d = _Params(), _Derived()
    rc = lib.orc_derive(ctypes.byref(p.to_c()), ctypes.byref(out), ctypes.byref(d))
    if rc != 0:
        raise ValueError(f"invalid parameters {p}")
    return dict(delta=d.delta, tau=d.tau, hot_min=d.hot_min, row_len2=d.row_len2, rho=d.rho,
                w_theta=d.w_theta)


def splitmix64(state: int, n: int) -> list[int]:
    lib = _load()
    s = ctypes.c_uint64(state)
    return [int(lib.orc_splitmix64(ctypes.byref(s))) for _ in range(n)]


def lsb(x: int) -> int:
    return int(_load().orc_lsb(x))


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


class Oracle:
    """One estimator (one router's RSRA + SLEA) in the paper's encoding."""

    def __init__(self, p: Params, track_exact: bool = False):
        self.p = p
        self._lib = _load()
        self.d = derive(p)
        self.delta = self.d["delta"]
        self._h = ctypes.c_void_p()
        rc = self._lib.orc_create(ctypes.byref(p.to_c()), int(track_exact), ctypes.byref(self._h))
        if rc != 0:
            raise ValueError(f"invalid parameters {p}")
        self.row_len2 = self.d["row_len2"]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_destroy(h)
            self._h = None

    # -- hashes ---------------------------------------------------------------
    def hash(self, which: int, x: int) -> int:
        return int(self._lib.orc_hash(self._h, which, x))

    def h1(self, bip): return self.hash(0, bip)
    def h2(self, bip): return self.hash(1, bip)
    def h3(self, bip): return self.hash(2, bip)
    def rhfg0(self, aip): return self.hash(3, aip)
    def lh(self, i, aip): return self.hash(4 + i, aip)

    def rhfg(self, i: int, aip: int) -> int:
        return int(self._lib.orc_rhfg(self._h, i, aip))

    def keys(self) -> np.ndarray:
        out = np.zeros(2 * (4 + self.p.r2), dtype=np.uint64)
        self._lib.orc_keys(self._h, out.ctypes.data)
        return out

    # -- stream ---------------------------------------------------------------
    @property
    def slice(self) -> int:
        return int(self._lib.orc_slice(self._h))

    def scan(self, pairs: np.ndarray) -> None:
        a = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
        self._lib.orc_scan(self._h, a.ctypes.data, a.shape[0])

    def advance(self) -> None:
        self._lib.orc_advance(self._h)

    # -- state ----------------------------------------------------------------
    def raw(self) -> tuple[np.ndarray, np.ndarray]:
        p = self.p
        sre = np.zeros((p.r, 1 << p.q, p.eta), dtype=np.uint16)
        sle = np.zeros((p.r2, self.row_len2), dtype=np.uint16)
        self._lib.orc_raw(self._h, sre.ctypes.data, sle.ctypes.data)
        return sre, sle

    def set_raw(self, sre: np.ndarray | None, sle: np.ndarray | None) -> None:
        s = None if sre is None else np.ascontiguousarray(sre, dtype=np.uint16)
        l = None if sle is None else np.ascontiguousarray(sle, dtype=np.uint16)
        self._lib.orc_set_raw(self._h, _ptr(s), _ptr(l))

    def canonical(self) -> tuple[np.ndarray, np.ndarray]:
        """Per cell: its distance (age in slices) when active (< k), else 255."""
        p = self.p
        sre = np.zeros((p.r, 1 << p.q, p.eta), dtype=np.uint8)
        sle = np.zeros((p.r2, self.row_len2), dtype=np.uint8)
        self._lib.orc_canonical(self._h, sre.ctypes.data, sle.ctypes.data)
        return sre, sle

    def hot(self) -> np.ndarray:
        out = np.zeros((self.p.r, 1 << self.p.q), dtype=np.uint8)
        self._lib.orc_hot(self._h, out.ctypes.data)
        return out

    def row_counts(self) -> np.ndarray:
        out = np.zeros(self.p.r2, dtype=np.uint64)
        self._lib.orc_row_counts(self._h, out.ctypes.data)
        return out

    # -- detection ------------------------------------------------------------
    def candidates(self) -> np.ndarray:
        n = int(self._lib.orc_candidates(self._h, None, 0))
        out = np.zeros(n, dtype=np.uint32)
        if n:
            self._lib.orc_candidates(self._h, out.ctypes.data, n)
        return out

    def candidates_brute(self, threads: int | None = None) -> np.ndarray:
        t = threads or max(1, os.cpu_count() or 1)
        cap = 1 << 20
        out = np.zeros(cap, dtype=np.uint32)
        n = int(self._lib.orc_candidates_brute(self._h, out.ctypes.data, cap, t))
        if n > cap:
            out = np.zeros(n, dtype=np.uint32)
            self._lib.orc_candidates_brute(self._h, out.ctypes.data, n, t)
        return out[:n].copy()

    def estimate(self, hosts, hist: bool = False) -> dict:
        h = np.ascontiguousarray(hosts, dtype=np.uint32).reshape(-1)
        n = h.size
        w = np.zeros(n, np.float64)
        est = np.zeros(n, np.float64)
        U = np.zeros(n, np.uint32)
        flags = np.zeros(n, np.uint8)
        hh = np.zeros((n, self.p.k), np.uint32) if hist else None
        self._lib.orc_estimate(self._h, h.ctypes.data, n, w.ctypes.data, est.ctypes.data,
                               U.ctypes.data, flags.ctypes.data, _ptr(hh))
        out = dict(w=w, est=est, U=U, flags=flags)
        if hist:
            out["hist"] = hh
        return out

    def detect(self) -> dict:
        """All candidates (ascending) with w^, estimate and flags."""
        n = int(self._lib.orc_candidates(self._h, None, 0))
        hosts = np.zeros(n, np.uint32)
        w = np.zeros(n, np.float64)
        est = np.zeros(n, np.float64)
        flags = np.zeros(n, np.uint8)
        if n:
            self._lib.orc_detect(self._h, hosts.ctypes.data, w.ctypes.data, est.ctypes.data,
                                 flags.ctypes.data, n)
        return dict(hosts=hosts, w=w, est=est, flags=flags)

    def sre_weights(self, hosts) -> np.ndarray:
        """|SRE_i|^k of each host's r rough estimators, shape [n, r]."""
        h = np.ascontiguousarray(hosts, dtype=np.uint32).reshape(-1)
        out = np.zeros((h.size, self.p.r), np.uint32)
        if h.size:
            self._lib.orc_sre_weights(self._h, h.ctypes.data, h.size, out.ctypes.data)
        return out

    def features(self, hosts) -> np.ndarray:
        """Learned-correction inputs (FP64): log1p of the union SLE's active cells per
        distance 0..k-1, then log1p of the sum and of the minimum of the SRE weights."""
        e = self.estimate(hosts, hist=True)
        w = self.sre_weights(hosts).astype(np.float64)
        return np.log1p(np.concatenate([e["hist"].astype(np.float64), w.sum(1, keepdims=True),
                                        w.min(1, keepdims=True)], axis=1))

    def merge(self, others: list["Oracle"]) -> None:
        arr = (ctypes.c_void_p * len(others))(*[o._h.value for o in others])
        rc = self._lib.orc_merge(self._h, arr, len(others))
        if rc != 0:
            raise ValueError("merge of mismatched estimators")

    # -- ground truth ---------------------------------------------------------
    def exact_counts(self, hosts) -> np.ndarray:
        h = np.ascontiguousarray(hosts, dtype=np.uint32).reshape(-1)
        out = np.zeros(h.size, np.uint32)
        if self._lib.orc_exact_counts(self._h, h.ctypes.data, h.size, out.ctypes.data) != 0:
            raise RuntimeError("exact tracking is off")
        return out

    def exact_super(self, theta: int | None = None) -> tuple[np.ndarray, np.ndarray]:
        th = self.p.theta if theta is None else theta
        n = int(self._lib.orc_exact_super(self._h, th, None, None, 0))
        if n < 0:
            raise RuntimeError("exact tracking is off")
        hosts = np.zeros(n, np.uint32)
        card = np.zeros(n, np.uint32)
        if n:
            self._lib.orc_exact_super(self._h, th, hosts.ctypes.data, card.ctypes.data, n)
        return hosts, card
