"""Python binding of libsse (include/sse.h): argument marshalling only.

Every computation runs in the CUDA library. PyTorch supplies device memory (tensors
whose ``data_ptr()`` is passed through) and the CUDA stream. Using this module on a
machine without the built library or without a CUDA device raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsse.so")

SSE_OK = 0
FLAG_SUPER = 1
FLAG_SATURATED = 2
ERR_CAPACITY = -3
ERR_TIMEOUT = -6
UPDATE_AUTO, UPDATE_DIRECT, UPDATE_TILED = 0, 1, 2
JOIN_AUTO, JOIN_FORWARD, JOIN_BACKWARD = 0, 1, 2
BATCH_DETECT, BATCH_ROUTERS, BATCH_SCAN = 0, 1, 2
DIR_SRC, DIR_DST, DIR_BOTH = 0, 1, 2


class SSEError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_strerror(code)} ({code})")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("r", "q", "delta", "eta", "r2", "q2", "delta2", "eta2", "k", "theta",
                 "stamp_bits", "max_candidates", "rhfg_hash", "reserved")] + [("seed", ctypes.c_uint64)]


class _Derived(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_uint32), ("tau", ctypes.c_uint32), ("hot_min", ctypes.c_uint32),
                ("lg_eta2", ctypes.c_uint32), ("row_len2", ctypes.c_uint64), ("row_pitch2", ctypes.c_uint64),
                ("sre_bytes", ctypes.c_uint64), ("sle_bytes", ctypes.c_uint64), ("w_theta", ctypes.c_double)]


class _Report(ctypes.Structure):
    _fields_ = [("slice", ctypes.c_uint64), ("n_candidates", ctypes.c_uint32), ("n_super", ctypes.c_uint32),
                ("cap", ctypes.c_uint32), ("truncated", ctypes.c_uint32), ("hosts", ctypes.c_void_p),
                ("est", ctypes.c_void_p), ("flags", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("slice", ctypes.c_uint64), ("hot", ctypes.c_uint32 * 16), ("active2", ctypes.c_uint32 * 16),
                ("join_pairs", ctypes.c_uint64), ("n_candidates", ctypes.c_uint32), ("n_super", ctypes.c_uint32)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("n_routers", ctypes.c_uint32), ("slots", ctypes.c_uint32), ("slot_pairs", ctypes.c_uint64),
                ("memory_budget", ctypes.c_uint64), ("slice_seconds", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("pairs", ctypes.c_uint64), ("slices_closed", ctypes.c_uint64),
                ("slot_waits", ctypes.c_uint64), ("current_slice", ctypes.c_uint64),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double)]


@dataclass
class Params:
    """Symbols of the paper; defaults are the 8-slice small trace configuration."""
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
    stamp_bits: int = 8
    max_candidates: int = 1 << 16
    seed: int = 0
    rhfg_hash: int = 0  # 0: multiply-add-shift, 1: simple tabulation (RHFG[0])

    def to_c(self) -> _Params:
        return _Params(self.r, self.q, self.delta, self.eta, self.r2, self.q2, self.delta2, self.eta2,
                       self.k, self.theta, self.stamp_bits, self.max_candidates, self.rhfg_hash, 0, self.seed)


def core_link_params(k: int = 8, seed: int = 0) -> Params:
    """Core-link scale: SRE rows of 2^20, SLEA 2^16 SLEs of 2^12 cells, window 8."""
    return Params(q=20, q2=16, eta2=4096, k=k, seed=seed)


def paper_params(k: int = 300) -> Params:
    """The parameter set of the paper's experiments (Section 5), 16-bit stamps; k defaults to
    the paper's sliding-window length."""
    p = _Params()
    lib().sse_params_default(ctypes.byref(p))
    return Params(r=p.r, q=p.q, delta=p.delta, eta=p.eta, r2=p.r2, q2=p.q2, delta2=p.delta2, eta2=p.eta2,
                  k=k, theta=p.theta, stamp_bits=p.stamp_bits, max_candidates=p.max_candidates, seed=p.seed,
                  rhfg_hash=p.rhfg_hash)


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libsse.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsse.so is not built ({LIB_PATH}); run paper_1805_09246_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        sig = {
            "sse_params_default": (None, [vp]),
            "sse_derive": (i32, [vp, vp]),
            "sse_init": (i32, [vp, vp, ctypes.POINTER(vp)]),
            "sse_destroy": (None, [vp]),
            "sse_update": (i32, [vp, vp, u64]),
            "sse_update_host": (i32, [vp, vp, u64]),
            "sse_set_update_mode": (i32, [vp, i32]),
            "sse_set_direction": (i32, [vp, i32]),
            "sse_set_update_variant": (i32, [vp, i32]),
            "sse_update_variant_count": (i32, []),
            "sse_autotune_update": (i32, [vp, vp, u64, i32, vp, ctypes.POINTER(i32)]),
            "sse_close_slice": (i32, [vp, vp]),
            "sse_advance": (i32, [vp]),
            "sse_merge": (i32, [vp, ctypes.POINTER(vp), i32]),
            "sse_query": (i32, [vp, vp, u32, vp, vp, vp]),
            "sse_get_stats": (i32, [vp, vp]),
            "sse_get_hot_bitmap": (i32, [vp, vp, ctypes.c_size_t]),
            "sse_export_state": (i32, [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "sse_import_state": (i32, [vp, vp, ctypes.c_size_t]),
            "sse_read_stamps": (i32, [vp, vp, ctypes.c_size_t, vp, ctypes.c_size_t]),
            "sse_current_slice": (u64, [vp]),
            "sse_kernel_launches": (u64, [vp]),
            "sse_sync": (i32, [vp]),
            "sse_strerror": (ctypes.c_char_p, [i32]),
            "sse_batch_create": (i32, [vp, i32, u64, ctypes.POINTER(vp)]),
            "sse_batch_destroy": (None, [vp]),
            "sse_batch_input": (vp, [vp, i32]),
            "sse_batch_stream": (vp, [vp]),
            "sse_batch_load": (i32, [vp, i32, vp, u64, i32]),
            "sse_batch_router": (i32, [vp, i32, ctypes.POINTER(vp)]),
            "sse_batch_global": (i32, [vp, ctypes.POINTER(vp)]),
            "sse_batch_use_graph": (i32, [vp, i32]),
            "sse_batch_configure": (i32, [vp, u32, i32]),
            "sse_debug_sort_barrier": (i32, [vp, u32, u32]),
            "sse_set_join": (i32, [vp, i32]),
            "sse_microbench": (i32, [vp, u64, vp, vp]),
            "sse_batch_tune": (i32, [vp, vp, vp, i32, vp, ctypes.POINTER(i32)]),
            "sse_batch_step": (i32, [vp, vp, vp]),
            "sse_batch_step_from": (i32, [vp, vp, vp, vp]),
            "sse_batch_step_async": (i32, [vp, vp, vp]),
            "sse_batch_step_wait": (i32, [vp, vp]),
            "sse_batch_pending": (i32, [vp]),
            "sse_batch_kernel_launches": (u64, [vp]),
            "sse_server_config_default": (None, [vp]),
            "sse_server_create": (i32, [vp, vp, ctypes.POINTER(vp)]),
            "sse_server_destroy": (None, [vp]),
            "sse_server_submit": (i32, [vp, u32, ctypes.c_double, vp, u64]),
            "sse_server_flush": (i32, [vp]),
            "sse_server_poll": (i32, [vp, vp, ctypes.POINTER(ctypes.c_double)]),
            "sse_server_get_stats": (i32, [vp, vp]),
            "sse_server_router": (i32, [vp, u32, ctypes.POINTER(vp)]),
            "sse_server_global": (i32, [vp, ctypes.POINTER(vp)]),
            "sse_cuda_error": (ctypes.c_char_p, [vp]),
            "sse_reset": (i32, [vp]),
            "sse_close_use_graph": (i32, [vp, i32]),
            "sse_close_slice_async": (i32, [vp]),
            "sse_close_slice_wait": (i32, [vp, vp]),
            "sse_batch_set_mode": (i32, [vp, i32]),
            "sse_batch_reset": (i32, [vp]),
            "sse_features": (i32, [vp, vp, u32, vp]),
            "sse_mlp_create": (i32, [u32, u32, u32, u64, ctypes.POINTER(vp)]),
            "sse_mlp_destroy": (None, [vp]),
            "sse_mlp_param_count": (u32, [vp]),
            "sse_mlp_kernel_launches": (u64, [vp]),
            "sse_mlp_set_params": (i32, [vp, vp]),
            "sse_mlp_get_params": (i32, [vp, vp, vp, vp]),
            "sse_mlp_set_feature_max": (i32, [vp, vp]),
            "sse_mlp_set_gate": (i32, [vp, u32]),
            "sse_mlp_forward": (i32, [vp, vp, u32, vp, vp]),
            "sse_mlp_gradients": (i32, [vp, vp, vp, vp, u32, vp, vp]),
            "sse_mlp_adam": (i32, [vp, ctypes.c_float, vp]),
            "sse_mlp_train_epoch": (i32, [vp, vp, vp, vp, u32, u32, ctypes.c_float, vp, vp]),
            "sse_query_learned": (i32, [vp, vp, vp, u32, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class _MicrobenchResult(ctypes.Structure):
    _fields_ = [("l2_random_byte_stores_per_s", ctypes.c_double), ("smem_random_atomics_per_s", ctypes.c_double),
                ("l2_stream_load_bytes_per_s", ctypes.c_double), ("hbm_stream_load_bytes_per_s", ctypes.c_double),
                ("tiled_skeleton_pairs_per_s", ctypes.c_double), ("sms", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


MICROBENCH_MIN_BYTES = (1 << 30) + 4096


def microbench(stream=None) -> dict:
    """Peak rates of the update's memory units on the current device (sse_microbench): random
    one-byte L2 stores/s, random shared-memory atomic ORs/s, streaming 128-bit load bytes/s
    from L2 and from HBM, and the tiled update's skeleton in pairs/s."""
    torch = _torch()
    buf = torch.empty(MICROBENCH_MIN_BYTES, dtype=torch.uint8, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    out = _MicrobenchResult()
    _check(lib().sse_microbench(ctypes.c_void_p(buf.data_ptr()), buf.numel(), ctypes.c_void_p(st.cuda_stream),
                                ctypes.byref(out)), "sse_microbench")
    del buf
    return {name: getattr(out, name) for name, _ in _MicrobenchResult._fields_ if name != "reserved"}


def update_variant_count() -> int:
    return int(lib().sse_update_variant_count())


def _strerror(code: int) -> str:
    try:
        return lib().sse_strerror(code).decode()
    except Exception:  # library missing: still produce a message
        return "error"


def _check(code: int, what: str, handle=None) -> int:
    if code != SSE_OK:
        detail = ""
        if handle is not None and handle.value:
            detail = lib().sse_cuda_error(handle).decode()
        raise SSEError(code, f"{what} [{detail}]" if detail else what)
    return code


def derive(p: Params) -> dict:
    d = _Derived()
    _check(lib().sse_derive(ctypes.byref(p.to_c()), ctypes.byref(d)), "sse_derive")
    return {name: getattr(d, name) for name, _ in _Derived._fields_}


@dataclass
class Report:
    slice: int
    n_candidates: int
    n_super: int
    truncated: bool
    hosts: np.ndarray
    est: np.ndarray
    flags: np.ndarray
    status: int = SSE_OK

    @property
    def super_points(self) -> np.ndarray:
        return self.hosts[(self.flags & FLAG_SUPER) != 0]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsse needs a CUDA device; no CPU fallback exists")
    return torch


def _dev_ptr(t, dtype_bytes: int | None = None) -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype_bytes is not None and t.element_size() != dtype_bytes:
        raise TypeError(f"expected {dtype_bytes}-byte elements")
    return t.data_ptr()


class Estimator:
    """One router's estimator (RSRA + SLEA) resident on the current CUDA device."""

    @classmethod
    def _borrowed(cls, params: Params, handle: ctypes.c_void_p) -> "Estimator":
        """A view of an estimator owned elsewhere (a batch's router or global estimator)."""
        e = cls.__new__(cls)
        e.params = params
        e._lib = lib()
        e.derived = derive(params)
        e.stream = None
        e._h = handle
        e._borrowed_handle = True
        return e

    def __init__(self, params: Params | None = None, stream=None):
        torch = _torch()
        self.params = params or Params()
        self._lib = lib()
        self.derived = derive(self.params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        _check(self._lib.sse_init(ctypes.byref(self.params.to_c()), ctypes.c_void_p(self.stream.cuda_stream),
                                  ctypes.byref(self._h)), "sse_init")

    def close(self) -> None:
        if getattr(self, "_borrowed_handle", False):
            self._h = None
            return
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def slice(self) -> int:
        return int(self._lib.sse_current_slice(self._h))

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.sse_kernel_launches(self._h))

    def set_update_mode(self, mode: int) -> None:
        _check(self._lib.sse_set_update_mode(self._h, mode), "sse_set_update_mode")

    def set_join(self, mode: int) -> None:
        """JOIN_AUTO, JOIN_FORWARD (rows 0, 1, 2 up) or JOIN_BACKWARD (rows 0 and r-1 down);
        identical candidates (sse_set_join)."""
        _check(self._lib.sse_set_join(self._h, mode), "sse_set_join")

    def set_direction(self, direction: int) -> None:
        """DIR_SRC (aip = source, default), DIR_DST (aip = destination) or DIR_BOTH (Definition 1)."""
        _check(self._lib.sse_set_direction(self._h, direction), "sse_set_direction")

    def set_update_variant(self, variant: int) -> None:
        _check(self._lib.sse_set_update_variant(self._h, variant), "sse_set_update_variant")

    def autotune_update(self, pairs, reps: int = 3) -> tuple[int, list[float]]:
        """Time every update variant on these (current-slice) pairs and keep the fastest."""
        nv = int(self._lib.sse_update_variant_count())
        times = (ctypes.c_float * nv)()
        chosen = ctypes.c_int(-1)
        _check(self._lib.sse_autotune_update(self._h, ctypes.c_void_p(_dev_ptr(pairs, 4)), pairs.numel() // 2,
                                             reps, times, ctypes.byref(chosen)), "sse_autotune_update", self._h)
        return chosen.value, [float(t) for t in times]

    def update(self, pairs) -> None:
        """Scan the pairs of a CUDA tensor of shape (n, 2), 32-bit elements {src, dst}."""
        n = pairs.numel() // 2
        if n == 0:
            return
        _check(self._lib.sse_update(self._h, ctypes.c_void_p(_dev_ptr(pairs, 4)), n), "sse_update", self._h)

    def update_host(self, pairs) -> None:
        """Scan pairs held in host memory (numpy array or CPU tensor, (n, 2) 32-bit)."""
        if isinstance(pairs, np.ndarray):
            a = np.ascontiguousarray(pairs).view(np.uint32).reshape(-1)
            ptr, n = a.ctypes.data, a.size // 2
        else:
            if pairs.is_cuda or not pairs.is_contiguous() or pairs.element_size() != 4:
                raise TypeError("expected a contiguous CPU tensor of 32-bit elements")
            ptr, n = pairs.data_ptr(), pairs.numel() // 2
        if n:
            _check(self._lib.sse_update_host(self._h, ctypes.c_void_p(ptr), n), "sse_update_host")

    def close_slice(self, cap: int | None = None, raise_on_capacity: bool = True) -> Report:
        """Detect the sliding super points of the window ending at the current slice."""
        return self._collect(self._lib.sse_close_slice, "sse_close_slice", cap, raise_on_capacity)

    def _collect(self, fn, what: str, cap: int | None, raise_on_capacity: bool) -> Report:
        cap = self.params.max_candidates if cap is None else cap
        bufs = getattr(self, "_report_bufs", None)
        if bufs is None or len(bufs[0]) != cap:
            # reused across slices, with their report struct: allocating the arrays, and even
            # reading their addresses through numpy's ctypes attribute, costs more than the copy
            h, e, f = np.empty(cap, np.uint32), np.empty(cap, np.float32), np.empty(cap, np.uint8)
            bufs = self._report_bufs = (h, e, f, _Report(0, 0, 0, cap, 0, h.ctypes.data, e.ctypes.data, f.ctypes.data))
        hosts, est, flags, rep = bufs
        rep.slice = rep.n_candidates = rep.n_super = rep.truncated = 0
        rep.cap = cap
        rc = fn(self._h, ctypes.byref(rep))
        if rc != SSE_OK and (rc != ERR_CAPACITY or raise_on_capacity):
            _check(rc, what, self._h)
        m = min(rep.n_candidates, cap, self.params.max_candidates)
        return Report(slice=rep.slice, n_candidates=rep.n_candidates, n_super=rep.n_super,
                      truncated=bool(rep.truncated), hosts=hosts[:m].copy(), est=est[:m].copy(),
                      flags=flags[:m].copy(), status=rc)

    def close_slice_async(self) -> None:
        """Enqueue the close of the current slice (see sse_close_slice_async); the report is
        collected by close_slice_wait()."""
        _check(self._lib.sse_close_slice_async(self._h), "sse_close_slice_async", self._h)

    def close_slice_wait(self, cap: int | None = None, raise_on_capacity: bool = True) -> Report:
        return self._collect(self._lib.sse_close_slice_wait, "sse_close_slice_wait", cap, raise_on_capacity)

    def advance(self) -> None:
        _check(self._lib.sse_advance(self._h), "sse_advance")

    def merge(self, others: list["Estimator"]) -> None:
        arr = (ctypes.c_void_p * len(others))(*[o._h.value for o in others])
        _check(self._lib.sse_merge(self._h, arr, len(others)), "sse_merge")

    def query(self, hosts, hist: bool = False):
        """Estimates (float32), flags (uint8) and optionally per-distance histograms
        (32-bit, [n, k]) of the hosts in a CUDA tensor of 32-bit addresses."""
        torch = _torch()
        n = hosts.numel()
        dev = hosts.device
        est = torch.empty(n, dtype=torch.float32, device=dev)
        flags = torch.empty(n, dtype=torch.uint8, device=dev)
        hh = torch.empty((n, self.params.k), dtype=torch.int32, device=dev) if hist else None
        _check(self._lib.sse_query(self._h, ctypes.c_void_p(_dev_ptr(hosts, 4)), n, ctypes.c_void_p(est.data_ptr()),
                                   ctypes.c_void_p(flags.data_ptr()),
                                   ctypes.c_void_p(hh.data_ptr() if hist else 0)), "sse_query")
        return (est, flags, hh) if hist else (est, flags)

    def stats(self) -> dict:
        s = _Stats()
        _check(self._lib.sse_get_stats(self._h, ctypes.byref(s)), "sse_get_stats")
        return dict(slice=s.slice, hot=list(s.hot)[: self.params.r], active2=list(s.active2)[: self.params.r2],
                    join_pairs=s.join_pairs, n_candidates=s.n_candidates, n_super=s.n_super)

    def hot_bitmap(self) -> np.ndarray:
        """Hot flags of the last close as uint8 [r, 2^q]."""
        p = self.params
        words = np.zeros(((p.r << p.q) + 31) // 32, np.uint32)
        _check(self._lib.sse_get_hot_bitmap(self._h, ctypes.c_void_p(words.ctypes.data), words.nbytes),
               "sse_get_hot_bitmap")
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")
        return bits[: p.r << p.q].reshape(p.r, 1 << p.q)

    def read_stamps(self) -> tuple[np.ndarray, np.ndarray]:
        """Raw stamps: RSRA [r, 2^q, 8] and SLEA [r', row_len2], uint8 or uint16 cells."""
        p, d = self.params, self.derived
        dt = np.uint8 if p.stamp_bits == 8 else np.uint16
        sre = np.zeros((p.r, 1 << p.q, p.eta), dt)
        sle = np.zeros((p.r2, d["row_pitch2"]), dt)
        _check(self._lib.sse_read_stamps(self._h, ctypes.c_void_p(sre.ctypes.data), sre.nbytes,
                                         ctypes.c_void_p(sle.ctypes.data), sle.nbytes), "sse_read_stamps")
        return sre, sle[:, : d["row_len2"]]

    def export_state(self) -> bytes:
        used = ctypes.c_size_t(0)
        _check(self._lib.sse_export_state(self._h, None, 0, ctypes.byref(used)), "sse_export_state")
        buf = ctypes.create_string_buffer(used.value)
        _check(self._lib.sse_export_state(self._h, buf, used.value, ctypes.byref(used)), "sse_export_state")
        return buf.raw

    def import_state(self, blob: bytes) -> None:
        _check(self._lib.sse_import_state(self._h, blob, len(blob)), "sse_import_state")

    def sync(self) -> None:
        _check(self._lib.sse_sync(self._h), "sse_sync")

    def debug_sort_barrier(self, spin_limit: int, extra_arrivals: int) -> None:
        """Failure-detection hook: bound the candidate sort's barrier waits to spin_limit polls
        (0: default); extra_arrivals = 1 makes every wait run out (sse_debug_sort_barrier)."""
        _check(self._lib.sse_debug_sort_barrier(self._h, spin_limit, extra_arrivals), "sse_debug_sort_barrier",
               self._h)

    def close_use_graph(self, enable: bool) -> None:
        """Replay sse_close_slice from a CUDA graph (default) or launch its kernels one by one."""
        _check(self._lib.sse_close_use_graph(self._h, 1 if enable else 0), "sse_close_use_graph")

    def reset(self) -> None:
        """Back to the initial state at slice 0."""
        _check(self._lib.sse_reset(self._h), "sse_reset", self._h)

    def features(self, hosts, out=None):
        """Learned-correction features of the hosts (CUDA tensor of 32-bit addresses):
        float32 [n, k + 2], log(1 + v) of the union SLE's per-distance active cells and of the
        sum and minimum of the host's SRE weights. Asynchronous on the estimator's stream."""
        torch = _torch()
        n = hosts.numel()
        x = torch.empty((n, self.params.k + 2), dtype=torch.float32, device=hosts.device) if out is None else out
        _check(self._lib.sse_features(self._h, ctypes.c_void_p(_dev_ptr(hosts, 4)), n,
                                      ctypes.c_void_p(_dev_ptr(x, 4))), "sse_features", self._h)
        return x

    def query_learned(self, mlp: "MLP", hosts):
        """(learned estimate, linear-counting estimate, flags) of the hosts."""
        torch = _torch()
        n = hosts.numel()
        est = torch.empty(n, dtype=torch.float32, device=hosts.device)
        lc = torch.empty(n, dtype=torch.float32, device=hosts.device)
        flags = torch.empty(n, dtype=torch.uint8, device=hosts.device)
        _check(self._lib.sse_query_learned(self._h, mlp._m, ctypes.c_void_p(_dev_ptr(hosts, 4)), n,
                                           ctypes.c_void_p(est.data_ptr()), ctypes.c_void_p(lc.data_ptr()),
                                           ctypes.c_void_p(flags.data_ptr())), "sse_query_learned", self._h)
        return est, lc, flags


class Batch:
    """R routers' estimators plus their merged global estimator, advanced slice by slice
    with one persistent update launch per slice and a CUDA-graph-captured step."""

    def __init__(self, params: Params, n_routers: int, capacity_pairs: int, use_graph: bool = True):
        _torch()
        self.params = params
        self.n = n_routers
        self.capacity = capacity_pairs
        self._lib = lib()
        self._b = ctypes.c_void_p()
        _check(self._lib.sse_batch_create(ctypes.byref(params.to_c()), n_routers, capacity_pairs,
                                          ctypes.byref(self._b)), "sse_batch_create")
        self._lib.sse_batch_use_graph(self._b, 1 if use_graph else 0)
        self._views = {}

    def close(self) -> None:
        if getattr(self, "_b", None) is not None and self._b.value:
            for v in self._views.values():
                v.close()
            self._lib.sse_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream_ptr(self) -> int:
        return int(self._lib.sse_batch_stream(self._b) or 0)

    def load(self, router: int, pairs) -> int:
        """Copy a router's pairs (CUDA tensor, numpy array or CPU tensor) into its input."""
        if isinstance(pairs, np.ndarray):
            a = np.ascontiguousarray(pairs).view(np.uint32).reshape(-1)
            ptr, n, host = a.ctypes.data, a.size // 2, 1
            self._keep = a
        elif pairs.is_cuda:
            _torch().cuda.current_stream().synchronize()  # the batch copies on its own stream
            ptr, n, host = _dev_ptr(pairs, 4), pairs.numel() // 2, 0
        else:
            ptr, n, host = pairs.data_ptr(), pairs.numel() // 2, 1
        _check(self._lib.sse_batch_load(self._b, router, ctypes.c_void_p(ptr), n, host), "sse_batch_load")
        return n

    def configure(self, item_pairs: int, unroll: int) -> None:
        _check(self._lib.sse_batch_configure(self._b, item_pairs, unroll), "sse_batch_configure")

    @staticmethod
    def _ptrs(tensors):
        if tensors is None:
            return None
        arr = (ctypes.c_void_p * len(tensors))(*[_dev_ptr(t, 4) if t.numel() else 0 for t in tensors])
        return arr

    def tune(self, counts, reps: int = 2, inputs=None) -> tuple[int, list[float]]:
        """Tune the persistent update on the loaded inputs, or on `inputs` (CUDA tensors)."""
        if inputs is not None:
            counts = [t.numel() // 2 for t in inputs]
            _torch().cuda.current_stream().synchronize()
        c = np.ascontiguousarray(counts, dtype=np.uint64)
        times = (ctypes.c_float * 9)()
        chosen = ctypes.c_int(-1)
        _check(self._lib.sse_batch_tune(self._b, self._ptrs(inputs), ctypes.c_void_p(c.ctypes.data), reps, times,
                                        ctypes.byref(chosen)), "sse_batch_tune")
        return chosen.value, [float(t) for t in times]

    def _report_buffers(self, cap: int):
        """(hosts, est, flags) arrays of `cap` entries, one set per step parity, reused."""
        sets = getattr(self, "_report_bufs", None)
        if sets is None or len(sets[0][0]) != cap:
            sets = []
            for _ in range(2):  # with their report struct (numpy's ctypes attribute is slow)
                h, e, f = np.empty(cap, np.uint32), np.empty(cap, np.float32), np.empty(cap, np.uint8)
                sets.append((h, e, f, _Report(0, 0, 0, cap, 0, h.ctypes.data, e.ctypes.data, f.ctypes.data)))
            self._report_bufs = sets
        self._parity = getattr(self, "_parity", 0) ^ 1
        hosts, est, flags, rep = sets[self._parity]
        rep.slice = rep.n_candidates = rep.n_super = rep.truncated = 0
        rep.cap = cap
        return sets[self._parity]

    def _report(self, rc: int, rep, bufs, cap: int, what: str) -> Report:
        if rc != SSE_OK and rc != ERR_CAPACITY:
            _check(rc, what)
        hosts, est, flags, _ = bufs
        m = min(rep.n_candidates, cap, self.params.max_candidates)
        return Report(slice=rep.slice, n_candidates=rep.n_candidates, n_super=rep.n_super,
                      truncated=bool(rep.truncated), hosts=hosts[:m].copy(), est=est[:m].copy(),
                      flags=flags[:m].copy(), status=rc)

    def step(self, counts=None, cap: int | None = None, inputs=None) -> Report:
        """One slice. Without `inputs`, router r scans counts[r] pairs of its loaded input
        buffer; with `inputs` (one CUDA tensor (n_r, 2) per router, already written), it scans
        those tensors in place."""
        if inputs is not None:
            counts = [t.numel() // 2 for t in inputs]
            _torch().cuda.current_stream().synchronize()  # producers finish before the batch stream reads
        c = np.ascontiguousarray(counts, dtype=np.uint64)
        cap = self.params.max_candidates if cap is None else cap
        bufs = self._report_buffers(cap)
        rep = bufs[3]
        if inputs is not None:
            rc = self._lib.sse_batch_step_from(self._b, self._ptrs(inputs), ctypes.c_void_p(c.ctypes.data),
                                               ctypes.byref(rep))
        else:
            rc = self._lib.sse_batch_step(self._b, ctypes.c_void_p(c.ctypes.data), ctypes.byref(rep))
        return self._report(rc, rep, bufs, cap, "sse_batch_step")

    def step_async(self, inputs=None, counts=None) -> None:
        """Enqueue one slice (see sse_batch_step_async) and return; `inputs`: one CUDA tensor
        (n_r, 2) per router, unchanged until the step is collected, or None for the loaded
        input buffers with `counts`. At most two steps may wait for step_wait()."""
        if inputs is not None:
            counts = [t.numel() // 2 for t in inputs]
            _torch().cuda.current_stream().synchronize()  # producers finish before the batch stream reads
        c = np.ascontiguousarray(counts, dtype=np.uint64)
        _check(self._lib.sse_batch_step_async(self._b, self._ptrs(inputs), ctypes.c_void_p(c.ctypes.data)),
               "sse_batch_step_async")

    def step_wait(self, cap: int | None = None) -> Report:
        """The report of the oldest enqueued slice (blocks until it is on the host)."""
        cap = self.params.max_candidates if cap is None else cap
        bufs = self._report_buffers(cap)
        rep = bufs[3]
        rc = self._lib.sse_batch_step_wait(self._b, ctypes.byref(rep))
        return self._report(rc, rep, bufs, cap, "sse_batch_step_wait")

    @property
    def pending(self) -> int:
        return int(self._lib.sse_batch_pending(self._b))

    def router(self, r: int) -> Estimator:
        if r not in self._views:
            h = ctypes.c_void_p()
            _check(self._lib.sse_batch_router(self._b, r, ctypes.byref(h)), "sse_batch_router")
            self._views[r] = Estimator._borrowed(self.params, h)
        return self._views[r]

    def global_estimator(self) -> Estimator:
        if "global" not in self._views:
            h = ctypes.c_void_p()
            _check(self._lib.sse_batch_global(self._b, ctypes.byref(h)), "sse_batch_global")
            self._views["global"] = Estimator._borrowed(self.params, h)
        return self._views["global"]

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.sse_batch_kernel_launches(self._b))

    def set_mode(self, mode: int) -> None:
        """BATCH_DETECT (default), BATCH_ROUTERS or BATCH_SCAN (see sse_batch_set_mode)."""
        _check(self._lib.sse_batch_set_mode(self._b, mode), "sse_batch_set_mode")

    def reset(self) -> None:
        """Every estimator back to slice 0."""
        _check(self._lib.sse_batch_reset(self._b), "sse_batch_reset")


class MLP:
    """The learned correction's network (sse_mlp_*): n_in -> hidden -> hidden -> 1, BF16
    weights, FP32 sums, trained with the library's own kernels."""

    def __init__(self, n_in: int, hidden: int = 64, max_batch: int = 1 << 16, seed: int = 0):
        _torch()
        self._lib = lib()
        self._m = ctypes.c_void_p()
        _check(self._lib.sse_mlp_create(n_in, hidden, max_batch, seed, ctypes.byref(self._m)), "sse_mlp_create")
        self.n_in, self.hidden, self.max_batch = n_in, hidden, max_batch
        self.n_params = int(self._lib.sse_mlp_param_count(self._m))

    def close(self) -> None:
        if getattr(self, "_m", None) is not None and self._m.value:
            self._lib.sse_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream():
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)

    def set_params(self, w: np.ndarray) -> None:
        a = np.ascontiguousarray(w, dtype=np.float32)
        assert a.size == self.n_params
        _check(self._lib.sse_mlp_set_params(self._m, ctypes.c_void_p(a.ctypes.data)), "sse_mlp_set_params")

    def params(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(FP32 parameters, BF16 parameters as uint16 bits, last gradients)."""
        _torch().cuda.current_stream().synchronize()
        f = np.zeros(self.n_params, np.float32)
        b = np.zeros(self.n_params, np.uint16)
        g = np.zeros(self.n_params, np.float32)
        _check(self._lib.sse_mlp_get_params(self._m, ctypes.c_void_p(f.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                            ctypes.c_void_p(g.ctypes.data)), "sse_mlp_get_params")
        return f, b, g

    def set_feature_max(self, xmax) -> None:
        a = np.ascontiguousarray(xmax, dtype=np.float32)
        assert a.size == self.n_in
        _check(self._lib.sse_mlp_set_feature_max(self._m, ctypes.c_void_p(a.ctypes.data)),
               "sse_mlp_set_feature_max")

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.sse_mlp_kernel_launches(self._m))

    def set_gate(self, min_active: int) -> None:
        """Use the network only for hosts with at least min_active active union-SLE cells."""
        _check(self._lib.sse_mlp_set_gate(self._m, int(min_active)), "sse_mlp_set_gate")

    def forward(self, x):
        torch = _torch()
        n = x.shape[0]
        y = torch.empty(n, dtype=torch.float32, device=x.device)
        _check(self._lib.sse_mlp_forward(self._m, ctypes.c_void_p(_dev_ptr(x, 4)), n,
                                         ctypes.c_void_p(y.data_ptr()), self._stream()), "sse_mlp_forward")
        return y

    def gradients(self, x, t, rows=None) -> float:
        """Gradients of the mean squared error over `rows` (or all rows); returns the loss."""
        n = rows.numel() if rows is not None else x.shape[0]
        loss = ctypes.c_float(0)
        _check(self._lib.sse_mlp_gradients(self._m, ctypes.c_void_p(_dev_ptr(x, 4)), ctypes.c_void_p(_dev_ptr(t, 4)),
                                           ctypes.c_void_p(_dev_ptr(rows, 4) if rows is not None else 0), n,
                                           ctypes.byref(loss), self._stream()), "sse_mlp_gradients")
        return float(loss.value)

    def adam(self, lr: float) -> None:
        _check(self._lib.sse_mlp_adam(self._m, ctypes.c_float(lr), self._stream()), "sse_mlp_adam")

    def train_epoch(self, x, t, perm, batch: int, lr: float) -> float:
        loss = ctypes.c_float(0)
        _check(self._lib.sse_mlp_train_epoch(self._m, ctypes.c_void_p(_dev_ptr(x, 4)), ctypes.c_void_p(_dev_ptr(t, 4)),
                                             ctypes.c_void_p(_dev_ptr(perm, 4)), perm.numel(), batch,
                                             ctypes.c_float(lr), ctypes.byref(loss), self._stream()),
               "sse_mlp_train_epoch")
        return float(loss.value)


class Server:
    """Request loop over many routers (see sse_server_* in include/sse.h)."""

    def __init__(self, params: Params, n_routers: int = 32, slots: int = 16, slot_pairs: int = 1 << 22,
                 memory_budget: int = 40 << 30, slice_seconds: float | None = None):
        _torch()
        self.params = params
        self._lib = lib()
        cfg = _ServerConfig()
        self._lib.sse_server_config_default(ctypes.byref(cfg))
        cfg.n_routers, cfg.slots, cfg.slot_pairs, cfg.memory_budget = n_routers, slots, slot_pairs, memory_budget
        if slice_seconds is not None:
            cfg.slice_seconds = slice_seconds
        self.slice_seconds = cfg.slice_seconds
        self._s = ctypes.c_void_p()
        _check(self._lib.sse_server_create(ctypes.byref(params.to_c()), ctypes.byref(cfg), ctypes.byref(self._s)),
               "sse_server_create")
        self._views = {}

    def close(self) -> None:
        if getattr(self, "_s", None) is not None and self._s.value:
            for v in self._views.values():
                v.close()
            self._lib.sse_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, router: int, t_arrival: float, pairs: np.ndarray) -> None:
        a = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1)
        _check(self._lib.sse_server_submit(self._s, router, float(t_arrival), ctypes.c_void_p(a.ctypes.data),
                                           a.size // 2), "sse_server_submit")

    def flush(self) -> None:
        _check(self._lib.sse_server_flush(self._s), "sse_server_flush")

    def poll(self, cap: int | None = None):
        """All ready reports as (Report, latency_ms)."""
        cap = self.params.max_candidates if cap is None else cap
        out = []
        while True:
            hosts = np.zeros(cap, np.uint32)
            est = np.zeros(cap, np.float32)
            flags = np.zeros(cap, np.uint8)
            rep = _Report(0, 0, 0, cap, 0, hosts.ctypes.data, est.ctypes.data, flags.ctypes.data)
            lat = ctypes.c_double(0)
            rc = self._lib.sse_server_poll(self._s, ctypes.byref(rep), ctypes.byref(lat))
            if rc == -7:  # nothing ready
                return out
            if rc != SSE_OK and rc != ERR_CAPACITY:
                _check(rc, "sse_server_poll")
            m = min(rep.n_candidates, cap)
            out.append((Report(slice=rep.slice, n_candidates=rep.n_candidates, n_super=rep.n_super,
                               truncated=bool(rep.truncated), hosts=hosts[:m].copy(), est=est[:m].copy(),
                               flags=flags[:m].copy(), status=rc), lat.value))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(self._lib.sse_server_get_stats(self._s, ctypes.byref(st)), "sse_server_get_stats")
        return {name: getattr(st, name) for name, _ in _ServerStats._fields_}

    def router(self, r: int) -> Estimator:
        if r not in self._views:
            h = ctypes.c_void_p()
            _check(self._lib.sse_server_router(self._s, r, ctypes.byref(h)), "sse_server_router")
            self._views[r] = Estimator._borrowed(self.params, h)
        return self._views[r]

    def global_estimator(self) -> Estimator:
        if "global" not in self._views:
            h = ctypes.c_void_p()
            _check(self._lib.sse_server_global(self._s, ctypes.byref(h)), "sse_server_global")
            self._views["global"] = Estimator._borrowed(self.params, h)
        return self._views["global"]
