"""The allocation-free query (sse_query_noalloc), called through the C ABI.

It is meant for callers that may not allocate device memory themselves (for instance a
data-plane process given fixed device buffers by its framework). Its results must equal
those of sse_query() on an estimator holding the same stamps, on consecutive calls that
reuse the library's shared scratch counters. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers
from tests.test_gpu_parity import oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EST_RTOL = 1e-6


def noalloc_fn():
    from paper_1805_09246_b300 import sse
    fn = sse.lib().sse_query_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def test_noalloc_query_matches_query_on_two_calls():
    from paper_1805_09246_b300 import sse
    fn = noalloc_fn()
    p = sse.Params(seed=21)
    tr = synth.Traffic(synth.small_trace(seed=21))
    est = sse.Estimator(p)
    orc = oracle.Oracle(oracle_params(p))
    stream = torch.cuda.current_stream()
    ip, _ = tr.planted()
    rng = np.random.default_rng(21)
    for call in range(2):
        # a different window for each call: the scratch must not keep the first call's counts
        for t in range(3 * call, 3 * call + 3):
            est.update(helpers.to_device(tr.slice(0, t)))
            orc.scan(tr.slice(0, t))
            if t < 3 * call + 2:
                est.advance()
                orc.advance()
        _, sle = est.read_stamps()
        sle_padded = np.zeros((p.r2, est.derived["row_pitch2"]), np.uint8)
        sle_padded[:, : sle.shape[1]] = sle
        d_sle = torch.from_numpy(sle_padded).cuda()
        hosts = np.concatenate([ip, tr.slice(0, 0)[:300, 0],
                                rng.integers(0, 2**32, 200, dtype=np.uint64).astype(np.uint32)])
        d_hosts = helpers.to_device(hosts)
        n = len(hosts)
        d_est = torch.empty(n, dtype=torch.float32, device="cuda")
        d_flags = torch.empty(n, dtype=torch.uint8, device="cuda")
        rc = fn(ctypes.byref(p.to_c()), d_sle.data_ptr(), est.slice, d_hosts.data_ptr(), n, d_est.data_ptr(),
                d_flags.data_ptr(), stream.cuda_stream)
        assert rc == 0
        ref_est, ref_flags = est.query(d_hosts)
        torch.cuda.synchronize()
        got, ref = d_est.cpu().numpy().astype(np.float64), ref_est.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= EST_RTOL * np.maximum(np.abs(ref), 1e-30))
        assert np.array_equal(d_flags.cpu().numpy(), ref_flags.cpu().numpy())
        assert (ref_flags.cpu().numpy() & sse.FLAG_SUPER).any()
        # and directly against the oracle's Algorithm 8 on the same window
        want = orc.estimate(hosts)
        assert np.all(np.abs(got - want["est"]) <= EST_RTOL * np.maximum(want["est"], 1e-30))
        assert np.array_equal(d_flags.cpu().numpy(), want["flags"])


def test_noalloc_query_rejects_rows_beyond_the_validator_limit_and_16bit_stamps():
    """r' = 17 fails parameter validation (the scratch array holds a counter for every r'
    that validation accepts); 16-bit stamps are refused with INVALID_PARAM."""
    from paper_1805_09246_b300 import sse
    fn = noalloc_fn()
    assert fn(ctypes.byref(sse.Params(r2=17).to_c()), None, 0, None, 1, None, None, None) == -1
    p16 = sse.Params(stamp_bits=16)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert fn(ctypes.byref(p16.to_c()), dummy.data_ptr(), 0, dummy.data_ptr(), 1, dummy.data_ptr(),
              None, None) == -1
