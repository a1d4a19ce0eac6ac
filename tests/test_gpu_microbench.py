"""The roof microbenchmarks (sse_microbench) run through the C ABI and return rates in the
ranges a B300 allows; bad arguments are refused before any launch."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_microbench_rates_are_positive_and_ordered():
    from paper_1805_09246_b300 import sse
    mb = sse.microbench()
    assert mb["sms"] > 0
    for key in ("l2_random_byte_stores_per_s", "smem_random_atomics_per_s", "l2_stream_load_bytes_per_s",
                "hbm_stream_load_bytes_per_s", "tiled_skeleton_pairs_per_s"):
        assert mb[key] > 0, key
    # L2-resident loads are faster than loads from HBM; the skeleton's five loads and atomics per
    # pair cannot outrun either unit alone
    assert mb["l2_stream_load_bytes_per_s"] > mb["hbm_stream_load_bytes_per_s"]
    assert mb["tiled_skeleton_pairs_per_s"] < mb["smem_random_atomics_per_s"] / 5 * 1.5
    assert mb["tiled_skeleton_pairs_per_s"] * 5 * 8 < mb["l2_stream_load_bytes_per_s"] * 1.5


def test_microbench_rejects_small_or_misaligned_buffers():
    from paper_1805_09246_b300 import sse
    out = sse._MicrobenchResult()
    small = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    fn = sse.lib().sse_microbench
    assert fn(ctypes.c_void_p(small.data_ptr()), small.numel(), None, ctypes.byref(out)) == -1
    big = torch.empty(sse.MICROBENCH_MIN_BYTES + 256, dtype=torch.uint8, device="cuda")
    assert fn(ctypes.c_void_p(big.data_ptr() + 16), sse.MICROBENCH_MIN_BYTES, None, ctypes.byref(out)) == -1
    assert fn(None, sse.MICROBENCH_MIN_BYTES, None, ctypes.byref(out)) == -1
