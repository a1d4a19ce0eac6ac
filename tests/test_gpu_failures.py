"""Failure detection without a GPU fault: a bounded device-side wait that runs out is
reported as SSE_ERR_TIMEOUT and leaves the handle usable.

The ordering of more than 4096 candidates is one cooperative launch whose blocks meet at
grid-wide barriers; every wait there polls a bounded number of times. The test hook
sse_debug_sort_barrier makes each barrier wait for a block that does not exist, with a
short poll limit, so the waits run out (nothing faults, traps or hangs); the next close,
with the hook off, must equal the oracle.
"""
import numpy as np
import pytest

import oracle
from tests import helpers
from tests.test_gpu_parity import compare_report, compare_state, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sse():
    from paper_1805_09246_b300 import sse as mod
    return mod


def heavy_hosts_traffic(rng, hosts, per_host=8):
    """Every host sends to per_host random destinations."""
    dst = rng.integers(0, 2**32, per_host * len(hosts), dtype=np.uint64).astype(np.uint32)
    return np.stack([np.repeat(hosts, per_host), dst], axis=1)


@pytest.mark.parametrize("graph", [True, False])
def test_sort_barrier_timeout_is_reported_and_the_handle_recovers(graph):
    S = sse()
    # theta = eta = 8 gives tau = 0: every pair reaches the RSRA, so ~6000 hosts with 8
    # destinations each are all hot in all five rows (q = 20 keeps false candidates out)
    p = S.Params(q=20, theta=8, seed=51)
    rng = np.random.default_rng(51)
    hosts = np.unique(rng.integers(0, 2**32, 6000, dtype=np.uint64).astype(np.uint32))
    est = S.Estimator(p)
    est.close_use_graph(graph)
    orc = oracle.Oracle(oracle_params(p))

    pairs = heavy_hosts_traffic(rng, hosts)
    est.update(helpers.to_device(pairs))
    orc.scan(pairs)
    est.debug_sort_barrier(1000, 1)  # every barrier wait runs out after 1000 polls
    with pytest.raises(S.SSEError) as err:
        est.close_slice()
    assert err.value.code == S.ERR_TIMEOUT
    assert est.slice == 1  # the slice was closed all the same
    assert est.stats()["n_candidates"] > 4096  # the sort did reach its barriers

    est.debug_sort_barrier(0, 0)
    orc.advance()
    pairs = heavy_hosts_traffic(rng, hosts)
    est.update(helpers.to_device(pairs))
    orc.scan(pairs)
    rep = est.close_slice()
    # Algorithms 4-5 by their definition (the oracle's tuple growth is cubic in the ~6000
    # hot SREs per row): every 32-bit address whose r SREs are hot, then Algorithm 8
    want = orc.candidates_brute()
    assert len(want) > 4096
    det = orc.estimate(want)
    det["hosts"] = want
    compare_report(rep, det)
    compare_state(est, orc, p, 1)
    assert np.array_equal(est.hot_bitmap(), orc.hot())


def test_debug_sort_barrier_rejects_more_than_one_missing_block():
    S = sse()
    est = S.Estimator(S.Params(seed=52))
    with pytest.raises(S.SSEError) as err:
        est.debug_sort_barrier(1000, 2)
    assert err.value.code == -1
