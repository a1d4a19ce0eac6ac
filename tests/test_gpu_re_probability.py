"""The GPU estimator's rough-estimator detection rate against the paper's Eq. 5 on tens of
thousands of lone hosts (one slice, k = 1): the share of hosts whose row-0 SRE is hot."""
import math

import numpy as np
import pytest

import oracle
from oracle import re_probability as rp
from tests import helpers
from tests.test_gpu_parity import oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_dst", [512, 1024, 1536])
def test_gpu_hot_rate_matches_eq5(n_dst):
    from paper_1805_09246_b300 import sse
    p = sse.Params(q=20, q2=16, eta2=4096, k=1, theta=1024, seed=41 + n_dst)
    rng = np.random.default_rng(n_dst)
    hosts = np.unique(rng.integers(0, 2**32, 20000, dtype=np.uint64).astype(np.uint32))
    pairs = np.stack([np.repeat(hosts, n_dst),
                      rng.integers(0, 2**32, len(hosts) * n_dst, dtype=np.uint64).astype(np.uint32)], 1)
    est = sse.Estimator(p)
    est.update(helpers.to_device(pairs))
    est.close_slice()
    hot = est.hot_bitmap()[0]
    orc = oracle.Oracle(oracle_params(p))  # the hash functions only (nothing scanned)
    cols = np.array([orc.rhfg(0, int(h)) for h in hosts])
    _, inv, counts = np.unique(cols, return_inverse=True, return_counts=True)
    lone = counts[inv] == 1
    got = hot[cols[lone]].mean()
    q = rp.pr_reported(n_dst, 8, sse.derive(p)["tau"], 3, alpha_max=400)
    m = lone.sum()
    assert abs(got - q) <= 4.5 * math.sqrt(q * (1 - q) / m), (got, q, m)
