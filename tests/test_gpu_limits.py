"""The estimator at the largest sizes that parameter validation accepts, against the oracle.

q = 26: RSRA of 5 x 2^26 SREs of 8 cells (2.7 G 8-bit cells, past 2^31 in the close pass).
q' = 24 with eta' = 65536: SLEA rows of 2^28 + 65520 cells (1.34 G cells in all), so the tiled
update splits every row into 164 bitmap pieces and the estimate gathers SLEs of 64 Ki cells.
Small traffic (three slices of 2^17 pairs with 20 planted super points) keeps the oracle's
part to seconds; state, hot SREs, row counts and reports are compared as everywhere else,
for both update strategies.
"""
import numpy as np
import pytest

import oracle
from paper_1805_09246_b300 import synth
from tests import helpers
from tests.test_gpu_parity import DIRECT, TILED, compare_report, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHUNK = 1 << 26


def canonical_lut(slice_index: int, k: int) -> np.ndarray:
    """8-bit stamp -> the oracle's canonical cell (its age when active, else 255)."""
    s = np.arange(256)
    age = (helpers.stamp(slice_index) - s) % helpers.modulus(8)
    return np.where((s != 0) & (age < k), age, 255).astype(np.uint8)


def same_cells(stamps: np.ndarray, want: np.ndarray, lut: np.ndarray) -> None:
    for i in range(0, stamps.size, CHUNK):
        assert np.array_equal(lut[stamps[i:i + CHUNK]], want[i:i + CHUNK])


@pytest.mark.parametrize("mode", [DIRECT, TILED])
@pytest.mark.parametrize("shape", ["rsra_q26", "slea_q24_eta64k"])
def test_largest_dimensions_match_oracle(shape, mode):
    from paper_1805_09246_b300 import sse as S
    if shape == "rsra_q26":
        p = S.Params(q=26, k=3, seed=31)
    else:
        p = S.Params(q=14, q2=24, eta2=65536, k=3, seed=37)
    tr = synth.Traffic(synth.small_trace(seed=p.seed))
    est = S.Estimator(p)
    est.set_update_mode(mode)
    orc = oracle.Oracle(oracle_params(p))
    for t in range(3):
        if t:
            orc.advance()
        pairs = tr.slice(0, t)
        est.update(helpers.to_device(pairs))
        orc.scan(pairs)
        rep = est.close_slice()
    det = orc.detect()
    compare_report(rep, det)
    assert rep.n_super >= 15
    assert np.array_equal(est.hot_bitmap(), orc.hot())
    assert est.stats()["active2"] == orc.row_counts().tolist()
    lut = canonical_lut(2, p.k)
    g_sre, g_sle = est.read_stamps()
    o_sre, o_sle = orc.canonical()
    same_cells(g_sre.reshape(-1), o_sre.reshape(-1), lut)
    del g_sre, o_sre
    for row in range(p.r2):
        same_cells(g_sle[row], o_sle[row], lut)


@pytest.mark.parametrize("mode", [DIRECT, TILED])
def test_most_rows_match_oracle(mode):
    """r = r' = 16, the most rows validation accepts (delta = 2 at q = 14: a chain's 16 rows
    each add two address bits), over four slices of the small trace: state, hot SREs, row
    counts and reports every slice."""
    from paper_1805_09246_b300 import sse as S
    from tests.test_gpu_parity import run_both
    p = S.Params(r=16, q=14, r2=16, seed=43)
    tr = synth.Traffic(synth.small_trace(seed=43))
    _, _, reports = run_both(p, [tr.slice(0, t) for t in range(4)], mode=mode)
    assert reports[-1].n_super >= 15
