"""The C ABI library loads without a GPU and exports every entry point of include/sse.h;
host-only logic (parameter validation and derivation) agrees with the oracle's."""
import ctypes
import os
import re

import pytest

import oracle
from paper_1805_09246_b300 import build as sse_build
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "sse.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))


def declared_symbols(path):
    text = open(path).read()
    return sorted(set(re.findall(r"^SSE_API [^(]*?\b(\w+)\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libsse():
    return ctypes.CDLL(sse_build.build())


def test_header_declares_the_boundary():
    names = declared_symbols(HEADER)
    for want in ("sse_init", "sse_update", "sse_close_slice", "sse_merge", "sse_query", "sse_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(libsse):
    assert len(HEADERS) >= 2
    for path in HEADERS:
        for name in declared_symbols(path):
            assert hasattr(libsse, name), f"{os.path.basename(path)}: {name}"


def _params(**kw):
    from paper_1805_09246_b300.sse import Params
    return Params(**kw)


def test_derivation_matches_oracle(libsse):
    from paper_1805_09246_b300 import sse
    cases = [dict(), dict(q=17, q2=17, eta2=1 << 14, k=8), dict(q=20, q2=16, eta2=4096, k=8),
             dict(theta=1, eta2=64, q2=4), dict(theta=5000, r=6, q=12)]
    fields = oracle.Params.__dataclass_fields__
    for kw in cases:
        mine = sse.derive(_params(**kw))
        theirs = oracle.derive(oracle.Params(**{k: v for k, v in _params(**kw).__dict__.items() if k in fields}))
        assert mine["delta"] == theirs["delta"]
        assert mine["tau"] == theirs["tau"]
        assert mine["hot_min"] == theirs["hot_min"]
        assert mine["row_len2"] == theirs["row_len2"]
        assert mine["w_theta"] == theirs["w_theta"]  # same double, computed on the host
        assert mine["row_pitch2"] % 4096 == 0 and mine["row_pitch2"] >= mine["row_len2"]


def test_invalid_parameters_rejected(libsse):
    from paper_1805_09246_b300 import sse
    bad = [dict(r=2), dict(q=4), dict(q=14, delta=5), dict(eta=16), dict(eta2=1000), dict(k=0), dict(k=255),
           dict(theta=0), dict(stamp_bits=12), dict(stamp_bits=16, k=65535), dict(max_candidates=0), dict(r2=17),
           dict(delta2=0)]
    for kw in bad:
        with pytest.raises(sse.SSEError):
            sse.derive(_params(**kw))


def test_paper_defaults(libsse):
    from paper_1805_09246_b300 import sse
    p = sse.paper_params()
    assert (p.r, p.q, p.delta, p.eta, p.r2, p.q2, p.delta2, p.eta2, p.theta) == (5, 17, 5, 8, 5, 17, 16, 1 << 14, 1024)
    assert (p.k, p.stamp_bits) == (300, 16)  # the sliding-window experiment (Section 5)
    d = sse.derive(p)
    assert d["sre_bytes"] == 5 * (1 << 17) * 8 * 2 and d["sle_bytes"] == 5 * d["row_pitch2"] * 2
