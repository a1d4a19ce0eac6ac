"""Host-side check of the searches that regain uses in the join (regain_search and
regain_search_bucketed in csrc/sse_internal.cuh): for a complete chain, the low address bits whose multiply-add-shift
RHFG[0] value lands on he_0 are those low < 2^delta with (v + a*low) mod 2^64 below
2^(64-q). The search over the sorted a*low table is compared, case by case, with the plain
loop over every low: random multipliers and offsets, offsets placed just inside and just
outside the interval's ends, every delta 0..5 and q 5..26. Compiled by nvcc as host code;
no GPU needed."""
import os
import shutil
import subprocess

import pytest

from tests.conftest import ROOT

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

PROGRAM = r"""
#include <algorithm>
#include <cstdio>
#include <vector>
#include "sse_internal.cuh"
using namespace sse;
static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next64() {  // xorshift64*
  state ^= state >> 12; state ^= state << 25; state ^= state >> 27;
  return state * 0x2545F4914F6CDD1Dull;
}
int main() {
  long checked = 0, bad = 0, hits = 0;
  for (uint32_t delta = 0; delta <= 5; ++delta)
    for (uint32_t q = 5; q <= 26; ++q)
      for (int rep = 0; rep < 400; ++rep) {
        const uint32_t n = 1u << delta;
        const uint64_t a = next64() | 1ull, width = 1ull << (64 - q);
        std::vector<std::pair<uint64_t, uint32_t>> t;
        for (uint32_t low = 0; low < n; ++low) t.push_back({a * low, low});
        std::sort(t.begin(), t.end());
        uint64_t d[32];
        uint32_t lows[32];
        for (uint32_t i = 0; i < n; ++i) { d[i] = t[i].first; lows[i] = t[i].second; }
        for (int k = 0; k < 8; ++k) {
          uint64_t v = next64();
          const uint64_t edge = 0ull - a * (next64() % n);  // v + a*low lands on 0 for that low
          if (k == 1) v = edge;                  // at the interval's start
          if (k == 2) v = edge - 1;              // just before it
          if (k == 3) v = edge + width - 1;      // at its last value
          if (k == 4) v = edge + width;          // just past it
          if (k == 5) v = edge - (width >> 1);   // halfway outside
          uint32_t want = 0, got = 0;
          for (uint32_t low = 0; low < n; ++low)
            if (v + a * low < width) want |= 1u << low;
          regain_search(d, lows, n, v, width, [&](uint32_t low) {
            if (got & (1u << low)) ++bad;  // each low once
            got |= 1u << low;
          });
          // the bucketed search: entries below each 2^58-wide bucket
          uint8_t first[65];
          for (uint32_t j = 0; j <= 64; ++j) {
            uint32_t below = 0;
            for (uint32_t i = 0; i < n; ++i) below += (d[i] >> 58) < j ? 1u : 0u;
            first[j] = (uint8_t)below;
          }
          uint32_t got2 = 0;
          regain_search_bucketed(d, lows, first, n, v, width, [&](uint32_t low) {
            if (got2 & (1u << low)) ++bad;
            got2 |= 1u << low;
          });
          ++checked;
          if (got != want || got2 != want) ++bad;
          if (want) ++hits;
        }
      }
  printf("%ld %ld %ld\n", checked, bad, hits);
  return bad != 0;
}
"""


@pytest.mark.skipif(not os.path.exists(NVCC) and shutil.which("nvcc") is None, reason="nvcc not available")
def test_regain_search_equals_the_loop_over_every_low(tmp_path):
    src = tmp_path / "regain.cu"
    exe = tmp_path / "regain"
    src.write_text(PROGRAM)
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-I",
                    os.path.join(ROOT, "paper_1805_09246_b300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad, hits = map(int, out.stdout.split())
    assert checked == 6 * 22 * 400 * 8 and bad == 0
    assert hits > 1000  # the boundary cases put lows inside the interval
    assert out.returncode == 0
