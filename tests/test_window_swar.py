"""Host-side check of the byte-wise window test the close and estimate kernels use
(active_hi8 in csrc/sse_internal.cuh): compiled by nvcc as host code and compared, for every
window k, current stamp and stamp value, with the plain definition of an active 8-bit cell
(set, and its cyclic age (cs - s) mod 255 below k). Runs on the CPU; no GPU needed."""
import os
import shutil
import subprocess

import pytest

from tests.conftest import ROOT

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

PROGRAM = r"""
#include <cstdio>
#include "sse_internal.cuh"
using namespace sse;
static unsigned plain_active(unsigned s, unsigned cs, unsigned k) {
  if (s == 0) return 0;
  return ((cs + 255 - s) % 255) < k ? 1u : 0u;
}
int main() {
  long bad = 0, checked = 0;
  for (unsigned k = 1; k <= 254; ++k)
    for (unsigned cs = 1; cs <= 255; ++cs) {
      const Window8 w = window8(cs, k);
      for (unsigned s0 = 0; s0 < 256; ++s0) {
        // four different stamps per word, so that neighbouring bytes interact
        const unsigned st[4] = {s0, (s0 * 7 + 3) & 255u, s0 ^ 0x5Au, 255u - s0};
        const unsigned word = st[0] | (st[1] << 8) | (st[2] << 16) | (st[3] << 24);
        const unsigned a = active_hi8(word, w);
        for (int b = 0; b < 4; ++b) {
          ++checked;
          if (((a >> (8 * b + 7)) & 1u) != plain_active(st[b], cs, k)) ++bad;
          if ((a >> (8 * b)) & 0x7Fu) ++bad;  // only the top bit of a byte may be set
        }
      }
    }
  printf("%ld %ld\n", checked, bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(not os.path.exists(NVCC) and shutil.which("nvcc") is None, reason="nvcc not available")
def test_byte_window_test_matches_the_definition(tmp_path):
    src = tmp_path / "window.cu"
    exe = tmp_path / "window"
    src.write_text(PROGRAM)
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1805_09246_b300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, out.stdout.split())
    assert checked == 254 * 255 * 256 * 4 and bad == 0
    assert out.returncode == 0
