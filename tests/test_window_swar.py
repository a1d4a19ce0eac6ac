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


PROGRAM16 = r"""
#include <cstdio>
#include "sse_internal.cuh"
using namespace sse;
static unsigned plain_active(unsigned s, unsigned cs, unsigned k) {
  if (s == 0) return 0;
  return ((cs + 65535 - s) % 65535) < k ? 1u : 0u;
}
static unsigned long long state = 88172645463325252ull;
static unsigned next32() { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return (unsigned)state; }
int main() {
  long bad = 0, checked = 0;
  // windows: every k up to 300 (the paper's) and a spread of larger ones up to 65534
  unsigned ks[400];
  int nk = 0;
  for (unsigned k = 1; k <= 300; ++k) ks[nk++] = k;
  for (int i = 0; i < 60; ++i) ks[nk++] = 301 + next32() % 65234;
  ks[nk++] = 65534;
  for (int ik = 0; ik < nk; ++ik) {
    const unsigned k = ks[ik];
    // current stamps: the ends of the cycle, around k, and random ones
    unsigned css[40];
    int nc = 0;
    const unsigned fixed[] = {1, 2, 3, k - 1 ? k - 1 : 1, k, k + 1 <= 65535 ? k + 1 : 65535, 65533, 65534, 65535};
    for (unsigned c : fixed) css[nc++] = c;
    for (int i = 0; i < 24; ++i) css[nc++] = 1 + next32() % 65535;
    for (int ic = 0; ic < nc; ++ic) {
      const unsigned cs = css[ic];
      const Window16 w = window16(cs, k);
      // stamps: unset, the window's ends and their neighbours, the cycle's ends, random ones
      unsigned st[64];
      int ns = 0;
      const unsigned L = cs >= k ? cs - k + 1 : cs + 65535 - k + 1;
      const unsigned near[] = {0, 1, 2, 65534, 65535, cs, cs - 1, cs + 1, L, L - 1, L + 1};
      for (unsigned x : near) st[ns++] = x & 0xFFFFu;
      for (int i = 0; i < 40; ++i) st[ns++] = next32() & 0xFFFFu;
      for (int a = 0; a < ns; ++a)
        for (int b = 0; b < ns; b += 3) {  // pairs of halves, so that the halves interact
          const unsigned word = st[a] | (st[b] << 16);
          const unsigned got = active_hi16(word, w);
          ++checked;
          if (((got >> 15) & 1u) != plain_active(st[a], cs, k)) ++bad;
          if (((got >> 31) & 1u) != plain_active(st[b], cs, k)) ++bad;
          if (got & 0x7FFF7FFFu) ++bad;  // only the top bit of a half may be set
        }
    }
  }
  printf("%ld %ld\n", checked, bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(not os.path.exists(NVCC) and shutil.which("nvcc") is None, reason="nvcc not available")
def test_half_word_window_test_matches_the_definition(tmp_path):
    """active_hi16 (two 16-bit stamps per word) against the plain definition: every window
    up to the paper's 300 slices and a spread of larger ones, current stamps at the ends of
    the 65535-slice cycle, around k and random, stamps at the window's edges and random."""
    src = tmp_path / "window16.cu"
    exe = tmp_path / "window16"
    src.write_text(PROGRAM16)
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1805_09246_b300", "csrc"),
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, out.stdout.split())
    assert checked > 1_000_000 and bad == 0
    assert out.returncode == 0
