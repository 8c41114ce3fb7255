"""The flag kernel's ticket decode divides by the blocks per MCS, the blocks
per coarse phase and half the blocks per row with host-computed reciprocals
(div_rcp32 / div_by_rcp in csrc/escg_types.h) instead of the device's
division.  The helpers are plain host C++ as well, so they are checked here
against exact integer division: every numerator below 20000, random 32-bit
numerators, the numerators on both sides of multiples of the divisor, and
2^32 - 1, for divisors 1..4000 and a geometric sweep up to 2^31."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_16639_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "escg_types.h"
using namespace escg_impl;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint32_t next_u32() {   // splitmix64
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (uint32_t)(z ^ (z >> 31));
}

int main() {
  long bad = 0, checked = 0;
  auto check = [&](uint32_t n, uint32_t d, uint32_t rcp) {
    uint32_t r = 0;
    const uint32_t q = div_by_rcp(n, d, rcp, r);
    if (q != n / d || r != n % d) {
      if (bad < 5) std::printf("n=%u d=%u: q=%u r=%u\n", n, d, q, r);
      ++bad;
    }
    ++checked;
  };
  for (uint64_t dd = 1; dd <= 0x80000000ull; dd = dd < 4000 ? dd + 1 : dd * 5 / 4 + 7) {
    const uint32_t d = (uint32_t)dd, rcp = div_rcp32(d);
    for (uint32_t n = 0; n < 20000; ++n) check(n, d, rcp);
    for (int i = 0; i < 4000; ++i) check(next_u32(), d, rcp);
    for (uint32_t k = 1; k <= 64; ++k) {
      const uint64_t base = (uint64_t)d * (0xFFFFFFFFull / d / 64) * k;
      for (int e = -1; e <= 1; ++e)
        if (base + e <= 0xFFFFFFFFull) check((uint32_t)(base + e), d, rcp);
    }
    check(0xFFFFFFFFu, d, rcp);
  }
  std::printf("checked %ld bad %ld\n", checked, bad);
  return bad != 0;
}
"""


def test_reciprocal_division_is_exact(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "div_check.cpp"
    exe = tmp_path / "div_check"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "bad 0" in out.stdout
