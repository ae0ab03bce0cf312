"""The exact-slice peel's final rounding, RN_fp32(q 2^e) in integer
arithmetic (csrc/rn_scaled.cuh), compiled for the host and checked bit for
bit against the C library's rounding of the exact FP64 value (float)(double)
ldexp(q, e) -- exact in FP64 for |q| < 2^53 -- over random and structured
(q, e): halfway ties, carries into the exponent, subnormal results,
underflow to zero and overflow to infinity."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_11563_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include "rn_scaled.cuh"

static unsigned bits(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }

int main() {
  std::mt19937_64 g(20261203);
  long bad = 0, n = 0, sub = 0, inf = 0, zero = 0, ties = 0;
  auto check = [&](long long q, int e) {
    const float want = static_cast<float>(std::ldexp(static_cast<double>(q), e));
    const float got = bpx::rn_float_scaled(q, e);
    ++n;
    if (std::isinf(want)) ++inf;
    else if (want == 0.f && q != 0) ++zero;
    else if (std::fpclassify(want) == FP_SUBNORMAL) ++sub;
    if (bits(want) != bits(got)) {
      if (bad < 5) std::printf("MISMATCH q=%lld e=%d want=%a got=%a\n", q, e, want, got);
      ++bad;
    }
  };
  for (int it = 0; it < 3000000; ++it) {
    const int nb = static_cast<int>(g() % 54);
    long long q = nb ? static_cast<long long>(g() & ((1ull << nb) - 1)) : 0;
    if (g() & 1) q = -q;
    check(q, static_cast<int>(g() % 420) - 260);
  }
  // halfway cases: 24 kept bits, then a 1 followed by zeros (ties to even) or
  // by a sticky bit, with the kept part odd or even
  for (int sh = 1; sh < 29; ++sh)
    for (int odd = 0; odd < 2; ++odd)
      for (int sticky = 0; sticky < 2; ++sticky)
        for (int e = -200; e <= 110; e += 3) {
          const long long kept = (1ll << 23) | static_cast<long long>(g() % (1 << 23) & ~1ll) | odd;
          const long long q = (kept << sh) | (1ll << (sh - 1)) | (sticky && sh > 1 ? 1ll : 0ll);
          check(q, e);
          check(-q, e);
          ++ties;
        }
  // carries: all ones below the kept bits round up into the exponent
  for (int sh = 1; sh < 29; ++sh)
    for (int e = -180; e <= 110; ++e) check(((1ll << (24 + sh)) - 1), e);
  std::printf("checked %ld bad %ld subnormal %ld inf %ld zero %ld ties %ld\n", n, bad, sub, inf, zero, ties);
  return bad != 0;
}
"""


def test_rn_float_scaled_matches_library_rounding(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "rn_check.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "rn_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True, timeout=300)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    stats = dict(zip(out.stdout.split()[0::2], out.stdout.split()[1::2]))
    assert int(stats["bad"]) == 0
    # the structured cases reached every regime
    assert int(stats["subnormal"]) > 1000 and int(stats["inf"]) > 1000 and int(stats["zero"]) > 1000
    assert int(stats["ties"]) > 1000
