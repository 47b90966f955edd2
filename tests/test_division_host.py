"""The generation kernels split a connection index i into (primary, slot) =
(i / K, i % K) with a multiply-high and two shifts (Granlund & Montgomery
1994, Fig. 4.1) instead of the compiler's division sequence.  The host
computes the multiplier and shifts (division_magic in snc_internal.h); this
test compiles that function with the host compiler and checks the quotient
formula against integer division for divisors 1..4096, the powers of two and
their neighbours up to 2^32 - 1, and random divisors, at dividends 0, 1, the
multiples of d and their neighbours, 2^32 - 1 and random values."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <cstdio>
#include <cstdint>
#include <random>
#include "snc_internal.h"

static int check(uint32_t d, uint32_t n) {
  uint32_t mul, sh1, sh2;
  snc::division_magic(d, &mul, &sh1, &sh2);
  const uint32_t t = static_cast<uint32_t>((static_cast<uint64_t>(n) * mul) >> 32);
  const uint32_t q = (t + ((n - t) >> sh1)) >> sh2;
  if (q != n / d) {
    std::printf("d=%u n=%u q=%u want=%u\n", d, n, q, n / d);
    return 1;
  }
  return 0;
}

int main() {
  std::mt19937_64 rng(7);
  std::vector<uint32_t> ds;
  for (uint32_t d = 1; d <= 4096; ++d) ds.push_back(d);
  for (int b = 1; b < 32; ++b) {
    const uint64_t p = 1ull << b;
    for (int64_t o = -2; o <= 2; ++o)
      if (p + o >= 1 && p + o <= 0xFFFFFFFFull) ds.push_back(static_cast<uint32_t>(p + o));
  }
  ds.push_back(0xFFFFFFFFu);
  ds.push_back(0xFFFFFFFEu);
  for (int k = 0; k < 2000; ++k) ds.push_back(static_cast<uint32_t>(rng() % 0xFFFFFFFFull) + 1u);
  int bad = 0;
  for (uint32_t d : ds) {
    const uint32_t fixed[] = {0u, 1u, 2u, d - 1u, d, d + 1u, 0xFFFFFFFFu, 0xFFFFFFFEu, 0x80000000u, 0x7FFFFFFFu};
    for (uint32_t n : fixed) bad += check(d, n);
    const uint64_t top = 0xFFFFFFFFull / d;
    for (int k = 0; k < 64; ++k) {
      const uint64_t m = (top ? rng() % (top + 1) : 0) * d;
      for (int64_t o = -1; o <= 1; ++o)
        if (static_cast<int64_t>(m) + o >= 0 && m + o <= 0xFFFFFFFFull) bad += check(d, static_cast<uint32_t>(m + o));
      bad += check(d, static_cast<uint32_t>(rng()));
    }
    if (bad > 10) break;
  }
  std::printf("%s\n", bad ? "FAIL" : "OK");
  return bad ? 1 : 0;
}
'''


def test_division_magic_equals_integer_division(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    src = tmp_path / "div.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "div"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2306_09855_gb300", "csrc"),
                    "-I", inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:]
