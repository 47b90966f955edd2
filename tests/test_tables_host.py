"""The library's host threshold tables (csrc/tables.cpp: delay steps, R2;
binomial counts, R8) equal the oracle's, bit for bit, with the same status,
over a grid of parameters and their edge cases (one-step and very wide delay
laws, tables above the size limit, n from 0 to 10^7, p near 0 and 1).  Both
sides run on this host, so any libm they share gives both the same erfc.
Host code only (no GPU): a small program compiled with g++ calls the
library's table builders."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_09855_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "snc_internal.h"

// Lines "d mu sigma dt" or "b n p"; prints "status base t0 t1 ..." per line.
int main() {
  char kind;
  while (std::scanf(" %c", &kind) == 1) {
    std::vector<uint32_t> thr;
    int st;
    unsigned long long base = 0;
    if (kind == 'd') {
      double mu, sigma, dt;
      if (std::scanf("%lf %lf %lf", &mu, &sigma, &dt) != 3) return 2;
      uint32_t b = 0;
      st = snc::delay_thresholds(mu, sigma, dt, thr, b);
      base = b;
    } else {
      unsigned long long n;
      double p;
      if (std::scanf("%llu %lf", &n, &p) != 2) return 2;
      uint64_t b = 0;
      st = snc::binomial_thresholds(n, p, thr, b);
      base = b;
    }
    std::printf("%d %llu", st, st == 0 ? base : 0ull);
    if (st == 0)
      for (uint32_t t : thr) std::printf(" %u", t);
    std::printf("\n");
  }
  return 0;
}
"""

DELAYS = ([(mu, sigma, dt) for mu, sigma, dt in itertools.product((0.1, 0.75, 1.5, 5.0, 20.0), (0.01, 0.375, 0.75, 3.0),
                                                                    (0.1, 0.05, 1.0))] +
          [(1.5, 1e-9, 0.1), (0.0, 0.5, 0.1), (-3.0, 1.0, 0.1), (1.5, 200.0, 0.1), (6000.0, 10.0, 0.1),
           (7000.0, 1.0, 0.1), (1.5, 0.75, 1e-4)])
BINOMS = ([(n, p) for n, p in itertools.product((0, 1, 2, 10, 100, 1999, 100_000, 10_000_000),
                                                (0.0, 1e-9, 1e-4, 0.01, 0.3, 0.5, 0.99, 1 - 1e-9, 1.0))] +
          [(4_000_000_000, 0.5), (50, 0.02)])


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2306_09855_gb300 import _build
    lib = _build.build()
    d = tmp_path_factory.mktemp("tables")
    (d / "tables.cpp").write_text(PROGRAM)
    exe = d / "tables"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", cuda_inc, str(d / "tables.cpp"), "-o", str(exe),
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    lines = ["d %r %r %r" % c for c in DELAYS] + ["b %d %r" % c for c in BINOMS]
    r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stderr)
    rows = [list(map(int, ln.split())) for ln in r.stdout.strip().split("\n")]
    assert len(rows) == len(lines)
    return rows[:len(DELAYS)], rows[len(DELAYS):]


def _oracle(fn, *args):
    import oracle
    try:
        base, thr = fn(*args)
        return 0, base, thr
    except oracle.OracleError as e:
        return e.status, None, None


def test_delay_tables_equal_the_oracle(tables, oracle_mod):
    rows, _ = tables
    statuses = set()
    for (mu, sigma, dt), row in zip(DELAYS, rows):
        st, base, thr = _oracle(oracle_mod.delay_table, mu, sigma, dt)
        assert row[0] == st, (mu, sigma, dt, row[0], st)
        statuses.add(st)
        if st == 0:
            assert row[1] == base, (mu, sigma, dt)
            np.testing.assert_array_equal(np.array(row[2:], dtype=np.uint64), thr.astype(np.uint64))
    assert statuses == {0, 6}  # accepted laws and laws beyond the table or step limits


def test_binomial_tables_equal_the_oracle(tables, oracle_mod):
    _, rows = tables
    for (n, p), row in zip(BINOMS, rows):
        st, base, thr = _oracle(oracle_mod.binom_table, n, p)
        assert row[0] == st, (n, p, row[0], st)
        if st == 0:
            assert row[1] == base, (n, p, row[1], base)
            np.testing.assert_array_equal(np.array(row[2:], dtype=np.uint64), thr.astype(np.uint64))
