"""The served form's admission decision (snc_server.cpp admit_from_front) on
fake queues, host code only (no GPU): on seeded random queues the requests
that start are a front run of the queue that fits the memory budget; a batch
(more than one) holds only small requests, none built alone, within the
network, connection and key-width limits; and the run stops only where the
next request breaks one of those limits.  A small program compiled with g++
calls the library's function."""
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

// Per case: "n budget reserved batch_max_syn batch_max_nets" then n lines
// "peak n_syn n_nodes max_step alone"; prints "take reserve".
int main() {
  unsigned long long n, budget, reserved, max_syn;
  int max_nets;
  while (std::scanf("%llu %llu %llu %llu %d", &n, &budget, &reserved, &max_syn, &max_nets) == 5) {
    std::vector<snc::AdmitRequest> q(n);
    for (auto& r : q) {
      unsigned long long peak, syn, nodes;
      unsigned step, alone;
      if (std::scanf("%llu %llu %llu %u %u", &peak, &syn, &nodes, &step, &alone) != 5) return 2;
      r = {peak, syn, nodes, step, alone != 0};
    }
    uint64_t reserve = 0;
    const size_t take = snc::admit_from_front(q.data(), q.size(), {budget, reserved, max_syn, max_nets}, &reserve);
    std::printf("%zu %llu\n", take, static_cast<unsigned long long>(reserve));
  }
  return 0;
}
"""


def _bits(v):
    return int(v).bit_length()


def _cases(seed=3, count=2000):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(0, 12))
        budget = int(rng.integers(1, 1000))
        reserved = int(rng.integers(0, budget + 1))
        max_syn = int(rng.integers(1, 400))
        max_nets = int(rng.integers(1, 8))
        q = []
        for _ in range(n):
            big_nodes = rng.random() < 0.1
            q.append((int(rng.integers(1, budget // 2 + 2)), int(rng.integers(0, max_syn)),
                      int(rng.integers(1, 2**31 if big_nodes else 5000)),
                      int(rng.choice([1, 40, 65535])), int(rng.random() < 0.1)))
        out.append((budget, reserved, max_syn, max_nets, q))
    return out


def _fits_batch(batch, nxt, budget, reserved, max_syn, max_nets):
    """Whether request nxt may join the batch (the limits of the header)."""
    small = max_syn // 2
    members = batch + [nxt]
    if len(members) > max_nets or any(r[4] for r in members) or any(r[1] > small for r in members):
        return False
    if sum(r[1] for r in members) > max_syn or reserved + sum(r[0] for r in members) > budget:
        return False
    nodes = sum(r[2] for r in members)
    if nodes > 0xFFFFFFFF:
        return False
    return _bits(nodes - 1) + _bits(max(r[2] for r in members) - 1) + _bits(max(r[3] for r in members)) <= 64


@pytest.fixture(scope="module")
def admit(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2306_09855_gb300 import _build
    lib = _build.build()
    d = tmp_path_factory.mktemp("admit")
    (d / "admit.cpp").write_text(PROGRAM)
    exe = d / "admit"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", cuda_inc, str(d / "admit.cpp"), "-o", str(exe), lib,
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)

    def run(cases):
        lines = []
        for budget, reserved, max_syn, max_nets, q in cases:
            lines.append("%d %d %d %d %d" % (len(q), budget, reserved, max_syn, max_nets))
            lines += ["%d %d %d %d %d" % r for r in q]
        r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, (r.returncode, r.stderr)
        return [tuple(map(int, ln.split())) for ln in r.stdout.strip().split("\n")]
    return run


def test_admission_follows_its_limits(admit):
    cases = _cases()
    got = admit(cases)
    assert len(got) == len(cases)
    sizes = set()
    for (budget, reserved, max_syn, max_nets, q), (take, reserve) in zip(cases, got):
        sizes.add(take)
        if not q or reserved + q[0][0] > budget:
            assert take == 0 and reserve == 0
            continue
        assert 1 <= take <= len(q)
        batch = q[:take]
        assert reserve == sum(r[0] for r in batch)
        assert reserved + reserve <= budget
        if take > 1:
            for i in range(1, take):
                assert _fits_batch(batch[:i], batch[i], budget, reserved, max_syn, max_nets)
        # the run stops only at a request that may not join
        if take < len(q):
            head_batchable = max_nets > 1 and q[0][1] <= max_syn // 2 and not q[0][4]
            assert not head_batchable or not _fits_batch(batch, q[take], budget, reserved, max_syn, max_nets)
    assert {0, 1} <= sizes and max(sizes) >= 4  # the cases reach refusals, single builds and batches
