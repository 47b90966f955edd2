"""The library's host checks of Connect calls with explicit arrays
(csrc/arrays.cpp, Sec. 2.1) against the oracle, on seeded random cases: the
same status for every case (ids out of range, repeated ids where the reading
forbids them, degree and pair limits, array lengths, bad delays), the same
connection count for accepted deterministic rules, and the same delay step
for every element of a delay array.  Host code only (no GPU): a small program
compiled with g++ runs the library's checks on the cases written to a file."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_09855_gb300", "csrc")
RULES = ["one_to_one", "all_to_all", "fixed_indegree", "fixed_outdegree", "fixed_total_number",
         "pairwise_bernoulli"]
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "STATE", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "UNSUPPORTED"}

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "arrays.h"

// Case format (whitespace separated): n_nodes dt rule aut mult k p
// src_first src_n tgt_first tgt_n has_src has_tgt has_w has_d n_conn,
// then the src ids, tgt ids, weights and delays that are present.
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "r");
  if (!f) return 2;
  int n_cases = 0;
  if (std::fscanf(f, "%d", &n_cases) != 1) return 3;
  for (int c = 0; c < n_cases; ++c) {
    unsigned n_nodes, rule, aut, mult, sf, sn, tf, tn, hs, ht, hw, hd;
    unsigned long long k, n_conn;
    double dt, p;
    if (std::fscanf(f, "%u %lf %u %u %u %llu %lf %u %u %u %u %u %u %u %u %llu", &n_nodes, &dt, &rule, &aut, &mult,
                    &k, &p, &sf, &sn, &tf, &tn, &hs, &ht, &hw, &hd, &n_conn) != 16)
      return 4;
    // A given array has a non-null address even when it is empty.
    std::vector<uint32_t> s(sn + 1), t(tn + 1);
    std::vector<float> w(n_conn + 1), d(n_conn + 1);
    for (unsigned i = 0; hs && i < sn; ++i) if (std::fscanf(f, "%u", &s[i]) != 1) return 5;
    for (unsigned i = 0; ht && i < tn; ++i) if (std::fscanf(f, "%u", &t[i]) != 1) return 5;
    char tok[64];
    for (unsigned long long i = 0; hw && i < n_conn; ++i) {
      if (std::fscanf(f, "%63s", tok) != 1) return 5;
      w[i] = std::strtof(tok, nullptr);
    }
    for (unsigned long long i = 0; hd && i < n_conn; ++i) {
      if (std::fscanf(f, "%63s", tok) != 1) return 5;
      d[i] = std::strtof(tok, nullptr);
    }
    snc_range src{sf, sn}, tgt{tf, tn};
    snc_conn_rule r{};
    r.kind = static_cast<snc_rule_kind>(rule);
    r.allow_autapses = static_cast<int32_t>(aut);
    r.allow_multapses = static_cast<int32_t>(mult);
    r.k = k;
    r.p = p;
    snc::ConnectArrays a;
    a.src_ids = hs ? s.data() : nullptr;
    a.tgt_ids = ht ? t.data() : nullptr;
    a.weights = hw ? w.data() : nullptr;
    a.delays_ms = hd ? d.data() : nullptr;
    a.n_conn = n_conn;
    snc::ArrayPlan plan;
    std::string why;
    const snc_status st = snc::check_connect_arrays(n_nodes, dt, src, tgt, r, a, &plan, &why);
    std::printf("%d %llu %llu %u", static_cast<int>(st), static_cast<unsigned long long>(plan.count),
                static_cast<unsigned long long>(plan.equal_pairs), plan.max_step);
    for (uint16_t x : plan.steps) std::printf(" %u", static_cast<unsigned>(x));
    std::printf("\n");
  }
  return 0;
}
"""


def _numbered(rule, ns, nt, k):
    return {"one_to_one": ns, "all_to_all": ns * nt, "fixed_indegree": nt * k, "fixed_outdegree": ns * k,
            "fixed_total_number": k, "pairwise_bernoulli": 0}[rule]


def _ids(rng, n, n_nodes, repeats):
    if repeats or n > n_nodes:
        return rng.integers(0, n_nodes, n).astype(np.uint32)
    return rng.permutation(n_nodes)[:n].astype(np.uint32)


def _cases(seed=21, count=600):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n_nodes = int(rng.integers(3, 30))
        rule = RULES[int(rng.integers(0, 6))]
        aut, mult = bool(rng.integers(0, 2)), bool(rng.integers(0, 2))
        ns, nt = int(rng.integers(0, n_nodes + 1)), int(rng.integers(0, n_nodes + 1))
        if rule == "one_to_one" and rng.random() < 0.8:
            nt = ns
        src_ids = _ids(rng, ns, n_nodes, rng.random() < 0.3) if rng.random() < 0.7 else None
        tgt_ids = _ids(rng, nt, n_nodes, rng.random() < 0.3) if rng.random() < 0.7 else None
        if src_ids is not None and rng.random() < 0.05:
            src_ids = src_ids.copy()
            if ns:
                src_ids[int(rng.integers(0, ns))] = n_nodes  # out of range
        sf = 0 if src_ids is not None else int(rng.integers(0, n_nodes - ns + 1 + int(rng.random() < 0.05)))
        tf = 0 if tgt_ids is not None else int(rng.integers(0, n_nodes - nt + 1 + int(rng.random() < 0.05)))
        k = {"fixed_indegree": int(rng.integers(0, ns + 3)), "fixed_outdegree": int(rng.integers(0, nt + 3)),
             "fixed_total_number": int(rng.integers(0, ns * nt + 3))}.get(rule, 0)
        p = float(rng.choice([0.0, 0.4, 1.0, 1.5]))
        n_conn = _numbered(rule, ns, nt, k) + (int(rng.integers(-1, 2)) if rng.random() < 0.1 else 0)
        n_conn = max(0, n_conn)
        weights = rng.normal(0, 1, n_conn).astype(np.float32) if rng.random() < 0.4 else None
        delays = None
        if rng.random() < 0.4:
            delays = rng.uniform(-0.5, 6.0, n_conn).astype(np.float32)
            if n_conn and rng.random() < 0.15:
                delays[int(rng.integers(0, n_conn))] = rng.choice([np.nan, np.inf, -np.inf, 7000.0, 6553.6])
        out.append(dict(n_nodes=n_nodes, dt=0.1, rule=rule, aut=aut, mult=mult, k=k, p=p, src=(sf, ns),
                        tgt=(tf, nt), src_ids=src_ids, tgt_ids=tgt_ids, weights=weights, delays=delays,
                        n_conn=n_conn))
    return out


def _write(cases, path):
    with open(path, "w") as f:
        f.write("%d\n" % len(cases))
        for c in cases:
            f.write("%d %r %d %d %d %d %r %d %d %d %d %d %d %d %d %d\n" % (
                c["n_nodes"], c["dt"], RULES.index(c["rule"]), c["aut"], c["mult"], c["k"], c["p"],
                c["src"][0], c["src"][1], c["tgt"][0], c["tgt"][1], c["src_ids"] is not None,
                c["tgt_ids"] is not None, c["weights"] is not None, c["delays"] is not None, c["n_conn"]))
            for key in ("src_ids", "tgt_ids"):
                if c[key] is not None:
                    f.write(" ".join(str(int(x)) for x in c[key]) + "\n")
            for key in ("weights", "delays"):
                if c[key] is not None:
                    f.write(" ".join(np.format_float_scientific(x, unique=True) if np.isfinite(x) else
                                     ("nan" if np.isnan(x) else ("inf" if x > 0 else "-inf"))
                                     for x in c[key]) + "\n")


def _spec(c):
    pj = Projection(src=c["src"], tgt=c["tgt"], rule=c["rule"], k=c["k"], p=c["p"], autapses=c["aut"],
                    multapses=c["mult"], weight=Dist("const", 1.0), delay=Dist("const", 1.0),
                    src_ids=c["src_ids"], tgt_ids=c["tgt_ids"], weights=c["weights"], delays=c["delays"])
    return NetworkSpec(seed=5, dt=c["dt"], populations=[c["n_nodes"]], projections=[pj])


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if gxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    from paper_2306_09855_gb300 import _build
    lib = _build.build()
    d = tmp_path_factory.mktemp("arrays")
    (d / "check.cpp").write_text(PROGRAM)
    exe = d / "check"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                    str(d / "check.cpp"), "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)

    def run(cases):
        path = d / "cases.txt"
        _write(cases, path)
        r = subprocess.run([str(exe), str(path)], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, (r.returncode, r.stderr)
        return [list(map(int, line.split())) for line in r.stdout.strip().split("\n")]
    return run


def test_host_checks_match_the_oracle(checker, oracle_mod):
    cases = _cases()
    got = checker(cases)
    assert len(got) == len(cases)
    seen = set()
    for i, (c, row) in enumerate(zip(cases, got)):
        status, count, _eq, max_step = row[:4]
        spec = _spec(c)
        ref = oracle_mod.check_projection(spec, 0)
        assert STATUS[status] == STATUS[ref], (i, c["rule"], STATUS[status], STATUS[ref])
        seen.add(STATUS[status])
        if status != 0:
            continue
        if c["rule"] != "pairwise_bernoulli":
            n, _ = oracle_mod.count(spec)
            assert count == n, (i, c["rule"], count, n)
        if c["delays"] is not None:
            steps = np.array(row[4:], dtype=np.int64)
            assert steps.size == c["n_conn"]
            if steps.size:
                assert max_step == steps.max()
                # the oracle's steps: a one_to_one network carrying the same delay array
                n = steps.size
                one = NetworkSpec(seed=1, dt=c["dt"], populations=[2 * n], projections=[Projection(
                    src=(0, n), tgt=(n, n), rule="one_to_one", delays=c["delays"])])
                np.testing.assert_array_equal(steps, oracle_mod.generate(one)["delay"].astype(np.int64))
    assert {"OK", "INVALID_ARG", "UNSUPPORTED"} <= seen  # the cases reach every outcome
