"""Parity at full size (the rule sweep's 2 x 100,000 nodes with about 4e8
connections per network, and the microcircuit shape's 3e8; the
configurations the bench times): the sorted
index properties on the whole network, and the connections of sampled
primary nodes against the oracle's generation of those nodes alone; for
fixed_total_number without multapses (no per-node decomposition), its
defining properties.  The same checks run on the CPU on the oracle's own
small networks, so the comparison code is tested without a GPU."""
import numpy as np
import pytest

from fullsize_checks import (check_index, check_projection_counts, check_source_primary, check_target_primary,
                             check_total_no_multapses)
from paper_2306_09855_gb300 import workloads as W

CASES = [("fixed_indegree", True), ("fixed_outdegree", False), ("pairwise_bernoulli", True),
         ("fixed_total_number", False), ("microcircuit", True)]


def _samples(n, k=4, seed=0):
    rng = np.random.default_rng(seed)
    return sorted({0, n - 1, *rng.integers(0, n, k).tolist()})


def _run_checks(torch, t, n_syn, oracle_mod, spec, rule):
    src = check_index(torch, t, n_syn)
    if rule == "microcircuit":  # 64 fixed_total_number calls with multapses: counts per call
        check_projection_counts(torch, t, src, spec)
        return
    if rule == "fixed_total_number":
        check_total_no_multapses(torch, t, src, spec)
        return
    for proj, pj in enumerate(spec.projections):
        if rule == "fixed_outdegree":
            for a in _samples(pj.src[1], seed=proj):
                check_source_primary(torch, t, oracle_mod, spec, proj, a)
        else:
            for b in _samples(pj.tgt[1], seed=proj):
                check_target_primary(torch, t, oracle_mod, spec, proj, b)


@pytest.mark.parametrize("rule,mult", CASES, ids=[r for r, _ in CASES])
def test_checks_on_oracle_networks(oracle_mod, rule, mult):
    torch = pytest.importorskip("torch")
    spec = W.microcircuit(scale=0.02) if rule == "microcircuit" else W.rule_sweep(rule, mult, scale=0.02)
    ref = oracle_mod.build(spec)
    t = {"row_ptr": torch.from_numpy(ref["row_ptr"].astype(np.int64)),
         "target": torch.from_numpy(ref["tgt"].astype(np.int32)),
         "delay": torch.from_numpy(ref["delay"].view(np.int16)),
         "weight": torch.from_numpy(ref["weight"]),
         "group_ptr": torch.from_numpy(ref["group_ptr"].astype(np.int64)),
         "group_first": torch.from_numpy(ref["group_first"].astype(np.int64))}
    _run_checks(torch, t, int(ref["src"].size), oracle_mod, spec, rule)


@pytest.mark.gpu
@pytest.mark.parametrize("rule,mult", CASES, ids=[r for r, _ in CASES])
def test_full_size_sampled(oracle_mod, rule, mult):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc
    snc.load()
    spec = W.microcircuit() if rule == "microcircuit" else W.rule_sweep(rule, mult)
    net = snc.Network(spec).finalize()
    try:
        v = net.view()
        assert int(v.n_nodes) == spec.n_nodes
        _run_checks(torch, net.tensors(), int(v.n_syn), oracle_mod, spec, rule)
    finally:
        net.close()
