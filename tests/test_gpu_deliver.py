"""Spike delivery through the index (Sec. 2.3) on the GPU against the
oracle's delivery on its own network: every target's input within the
bound of fp32 summation in any order, (terms + 1) * 2^-24 * sum |w * m|,
plus the weights' own parity tolerance (4 fp32 ulp, at most 4 * 2^-23 of
each |w|) carried through the sum."""
import numpy as np
import pytest

from paper_2306_09855_gb300 import workloads as W
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


def _spikes(rng, ref, n_nodes, n):
    g = np.diff(ref["group_ptr"].astype(np.int64))
    have = np.flatnonzero(g > 0)
    src = rng.choice(have, n).astype(np.uint32)
    grp = (rng.random(n) * g[src]).astype(np.uint32)
    mult = rng.uniform(0.5, 2.0, n).astype(np.float32)
    return src, grp, mult


def _deliver_gpu(net, src, grp, mult, n_nodes):
    import torch
    inp = torch.zeros(n_nodes, dtype=torch.float32, device="cuda")
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (src.view(np.int32), grp.view(np.int32), mult)]
    net.deliver(t[0], t[1], t[2], inp)
    return inp.cpu().numpy()


def _check(got, ref):
    tol = ((ref["terms"].astype(np.float64) + 1.0) * 2.0 ** -24 + 4.0 * 2.0 ** -23) * ref["abs"] * 1.01 + 1e-30
    err = np.abs(got.astype(np.float64) - ref["input"])
    assert np.all(err <= tol), (float(err.max()), int(np.argmax(err - tol)))


@pytest.mark.parametrize("spec", [
    W.plain_indegree(),
    W.rule_sweep("fixed_total_number", False, scale=0.05),
    W.rule_sweep("fixed_outdegree", True, scale=0.05),
    W.microcircuit(scale=0.05),
], ids=["plain", "total_nomult", "outdegree", "microcircuit"])
def test_delivery_matches_oracle(snc, oracle_mod, spec):
    rng = np.random.default_rng(11)
    ref_net = oracle_mod.build(spec)
    net = snc.Network(spec).finalize()
    try:
        for n in (1, 1000, 50_000):
            src, grp, mult = _spikes(rng, ref_net, spec.n_nodes, n)
            got = _deliver_gpu(net, src, grp, mult, spec.n_nodes)
            ref = oracle_mod.deliver(ref_net, spec.n_nodes, src, grp, mult)
            assert ref["bad"] == 0
            _check(got, ref)
    finally:
        net.close()


def test_every_group_once_and_bad_entries(snc, oracle_mod):
    spec = NetworkSpec(seed=8, dt=0.1, populations=[400, 300], projections=[
        Projection(src=(0, 400), tgt=(400, 300), rule="fixed_indegree", k=25,
                   weight=Dist("normal", 5.0, 1.0), delay=Dist("normal", 1.5, 0.75)),
        Projection(src=(400, 300), tgt=(0, 700), rule="all_to_all", autapses=False,
                   weight=Dist("normal", -20.0, 2.0), delay=Dist("normal", 0.75, 0.375))])
    ref_net = oracle_mod.build(spec)
    g = np.diff(ref_net["group_ptr"].astype(np.int64))
    src = np.repeat(np.arange(g.size, dtype=np.uint32), g)
    grp = np.concatenate([np.arange(k, dtype=np.uint32) for k in g])
    mult = np.ones(src.size, np.float32)
    net = snc.Network(spec).finalize()
    try:
        _check(_deliver_gpu(net, src, grp, mult, spec.n_nodes),
               oracle_mod.deliver(ref_net, spec.n_nodes, src, grp, mult))
        # Entries naming no group: INVALID_ARG, the others still delivered.
        bad_src = np.concatenate([src[:5], np.array([spec.n_nodes, 0], np.uint32)])
        bad_grp = np.concatenate([grp[:5], np.array([0, g[0]], np.uint32)])
        bad_mult = np.ones(bad_src.size, np.float32)
        with pytest.raises(snc.SncError) as e:
            _deliver_gpu(net, bad_src, bad_grp, bad_mult, spec.n_nodes)
        assert e.value.name == "INVALID_ARG"
        import torch
        inp = torch.zeros(spec.n_nodes, dtype=torch.float32, device="cuda")
        t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
             (bad_src.view(np.int32), bad_grp.view(np.int32), bad_mult)]
        with pytest.raises(snc.SncError):
            net.deliver(t[0], t[1], t[2], inp)
        _check(inp.cpu().numpy(), oracle_mod.deliver(ref_net, spec.n_nodes, bad_src, bad_grp, bad_mult))
        # An empty spike array is a no-op.
        z = torch.zeros(0, dtype=torch.int32, device="cuda")
        net.deliver(z, z, torch.zeros(0, dtype=torch.float32, device="cuda"), inp)
    finally:
        net.close()


def test_batch_member_delivery(snc, oracle_mod):
    specs = [W.two_population(600, "fixed_indegree", k=40, seed=31),
             W.two_population(900, "pairwise_bernoulli", p=0.02, seed=32)]
    nets = snc.Network.batch(specs)
    rng = np.random.default_rng(5)
    try:
        for sp, net in zip(specs, nets):
            ref_net = oracle_mod.build(sp)
            src, grp, mult = _spikes(rng, ref_net, sp.n_nodes, 5000)
            _check(_deliver_gpu(net, src, grp, mult, sp.n_nodes),
                   oracle_mod.deliver(ref_net, sp.n_nodes, src, grp, mult))
    finally:
        for net in reversed(nets):
            net.close()


@pytest.mark.parametrize("spec", [
    W.rule_sweep("fixed_indegree", True, scale=0.05),
    W.microcircuit(scale=0.05),
], ids=["indegree", "microcircuit"])
def test_delivery_on_the_gpus_own_network(snc, oracle_mod, spec):
    """The oracle's delivery run on the arrays the GPU built (row_ptr,
    group_ptr, group_first, target, weight), so both sums add the same fp32
    weights: only the summation order differs, and the bound is that of fp32
    summation alone, (terms + 1) * 2^-24 * sum |w * m|, with no weight term."""
    net = snc.Network(spec).finalize()
    try:
        gpu_net = net.to_host()
        rng = np.random.default_rng(23)
        for n in (1000, 50_000):
            src, grp, mult = _spikes(rng, gpu_net, spec.n_nodes, n)
            got = _deliver_gpu(net, src, grp, mult, spec.n_nodes)
            ref = oracle_mod.deliver(gpu_net, spec.n_nodes, src, grp, mult)
            assert ref["bad"] == 0
            tol = (ref["terms"].astype(np.float64) + 1.0) * 2.0 ** -24 * ref["abs"] * 1.01 + 1e-30
            err = np.abs(got.astype(np.float64) - ref["input"])
            assert np.all(err <= tol), (float(err.max()), int(np.argmax(err - tol)))
    finally:
        net.close()
