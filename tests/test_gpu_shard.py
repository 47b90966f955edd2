"""Target-sharded builds (Sec. 4 names target-distributed construction as
future work), ranks emulated one after another on one GPU: each rank's build
equals the oracle's whole network restricted to the rank's targets, in the
same (source, delay, generation) order, with no exchange between ranks."""
import numpy as np
import pytest

from gpu_helpers import assert_network_equal
from paper_2306_09855_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09855_gb300 import snc as mod
    mod.load()
    return mod


SPECS = [W.plain_indegree(),
         W.rule_sweep("fixed_indegree", False, scale=0.05),
         W.rule_sweep("fixed_outdegree", True, scale=0.05),
         W.rule_sweep("fixed_total_number", False, scale=0.05),
         W.rule_sweep("pairwise_bernoulli", True, scale=0.05),
         W.rule_sweep("all_to_all", False, scale=0.05),
         W.microcircuit(scale=0.05)]


@pytest.mark.parametrize("ranks", [2, 3])
@pytest.mark.parametrize("spec", SPECS, ids=["plain", "indegree_nomult", "outdegree", "total_nomult", "bernoulli",
                                             "all_to_all", "microcircuit"])
def test_shards_are_the_network_restricted(snc, oracle_mod, spec, ranks):
    g = oracle_mod.generate(spec)  # generation order
    bounds = np.linspace(0, spec.n_nodes, ranks + 1).astype(np.int64)
    total = 0
    for r in range(ranks):
        first, n = int(bounds[r]), int(bounds[r + 1] - bounds[r])
        net = snc.Network(spec, target_shard=(first, n)).finalize()
        got = net.to_host()
        net.close()
        keep = (g["tgt"] >= first) & (g["tgt"] < first + n)
        ref = oracle_mod.sort_index(spec.n_nodes, g["src"][keep], g["tgt"][keep], g["delay"][keep],
                                    g["weight"][keep])
        assert_network_equal(got, ref, f"rank {r} of {ranks}")
        total += got["src"].size
    assert total == g["src"].size


def test_shard_errors(snc):
    spec = W.plain_indegree()
    net = snc.Network(spec, target_shard=(spec.n_nodes - 10, 11))
    with pytest.raises(snc.SncError) as e:
        net.finalize()
    assert e.value.name == "INVALID_ARG"
    net.close()
    net = snc.Network(spec, target_shard=(0, 0)).finalize()  # an empty shard
    assert int(net.view().n_syn) == 0
    with pytest.raises(snc.SncError) as e:
        snc.snc_set_target_shard(net.ctx, 0, 5)
    assert e.value.name == "STATE"
    net.close()
    a = snc.Network(spec, target_shard=(0, 100))
    b = snc.Network(W.plain_indegree(seed=3))
    with pytest.raises(snc.SncError) as e:
        snc.snc_batch_finalize([a.ctx, b.ctx])
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(snc.SncError) as e:
        snc.snc_batch_finalize_graph([a.ctx])
    assert e.value.name == "INVALID_ARG"
    a.close()
    b.close()


@pytest.mark.parametrize("rule,kw", [("fixed_indegree", dict(k=1000)), ("pairwise_bernoulli", dict(p=0.02))])
def test_shards_divide_the_generation(snc, rule, kw):
    """Target-primary rules: a rank generates only its own targets'
    connections, so its generation time falls about as 1 / ranks (stage
    timers, best of three builds; bound 0.45 for four ranks)."""
    spec = W.two_population(50_000, rule, autapses=False, seed=9, **kw)

    def gen_ms(shard):
        best = float("inf")
        for _ in range(3):
            net = snc.Network(spec, target_shard=shard).finalize()
            times, _ = net.stage_times()
            n = int(net.view().n_syn)
            net.close()
            best = min(best, times[0] + times[1])
        return best, n

    full_ms, full_n = gen_ms(None)
    ranks = 4
    per = spec.n_nodes // ranks
    for r in range(ranks):
        ms, n = gen_ms((r * per, per))
        assert n < 0.3 * full_n
        assert ms < 0.45 * full_ms, (r, ms, full_ms)
