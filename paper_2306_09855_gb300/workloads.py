"""Seeded synthetic network specifications.

This module holds only parameters: population sizes, Connect calls, rule
parameters, weight and delay distributions and seeds.  It contains none of the
construction arithmetic, so that both the CUDA library and the CPU oracle can
be driven from the same specification without sharing any method code.

Shapes follow the two models of the paper (Sec. 2.4):
  * a two-population network connected in four Connect calls, used for the
    scaling study (E->E, E->I, I->E, I->I);
  * a cortical-microcircuit-shaped network of eight populations connected by
    fixed_total_number with autapses and multapses allowed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

RULES = ("one_to_one", "all_to_all", "fixed_indegree", "fixed_outdegree",
         "fixed_total_number", "pairwise_bernoulli")
RULE_ID = {name: i for i, name in enumerate(RULES)}
DIST_ID = {"const": 0, "normal": 1}


@dataclass(frozen=True)
class Dist:
    """Constant value (std ignored) or normal distribution N(mean, std)."""
    kind: str
    mean: float
    std: float = 0.0


@dataclass(frozen=True)
class Projection:
    """One Connect(sources, targets, conn_dict, syn_dict) call.

    src, tgt: (first global node id, count) of a node range.
    k: in-degree / out-degree K, or the total number N of fixed_total_number.
    p: connection probability of pairwise_bernoulli.
    src_ids, tgt_ids: explicit node ids (uint32) in place of the range; the
        range's count must then equal the array's length (its first id is
        unused).
    weights, delays: per-connection values (float32; delays in ms) in place
        of the distributions, one per connection number of the rule.
    """
    src: Tuple[int, int]
    tgt: Tuple[int, int]
    rule: str
    k: int = 0
    p: float = 0.0
    autapses: bool = True
    multapses: bool = True
    weight: Dist = Dist("const", 1.0)
    delay: Dist = Dist("const", 1.0)
    src_ids: Optional[np.ndarray] = field(default=None, compare=False, repr=False)
    tgt_ids: Optional[np.ndarray] = field(default=None, compare=False, repr=False)
    weights: Optional[np.ndarray] = field(default=None, compare=False, repr=False)
    delays: Optional[np.ndarray] = field(default=None, compare=False, repr=False)

    @property
    def has_arrays(self) -> bool:
        return any(a is not None for a in (self.src_ids, self.tgt_ids, self.weights, self.delays))


@dataclass
class NetworkSpec:
    seed: int
    dt: float
    populations: List[int]
    projections: List[Projection] = field(default_factory=list)
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(sum(self.populations))

    def pop_range(self, i: int) -> Tuple[int, int]:
        first = int(sum(self.populations[:i]))
        return (first, int(self.populations[i]))


# Synaptic parameters of the two-population model (pA, ms).
W_EXC = Dist("normal", 50.0, 5.0)
W_INH = Dist("normal", -250.0, 25.0)
D_TWO_POP = Dist("normal", 1.5, 0.75)


def two_population(n: int, rule: str, *, k: int = 0, p: float = 0.0,
                   autapses: bool = True, multapses: bool = True,
                   seed: int = 1234, dt: float = 0.1, name: str = "") -> NetworkSpec:
    """Two populations of n nodes (E then I) connected by four calls of one rule.

    Weights N(50, 5) pA from E sources and N(-250, 25) pA from I sources;
    delays N(1.5 ms, 0.75 ms), quantised in steps of dt with a one-step minimum.
    """
    spec = NetworkSpec(seed=seed, dt=dt, populations=[n, n], name=name or f"two_pop_{rule}")
    for src_pop, tgt_pop in ((0, 0), (0, 1), (1, 0), (1, 1)):
        spec.projections.append(Projection(
            src=spec.pop_range(src_pop), tgt=spec.pop_range(tgt_pop), rule=rule, k=k, p=p,
            autapses=autapses, multapses=multapses,
            weight=W_EXC if src_pop == 0 else W_INH, delay=D_TWO_POP))
    return spec


def plain_indegree(n: int = 1000, k: int = 100, seed: int = 1234) -> NetworkSpec:
    """2 x 1,000 nodes, fixed_indegree K=100 on all four projections, no
    autapses, multapses allowed: 400,000 synapses."""
    return two_population(n, "fixed_indegree", k=k, autapses=False, multapses=True,
                          seed=seed, name="plain_indegree_2x%d_K%d" % (n, k))


def rule_sweep(rule: str, multapses: bool, scale: float = 1.0, seed: int = 1234) -> NetworkSpec:
    """Two-population rule sweep: 2 x 100,000 nodes, four calls of one rule.

    fixed_indegree / fixed_outdegree K=1,000; fixed_total_number 1e8 per call;
    pairwise_bernoulli p=0.01; all_to_all on 2 x 10,000; one_to_one on
    2 x 100,000.  Run with multapses and autapses both allowed (the paper's
    setting) or both forbidden.  `scale` shrinks node counts (and the
    total-number count with the square) for tests; the in/out-degree stays.
    """
    autapses = multapses
    tag = "mult" if multapses else "nomult"
    if rule == "all_to_all":
        n = max(2, int(round(10_000 * scale)))
        return two_population(n, rule, autapses=autapses, multapses=multapses, seed=seed,
                              name=f"sweep_{rule}_{tag}_2x{n}")
    n = max(2, int(round(100_000 * scale)))
    kw = {}
    if rule in ("fixed_indegree", "fixed_outdegree"):
        kw["k"] = min(1000, n - 1)
    elif rule == "fixed_total_number":
        kw["k"] = int(round(1e8 * scale * scale))
    elif rule == "pairwise_bernoulli":
        kw["p"] = 0.01
    return two_population(n, rule, autapses=autapses, multapses=multapses, seed=seed,
                          name=f"sweep_{rule}_{tag}_2x{n}", **kw)


RULE_SWEEP_RUNS = [(r, m) for r in ("fixed_indegree", "fixed_outdegree", "fixed_total_number",
                                    "pairwise_bernoulli", "all_to_all", "one_to_one")
                   for m in (True, False)]

MICROCIRCUIT_SIZES = [20683, 5834, 21915, 5479, 4850, 1065, 14395, 2948]


def microcircuit(seed: int = 1234, total: float = 3.0e8, scale: float = 1.0) -> NetworkSpec:
    """Eight populations shaped like the cortical microcircuit (Sec. 2.4).

    Connection probabilities p[a][b] (target a, source b) are drawn seeded
    uniform in [0.01, 0.15] and rescaled so that the total is `total`; each
    pair gets round(c * p * N_a * N_b) connections by fixed_total_number with
    autapses and multapses allowed.  Weights N(87.8, 8.78) pA, scaled by -4
    for inhibitory (odd-index) sources; delays N(1.5, 0.75) ms from excitatory
    and N(0.75, 0.375) ms from inhibitory sources; dt = 0.1 ms.
    """
    sizes = [max(1, int(round(s * scale))) for s in MICROCIRCUIT_SIZES]
    rng = np.random.default_rng(1234)
    p = rng.uniform(0.01, 0.15, (8, 8))
    n = np.asarray(sizes, dtype=np.float64)
    c = (total * scale * scale) / float(np.sum(p * n[:, None] * n[None, :]))
    counts = np.rint(c * p * n[:, None] * n[None, :]).astype(np.int64)
    spec = NetworkSpec(seed=seed, dt=0.1, populations=sizes, name="microcircuit")
    for a in range(8):
        for b in range(8):
            exc = b % 2 == 0
            w = Dist("normal", 87.8, 8.78) if exc else Dist("normal", -4 * 87.8, 4 * 8.78)
            d = Dist("normal", 1.5, 0.75) if exc else Dist("normal", 0.75, 0.375)
            spec.projections.append(Projection(
                src=spec.pop_range(b), tgt=spec.pop_range(a), rule="fixed_total_number",
                k=int(counts[a, b]), autapses=True, multapses=True, weight=w, delay=d))
    return spec


def _log_uniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def batched_sweep(count: int = 64, seed: int = 1234, scale: float = 1.0) -> List[NetworkSpec]:
    """Independent two-population networks of uneven size, as in a parameter scan.

    N per population log-uniform in [2,000, 50,000]; the rule is one of
    fixed_indegree (K log-uniform in [50, 2,000]), fixed_total_number
    (K * N per call) or pairwise_bernoulli (p log-uniform in [0.005, 0.05]);
    multapses (and autapses with them) allowed with probability 1/2 where the
    rule distinguishes them.  Instance i is seeded 1234 + i.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = max(4, int(_log_uniform(rng, 2000, 50000) * scale))
        rule = ("fixed_indegree", "fixed_total_number", "pairwise_bernoulli")[int(rng.integers(0, 3))]
        k = int(_log_uniform(rng, 50, 2000))
        p = _log_uniform(rng, 0.005, 0.05)
        mult = bool(rng.integers(0, 2))
        k = min(k, n - 1)
        if rule == "fixed_indegree":
            spec = two_population(n, rule, k=k, autapses=mult, multapses=mult, seed=1234 + i)
        elif rule == "fixed_total_number":
            # at most a quarter of the pairs, so that the no-multapse redraws stay short
            spec = two_population(n, rule, k=min(k, n // 4) * n, autapses=mult, multapses=mult, seed=1234 + i)
        else:
            spec = two_population(n, rule, p=p, autapses=mult, multapses=True, seed=1234 + i)
        spec.name = f"batch{i}_{rule}_2x{n}"
        out.append(spec)
    return out


def served_request(size: float, rule: str, multapses: bool, seed: int) -> NetworkSpec:
    """A two-population construction request of about `size` synapses."""
    s4 = size / 4.0
    if rule == "one_to_one":
        n = max(2, int(s4))
        return two_population(n, rule, autapses=multapses, multapses=multapses, seed=seed)
    if rule == "all_to_all":
        n = max(2, int(math.ceil(math.sqrt(s4))))
        return two_population(n, rule, autapses=multapses, multapses=multapses, seed=seed)
    k = 100 if s4 < 1e7 else 1000
    n = max(k + 2, int(s4 / k))
    if rule in ("fixed_indegree", "fixed_outdegree"):
        return two_population(n, rule, k=k, autapses=multapses, multapses=multapses, seed=seed)
    if rule == "fixed_total_number":
        return two_population(n, rule, k=int(s4), autapses=multapses, multapses=multapses, seed=seed)
    return two_population(n, rule, p=k / n, autapses=multapses, multapses=True, seed=seed)


def served_stream(count: int = 2000, seed: int = 1234, lo: float = 1e5, hi: float = 5e8):
    """Poisson-arrival request stream: (arrival offset in units of the mean
    inter-arrival time, spec).  Sizes log-uniform in [lo, hi]; rule uniform
    over the six; multapse flag Bernoulli(1/2)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0))
        size = _log_uniform(rng, lo, hi)
        rule = RULES[int(rng.integers(0, 6))]
        mult = bool(rng.integers(0, 2))
        out.append((t, served_request(size, rule, mult, 1234 + i)))
    return out


def with_seed(spec: NetworkSpec, seed: int) -> NetworkSpec:
    return replace(spec, seed=seed, projections=list(spec.projections))
