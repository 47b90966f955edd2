"""Checks of a built network at any size, on torch tensors of either device
(comparison only, no method code): the sorted-index properties of
Sec. 2.2, and the connections of sampled primary nodes against the
oracle's generation of those nodes alone."""
import numpy as np

from gpu_helpers import ulp_diff, WEIGHT_ULP


def sources(torch, t):
    """Source of every position, expanded from row_ptr."""
    row = t["row_ptr"]
    n_nodes = row.numel() - 1
    return torch.repeat_interleave(torch.arange(n_nodes, device=row.device), row[1:] - row[:-1])


def check_index(torch, t, n_syn):
    """row_ptr, the (source, delay) order, group starts and p_i."""
    row, delay = t["row_ptr"], t["delay"].to(torch.int64) & 0xFFFF
    assert int(row[0]) == 0 and int(row[-1]) == n_syn
    assert bool(torch.all(row[1:] >= row[:-1]))
    src = sources(torch, t)
    key = src * 65536 + delay
    if n_syn > 1:
        assert bool(torch.all(key[1:] >= key[:-1])), "not sorted by (source, delay)"
    starts = torch.ones(n_syn, dtype=torch.bool, device=row.device)
    if n_syn > 1:
        starts[1:] = key[1:] != key[:-1]
    first = torch.nonzero(starts).flatten()
    gf = t["group_first"].to(torch.int64)
    assert first.numel() == gf.numel() and bool(torch.all(first == gf)), "group starts"
    per_src = torch.bincount(src[first], minlength=row.numel() - 1)
    gp = t["group_ptr"].to(torch.int64)
    assert int(gp[0]) == 0 and bool(torch.all(gp[1:] - gp[:-1] == per_src)), "p_i"
    return src


def _expect_by_source_delay(ref):
    """The oracle's connections of one primary in slot order, ordered as the
    sorted network holds them: by (source, delay), slots in order."""
    order = np.lexsort((np.arange(ref["src"].size), ref["delay"], ref["src"]))
    return {k: v[order] for k, v in ref.items()}


def check_target_primary(torch, t, oracle_mod, spec, proj, b):
    """Connections onto target t0 + b from projection proj (in/Bernoulli
    rules: the primary is the target) equal the oracle's, in order."""
    pj = spec.projections[proj]
    tgt = pj.tgt[0] + b
    pos = torch.nonzero(t["target"].to(torch.int64) == tgt).flatten()
    row = t["row_ptr"]
    src = torch.searchsorted(row, pos, right=True) - 1
    keep = (src >= pj.src[0]) & (src < pj.src[0] + pj.src[1])
    pos, src = pos[keep], src[keep]
    got = {"src": src.cpu().numpy(), "delay": (t["delay"][pos].to(torch.int64) & 0xFFFF).cpu().numpy(),
           "weight": t["weight"][pos].cpu().numpy()}
    ref = _expect_by_source_delay(oracle_mod.generate_primary(spec, proj, b))
    np.testing.assert_array_equal(got["src"], ref["src"].astype(np.int64), err_msg=f"proj {proj} target {tgt}")
    np.testing.assert_array_equal(got["delay"], ref["delay"].astype(np.int64))
    assert ulp_diff(got["weight"], ref["weight"]).max(initial=0) <= WEIGHT_ULP
    return ref["src"].size


def check_source_primary(torch, t, oracle_mod, spec, proj, a):
    """Connections from source s0 + a of projection proj (out-degree rule:
    the primary is the source) equal the oracle's, in order."""
    pj = spec.projections[proj]
    s = pj.src[0] + a
    row = t["row_ptr"]
    lo, hi = int(row[s]), int(row[s + 1])
    tg = t["target"][lo:hi].to(torch.int64)
    keep = (tg >= pj.tgt[0]) & (tg < pj.tgt[0] + pj.tgt[1])
    got = {"tgt": tg[keep].cpu().numpy(), "delay": (t["delay"][lo:hi][keep].to(torch.int64) & 0xFFFF).cpu().numpy(),
           "weight": t["weight"][lo:hi][keep].cpu().numpy()}
    ref = _expect_by_source_delay(oracle_mod.generate_primary(spec, proj, a))
    np.testing.assert_array_equal(got["tgt"], ref["tgt"].astype(np.int64), err_msg=f"proj {proj} source {s}")
    np.testing.assert_array_equal(got["delay"], ref["delay"].astype(np.int64))
    assert ulp_diff(got["weight"], ref["weight"]).max(initial=0) <= WEIGHT_ULP
    return ref["tgt"].size


def check_projection_counts(torch, t, src, spec):
    """Every projection holds its count (fixed_total_number: N)."""
    tg = t["target"].to(torch.int64)
    for pj in spec.projections:
        inside = ((src >= pj.src[0]) & (src < pj.src[0] + pj.src[1]) &
                  (tg >= pj.tgt[0]) & (tg < pj.tgt[0] + pj.tgt[1]))
        assert int(inside.sum()) == pj.k


def check_total_no_multapses(torch, t, src, spec):
    """fixed_total_number without autapses or multapses: per projection N
    connections, no autapse, no pair twice."""
    tg = t["target"].to(torch.int64)
    assert not bool(torch.any(src == tg)), "autapse"
    pair = torch.sort(src * (1 << 32) + tg).values
    assert not bool(torch.any(pair[1:] == pair[:-1])), "multapse"
    for pj in spec.projections:
        inside = ((src >= pj.src[0]) & (src < pj.src[0] + pj.src[1]) &
                  (tg >= pj.tgt[0]) & (tg < pj.tgt[0] + pj.tgt[1]))
        assert int(inside.sum()) == pj.k
