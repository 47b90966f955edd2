"""Target shards built by separate processes (world size 2, gloo): each rank
builds the connections onto its own target range and the ranks exchange
only their counts; the union of the shards is the single build.

On the CPU each rank's shard comes from the oracle (the whole network's
connections onto the rank's targets, sorted and indexed); with a GPU the
ranks build their shards with the library (snc_set_target_shard), which
generates only the target-primary projections' own targets."""
import os
import socket

import numpy as np
import pytest

from gpu_helpers import WEIGHT_ULP, ulp_diff
from paper_2306_09855_gb300.workloads import Dist, NetworkSpec, Projection

WD = dict(weight=Dist("normal", 1.0, 0.1), delay=Dist("normal", 1.5, 0.75))


def _spec():
    return NetworkSpec(seed=21, dt=0.1, populations=[700, 500], projections=[
        Projection(src=(0, 700), tgt=(0, 1200), rule="fixed_indegree", k=30, autapses=False, **WD),
        Projection(src=(0, 1200), tgt=(200, 900), rule="pairwise_bernoulli", p=0.02, multapses=False, **WD),
        Projection(src=(100, 900), tgt=(0, 1200), rule="fixed_outdegree", k=25, multapses=False, **WD),
        Projection(src=(0, 1200), tgt=(0, 1200), rule="fixed_total_number", k=40_000, autapses=False, **WD),
        Projection(src=(50, 150), tgt=(500, 300), rule="all_to_all", **WD),
        Projection(src=(0, 400), tgt=(650, 400), rule="one_to_one", **WD),
    ])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_shard(spec, first, n):
    import oracle
    g = oracle.generate(spec)
    keep = (g["tgt"] >= first) & (g["tgt"] < first + n)
    return oracle.sort_index(spec.n_nodes, g["src"][keep], g["tgt"][keep], g["delay"][keep], g["weight"][keep])


def _library_shard(spec, first, n):
    import torch
    torch.cuda.set_device(0)
    from paper_2306_09855_gb300 import snc
    net = snc.Network(spec, target_shard=(first, n)).finalize()
    out = net.to_host()
    net.close()
    return out


def _rank_main(rank, world, port, out_path, builder):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2306_09855_gb300 import replicas
    replicas.init("gloo")
    spec = _spec()
    first, n = replicas.shard_ranges(spec.n_nodes, world)[rank]
    net = (_library_shard if builder == "library" else _oracle_shard)(spec, first, n)
    counts, firsts = replicas.gather_shard_counts(int(net["src"].size))
    np.savez(out_path + ".%d.npz" % rank, first=first, n=n, counts=np.asarray(counts), firsts=np.asarray(firsts),
             **{k: net[k] for k in ("src", "tgt", "delay", "weight", "row_ptr", "group_ptr", "group_first")})
    replicas.barrier()
    import torch.distributed as dist
    dist.destroy_process_group()


def _run(tmp_path, builder, world=2):
    import torch.multiprocessing as mp
    out = str(tmp_path / "shard")
    mp.start_processes(_rank_main, args=(world, _free_port(), out, builder), nprocs=world, start_method="spawn",
                       join=True)
    return [dict(np.load(out + ".%d.npz" % r)) for r in range(world)]


def _check_union(oracle_mod, parts):
    spec = _spec()
    full = oracle_mod.build(spec)
    counts = [int(p["src"].size) for p in parts]
    covered = 0
    for r, p in enumerate(parts):
        # the all-gather gave every rank the same counts and global offsets
        assert list(p["counts"]) == counts and int(p["firsts"][r]) == sum(counts[:r])
        first, n = int(p["first"]), int(p["n"])
        assert first == covered
        covered += n
        assert np.all((p["tgt"] >= first) & (p["tgt"] < first + n))
        keep = (full["tgt"] >= first) & (full["tgt"] < first + n)
        # the shard is the whole network restricted to its targets, in order
        # (weights: the library's fp32 within 4 ulp of the oracle's double)
        for f in ("src", "tgt", "delay"):
            np.testing.assert_array_equal(p[f], full[f][keep], err_msg=f"rank {r}: {f}")
        assert ulp_diff(p["weight"], full["weight"][keep]).max(initial=0) <= WEIGHT_ULP
    assert covered == spec.n_nodes
    assert sum(counts) == full["src"].size
    # the union, merged back into the whole network's positions
    merged = np.zeros(full["src"].size, dtype=np.int64)
    for p in parts:
        keep = (full["tgt"] >= int(p["first"])) & (full["tgt"] < int(p["first"]) + int(p["n"]))
        merged[keep] += 1
    assert np.all(merged == 1)


def test_two_ranks_oracle_shards_union_is_the_network(tmp_path, oracle_mod):
    _check_union(oracle_mod, _run(tmp_path, "oracle"))


@pytest.mark.gpu
def test_two_ranks_library_shards_union_is_the_network(tmp_path, oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _check_union(oracle_mod, _run(tmp_path, "library"))


def test_shard_ranges_cover_the_nodes():
    from paper_2306_09855_gb300 import replicas
    for n_nodes, world in ((10, 3), (7, 7), (5, 8), (200_000, 4)):
        r = replicas.shard_ranges(n_nodes, world)
        assert len(r) == world and r[0][0] == 0
        assert sum(n for _, n in r) == n_nodes
        assert all(r[i][0] + r[i][1] == r[i + 1][0] for i in range(world - 1))
        assert max(n for _, n in r) - min(n for _, n in r) <= 1
