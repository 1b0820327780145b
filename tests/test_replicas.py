"""Multi-GPU runs are replicas over independent units: the sharding, routing
and timing reductions are host logic, checked here on CPU with world_size-2
gloo process groups (the unit solves stand in with the CPU oracle)."""
import os
import socket

import numpy as np
import pytest

from paper_2310_16298_gb300 import replicas


@pytest.mark.parametrize("n", [0, 1, 5, 6, 1024, 1031])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_owns_every_unit_once(n, world):
    seen = []
    sizes = []
    for rank in range(world):
        s = replicas.shard(n, rank, world)
        seen.extend(s)
        sizes.append(len(s))
    assert sorted(seen) == list(range(n))
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard(-1, 0, 1)


def test_routing_is_round_robin_and_complete():
    items = list(range(17))
    parts = [replicas.routed(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert parts[1] == [1, 4, 7, 10, 13, 16]


def test_field_seeds_distinct_and_rank0_unchanged():
    seeds = [replicas.field_seed(2, r) for r in range(8)]
    assert seeds[0] == 2 and len(set(seeds)) == 8


def test_reductions_are_identity_without_process_group():
    assert replicas.max_over_ranks(1.5) == 1.5
    assert replicas.sum_over_ranks(7) == 7.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import stencil_inputs as si
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    probs = si.batch_1024(6, lo=10, hi=20, steps_lo=2, steps_hi=4)
    mine = {i: float(oracle.gather(probs[i].field(), probs[i].r, probs[i].coeffs, probs[i].bc,
                                   probs[i].steps).sum())
            for i in replicas.shard(len(probs), rank, world)}
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t_max = replicas.max_over_ranks(1.0 + rank)
    n_tot = replicas.sum_over_ranks(len(mine))
    if rank == 0:
        merged = {}
        for d in gathered:
            assert not set(d) & set(merged), "a unit ran on two ranks"
            merged.update(d)
        np.save(os.path.join(out_dir, "sums.npy"), np.array([merged[i] for i in range(len(probs))]))
        np.save(os.path.join(out_dir, "red.npy"), np.array([t_max, n_tot]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_a_batch(tmp_path):
    import torch.multiprocessing as mp
    import stencil_inputs as si
    import oracle
    oracle.build()
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    sums = np.load(tmp_path / "sums.npy")
    t_max, n_tot = np.load(tmp_path / "red.npy")
    probs = si.batch_1024(6, lo=10, hi=20, steps_lo=2, steps_hi=4)
    want = [float(oracle.gather(p.field(), p.r, p.coeffs, p.bc, p.steps).sum()) for p in probs]
    assert list(sums) == want            # same units, same results, each exactly once
    assert t_max == 2.0 and n_tot == 6.0  # slowest rank; units of all ranks
