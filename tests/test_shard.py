"""Assignment of whole instances to ranks (host logic, CPU only).

The partition of samples into contiguous blocks must be the best any contiguous split can do
(checked against every split of small cases), must cover every sample once in rank order,
and must keep the sample-major instance numbering, so that each rank's oracle results equal
those of the same instances in one run. Two and three gloo ranks run their blocks of a small
nanoparticle batch through the oracle and the bench's timing reductions.
"""

import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from conftest import ROOT
from paper_1803_07030_gb300.shard import contiguous_shards, rank_shard, sample_costs


def best_max_cost(costs, world):
    """Smallest largest-block cost over every split of costs into `world` contiguous blocks."""
    n = len(costs)
    best = None
    for cuts in itertools.combinations_with_replacement(range(n + 1), world - 1):
        edges = (0,) + cuts + (n,)
        worst = max(sum(costs[edges[k]:edges[k + 1]]) for k in range(world))
        best = worst if best is None else min(best, worst)
    return best


def check_cover(shards, n, world):
    assert len(shards) == world
    pos = 0
    for b, e in shards:
        assert b == pos and e >= b
        pos = e
    assert pos == n


@pytest.mark.parametrize("seed", range(40))
def test_shards_are_the_best_contiguous_split(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 9))
    world = int(rng.integers(1, 5))
    costs = rng.integers(0, 20 if seed % 3 else 3, n).tolist()
    shards = contiguous_shards(costs, world)
    check_cover(shards, n, world)
    got = max((sum(costs[b:e]) for b, e in shards), default=0)
    assert got == (best_max_cost(costs, world) if n else 0)
    assert [rank_shard(costs, world, r) for r in range(world)] == shards


def test_shard_special_cases():
    assert contiguous_shards([4] * 12, 3) == [(0, 4), (4, 8), (8, 12)]  # equal costs: equal blocks
    assert contiguous_shards([7, 1, 1], 1) == [(0, 3)]
    assert contiguous_shards([9, 1, 1, 1], 2) == [(0, 1), (1, 4)]       # one sample outweighs the rest
    assert contiguous_shards([2, 3], 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]  # more ranks than samples
    assert contiguous_shards([], 3) == [(0, 0)] * 3
    for bad in (lambda: contiguous_shards([1], 0), lambda: contiguous_shards([1, -1], 2),
                lambda: rank_shard([1, 2], 2, 2)):
        with pytest.raises(ValueError):
            bad()


def test_nanoparticle_batch_balances_within_one_sample():
    """The 256 nanoparticles over 2-8 ranks: every rank's attempts are within the largest
    particle's of the mean, and the instance ranges follow the sample-major numbering."""
    sys.path.insert(0, ROOT)
    import bench
    from lattices import workload

    w = workload("np256", mcs=1)
    costs = sample_costs(w.samples, w.replicas, w.n_steps, w.mcs)
    assert sum(costs) == w.attempts()
    for world in (1, 2, 3, 4, 8):
        shares = [bench.workload_share(w, r, world) for r in range(world)]
        check_cover([s["range"] for s in shares], len(w.samples), world)
        mean = sum(costs) / world
        assert max(s["attempts"] for s in shares) <= mean + max(costs)
        for s in shares:
            b, e = s["range"]
            assert s["inst_base"] == b * w.replicas and s["scaling"] == "strong"
            assert s["job_attempts"] == w.attempts() and len(s["samples"]) == e - b
            assert np.array_equal(s["T"], w.T[b:e])
        assert shares[0]["max_over_mean"] == pytest.approx(max(s["attempts"] for s in shares) / mean)


def test_one_sample_workloads_run_as_copies():
    sys.path.insert(0, ROOT)
    import bench
    from lattices import workload

    w = workload("sc64_hyst", scale=0.125, mcs=2)
    shares = [bench.workload_share(w, r, 3) for r in range(3)]
    assert [s["inst_base"] for s in shares] == [0, 1, 2]
    assert all(s["scaling"] == "weak" and s["job_attempts"] == 3 * w.attempts() for s in shares)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import oracle
    from lattices import workload

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workload("np256", scale=0.03, mcs=4)
    share = bench.workload_share(w, rank, world)
    hist = []
    for k, smp in enumerate(share["samples"]):
        inst = share["inst_base"] + k * w.replicas
        res = oracle.run(smp, share["T"][k:k + 1], share["B"][k:k + 1], w.mcs, seed=w.seed, inst_base=inst)
        hist.append(res["history"][0])
    np.save(os.path.join(out_dir, f"range_{rank}.npy"), np.array(share["range"]))
    np.save(os.path.join(out_dir, f"hist_{rank}.npy"), np.array(hist, dtype=object), allow_pickle=True)
    slow = bench.slowest_rank_ms(5.0 + rank, world)
    total = bench.sum_over_ranks(float(share["attempts"]), world)
    np.save(os.path.join(out_dir, f"red_{rank}.npy"), np.array([slow, total]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_run_their_blocks_like_one_run(tmp_path, world):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    import oracle
    from lattices import workload

    w = workload("np256", scale=0.03, mcs=4)
    ranges = [tuple(np.load(tmp_path / f"range_{r}.npy")) for r in range(world)]
    check_cover(ranges, len(w.samples), world)
    for r, (b, e) in enumerate(ranges):
        got = np.load(tmp_path / f"hist_{r}.npy", allow_pickle=True)
        assert len(got) == e - b
        for k, p in enumerate(range(b, e)):
            ref = oracle.run(w.samples[p], w.T[p:p + 1], w.B[p:p + 1], w.mcs, seed=w.seed, inst_base=p)["history"][0]
            assert np.array_equal(got[k], ref), (r, p)
    for r in range(world):
        slow, total = np.load(tmp_path / f"red_{r}.npy")
        assert slow == 5.0 + world - 1 and total == w.attempts()
