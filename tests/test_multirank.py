"""Multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

Each rank sweeps its own block of replicas; instances are independent and every random
number is keyed by the instance id, so the ranks need no collective on the data path.
The test runs the oracle for each rank's instances of a small +-J glass, checks that the
two ranks' instance sets are disjoint and complete, that per-instance results equal a
single-process run of all instances, and that the timing reduction takes the slowest
rank.
"""

import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from lattices import sc_periodic

    dist.init_process_group("gloo", rank=rank, world_size=world)
    R = 4
    insts = bench.rank_instances(rank, world, replicas=R)
    s = sc_periodic(4, bimodal_seed=3)
    T = np.array([0.5 + 0.1 * i for i in insts])[:, None]
    res = oracle.run(s, T, np.zeros_like(T), 5, seed=1, inst_base=insts[0])
    np.save(os.path.join(out_dir, f"spins_{rank}.npy"), res["spins"])
    np.save(os.path.join(out_dir, f"insts_{rank}.npy"), np.array(insts))
    slow = bench.slowest_rank_ms(10.0 + rank, world)
    np.save(os.path.join(out_dir, f"slow_{rank}.npy"), np.array([slow]))
    total = torch.tensor([len(insts) * s.n_sites * 5], dtype=torch.float64)
    dist.all_reduce(total)
    np.save(os.path.join(out_dir, f"total_{rank}.npy"), total.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_instances_without_a_collective(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    import oracle
    from lattices import sc_periodic

    insts = [np.load(tmp_path / f"insts_{r}.npy") for r in range(world)]
    assert not set(insts[0]) & set(insts[1])
    assert sorted(np.concatenate(insts).tolist()) == list(range(8))
    s = sc_periodic(4, bimodal_seed=3)
    T = np.array([0.5 + 0.1 * i for i in range(8)])[:, None]
    whole = oracle.run(s, T, np.zeros_like(T), 5, seed=1, inst_base=0)["spins"]
    for r in range(world):
        got = np.load(tmp_path / f"spins_{r}.npy")
        assert np.array_equal(got, whole[insts[r]])
    for r in range(world):
        assert float(np.load(tmp_path / f"slow_{r}.npy")[0]) == 11.0  # the slowest rank's time
        assert float(np.load(tmp_path / f"total_{r}.npy")[0]) == 8 * s.n_sites * 5
