"""Assignment of whole instances to ranks, one process per GPU.

Instances (replicas, temperatures, samples) are independent Markov chains and every random
number is keyed by the instance id, so the path shards over instances with nothing exchanged
while the chains run. A rank sweeps one contiguous block of samples in its own context, with
`inst_base` set to the block's first instance id; its results are then those of the same
instances in a single context over all samples. The blocks are chosen to balance the work,
attempts = sites x replicas x steps x MCS per sample, over the ranks.
"""

from __future__ import annotations


def sample_costs(samples, replicas: int, n_steps: int, mcs: int) -> list:
    """Attempted updates per sample over a schedule: every site of every replica once per MCS."""
    return [int(s.n_sites) * int(replicas) * int(n_steps) * int(mcs) for s in samples]


def _blocks_needed(costs, bound: int) -> int:
    """Contiguous blocks a left-to-right greedy packing needs when no block may exceed bound."""
    blocks, load = 1, 0
    for c in costs:
        if load + c > bound:
            blocks += 1
            load = 0
        load += c
    return blocks


def contiguous_shards(costs, world: int) -> list:
    """Split samples 0..n-1 into `world` contiguous half-open ranges (begin, end), in rank
    order, so that the largest range cost is as small as any contiguous split allows.

    The smallest feasible bound is found by bisection over integers: a bound is feasible when
    the greedy packing (close a block just before it would exceed the bound) needs at most
    `world` blocks, and the greedy packing needs the fewest blocks of any split under that
    bound. The ranges are then that packing; ranks past its last block get empty ranges
    (begin == end). Costs are non-negative integers.
    """
    if world < 1:
        raise ValueError("world must be at least 1")
    costs = [int(c) for c in costs]
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    n = len(costs)
    if n == 0:
        return [(0, 0)] * world
    lo, hi = max(costs), sum(costs)
    while lo < hi:
        mid = (lo + hi) // 2
        if _blocks_needed(costs, mid) <= world:
            hi = mid
        else:
            lo = mid + 1
    shards, begin, load = [], 0, 0
    for i, c in enumerate(costs):
        if load + c > lo:
            shards.append((begin, i))
            begin, load = i, 0
        load += c
    shards.append((begin, n))
    shards += [(n, n)] * (world - len(shards))
    return shards


def rank_shard(costs, world: int, rank: int) -> tuple:
    """The half-open sample range of one rank."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return contiguous_shards(costs, world)[rank]
