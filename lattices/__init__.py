"""Seeded synthetic samples for the Metropolis sweep of the classical Heisenberg model.

This package builds inputs only: site lists, neighbour CSR with per-bond exchange,
per-site parameters and the temperature/field schedules of the workloads. It holds no
part of the Monte Carlo method itself (no energies, no trial moves, no random numbers
of the Markov chain). Random structure (bond signs, particle radii and centres) is drawn
from numpy's seeded PCG64 generator. Both the CPU oracle and the CUDA library consume
what it returns.
"""

from .generators import (  # noqa: F401
    Sample,
    chain_open,
    core_shell_particle,
    dimers,
    fcc_sphere,
    free_spins,
    nanoparticle_batch,
    random_graph,
    sc_periodic,
    triangles,
)
from .workloads import Workload, workload  # noqa: F401
