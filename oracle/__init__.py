"""CPU FP64 oracle of the Metropolis sweep and of the history analysis (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg import
this package. The CUDA library never does, and shares no code with it.
"""

from . import analysis  # noqa: F401
from .oracle import (  # noqa: F401
    ADAPTIVE,
    GAUSSIAN,
    HINZKE_NOWAK,
    QISING,
    RANDOM,
    SMALL_STEP,
    SPIN_FLIP,
    build,
    cap_height,
    delta_e,
    energy,
    greedy_colour,
    init_spins,
    ising_run,
    log,
    magnetisation,
    philox4x32_10,
    renormalise,
    run,
    sphere,
    trial,
    uniform,
)
