"""GB300 (sm_103a) Metropolis sweep of the classical Heisenberg model behind a C-ABI.

The compute path is the CUDA library built from csrc/ (libvegas.so); vegas.py is its ctypes
binding. Importing the package does not build anything; call build.build() first.
"""

from .build import LIB, build  # noqa: F401
from .shard import contiguous_shards, rank_shard, sample_costs  # noqa: F401
from .vegas import (  # noqa: F401
    AVG_FIELDS,
    POLICY_ADAPTIVE,
    POLICY_GAUSSIAN,
    POLICY_HINZKE_NOWAK,
    POLICY_QISING,
    POLICY_RANDOM,
    POLICY_SMALL_STEP,
    POLICY_SPIN_FLIP,
    Context,
    IsingContext,
    VegasError,
    load_library,
    reweight,
    thermal_averages,
    vegas_accept_history,
    vegas_accept_log,
    vegas_adaptive_width,
    vegas_create,
    vegas_default_options,
    vegas_destroy,
    vegas_get_snapshot,
    vegas_get_spins,
    vegas_greedy_colour,
    vegas_history,
    vegas_last_error,
    vegas_run,
    vegas_set_adaptive_width,
    vegas_set_mcs_counter,
    vegas_set_spins,
    vegas_sweep_noalloc,
    vegas_stats,
    vegas_type_history,
)
