"""Thin ctypes binding of the C-ABI in include/vegas.h (argument marshalling only).

Every step of the sweep runs in the CUDA library; this module only converts numpy arrays
to the C structs and back. The library must have been built (paper_1803_07030_gb300.build);
if it is missing, loading raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .build import LIB

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDEVICE, ESTATE = range(7)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EDEVICE", 6: "ESTATE"}

P = C.c_void_p


class vegas_sample(C.Structure):
    _fields_ = [
        ("n_sites", C.c_int32),
        ("n_policy_types", C.c_int32),
        ("n_edges", C.c_int64),
        ("row_ptr", P),
        ("col", P),
        ("J", P),
        ("type", P),
        ("spin_norm", P),
        ("field_axis", P),
        ("k_uni", P),
        ("e_uni", P),
        ("k_cub", P),
        ("color", P),
        ("init_spins", P),
        ("positions", P),
        ("type_policy", P),
        ("type_param", P),
    ]

# bits of vegas_stats_t.sweep_kernels (VEGAS_KERNEL_*)
KERNEL_BITS = {"pass64": 0x1, "pass32_direct": 0x2, "pass32_staged": 0x4, "pass32_r32": 0x8,
               "pass32_r32_policy": 0x10, "resident32": 0x20, "coop32": 0x40, "cluster32": 0x80, "wave32": 0x100,
               "pass32_r32_one_policy": 0x200, "resident32_smem": 0x400, "cluster32_smem": 0x800,
               "pass32_r32_renorm": 0x1000, "coop64": 0x2000}


def sweep_kernel_names(bits: int) -> list:
    """Names of the sweep kernels in a vegas_stats_t.sweep_kernels mask."""
    return [k for k, v in KERNEL_BITS.items() if bits & v]


# update policies (vegas_policy)
(POLICY_RANDOM, POLICY_SPIN_FLIP, POLICY_SMALL_STEP, POLICY_GAUSSIAN, POLICY_HINZKE_NOWAK, POLICY_ADAPTIVE,
 POLICY_QISING) = range(7)


class vegas_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("replicas", C.c_int32),
        ("seed", C.c_uint64),
        ("inst_base", C.c_int32),
        ("device", C.c_int32),
        ("cuda_stream", P),
        ("variant", C.c_int32),
        ("accept_log_mcs", C.c_int32),
        ("timing", C.c_int32),
        ("graphs", C.c_int32),
        ("max_blocks", C.c_int32),
        ("pipeline_depth", C.c_int32),
        ("timeout_ns", C.c_int64),
        ("fault_inject", C.c_int32),
        ("type_stats", C.c_int32),
        ("snapshots", C.c_int32),
        ("cluster_blocks", C.c_int32),
        ("cluster_threads", C.c_int32),
        ("group_threads", C.c_int32),
        ("group_sites", C.c_int32),
        ("cluster_split", C.c_int32),
        ("wave_lag", C.c_int32),
        ("wave_slab", C.c_int32),
        ("resident_smem", C.c_int32),
        ("renorm_fold", C.c_int32),
    ]


class vegas_stats_t(C.Structure):
    _fields_ = [
        ("n_samples", C.c_int32),
        ("n_instances", C.c_int32),
        ("replicas", C.c_int32),
        ("precision", C.c_int32),
        ("max_colours", C.c_int32),
        ("variant", C.c_int32),
        ("n_sites", C.c_int64),
        ("n_edges", C.c_int64),
        ("records", C.c_int64),
        ("mcs_done", C.c_uint32),
        ("device_error", C.c_uint32),
        ("kernel_launches", C.c_int64),
        ("sweep_launches", C.c_int64),
        ("sweep_ms", C.c_double),
        ("last_run_ms", C.c_double),
        ("device_bytes", C.c_int64),
        ("n_types", C.c_int32),
        ("pad_", C.c_int32),
        ("snapshot_steps", C.c_int64),
        ("block_threads", C.c_int32),
        ("cluster_blocks", C.c_int32),
        ("graph_launches", C.c_int64),
        ("split_sites", C.c_int32),
        ("group_threads", C.c_int32),
        ("group_sites", C.c_int32),
        ("sweep_kernels", C.c_uint32),
    ]


class vegas_ising_options(C.Structure):
    _fields_ = [
        ("dims", C.c_int32),
        ("L", C.c_int32),
        ("J", C.c_double),
        ("replicas", C.c_int32),
        ("inst_base", C.c_int32),
        ("seed", C.c_uint64),
        ("device", C.c_int32),
        ("cuda_stream", P),
        ("init_up", C.c_int32),
        ("timing", C.c_int32),
    ]


# every function declared in include/vegas.h, with its ctypes signature
SIGNATURES = {
    "vegas_default_options": (None, [P]),
    "vegas_create": (C.c_int, [P, C.c_int32, P, P]),
    "vegas_run": (C.c_int, [P, P, P, C.c_int32, C.c_int32]),
    "vegas_history": (C.c_int, [P, P, C.c_size_t, P]),
    "vegas_get_spins": (C.c_int, [P, C.c_int32, P]),
    "vegas_set_spins": (C.c_int, [P, C.c_int32, P]),
    "vegas_set_mcs_counter": (C.c_int, [P, C.c_uint32]),
    "vegas_accept_log": (C.c_int, [P, P, C.c_size_t, P]),
    "vegas_accept_history": (C.c_int, [P, P, C.c_size_t, P]),
    "vegas_adaptive_width": (C.c_int, [P, P]),
    "vegas_type_history": (C.c_int, [P, P, C.c_size_t, P]),
    "vegas_get_snapshot": (C.c_int, [P, C.c_int32, C.c_int64, P]),
    "vegas_set_adaptive_width": (C.c_int, [P, P]),
    "vegas_stats": (C.c_int, [P, P]),
    "vegas_greedy_colour": (C.c_int32, [C.c_int32, P, P, P]),
    "vegas_last_error": (C.c_char_p, [P]),
    "vegas_destroy": (None, [P]),
    "vegas_sweep_noalloc": (C.c_int, [P, P, P, P, C.c_int32, P, C.c_int32, C.c_int32, P, P, P, C.c_uint64,
                                      C.c_int32, C.c_uint32, P, P]),
    "vegas_noalloc_last_error": (C.c_char_p, []),
    "vegas_thermal_averages": (C.c_int, [P, C.c_int64, C.c_int64, C.c_int64, C.c_int32, P, P, P, P]),
    "vegas_reweight": (C.c_int, [P, P, C.c_int32, C.c_int64, C.c_int32, P, P, C.c_int32, C.c_int32, C.c_double, P,
                                 P, P, P]),
    "vegas_analysis_last_error": (C.c_char_p, []),
    "vegas_ising_default_options": (None, [P]),
    "vegas_ising_create": (C.c_int, [P, P]),
    "vegas_ising_run": (C.c_int, [P, P, P, C.c_int32, C.c_int32]),
    "vegas_ising_history": (C.c_int, [P, P, C.c_size_t, P]),
    "vegas_ising_get_spins": (C.c_int, [P, C.c_int32, P]),
    "vegas_ising_set_spins": (C.c_int, [P, C.c_int32, P]),
    "vegas_ising_set_mcs_counter": (C.c_int, [P, C.c_uint32]),
    "vegas_ising_stats": (C.c_int, [P, P]),
    "vegas_ising_last_error": (C.c_char_p, [P]),
    "vegas_ising_destroy": (None, [P]),
}

AVG_FIELDS = ("e", "e_err", "m", "m_err", "c", "c_err", "chi", "chi_err", "u4", "u4_err", "v1", "v2", "tau_e",
              "tau_m", "n", "bins")

_lib = None


def load_library(path: Optional[str] = None) -> C.CDLL:
    """Load libvegas.so (built in-tree); raises OSError if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise OSError(f"CUDA library not built: {p} (run paper_1803_07030_gb300.build.build())")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


class VegasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, ctx_ptr) -> None:
    if st != OK:
        msg = load_library().vegas_last_error(ctx_ptr)
        raise VegasError(st, msg.decode() if msg else "")


def _arr(a, dtype, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=dtype)
    return a if shape is None else a.reshape(shape)


def _ptr(a):
    return None if a is None else a.ctypes.data


def vegas_greedy_colour(row_ptr, col) -> tuple:
    """Host-only greedy colouring of the library (sites in index order)."""
    rp = _arr(row_ptr, np.int64)
    cl = _arr(col, np.int32)
    n = rp.shape[0] - 1
    out = np.zeros(max(n, 1), dtype=np.int32)
    nc = load_library().vegas_greedy_colour(n, _ptr(rp), _ptr(cl), _ptr(out))
    if nc < 0:
        raise ValueError("invalid CSR")
    return out[:n], int(nc)


def vegas_default_options() -> vegas_options:
    o = vegas_options()
    load_library().vegas_default_options(C.byref(o))
    return o


class _SampleArrays:
    """Keeps the numpy arrays a vegas_sample points into alive."""

    def __init__(self, s):
        n = int(np.asarray(s.row_ptr).shape[0] - 1)
        self.row_ptr = _arr(s.row_ptr, np.int64)
        self.col = _arr(s.col, np.int32)
        self.J = _arr(s.J, np.float64)
        g = lambda k: getattr(s, k, None)  # noqa: E731
        self.type = _arr(g("type"), np.int32)
        self.spin_norm = _arr(g("spin_norm"), np.float64)
        self.field_axis = _arr(g("field_axis"), np.float64, (n, 3) if g("field_axis") is not None else None)
        self.k_uni = _arr(g("k_uni"), np.float64)
        self.e_uni = _arr(g("e_uni"), np.float64, (n, 3) if g("e_uni") is not None else None)
        self.k_cub = _arr(g("k_cub"), np.float64)
        self.color = _arr(g("colour"), np.int32)
        self.init_spins = _arr(g("init_spins"), np.float64)
        self.positions = _arr(g("positions"), np.float64, (n, 3) if g("positions") is not None else None)
        self.type_policy = _arr(g("type_policy"), np.int32)
        self.type_param = _arr(g("type_param"), np.float64)
        nt = 0 if self.type_policy is None else int(self.type_policy.shape[0])
        self.c = vegas_sample(n, nt, int(self.col.shape[0]), _ptr(self.row_ptr), _ptr(self.col), _ptr(self.J),
                              _ptr(self.type), _ptr(self.spin_norm), _ptr(self.field_axis), _ptr(self.k_uni),
                              _ptr(self.e_uni), _ptr(self.k_cub), _ptr(self.color), _ptr(self.init_spins),
                              _ptr(self.positions), _ptr(self.type_policy), _ptr(self.type_param))


def vegas_create(samples: Sequence, options: vegas_options):
    """Returns an opaque context pointer (int). Raises VegasError on failure."""
    keep = [_SampleArrays(s) for s in samples]
    arr = (vegas_sample * len(keep))(*[k.c for k in keep])
    ctx = P()
    st = load_library().vegas_create(arr, len(keep), C.byref(options), C.byref(ctx))
    _check(st, None)
    return ctx.value


def vegas_run(ctx, T, B, n_steps: int, mcs: int) -> None:
    T = _arr(T, np.float64)
    B = _arr(B, np.float64)
    _check(load_library().vegas_run(ctx, _ptr(T), _ptr(B), n_steps, mcs), ctx)


def vegas_history(ctx) -> np.ndarray:
    lib = load_library()
    n = C.c_size_t()
    _check(lib.vegas_history(ctx, None, 0, C.byref(n)), ctx)
    out = np.zeros(n.value, dtype=np.float64)
    _check(lib.vegas_history(ctx, _ptr(out), n.value, C.byref(n)), ctx)
    return out


def vegas_get_spins(ctx, inst: int, n_sites: int) -> np.ndarray:
    out = np.zeros((n_sites, 3), dtype=np.float64)
    _check(load_library().vegas_get_spins(ctx, inst, _ptr(out)), ctx)
    return out


def vegas_set_spins(ctx, inst: int, spins) -> None:
    s = _arr(spins, np.float64)
    _check(load_library().vegas_set_spins(ctx, inst, _ptr(s)), ctx)


def vegas_set_mcs_counter(ctx, t: int) -> None:
    _check(load_library().vegas_set_mcs_counter(ctx, int(t)), ctx)


def vegas_accept_log(ctx) -> np.ndarray:
    lib = load_library()
    n = C.c_size_t()
    _check(lib.vegas_accept_log(ctx, None, 0, C.byref(n)), ctx)
    out = np.zeros(n.value, dtype=np.uint8)
    if n.value:
        _check(lib.vegas_accept_log(ctx, _ptr(out), n.value, C.byref(n)), ctx)
    return out


def vegas_accept_history(ctx) -> np.ndarray:
    lib = load_library()
    n = C.c_size_t()
    _check(lib.vegas_accept_history(ctx, None, 0, C.byref(n)), ctx)
    out = np.zeros(n.value, dtype=np.uint32)
    if n.value:
        _check(lib.vegas_accept_history(ctx, _ptr(out), n.value, C.byref(n)), ctx)
    return out


def vegas_type_history(ctx) -> np.ndarray:
    lib = load_library()
    n = C.c_size_t()
    _check(lib.vegas_type_history(ctx, None, 0, C.byref(n)), ctx)
    out = np.zeros(n.value, dtype=np.float64)
    if n.value:
        _check(lib.vegas_type_history(ctx, _ptr(out), n.value, C.byref(n)), ctx)
    return out


def vegas_get_snapshot(ctx, inst: int, step: int, n_sites: int) -> np.ndarray:
    out = np.zeros((n_sites, 3), dtype=np.float64)
    _check(load_library().vegas_get_snapshot(ctx, inst, step, _ptr(out)), ctx)
    return out


def vegas_adaptive_width(ctx, n_instances: int) -> np.ndarray:
    out = np.zeros(n_instances, dtype=np.float64)
    _check(load_library().vegas_adaptive_width(ctx, _ptr(out)), ctx)
    return out


def vegas_set_adaptive_width(ctx, widths) -> None:
    w = _arr(widths, np.float64)
    _check(load_library().vegas_set_adaptive_width(ctx, _ptr(w)), ctx)


def vegas_stats(ctx) -> dict:
    s = vegas_stats_t()
    _check(load_library().vegas_stats(ctx, C.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in vegas_stats_t._fields_}


def vegas_sweep_noalloc(spins_ptr: int, links_ptr: int, row_ptr_ptr: int, site_id_ptr: int, n_sites: int,
                        colour_start, replicas: int, beta, field, site_params=None, seed: int = 1, inst0: int = 0,
                        t: int = 0, out_ptr: int = 0, stream: Optional[int] = None) -> None:
    """One MCS on caller-owned device buffers (device pointers as ints); allocates nothing."""
    cs = _arr(colour_start, np.int32)
    b = _arr(beta, np.float64)
    f = _arr(field, np.float64)
    sp = _arr(site_params, np.float64)
    # the C side reads replicas entries of beta and field, 9 site parameters and
    # n_colours + 1 colour starts from these host arrays
    if cs is None or cs.ndim != 1 or cs.size < 2:
        raise ValueError("colour_start needs n_colours + 1 >= 2 entries")
    if b is None or f is None or b.size < replicas or f.size < replicas:
        raise ValueError("beta and field need one entry per replica")
    if sp is not None and sp.size != 9:
        raise ValueError("site_params holds 9 values (nx, ny, nz, s, ex, ey, ez, k, kc)")
    lib = load_library()
    st = lib.vegas_sweep_noalloc(spins_ptr, links_ptr, row_ptr_ptr, site_id_ptr, n_sites, _ptr(cs), len(cs) - 1,
                                 replicas, _ptr(b), _ptr(f), _ptr(sp), seed, inst0, t, out_ptr, stream)
    if st != OK:
        m = lib.vegas_noalloc_last_error()
        raise VegasError(st, m.decode() if m else "")


def _check_analysis(st: int) -> None:
    if st != OK:
        msg = load_library().vegas_analysis_last_error()
        raise VegasError(st, msg.decode() if msg else "")


def thermal_averages(series, cut: int, n_bins: int, T, n_sites, stream=None) -> np.ndarray:
    """series [n_series, len, 4] (E, Mx, My, Mz per MCS); T, n_sites per series (or scalars).
    Returns [n_series, 16] in the order of AVG_FIELDS, computed on the GPU."""
    h = _arr(series, np.float64)
    if h.ndim == 2:
        h = h[None]
    ns, ln = h.shape[0], h.shape[1]
    Tv = _arr(np.broadcast_to(np.asarray(T, dtype=np.float64), (ns,)), np.float64)
    Nv = _arr(np.broadcast_to(np.asarray(n_sites, dtype=np.float64), (ns,)), np.float64)
    out = np.zeros((ns, len(AVG_FIELDS)))
    _check_analysis(load_library().vegas_thermal_averages(_ptr(h), ns, ln, int(cut), int(n_bins), _ptr(Tv), _ptr(Nv),
                                                          _ptr(out), stream))
    return out


def reweight(E, O, betas_k, betas_out, max_iter: int = 10000, tol: float = 1e-12, stream=None):
    """E [K, n], O [K, n, n_obs]; returns (<O> at betas_out [n_out, n_obs], g [K], iterations)."""
    Ea = _arr(E, np.float64)
    K, n = Ea.shape
    Oa = _arr(O, np.float64).reshape(K, n, -1)
    n_obs = Oa.shape[2]
    bk = _arr(betas_k, np.float64)
    bo = _arr(np.atleast_1d(betas_out), np.float64)
    out = np.zeros((bo.shape[0], max(n_obs, 1)))
    g = np.zeros(K)
    it = C.c_int32()
    _check_analysis(load_library().vegas_reweight(_ptr(Ea), _ptr(Oa), K, n, n_obs, _ptr(bk), _ptr(bo), bo.shape[0],
                                                  int(max_iter), float(tol), _ptr(out), _ptr(g), C.byref(it), stream))
    return out[:, :n_obs], g, it.value


def vegas_last_error(ctx=None) -> str:
    m = load_library().vegas_last_error(ctx)
    return m.decode() if m else ""


def vegas_destroy(ctx) -> None:
    if ctx:
        load_library().vegas_destroy(ctx)


def _current_stream() -> Optional[int]:
    try:
        import torch

        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:  # torch missing or no device: the library makes its own stream
        return None
    return None


class Context:
    """One vegas context: samples x replicas instances on one GPU.

    samples: objects with numpy attributes row_ptr, col, J and optionally type, spin_norm,
    field_axis, k_uni, e_uni, k_cub, colour, init_spins, positions, type_policy, type_param
    (the vegas_sample fields).
    stream: a cudaStream_t as int, 'torch' for torch's current stream, or None (own stream).
    The other keywords are the vegas_options fields of the same names (include/vegas.h):
    variant (-1 automatic, 0 per class, 1 resident, 2 cooperative, 3 cluster, 4 wavefront),
    graphs (1 a run as one graph, 2 a graph per step, 0 none), the cluster and grouping shapes
    (cluster_blocks, cluster_threads, cluster_split, group_threads, group_sites; 0 =
    automatic or off), wave_lag, wave_slab, resident_smem (1: the resident sweep keeps spins in
    shared memory), renorm_fold (-1: the renormalisation always in a pass of its own), and the
    testing options max_blocks, pipeline_depth,
    timeout_ns, fault_inject. library: load another build (the debug build) for this and
    later contexts.
    """

    def __init__(self, samples: Sequence, precision: int = 32, replicas: int = 1, seed: int = 1,
                 inst_base: int = 0, device: int = -1, stream="torch", variant: int = -1,
                 accept_log_mcs: int = 0, timing: bool = False, graphs: int = 1, max_blocks: int = 0,
                 pipeline_depth: int = 0, timeout_ns: int = 0, fault_inject: int = 0,
                 type_stats: bool = False, snapshots: bool = False, cluster_blocks: int = 0,
                 cluster_threads: int = 0, cluster_split: int = 0, group_threads: int = 0, group_sites: int = 0,
                 wave_lag: int = 0, wave_slab: int = 0, resident_smem: int = 0, renorm_fold: int = 0,
                 library: Optional[str] = None):
        self.samples = list(samples)
        self.n_sites = [int(np.asarray(s.row_ptr).shape[0] - 1) for s in self.samples]
        if library is not None:
            global _lib
            _lib = load_library(library)
        o = vegas_default_options()
        o.precision = precision
        o.replicas = replicas
        o.seed = seed
        o.inst_base = inst_base
        o.device = device
        o.variant = variant
        o.accept_log_mcs = accept_log_mcs
        o.timing = 1 if timing else 0
        o.graphs = int(graphs)  # True = 1: a run as one graph; 2: a graph per step; False = 0
        o.max_blocks = max_blocks
        o.pipeline_depth = pipeline_depth
        o.timeout_ns = timeout_ns
        o.fault_inject = fault_inject
        o.type_stats = 1 if type_stats else 0
        o.snapshots = 1 if snapshots else 0
        o.cluster_blocks = cluster_blocks
        o.cluster_threads = cluster_threads
        o.cluster_split = cluster_split
        o.group_threads = group_threads
        o.group_sites = group_sites
        o.wave_lag = wave_lag
        o.wave_slab = wave_slab
        o.resident_smem = resident_smem
        o.renorm_fold = renorm_fold
        o.cuda_stream = _current_stream() if stream == "torch" else stream
        self.replicas = replicas
        self.ptr = None
        self.ptr = vegas_create(self.samples, o)

    @property
    def n_instances(self) -> int:
        return len(self.samples) * self.replicas

    def run(self, T, B, mcs: int) -> None:
        """T, B: scalars, per-step 1-D arrays, or [n_instances, n_steps] arrays."""
        T = np.asarray(T, dtype=np.float64)
        T = T.reshape(1, 1) if T.ndim == 0 else (T[None, :] if T.ndim == 1 else T)
        n_steps = T.shape[1]
        B = np.asarray(B, dtype=np.float64)
        B = np.full((1, n_steps), float(B)) if B.ndim == 0 else (B[None, :] if B.ndim == 1 else B)
        shape = (self.n_instances, n_steps)
        vegas_run(self.ptr, np.broadcast_to(T, shape), np.broadcast_to(B, shape), n_steps, mcs)

    def history(self) -> np.ndarray:
        """[n_instances, records, 4] = (E, Mx, My, Mz) after every MCS."""
        h = vegas_history(self.ptr)
        return h.reshape(self.n_instances, -1, 4)

    def spins(self, inst: int) -> np.ndarray:
        return vegas_get_spins(self.ptr, inst, self.n_sites[inst // self.replicas])

    def set_spins(self, inst: int, spins) -> None:
        if not 0 <= inst < self.n_instances:
            raise ValueError(f"instance {inst} outside [0, {self.n_instances})")
        a = _arr(spins, np.float64)
        n = self.n_sites[inst // self.replicas]
        if a.shape != (n, 3):  # the library reads n_sites x 3 doubles
            raise ValueError(f"spins of instance {inst} must have shape ({n}, 3), not {a.shape}")
        vegas_set_spins(self.ptr, inst, a)

    def set_mcs_counter(self, t: int) -> None:
        """Global MCS counter of the next MCS (keys its random numbers)."""
        vegas_set_mcs_counter(self.ptr, t)

    def checkpoint(self) -> dict:
        """Everything a new context over the same samples and options needs to continue the
        chain bit for bit: every instance's spins, the MCS counter and the adaptive widths."""
        return {"spins": [self.spins(i) for i in range(self.n_instances)], "mcs": self.stats()["mcs_done"],
                "widths": self.adaptive_width()}

    def restore(self, state: dict) -> None:
        """Load a checkpoint() of a context over the same samples and options."""
        if len(state["spins"]) != self.n_instances:
            raise ValueError("checkpoint has a different number of instances")
        for i, x in enumerate(state["spins"]):
            self.set_spins(i, x)
        w = np.asarray(state["widths"], dtype=np.float64)
        if np.any(w > 0):
            self.set_adaptive_width(np.where(w > 0, w, 1.0))
        self.set_mcs_counter(state["mcs"])

    def accept_log(self) -> np.ndarray:
        return vegas_accept_log(self.ptr)

    def accept_history(self) -> np.ndarray:
        """[n_instances, records] accepted attempts per MCS."""
        return vegas_accept_history(self.ptr).reshape(self.n_instances, -1)

    def type_history(self) -> np.ndarray:
        """[n_instances, records, n_types, 3] magnetization of every site type (type_stats)."""
        h = vegas_type_history(self.ptr)
        n_types = self.stats()["n_types"]
        return h.reshape(self.n_instances, -1, n_types, 3)

    def snapshot(self, inst: int, step: int) -> np.ndarray:
        """Spins of instance inst at the end of temperature/field step `step` (snapshots)."""
        return vegas_get_snapshot(self.ptr, inst, step, self.n_sites[inst // self.replicas])

    def adaptive_width(self) -> np.ndarray:
        return vegas_adaptive_width(self.ptr, self.n_instances)

    def set_adaptive_width(self, widths) -> None:
        vegas_set_adaptive_width(self.ptr, np.broadcast_to(np.asarray(widths, dtype=np.float64), (self.n_instances,)))

    def stats(self) -> dict:
        return vegas_stats(self.ptr)

    def close(self) -> None:
        if self.ptr:
            vegas_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class IsingContext:
    """Ising model (spin-flip policy) on a periodic square (dims 2) or cubic (dims 3) lattice,
    replicas multi-spin coded on the GPU (see include/vegas.h)."""

    def __init__(self, dims: int = 2, L: int = 64, J: float = 1.0, replicas: int = 32, seed: int = 1,
                 inst_base: int = 0, device: int = -1, stream=None, init_up: bool = False, timing: bool = False):
        lib = load_library()
        o = vegas_ising_options()
        lib.vegas_ising_default_options(C.byref(o))
        o.dims, o.L, o.J, o.replicas, o.seed, o.inst_base, o.device = dims, L, J, replicas, seed, inst_base, device
        o.cuda_stream = _current_stream() if stream == "torch" else stream
        o.init_up = 1 if init_up else 0
        o.timing = 1 if timing else 0
        self.dims, self.L, self.replicas = dims, L, replicas
        self.n_sites = L ** dims
        self.ptr = None
        ptr = P()
        st = lib.vegas_ising_create(C.byref(o), C.byref(ptr))
        if st != OK:
            msg = lib.vegas_ising_last_error(None)
            raise VegasError(st, msg.decode() if msg else "")
        self.ptr = ptr.value

    def _check(self, st):
        if st != OK:
            msg = load_library().vegas_ising_last_error(self.ptr)
            raise VegasError(st, msg.decode() if msg else "")

    def run(self, T, h, mcs: int) -> None:
        T = np.asarray(T, dtype=np.float64)
        T = T.reshape(1, 1) if T.ndim == 0 else (T[None, :] if T.ndim == 1 else T)
        n_steps = T.shape[1]
        T = np.ascontiguousarray(np.broadcast_to(T, (self.replicas, n_steps)))
        hv = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64).reshape(-1, n_steps)
                                                  if np.ndim(h) else np.full((1, n_steps), float(h)),
                                                  (self.replicas, n_steps)))
        self._check(load_library().vegas_ising_run(self.ptr, _ptr(T), _ptr(hv), n_steps, mcs))

    def history(self) -> np.ndarray:
        """[replicas, records, 2] = (E, M) after every MCS."""
        lib = load_library()
        n = C.c_size_t()
        self._check(lib.vegas_ising_history(self.ptr, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        if n.value:
            self._check(lib.vegas_ising_history(self.ptr, _ptr(out), n.value, C.byref(n)))
        return out.reshape(self.replicas, -1, 2)

    def spins(self, replica: int) -> np.ndarray:
        out = np.zeros(self.n_sites, dtype=np.int8)
        self._check(load_library().vegas_ising_get_spins(self.ptr, replica, _ptr(out)))
        return out

    def set_spins(self, replica: int, spins) -> None:
        s = np.ascontiguousarray(spins, dtype=np.int8)
        self._check(load_library().vegas_ising_set_spins(self.ptr, replica, _ptr(s)))

    def set_mcs_counter(self, t: int) -> None:
        """Global MCS counter of the next MCS (keys its random numbers)."""
        self._check(load_library().vegas_ising_set_mcs_counter(self.ptr, int(t)))

    def checkpoint(self) -> dict:
        """Every replica's spins and the MCS counter: what a new context with the same options
        needs to continue the chains bit for bit."""
        return {"spins": [self.spins(r) for r in range(self.replicas)], "mcs": self.stats()["mcs_done"]}

    def restore(self, state: dict) -> None:
        """Load a checkpoint() of a context with the same options."""
        if len(state["spins"]) != self.replicas:
            raise ValueError("checkpoint has a different number of replicas")
        for r, x in enumerate(state["spins"]):
            self.set_spins(r, x)
        self.set_mcs_counter(state["mcs"])

    def stats(self) -> dict:
        s = vegas_stats_t()
        self._check(load_library().vegas_ising_stats(self.ptr, C.byref(s)))
        return {k: getattr(s, k) for k, _ in vegas_stats_t._fields_}

    def close(self) -> None:
        if self.ptr:
            load_library().vegas_ising_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
