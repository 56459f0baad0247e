"""ctypes binding of the C oracle (vegas_oracle.c), built with gcc on first use.

Test infrastructure only: see the header of vegas_oracle.c for what is computed and which
passage of the paper each part follows.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vegas_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libvegas_oracle.so")
_lock = threading.Lock()
_lib = None

ERR_NAN = 1
ERR_SPHERE = 2


class _Sample(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("pad_", C.c_int32),
        ("row_ptr", C.c_void_p),
        ("col", C.c_void_p),
        ("J", C.c_void_p),
        ("spin_norm", C.c_void_p),
        ("field_axis", C.c_void_p),
        ("k_uni", C.c_void_p),
        ("e_uni", C.c_void_p),
        ("k_cub", C.c_void_p),
        ("type", C.c_void_p),
        ("type_policy", C.c_void_p),
        ("type_param", C.c_void_p),
        ("n_policy_types", C.c_int32),
        ("pad2_", C.c_int32),
    ]

RANDOM, SPIN_FLIP, SMALL_STEP, GAUSSIAN, HINZKE_NOWAK, ADAPTIVE, QISING = range(7)


class _Extra(C.Structure):
    _fields_ = [
        ("acc_hist", C.c_void_p),
        ("sigma_inout", C.c_void_p),
        ("type_hist", C.c_void_p),
        ("n_types", C.c_int32),
        ("pad_", C.c_int32),
        ("snaps", C.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with FMA contraction off; returns the path of the .so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _configure(lib):
    P = C.c_void_p
    lib.vo_philox4x32_10.argtypes = [P, P, P]
    lib.vo_sphere.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P]
    lib.vo_sphere.restype = C.c_int
    lib.vo_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
    lib.vo_uniform.restype = C.c_double
    lib.vo_greedy_colour.argtypes = [C.c_int32, P, P, P]
    lib.vo_greedy_colour.restype = C.c_int32
    lib.vo_energy.argtypes = [P, P, C.c_double]
    lib.vo_energy.restype = C.c_double
    lib.vo_magnetisation.argtypes = [C.c_int32, P, P]
    lib.vo_delta_e.argtypes = [P, P, C.c_int32, P, C.c_double]
    lib.vo_delta_e.restype = C.c_double
    lib.vo_renormalise.argtypes = [P, P]
    lib.vo_init_spins.argtypes = [P, C.c_uint64, C.c_int32, P]
    lib.vo_init_spins.restype = C.c_int
    lib.vo_run.argtypes = [P, P, C.c_uint64, C.c_int32, C.c_int32, P, P, C.c_int32, C.c_int32,
                           C.c_uint32, P, C.c_int32, P, P, C.c_int32, C.c_int32, C.c_int32]
    lib.vo_run.restype = C.c_int
    lib.vo_run_ex.argtypes = lib.vo_run.argtypes + [P]
    lib.vo_run_ex.restype = C.c_int
    lib.vo_log.argtypes = [C.c_double]
    lib.vo_log.restype = C.c_double
    lib.vo_cap_height.argtypes = [C.c_double]
    lib.vo_cap_height.restype = C.c_double
    lib.vo_trial.argtypes = [P, P, C.c_int32, C.c_uint64, C.c_uint32, C.c_int32, C.c_double, P]
    lib.vo_trial.restype = C.c_int
    lib.vo_ising_run.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_uint64, C.c_int32, C.c_int32, P, P, C.c_int32,
                                 C.c_int32, C.c_uint32, P, C.c_int32, P]
    lib.vo_ising_run.restype = C.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(C.CDLL(build()))
    return _lib


class use_library:
    """Context manager that points every oracle call at another build of vegas_oracle.c
    (the mutation tests compile deliberately broken copies and check that pins fail)."""

    def __init__(self, path: str):
        self.lib = _configure(C.CDLL(path))

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = self.lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_source(text: str, out_path: str) -> str:
    """Compile C source text with the oracle's flags into out_path (a shared library)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared", src,
                    "-o", out_path, "-lm", "-lpthread"], check=True)
    return out_path


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Bound:
    """Holds the contiguous arrays a _Sample points into, for the call's lifetime."""

    def __init__(self, s):
        def f64(a, shape=None):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            return a if shape is None else a.reshape(shape)

        n = s.n_sites
        self.row_ptr = np.ascontiguousarray(s.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(s.col, dtype=np.int32)
        self.J = f64(s.J)
        self.spin_norm = f64(s.spin_norm)
        self.field_axis = f64(s.field_axis, (n, 3))
        self.k_uni = f64(s.k_uni)
        self.e_uni = f64(s.e_uni, (n, 3))
        self.k_cub = f64(s.k_cub)
        tp = getattr(s, "type_policy", None)
        self.type = None if s.type is None else np.ascontiguousarray(s.type, dtype=np.int32)
        self.type_policy = None if tp is None else np.ascontiguousarray(tp, dtype=np.int32)
        self.type_param = None if tp is None else f64(s.type_param)
        nt = 0 if tp is None else int(self.type_policy.shape[0])
        self.c = _Sample(n, 0, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.J), _ptr(self.spin_norm),
                         _ptr(self.field_axis), _ptr(self.k_uni), _ptr(self.e_uni), _ptr(self.k_cub),
                         _ptr(self.type), _ptr(self.type_policy), _ptr(self.type_param), nt, 0)

    @property
    def ref(self):
        return C.byref(self.c)


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11) of a 4-word counter and 2-word key: the
    generator every random number of the chain comes from."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _load().vo_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def sphere(seed: int, c0: int, c1: int, c2: int, purpose: int):
    """Marsaglia (1972) point on the unit sphere from Philox candidates (purpose | k): the trial
    of the random policy (Sec. III.B). Returns (unit vector, candidates used)."""
    o = np.zeros(3)
    k = _load().vo_sphere(seed, c0, c1, c2, purpose, _ptr(o))
    return o, k


def uniform(seed: int, c0: int, c1: int, c2: int, c3: int) -> float:
    """53-bit uniform in [0, 1) from one Philox block: the acceptance draw of Eq. 4."""
    return _load().vo_uniform(seed, c0, c1, c2, c3)


def greedy_colour(sample):
    """Greedy colouring in site order (smallest colour no coloured neighbour has): the colour
    classes of the sweep. Returns (colours, number of colours)."""
    n = sample.n_sites
    rp = np.ascontiguousarray(sample.row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(sample.col, dtype=np.int32)
    out = np.zeros(max(n, 1), dtype=np.int32)
    nc = _load().vo_greedy_colour(n, _ptr(rp), _ptr(cl), _ptr(out))
    return out[:n], int(nc)


def energy(sample, S, B: float) -> float:
    """Total energy of Eq. 1-3 (each bond once) of spins S [n, 3] in field B."""
    b = _Bound(sample)
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(sample.n_sites, 3)
    return _load().vo_energy(b.ref, _ptr(S), float(B))


def magnetisation(S) -> np.ndarray:
    """M = sum_i S_i, the magnetization of the history (Sec. II)."""
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(-1, 3)
    o = np.zeros(3)
    _load().vo_magnetisation(S.shape[0], _ptr(S), _ptr(o))
    return o


def delta_e(sample, S, i: int, trial, B: float) -> float:
    """Energy change (Eq. 1-3) of replacing S_i by `trial`, in the oracle's fixed order."""
    b = _Bound(sample)
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(sample.n_sites, 3)
    t = np.ascontiguousarray(trial, dtype=np.float64)
    return _load().vo_delta_e(b.ref, _ptr(S), int(i), _ptr(t), float(B))


def renormalise(sample, S) -> np.ndarray:
    """S_i <- s_i S_i / |S_i| (once per temperature/field step); qIsing sites keep their length."""
    b = _Bound(sample)
    S = np.array(S, dtype=np.float64).reshape(sample.n_sites, 3)
    _load().vo_renormalise(b.ref, _ptr(S))
    return S


def init_spins(sample, seed: int, inst: int) -> np.ndarray:
    """Initial state of one instance: s_i times a Philox sphere point per site (Sec. III.B)."""
    b = _Bound(sample)
    S = np.zeros((sample.n_sites, 3))
    err = _load().vo_init_spins(b.ref, seed, inst, _ptr(S))
    if err:
        raise RuntimeError(f"oracle init error {err}")
    return S


def log(x: float) -> float:
    """The oracle's own natural logarithm (atanh series)."""
    return _load().vo_log(float(x))


def cap_height(theta: float) -> float:
    """h = 1 - cos(theta) of the small-step policy's cap (Sec. II)."""
    return _load().vo_cap_height(float(theta))


def trial(sample, S, i: int, seed: int, t: int, inst: int, sigma: float = 0.0):
    """Trial unit vector of site i under its policy (counters i, t, inst); returns (vector, err)."""
    b = _Bound(sample)
    S = np.ascontiguousarray(S, dtype=np.float64).reshape(sample.n_sites, 3)
    o = np.zeros(3)
    err = _load().vo_trial(b.ref, _ptr(S), int(i), seed, t, inst, float(sigma), _ptr(o))
    return o, err


def run(sample, T, B, mcs: int, seed: int = 1, spins=None, inst_base: int = 0, t0: int = 0,
        colour=None, log_mcs: int = 0, mode: int = 0, n_threads: int = 1, sigma=None, n_types: int = 0,
        snapshots: bool = False):
    """Run the chain for every instance in T's first axis.

    T, B: [n_inst, n_steps]. spins: None (Philox initial state) or [n_inst, n, 3].
    colour: the colour classes of the sweep, [n] (default: the sample's own colouring if it
    carries one, as the library takes it, else the greedy colouring in site order).
    sigma: None or [n_inst] starting widths of the adaptive policy (<= 0: the policy's
    parameter). n_types > 0: also the magnetization per site type after every MCS.
    snapshots: also the spins at the end of every step. Returns dict(spins=[n_inst,n,3],
    history=[n_inst, n_steps*mcs, 4], accepted=[n_inst, n_steps*mcs] int64, sigma=[n_inst],
    accept_log=[n_inst, log_mcs, n] uint8 or None, type_history=[n_inst, n_steps*mcs,
    n_types, 3] or None, snapshots=[n_inst, n_steps, n, 3] or None, err=int).
    """
    T = np.ascontiguousarray(np.atleast_2d(T), dtype=np.float64)
    B = np.ascontiguousarray(np.broadcast_to(np.atleast_2d(B), T.shape), dtype=np.float64)
    n_inst, n_steps = T.shape
    n = sample.n_sites
    b = _Bound(sample)
    init = 1 if spins is None else 0
    S = np.zeros((n_inst, n, 3)) if spins is None else np.array(spins, dtype=np.float64).reshape(n_inst, n, 3)
    hist = np.zeros((n_inst, n_steps * mcs, 4))
    alog = np.zeros((n_inst, log_mcs, n), dtype=np.uint8) if log_mcs > 0 else None
    if colour is None:
        colour = getattr(sample, "colour", None)
    cl = None if colour is None else np.ascontiguousarray(colour, dtype=np.int32)
    acc = np.zeros((n_inst, n_steps * mcs), dtype=np.int64)
    sg = np.zeros(n_inst) if sigma is None else np.array(np.broadcast_to(sigma, (n_inst,)), dtype=np.float64)
    th = np.zeros((n_inst, n_steps * mcs, n_types, 3)) if n_types > 0 else None
    snaps = np.zeros((n_inst, n_steps, n, 3)) if snapshots else None
    x = _Extra(_ptr(acc), _ptr(sg), _ptr(th), int(n_types), 0, _ptr(snaps))
    err = _load().vo_run_ex(b.ref, _ptr(cl), seed, n_inst, inst_base, _ptr(T), _ptr(B), n_steps, mcs, t0, _ptr(S),
                            init, _ptr(hist), _ptr(alog), log_mcs, mode, n_threads, C.byref(x))
    if err < 0:
        raise ValueError("oracle rejected its arguments")
    return {"spins": S, "history": hist, "accepted": acc, "sigma": sg, "accept_log": alog, "type_history": th,
            "snapshots": snaps, "err": err}


def ising_run(dims: int, L: int, J: float, T, h, mcs: int, seed: int = 1, inst_base: int = 0, spins=None,
              t0: int = 0):
    """Ising chain (spin flip) on the periodic square (dims 2) or cubic (dims 3) lattice.

    T, h: [n_rep, n_steps]. spins: None (Philox initial state) or int8 [n_rep, L^dims].
    Returns dict(spins=int8 [n_rep, n], history=[n_rep, n_steps*mcs, 2] = (E, M)).
    """
    T = np.ascontiguousarray(np.atleast_2d(T), dtype=np.float64)
    h = np.ascontiguousarray(np.broadcast_to(np.atleast_2d(h), T.shape), dtype=np.float64)
    n_rep, n_steps = T.shape
    n = L ** dims
    init = 1 if spins is None else 0
    S = np.zeros((n_rep, n), dtype=np.int8) if spins is None else np.array(spins, dtype=np.int8).reshape(n_rep, n)
    hist = np.zeros((n_rep, n_steps * mcs, 2))
    err = _load().vo_ising_run(dims, L, J, seed, n_rep, inst_base, _ptr(T), _ptr(h), n_steps, mcs, t0, _ptr(S), init,
                               _ptr(hist))
    if err < 0:
        raise ValueError("oracle rejected its arguments")
    return {"spins": S, "history": hist}
