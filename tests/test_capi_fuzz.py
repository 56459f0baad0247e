"""Randomised corruptions of valid samples are refused by vegas_create before any device
work (host only, no GPU).

Each case takes a valid sample (periodic sc, random graph, fcc sphere with its sublattice
colouring, frustrated triangles), applies one corruption drawn at random (a broken link, a
non-finite parameter, a bad row pointer, an improper colouring, a bad policy table, ...) at a
random place, and checks that the library answers VEGAS_EINVAL with a message and without
touching memory it was not given. The untouched samples pass validation (without a GPU the
call then stops at the device query). The exported greedy colouring gets the same treatment.
"""

import ctypes as C
import subprocess
import sys
import zlib

import numpy as np
import pytest

import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from conftest import ROOT
from lattices import fcc_sphere, random_graph, sc_periodic, triangles

MAKERS = [lambda: sc_periodic(4, k_uni=0.1), lambda: random_graph(40, 0.12, 5), lambda: fcc_sphere(3.0),
          lambda: triangles(6, J=-1.0)]


@pytest.fixture(scope="module")
def lib():
    vg.build()
    return vg.load_library()


def fresh(make):
    s = make()
    for k in ("row_ptr", "col", "J"):
        setattr(s, k, np.array(getattr(s, k)))
    return s


def rows(s):
    return np.repeat(np.arange(s.n_sites), np.diff(s.row_ptr))


def site_vector_field(name):
    def f(rng, s):
        v = np.tile([0.0, 0.0, 1.0], (s.n_sites, 1))
        v[rng.integers(s.n_sites), rng.integers(3)] = rng.choice([np.nan, np.inf, -np.inf])
        setattr(s, name, v)
    return f


def site_scalar_field(name, bad):
    def f(rng, s):
        v = np.ones(s.n_sites)
        v[rng.integers(s.n_sites)] = rng.choice(bad)
        setattr(s, name, v)
    return f


def asymmetric_J(rng, s):
    s.J[rng.integers(len(s.J))] += rng.choice([-0.5, 0.25, 1e-9])


def self_link(rng, s):
    e = rng.integers(len(s.col))
    s.col[e] = rows(s)[e]


def duplicate(rng, s):
    i = rng.choice(np.flatnonzero(np.diff(s.row_ptr) >= 2))
    b = s.row_ptr[i]
    s.col[b + 1] = s.col[b]


def out_of_range(rng, s):
    s.col[rng.integers(len(s.col))] = rng.choice([-1, s.n_sites, s.n_sites + 7, np.iinfo(np.int32).max])


def one_sided(rng, s):
    """Re-point one link at a site that does not link back."""
    e = rng.integers(len(s.col))
    i = rows(s)[e]
    linked = set(s.col[s.row_ptr[i]:s.row_ptr[i + 1]].tolist()) | {i}
    s.col[e] = rng.choice([j for j in range(s.n_sites) if j not in linked])


def row_ptr_start(rng, s):
    s.row_ptr[0] = rng.choice([1, -1])


def row_ptr_decreasing(rng, s):
    i = rng.choice(np.flatnonzero(np.diff(s.row_ptr) > 0))
    s.row_ptr[i + 1] = s.row_ptr[i] - 1


def row_ptr_end(rng, s):
    extra = rng.integers(1, 4)
    if rng.integers(2):  # more links given than the rows hold
        s.col = np.concatenate([s.col, np.zeros(extra, np.int32)])
        s.J = np.concatenate([s.J, np.ones(extra)])
    else:                # the last row runs past the links given
        s.row_ptr[-1] += extra


def nonfinite_J(rng, s):
    s.J[rng.integers(len(s.J))] = rng.choice([np.nan, np.inf])


def improper_colouring(rng, s):
    c = getattr(s, "colour", None)
    c = np.array(c if c is not None else vg.vegas_greedy_colour(s.row_ptr, s.col)[0])
    e = rng.integers(len(s.col))
    c[rows(s)[e]] = c[s.col[e]]
    s.colour = c.astype(np.int32)


def colour_range(rng, s):
    c = np.zeros(s.n_sites, np.int32) if getattr(s, "colour", None) is None else np.asarray(s.colour).copy()
    c[rng.integers(s.n_sites)] = rng.choice([-1, 64, 1000])
    s.colour = c


def bad_policy(rng, s):
    k = rng.integers(3)
    if k == 0:
        s.with_policy([rng.choice([7, -2, 99])], [0.1])
    elif k == 1:
        s.with_policy([vg.POLICY_SMALL_STEP], [rng.choice([0.0, -0.1, 4.0, np.nan])])
    else:
        s.type = np.full(s.n_sites, 1, np.int32)
        s.with_policy([vg.POLICY_RANDOM], [0.0])


CORRUPTIONS = {
    "asymmetric J": asymmetric_J, "self link": self_link, "duplicate": duplicate, "out of range": out_of_range,
    "one-sided link": one_sided, "row_ptr start": row_ptr_start, "row_ptr decreasing": row_ptr_decreasing,
    "row_ptr end": row_ptr_end, "non-finite J": nonfinite_J, "improper colouring": improper_colouring,
    "colour range": colour_range, "policy table": bad_policy,
    "spin_norm": site_scalar_field("spin_norm", [0.0, -1.0, np.nan, np.inf]),
    "k_uni": site_scalar_field("k_uni", [np.nan, np.inf]),
    "k_cub": site_scalar_field("k_cub", [np.nan, -np.inf]),
    "field_axis": site_vector_field("field_axis"), "e_uni": site_vector_field("e_uni"),
    "init_spins": site_vector_field("init_spins"), "positions": site_vector_field("positions"),
}


def create_status(lib, samples):
    keep = [vb._SampleArrays(s) for s in samples]
    arr = (vb.vegas_sample * len(keep))(*[k.c for k in keep])
    out = C.c_void_p(1)
    st = lib.vegas_create(arr, len(keep), None, C.byref(out))
    msg = lib.vegas_last_error(None).decode()
    if st == vb.OK:
        lib.vegas_destroy(out)
    else:
        assert not out.value  # *out is NULL on failure
    return st, msg


@pytest.mark.parametrize("make", MAKERS)
def test_valid_samples_pass_validation(lib, make):
    st, msg = create_status(lib, [fresh(make)])
    assert st in (vb.OK, vb.ECUDA), msg


@pytest.mark.parametrize("name", sorted(CORRUPTIONS))
def test_random_corruptions_are_refused(lib, name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    for trial in range(12):
        make = MAKERS[trial % len(MAKERS)]
        s = fresh(make)
        CORRUPTIONS[name](rng, s)
        good = fresh(MAKERS[(trial + 1) % len(MAKERS)])
        samples = [good, s] if trial % 3 == 0 else [s]  # a bad sample after a good one too
        st, msg = create_status(lib, samples)
        assert st == vb.EINVAL, (name, trial, st, msg)
        assert msg, (name, trial)


def test_greedy_colour_refuses_bad_csr(lib):
    s = sc_periodic(4)
    rp, col = np.array(s.row_ptr, np.int64), np.array(s.col, np.int32)
    out = np.zeros(s.n_sites, np.int32)

    def call(n, r, c, o):
        return lib.vegas_greedy_colour(n, vb._ptr(r), vb._ptr(c), vb._ptr(o))

    assert call(s.n_sites, rp, col, out) == 2
    bad_start = rp.copy()
    bad_start[0] = 3
    dec = rp.copy()
    dec[5] = dec[4] - 1
    oor = col.copy()
    oor[7] = s.n_sites
    assert call(s.n_sites, bad_start, col, out) == -1
    assert call(s.n_sites, dec, col, out) == -1
    assert call(s.n_sites, rp, oor, out) == -1
    assert call(-1, rp, col, out) == -1
    assert lib.vegas_greedy_colour(s.n_sites, vb._ptr(rp), None, vb._ptr(out)) == -1
    assert call(0, np.zeros(1, np.int64), col, out) == 0


CHILD = """
import ctypes as C, resource, sys
sys.path.insert(0, {root!r})
from paper_1803_07030_gb300 import vegas as vb
from lattices import sc_periodic
lib = vb.load_library()
keep = vb._SampleArrays(sc_periodic(4))
arr = (vb.vegas_sample * 1)(keep.c)
out = C.c_void_p(1)
vm = [int(l.split()[1]) * 1024 for l in open("/proc/self/status") if l.startswith("VmSize")][0]
resource.setrlimit(resource.RLIMIT_AS, (vm + (1 << 30), vm + (1 << 30)))
st = lib.vegas_create(arr, 2 ** 31 - 1, None, C.byref(out))
print(st, out.value is None, lib.vegas_last_error(None).decode())
"""


def test_failed_host_allocation_is_a_status_not_an_abort(lib):
    """A host allocation that fails inside an entry point (here the per-sample table of
    2^31 - 1 samples, in a process allowed 1 GB of address space beyond what it holds) comes back as
    VEGAS_ENOMEM with *out = NULL instead of an exception through the C boundary."""
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    st, null_out, msg = r.stdout.split(maxsplit=2)
    assert int(st) == vb.ENOMEM and null_out == "True" and "allocation" in msg
