"""C-ABI library on the host (no GPU): it builds, loads, exports what include/vegas.h
declares, colours like the oracle, and rejects invalid samples and options before it
touches a device."""

import os
import re

import numpy as np
import pytest

from conftest import ROOT

import oracle
import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import fcc_sphere, random_graph, sc_periodic, triangles


@pytest.fixture(scope="module")
def lib():
    vg.build()
    return vg.load_library()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "vegas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vegas_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_function(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(vb.SIGNATURES)


def test_struct_sizes_match_header(lib):
    import ctypes as C

    # vegas_sample: 2 int32 + int64 + one pointer per array field of the header's struct
    text = open(os.path.join(ROOT, "include", "vegas.h")).read()
    body = text[text.index("typedef struct {\n    int32_t n_sites;"):text.index("} vegas_sample;")]
    n_ptr = len(re.findall(r"^\s*const [a-z0-9_]+ \*[A-Za-z_]+;", body, flags=re.M))
    assert n_ptr == len(vb.vegas_sample._fields_) - 3
    assert C.sizeof(vb.vegas_sample) == 16 + n_ptr * 8
    o = vg.vegas_default_options()
    assert (o.precision, o.replicas, o.seed, o.device, o.variant, o.graphs) == (32, 1, 1, -1, -1, 1)


@pytest.mark.parametrize("make", [lambda: sc_periodic(6), lambda: sc_periodic((5, 4, 3)), lambda: triangles(7),
                                  lambda: fcc_sphere(3.7), lambda: random_graph(150, 0.04, 9)])
def test_greedy_colouring_matches_oracle(lib, make):
    s = make()
    c, nc = vg.vegas_greedy_colour(s.row_ptr, s.col)
    c2, nc2 = oracle.greedy_colour(s)
    assert nc == nc2 and np.array_equal(c, c2)


def _create_status(samples, **kw):
    o = vg.vegas_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    try:
        ctx = vb.vegas_create(samples, o)
    except vb.VegasError as e:
        return e.status, str(e)
    vb.vegas_destroy(ctx)
    return vb.OK, ""


def _bad(mut):
    s = sc_periodic(4)
    s.J = s.J.copy()
    s.col = s.col.copy()
    s.row_ptr = s.row_ptr.copy()
    mut(s)
    return s


@pytest.mark.parametrize(
    "name,mut,needle",
    [
        ("asymmetric J", lambda s: s.J.__setitem__(0, 0.5), "not symmetric"),
        ("self link", lambda s: s.col.__setitem__(0, 0), "self-link"),
        ("duplicate", lambda s: s.col.__setitem__(1, s.col[0]), "duplicate"),
        ("out of range", lambda s: s.col.__setitem__(2, 64), "out of range"),
        ("row_ptr start", lambda s: s.row_ptr.__setitem__(0, 1), "row_ptr[0]"),
        ("nan J", lambda s: s.J.__setitem__(5, np.nan), "non-finite J"),
        ("bad norm", lambda s: setattr(s, "spin_norm", np.zeros(64)), "spin_norm"),
        ("nan axis", lambda s: setattr(s, "field_axis", np.full((64, 3), np.nan)), "field_axis"),
        ("improper colouring", lambda s: setattr(s, "colour", np.zeros(64, dtype=np.int32)), "not proper"),
    ],
)
def test_invalid_samples_rejected(lib, name, mut, needle):
    st, msg = _create_status([_bad(mut)])
    assert st == vb.EINVAL, (name, st, msg)
    assert needle in msg


def _with_table(policies, params, types=None):
    s = sc_periodic(4)
    if types is not None:
        s.type = np.asarray(types, dtype=np.int32)
    return s.with_policy(policies, params)


@pytest.mark.parametrize(
    "name,make,needle",
    [
        ("unknown policy", lambda: _with_table([7], [0.0]), "unknown update policy"),
        ("negative policy", lambda: _with_table([-1], [0.0]), "unknown update policy"),
        ("cap angle zero", lambda: _with_table([2], [0.0]), "cap half-angle"),
        ("cap angle above pi", lambda: _with_table([4], [3.2]), "cap half-angle"),
        ("gaussian width zero", lambda: _with_table([3], [0.0]), "Gaussian width"),
        ("adaptive width nan", lambda: _with_table([5], [np.nan]), "Gaussian width"),
        ("type outside table", lambda: _with_table([0, 1], [0.0, 0.0], np.full(64, 2)), "outside the policy table"),
        ("negative type", lambda: _with_table([0, 1], [0.0, 0.0], np.full(64, -1)), "outside the policy table"),
    ],
)
def test_invalid_policy_tables_rejected(lib, name, make, needle):
    st, msg = _create_status([make()])
    assert st == vb.EINVAL, (name, st, msg)
    assert needle in msg, msg


def test_type_statistics_reject_bad_types(lib):
    s = sc_periodic(4)
    s.type = np.full(64, -1, dtype=np.int32)
    st, msg = _create_status([s], type_stats=1)
    assert st == vb.EINVAL and "site type outside [0, 64)" in msg
    s.type = np.full(64, 64, dtype=np.int32)
    st, msg = _create_status([s], type_stats=1)
    assert st == vb.EINVAL


def test_policy_table_without_params_rejected(lib):
    import ctypes as C

    s = sc_periodic(4)
    keep = vb._SampleArrays(s)
    pol = np.zeros(1, dtype=np.int32)
    keep.c.n_policy_types = 1
    keep.c.type_policy = pol.ctypes.data
    arr = (vb.vegas_sample * 1)(keep.c)
    out = C.c_void_p()
    st = lib.vegas_create(arr, 1, None, C.byref(out))
    assert st == vb.EINVAL and b"type_param is NULL" in lib.vegas_last_error(None)


@pytest.mark.parametrize("opt", [{"precision": 16}, {"replicas": 3}, {"replicas": 64}, {"variant": 7},
                                 {"accept_log_mcs": -1}, {"type_stats": 2}, {"snapshots": -1},
                                 {"variant": 2, "type_stats": 1}, {"graphs": 3}, {"graphs": -1},
                                 {"cluster_blocks": 1}, {"cluster_blocks": 17}, {"cluster_threads": 300},
                                 {"cluster_split": -1}, {"group_threads": 100}, {"group_sites": -1},
                                 {"wave_lag": -1}, {"variant": 5}, {"wave_slab": -2}, {"resident_smem": 2},
                                 {"resident_smem": -2}, {"resident_smem": 1, "variant": 0},
                                 {"resident_smem": 1, "variant": 2}, {"renorm_fold": 1}, {"renorm_fold": -2}])
def test_invalid_options_rejected(lib, opt):
    st, msg = _create_status([sc_periodic(4)], **opt)
    assert st == vb.EINVAL, (opt, msg)


@pytest.mark.parametrize("samples,opt,needle", [
    ("sc4", {"variant": 4}, "32 replicas"),
    ("sc4", {"variant": 4, "replicas": 32, "precision": 64}, "FP32"),
    ("sc4", {"variant": 4, "replicas": 32, "type_stats": 1}, "per-type"),
    ("two", {"variant": 4, "replicas": 32}, "one sample"),
    ("sc4", {"variant": 4, "replicas": 32, "wave_lag": -1}, "wave_lag"),
    ("sc5", {"variant": 4, "replicas": 32}, "two colour classes"),   # odd periodic sides: 3 colours
    ("graph", {"variant": 4, "replicas": 32}, "six links"),
    ("policy", {"variant": 4, "replicas": 32}, "policy table"),
])
def test_wavefront_requirements_checked_before_the_device(lib, samples, opt, needle):
    s = {"sc4": [sc_periodic(4)], "two": [sc_periodic(4), sc_periodic(4)], "sc5": [sc_periodic(5)],
         "graph": [random_graph(40, 0.1, 3)],
         "policy": [sc_periodic(4).with_policy([vg.POLICY_SMALL_STEP], [0.5])]}[samples]
    st, msg = _create_status(s, **opt)
    assert st == vb.EINVAL and needle in msg, (st, msg)


def test_wavefront_sample_passes_validation(lib):
    """A periodic even-sided sc lattice with 32 replicas is accepted: without a GPU the
    create call gets as far as the device query."""
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    st, msg = _create_status([sc_periodic((4, 6, 8))], variant=4, replicas=32)
    assert st == vb.ECUDA and "no CUDA device" in msg, msg


def test_null_safety(lib):
    import ctypes as C

    lib.vegas_destroy(None)
    assert isinstance(lib.vegas_last_error(None), bytes)
    assert lib.vegas_stats(None, None) == vb.EINVAL
    assert lib.vegas_run(None, None, None, 1, 1) == vb.EINVAL
    assert lib.vegas_set_mcs_counter(None, 5) == vb.EINVAL
    assert lib.vegas_ising_set_mcs_counter(None, 5) == vb.EINVAL
    out = C.c_void_p()
    assert lib.vegas_create(None, 0, None, C.byref(out)) == vb.EINVAL and not out.value


def test_no_device_is_an_error_not_a_fallback(lib):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    st, msg = _create_status([sc_periodic(4)])
    assert st == vb.ECUDA and "no CUDA device" in msg


def test_analysis_arguments_rejected_before_the_device(lib):
    import ctypes as C

    h = np.zeros((2, 50, 4))
    T = np.ones(2)
    N = np.ones(2)
    out = np.zeros((2, vb.AVG_FIELDS.__len__()))
    P = lambda a: a.ctypes.data  # noqa: E731
    for cut, nb, Tv in ((50, 10, T), (0, 1, T), (0, 65, T), (45, 10, T), (0, 10, np.array([1.0, 0.0]))):
        st = lib.vegas_thermal_averages(P(h), 2, 50, cut, nb, P(Tv), P(N), P(out), None)
        assert st == vb.EINVAL, (cut, nb)
    E = np.zeros((2, 10))
    O = np.zeros((2, 10, 9))
    bk = np.ones(2)
    bo = np.ones(1)
    assert lib.vegas_reweight(P(E), P(O), 2, 10, 9, P(bk), P(bo), 1, 10, 1e-9, P(out), None, None, None) == vb.EINVAL
    assert lib.vegas_reweight(P(E), P(O), 2, 10, 1, P(bk), P(bo), 1, 10, 0.0, P(out), None, None, None) == vb.EINVAL
    E[0, 3] = np.nan
    assert lib.vegas_reweight(P(E), P(O), 2, 10, 1, P(bk), P(bo), 1, 10, 1e-9, P(out), None, None, None) == vb.EINVAL
    assert b"non-finite" in lib.vegas_analysis_last_error()


def test_analysis_without_a_device_is_an_error(lib):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(vb.VegasError) as e:
        vb.thermal_averages(np.ones((1, 40, 4)), 0, 4, 1.0, 1.0)
    assert e.value.status == vb.ECUDA


def test_ising_options_rejected_before_the_device(lib):
    for kw in ({"L": 96}, {"L": 0}, {"replicas": 6}, {"replicas": 1024}, {"inst_base": 2}, {"dims": 1},
               {"J": float("nan")}, {"L": 65536}):
        with pytest.raises(vb.VegasError) as e:
            vb.IsingContext(**kw)
        assert e.value.status == vb.EINVAL, kw


def test_noalloc_refuses_misaligned_pointers_before_the_device(lib):
    """Misaligned device pointers would fault the GPU in the kernels' vector loads, so the
    allocation-free entry point refuses them on the host: these calls never reach CUDA
    (the pointer values are never dereferenced)."""
    import ctypes as C

    cs = np.array([0, 4, 8], dtype=np.int32)
    beta = np.ones(2)
    field = np.zeros(2)
    good = dict(spins=0x10000, links=0x20000, row_ptr=0x30000, site_id=0x40000, out=0x50000)
    for name, bad in (("spins", 0x10008), ("links", 0x20004), ("row_ptr", 0x30004), ("out", 0x50004),
                      ("site_id", 0x40002)):
        p = dict(good, **{name: bad})
        st = lib.vegas_sweep_noalloc(p["spins"], p["links"], p["row_ptr"], p["site_id"], 8, cs.ctypes.data, 2, 2,
                                     beta.ctypes.data, field.ctypes.data, None, 1, 0, 0, p["out"], None)
        assert st == vb.EINVAL, name
        assert "aligned" in lib.vegas_noalloc_last_error().decode(), name
    assert C.sizeof(C.c_void_p) == 8


def test_noalloc_binding_checks_host_array_lengths(lib):
    args = (0x10000, 0x20000, 0x30000, 0x40000, 8)
    with pytest.raises(ValueError):
        vg.vegas_sweep_noalloc(*args, [0, 4, 8], 4, np.ones(2), np.zeros(4), out_ptr=0x50000)
    with pytest.raises(ValueError):
        vg.vegas_sweep_noalloc(*args, [0, 4, 8], 2, np.ones(2), np.zeros(1), out_ptr=0x50000)
    with pytest.raises(ValueError):
        vg.vegas_sweep_noalloc(*args, [0, 4, 8], 2, np.ones(2), np.zeros(2), site_params=np.zeros(8),
                               out_ptr=0x50000)
    with pytest.raises(ValueError):
        vg.vegas_sweep_noalloc(*args, [8], 2, np.ones(2), np.zeros(2), out_ptr=0x50000)
