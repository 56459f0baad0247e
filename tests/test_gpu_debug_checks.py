"""The staged and wavefront sweeps with every index and alignment check on.

The debug build (VEGAS_DEBUG_CHECKS) checks every copy the staged kernels issue (link and
row addresses, link-slot and row-slot indices, caller ids, the 16-byte alignment of each
cp.async source) and every dependency the wavefront kernel reads; a failed check sets a
device error instead of touching memory. Small lattices with ragged classes (class sizes
that are not multiples of the 8-site block) run through the R = 32 per-class kernel (with
and without an update-policy table), the generic staged kernel (R = 4, depth 3) and the
wavefront kernel: no check may fail, and the spins must equal the normal build's.
"""

import numpy as np
import pytest

import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import sc_periodic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_lib():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    path = vg.build(debug=True)
    normal = vb.load_library()
    yield path
    vb._lib = normal  # later tests use the normal build again


def run(sample, library, **kw):
    """Run a context on one build and return its spins and device error bits; every call on
    the context goes to the build that created it."""
    saved = vb._lib
    try:
        if library is not None:
            vb._lib = vb.load_library(library)
        R = kw.pop("replicas")
        T = np.linspace(0.4, 2.5, R)[:, None] * np.array([[1.0, 0.8]])
        B = np.full_like(T, 0.15)
        with vg.Context([sample], replicas=R, stream=None, seed=51, **kw) as c:
            c.run(T, B, 4)
            st = c.stats()
            spins = [c.spins(i) for i in range(R)]
        return spins, st
    finally:
        vb._lib = saved


CASES = [
    ("r32", dict(replicas=32, variant=0)),
    ("r32_policy", dict(replicas=32, variant=0)),
    ("staged_r4", dict(replicas=4, variant=0, pipeline_depth=3)),
    ("wave", dict(replicas=32, variant=4, max_blocks=2)),
    ("wave_full", dict(replicas=32, variant=4)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_debug_build_checks_pass_and_spins_match(debug_lib, name, kw):
    s = sc_periodic((10, 6, 14), bimodal_seed=3, k_uni=0.2)  # 420 sites per class: 52.5 blocks
    if name == "r32_policy":
        s.type = (np.arange(s.n_sites) % 2).astype(np.int32)
        s.with_policy([vg.POLICY_RANDOM, vg.POLICY_SMALL_STEP], [0.0, 0.5])
    ref, st_ref = run(s, None, **dict(kw))
    got, st = run(s, debug_lib, **dict(kw))
    assert st["device_error"] == 0, hex(st["device_error"])
    assert st_ref["device_error"] == 0
    assert st["variant"] == kw["variant"]
    for i, (a, b) in enumerate(zip(ref, got)):
        assert np.array_equal(a, b), (name, i)


def _noalloc_call(torch, lay, s, R, T, B, library):
    saved = vb._lib
    try:
        vb._lib = vb.load_library(library) if library else saved
        out = torch.zeros((R, 4), dtype=torch.float64, device="cuda")
        vg.vegas_sweep_noalloc(lay["spins"].data_ptr(), lay["links"].data_ptr(), lay["row_ptr"].data_ptr(),
                               lay["site_id"].data_ptr(), s.n_sites, lay["colour_start"], R, 1.0 / T, B, seed=7,
                               inst0=0, t=0, out_ptr=out.data_ptr(), stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return out.cpu().numpy(), lay["spins"].cpu().numpy()
    finally:
        vb._lib = saved


def test_debug_build_checks_the_allocation_free_sweep(debug_lib):
    """The allocation-free entry point cannot validate device arrays on the host; its debug
    build checks every row and neighbour index in the kernel. Valid data: no flag, and the
    same sums and spins as the normal build. A neighbour index past the sites: the kernel
    skips that attempt and the call reports VEGAS_EDEVICE with the index flag (the bad index
    is never used to address memory)."""
    import torch
    from conftest import noalloc_device_layout

    s = sc_periodic((6, 4, 5), bimodal_seed=2)
    R = 4
    T = np.array([0.4, 0.9, 1.5, 2.2])
    B = np.array([0.0, 0.1, 0.2, 0.3])
    up = [np.tile([0.0, 0.0, 1.0], (s.n_sites, 1))] * R
    ref = _noalloc_call(torch, noalloc_device_layout(torch, s, up), s, R, T, B, None)
    got = _noalloc_call(torch, noalloc_device_layout(torch, s, up), s, R, T, B, debug_lib)
    assert np.array_equal(ref[1], got[1])
    assert np.allclose(ref[0], got[0], rtol=0, atol=1e-9 * s.n_sites)
    lay = noalloc_device_layout(torch, s, up)
    bad = lay["links_host"].copy()
    bad[5, 0] = s.n_sites + 3  # one link points past the last site
    lay["links"] = torch.from_numpy(bad).to("cuda")
    with pytest.raises(vb.VegasError) as e:
        _noalloc_call(torch, lay, s, R, T, B, debug_lib)
    assert e.value.status == vb.EDEVICE and "4" in str(e.value)
