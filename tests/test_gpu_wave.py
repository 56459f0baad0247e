"""Wavefront sweep (variant 4) against the per-class sweep (Sec. II, Eq. 4).

One launch per MCS runs both colour classes; a block of class-1 sites starts only after the
class-0 blocks it links to have finished. Every attempt then sees the neighbour values of
the per-class sweep and draws the same Philox counters, so the spins and the accept/reject
decisions must agree bit for bit; the history sums agree up to the order of the FP32 block
sums. The cases cover the three parameter modes, class sizes that are not multiples of the
8-site block, slab orders with periodic boundaries across slabs, grids from one block (many tasks per warp, long dependency waits) to the whole
device (about one task per warp), a tight and a default queueing lag, samples with and
without positions, and the bounded wait that reports a lost dependency instead of hanging.
"""

import numpy as np
import pytest

import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import sc_periodic

pytestmark = pytest.mark.gpu
R = 32


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ctx(samples, **kw):
    kw.setdefault("stream", None)
    kw.setdefault("replicas", R)
    return vg.Context(samples, **kw)


def schedule(n_steps):
    T = np.stack([0.3 * 8.0 ** (np.arange(R) / (R - 1.0)) * (1.0 - 0.1 * k) for k in range(n_steps)], axis=1)
    B = np.tile(np.linspace(0.2, -0.1, n_steps), (R, 1))
    return T, B


def random_axes(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def lattice(shape, mode, positions=True):
    s = sc_periodic(shape, bimodal_seed=5, k_uni=0.4 if mode == 1 else 0.0)
    if mode == 2:  # per-site field axes and anisotropy
        s.field_axis = random_axes(s.n_sites, 1)
        s.k_uni = np.random.default_rng(2).uniform(-0.5, 0.5, s.n_sites)
        s.e_uni = random_axes(s.n_sites, 3)
    if not positions:
        s.positions = None
    return s


def assert_same_chain(a, b, n_sites):
    for i in range(R):
        assert np.array_equal(a.spins(i), b.spins(i)), i
    assert np.array_equal(a.accept_history(), b.accept_history())
    Ha, Hb = a.history(), b.history()
    assert Ha.shape == Hb.shape
    assert np.all(np.abs(Ha - Hb) <= 2e-6 * n_sites), np.max(np.abs(Ha - Hb))


@pytest.mark.parametrize("shape,mode,max_blocks,lag", [
    ((16, 16, 16), 0, 0, 0),     # whole device: about one task per warp
    ((10, 6, 14), 1, 1, 0),      # 420 sites per class (52.5 blocks); one block of 8 warps
    ((10, 6, 14), 2, 3, 1),      # per-site parameters; lag 1: waits on almost every block
    ((24, 20, 16), 0, 2, 0),     # 3840 sites per class over 16 warps
    ((24, 20, 16), 2, 0, 5),
])
def test_wave_matches_per_class_sweep(shape, mode, max_blocks, lag):
    s = lattice(shape, mode)
    T, B = schedule(2)
    with ctx([s], seed=41, variant=0) as a, \
            ctx([s], seed=41, variant=4, max_blocks=max_blocks, wave_lag=lag) as b:
        a.run(T, B, 7)
        b.run(T, B, 7)
        assert b.stats()["variant"] == 4
        assert_same_chain(a, b, s.n_sites)


@pytest.mark.parametrize("shape,slab", [((24, 20, 16), 6), ((16, 12, 10), 4), ((16, 16, 16), -1)])
def test_wave_slab_orders_match_per_class_sweep(shape, slab):
    """Sites stored slab by slab along x (wave_slab in position units; -1 whole planes): the
    boundary columns of a slab, whose class-1 sites wait for the next slab's class-0 blocks,
    and the periodic wrap in every direction keep the per-class sweep's chain."""
    s = lattice(shape, 0)
    T, B = schedule(2)
    with ctx([s], seed=47, variant=0) as a, ctx([s], seed=47, variant=4, wave_slab=slab) as b:
        a.run(T, B, 5)
        b.run(T, B, 5)
        assert_same_chain(a, b, s.n_sites)


def test_wave_without_positions_and_with_timing():
    """Caller order (no positions) and the timed launch path give the same chain."""
    s = lattice((12, 12, 8), 1, positions=False)
    T, B = schedule(3)
    with ctx([s], seed=42, variant=0) as a, ctx([s], seed=42, variant=4, timing=True, max_blocks=2) as b:
        a.run(T, B, 5)
        b.run(T, B, 5)
        st = b.stats()
        assert st["sweep_launches"] == 15 and st["sweep_ms"] > 0.0
        assert_same_chain(a, b, s.n_sites)


def test_wave_continues_across_runs_and_set_spins():
    s = lattice((8, 8, 12), 0)
    T, B = schedule(2)
    with ctx([s], seed=43, variant=0) as a, ctx([s], seed=43, variant=4) as b:
        a.run(T, B, 4)
        b.run(T[:, :1], B[:, :1], 4)
        b.run(T[:, 1:], B[:, 1:], 4)
        assert_same_chain(a, b, s.n_sites)
        x = random_axes(s.n_sites, 9)
        a.set_spins(3, x)
        b.set_spins(3, x)
        a.run(T, B, 3)
        b.run(T, B, 3)
        assert_same_chain(a, b, s.n_sites)


def test_wave_run_is_one_graph_launch():
    s = lattice((8, 8, 12), 1)
    T, B = schedule(3)
    with ctx([s], seed=46, variant=4) as a, ctx([s], seed=46, variant=4, graphs=False) as b:
        a.run(T, B, 4)
        b.run(T, B, 4)
        assert a.stats()["graph_launches"] == 1 and b.stats()["graph_launches"] == 0
        assert_same_chain(a, b, s.n_sites)


def test_wave_accept_log_matches():
    s = lattice((8, 6, 10), 1)
    T, B = schedule(1)
    with ctx([s], seed=44, variant=0, accept_log_mcs=3) as a, ctx([s], seed=44, variant=4, accept_log_mcs=3) as b:
        a.run(T, B, 5)
        b.run(T, B, 5)
        assert np.array_equal(a.accept_log(), b.accept_log())


def test_wave_dependency_timeout_is_reported_not_hung():
    """The first class-0 block is never reported finished (host-requested fault injection):
    the class-1 blocks that link to it give up after timeout_ns, the run fails with ETIMEOUT
    and the context refuses further work. No trap, no hang."""
    s = lattice((8, 8, 8), 0)
    T, B = schedule(1)
    with ctx([s], seed=45, variant=4, max_blocks=1, timeout_ns=50_000_000, fault_inject=1) as c:
        with pytest.raises(vb.VegasError) as e:
            c.run(T, B, 3)
        assert e.value.status == vb.ETIMEOUT
        assert c.stats()["device_error"] & 8
        with pytest.raises(vb.VegasError) as e2:
            c.run(T, B, 1)
        assert e2.value.status == vb.ESTATE
    with ctx([s], seed=45, variant=4) as c:  # the device is fine afterwards
        c.run(T, B, 2)
