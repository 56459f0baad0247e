"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

FP64: spins, accept/reject decisions and history must match the oracle bit for bit
(history energy and magnetization to 1e-12 relative: the GPU sums per colour class in a
different order). FP32: bitwise independence of batching and of run splitting, the
history's E/N against the oracle's energy of the same spins (|d(E/N)| < 1e-3), the
observables <E>/N, <|M|>/N, C_v, chi against the FP64 oracle within 3 binned standard errors
(independent seeds; |d(E/N)| between the chains is printed per result), and closed forms
within 4 standard errors.
"""

import numpy as np
import pytest

from conftest import assert_statistically_equal, binned, chain_observables

import oracle
import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import (chain_open, core_shell_particle, dimers, fcc_sphere, free_spins, nanoparticle_batch,
                      random_graph, sc_periodic, triangles)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ctx(samples, **kw):
    kw.setdefault("stream", None)
    return vg.Context(samples, **kw)


def first_divergence(a, b):
    d = np.argwhere(a != b)
    return None if d.size == 0 else tuple(int(x) for x in d[0])


def assert_fp32_history_close(h, hr, n_sites):
    """FP32 history sums depend on which sites a thread sums in FP32 before its FP64
    accumulation (the grid shape), so they agree to ~1e-8 per site, not bit for bit."""
    assert np.all(np.abs(h - hr) <= 1e-6 * n_sites), np.max(np.abs(h - hr)) / n_sites


def assert_history_close(h, hr, n_sites, rel=1e-12):
    scale = np.maximum(np.abs(hr[..., 0]), 1.0)
    assert np.all(np.abs(h[..., 0] - hr[..., 0]) <= rel * scale), np.max(np.abs(h[..., 0] - hr[..., 0]) / scale)
    assert np.all(np.abs(h[..., 1:] - hr[..., 1:]) <= rel * n_sites)


# --------------------------------------------------------------------------- FP64 bit identity

def test_fp64_sc8_first_100_mcs_bitwise():
    s = sc_periodic(8)
    with ctx([s], precision=64, seed=1, accept_log_mcs=100) as c:
        c.run([[3.0]], [[0.0]], 100)
        ref = oracle.run(s, [[3.0]], [[0.0]], 100, seed=1, log_mcs=100)
        alog = c.accept_log().reshape(100, 512)
        assert first_divergence(alog, ref["accept_log"][0]) is None, first_divergence(alog, ref["accept_log"][0])
        assert np.array_equal(c.spins(0), ref["spins"][0])
        assert_history_close(c.history()[0], ref["history"][0], 512)
        assert 0.3 < alog.mean() < 0.9


def test_fp64_sc8_full_schedule_bitwise():
    """The 8^3 ferromagnet, 30 temperatures 3.0 -> 0.1, 1000 MCS each."""
    s = sc_periodic(8)
    T = np.linspace(3.0, 0.1, 30)[None, :]
    with ctx([s], precision=64, seed=1) as c:
        c.run(T, np.zeros_like(T), 1000)
        ref = oracle.run(s, T, np.zeros_like(T), 1000, seed=1)
        S = c.spins(0)
        d = first_divergence(S, ref["spins"][0])
        assert d is None, f"first spin divergence at {d}"
        h = c.history()[0]
        assert_history_close(h, ref["history"][0], 512)
        assert abs(h[-1, 0] - ref["history"][0, -1, 0]) <= 1e-12 * abs(ref["history"][0, -1, 0])


def _packed_samples():
    cs = core_shell_particle(seed=3, radius=5.0, core_radius=3.5)
    rg = random_graph(60, 0.1, 4)
    iso = free_spins(5, k_cub=0.7, spin_norm=1.3)
    return [sc_periodic((10, 9, 11)), fcc_sphere(4.3), cs, rg, chain_open(37), iso, free_spins(1)]


def test_fp64_packed_ragged_replicas_bitwise():
    samples = _packed_samples()
    R, base, mcs = 4, 5, 12
    Tl = np.array([2.0, 1.0, 0.4])
    Bl = np.array([0.3, -0.5, 1.0])
    n_inst = len(samples) * R
    T = np.stack([Tl * (1 + 0.1 * i) for i in range(n_inst)])
    B = np.stack([Bl * (1 - 0.05 * i) for i in range(n_inst)])
    with ctx(samples, precision=64, replicas=R, inst_base=base, seed=77) as c:
        c.run(T, B, mcs)
        H = c.history()
        for si, s in enumerate(samples):
            rows = slice(si * R, (si + 1) * R)
            ref = oracle.run(s, T[rows], B[rows], mcs, seed=77, inst_base=base + si * R)
            assert ref["err"] == 0
            for r in range(R):
                S = c.spins(si * R + r)
                assert first_divergence(S, ref["spins"][r]) is None, (s.name, r, first_divergence(S, ref["spins"][r]))
                assert_history_close(H[si * R + r], ref["history"][r], s.n_sites)


def test_fp64_given_initial_state_and_set_spins():
    s = random_graph(40, 0.15, 8)
    rng = np.random.Generator(np.random.PCG64(2))
    S0 = rng.normal(size=(40, 3))
    s.init_spins = S0
    with ctx([s], precision=64, seed=9) as c:
        assert np.array_equal(c.spins(0), S0)
        c.run([[1.1]], [[0.2]], 7)
        ref = oracle.run(s, [[1.1]], [[0.2]], 7, seed=9, spins=S0[None])
        assert np.array_equal(c.spins(0), ref["spins"][0])
        c.set_spins(0, S0)
        assert np.array_equal(c.spins(0), S0)


# --------------------------------------------------------------------------- chain continuation

@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("variant", [0, 2])
def test_run_splitting_is_bitwise_invisible(precision, variant):
    """A schedule run at once or in pieces: the same spins and histories bit for bit, for a
    given sweep (the history's sums keep one order per sweep, so the sweep is fixed here: with
    the automatic choice two contexts may keep different sweeps, whose spins agree bit for bit
    and histories to rounding)."""
    s = fcc_sphere(3.9)
    T = np.array([[2.5, 1.5, 0.7, 0.3]])
    B = np.array([[0.1, 0.4, -0.2, 0.0]])
    with ctx([s], precision=precision, seed=5, variant=variant) as a, \
            ctx([s], precision=precision, seed=5, variant=variant) as b:
        a.run(T, B, 9)
        b.run(T[:, :1], B[:, :1], 9)
        b.run(T[:, 1:3], B[:, 1:3], 9)
        b.run(T[:, 3:], B[:, 3:], 9)
        assert np.array_equal(a.spins(0), b.spins(0))
        assert np.array_equal(a.history(), b.history())


def test_graph_and_direct_launches_agree():
    s = sc_periodic(6, k_uni=0.1)
    with ctx([s], seed=3, graphs=True) as a, ctx([s], seed=3, graphs=False) as b, ctx([s], seed=3, timing=True) as t:
        for c in (a, b, t):
            c.run([[1.0, 0.5]], [[0.2, 0.3]], 11)
        assert np.array_equal(a.spins(0), b.spins(0)) and np.array_equal(a.spins(0), t.spins(0))
        assert np.array_equal(a.history(), b.history())
        assert t.stats()["sweep_ms"] > 0.0


# --------------------------------------------------------------------------- grid independence
# A small max_blocks makes every warp walk many groups (the steady state of the staged
# pipeline and of the grid-stride loops); results must not depend on the grid.

@pytest.mark.parametrize("R,max_blocks", [(32, 2), (1, 1), (4, 1)])
def test_fp32_staged_many_groups_per_warp(R, max_blocks):
    s = sc_periodic(24, bimodal_seed=7)
    T = np.linspace(0.2, 2.0, R)[:, None]
    with ctx([s], precision=32, replicas=R, seed=3, max_blocks=max_blocks) as a, \
            ctx([s], precision=32, replicas=R, seed=3) as b:
        a.run(T, np.zeros_like(T), 10)
        b.run(T, np.zeros_like(T), 10)
        Ha, Hb = a.history(), b.history()
        assert_fp32_history_close(Ha, Hb, s.n_sites)
        for i in sorted({0, R - 1}):
            S = a.spins(i)
            assert np.array_equal(S, b.spins(i))
            assert abs(Ha[i, -1, 0] - oracle.energy(s, S, 0.0)) < 1e-5 * s.n_sites


@pytest.mark.parametrize("precision,R", [(32, 32), (32, 1), (64, 2)])
def test_memory_order_from_positions_does_not_change_spins(precision, R):
    import copy

    s = sc_periodic(10, bimodal_seed=2)
    u = copy.copy(s)
    u.positions = None
    assert s.positions is not None
    T = np.linspace(0.3, 2.0, R)[:, None]
    with ctx([s], precision=precision, replicas=R, seed=9) as a, ctx([u], precision=precision, replicas=R, seed=9) as b:
        a.run(T, np.full_like(T, 0.1), 6)
        b.run(T, np.full_like(T, 0.1), 6)
        for i in sorted({0, R - 1}):
            assert np.array_equal(a.spins(i), b.spins(i))
        assert_fp32_history_close(a.history(), b.history(), s.n_sites)


def test_fp32_direct_kernel_many_items_per_thread():
    s = fcc_sphere(7.0)
    T = np.array([[0.5], [1.0], [1.5], [3.0]])
    with ctx([s], precision=32, replicas=4, seed=4, max_blocks=1) as a, ctx([s], precision=32, replicas=4, seed=4) as b:
        a.run(T, np.full_like(T, 0.2), 8)
        b.run(T, np.full_like(T, 0.2), 8)
        for i in range(4):
            assert np.array_equal(a.spins(i), b.spins(i))
        assert_fp32_history_close(a.history(), b.history(), s.n_sites)


def test_fp64_many_items_per_thread_bitwise():
    s = sc_periodic((10, 9, 11), k_uni=0.1)
    with ctx([s], precision=64, replicas=2, seed=6, max_blocks=1) as c:
        T, B = np.array([[1.2], [0.6]]), np.array([[0.3], [-0.2]])
        c.run(T, B, 6)
        ref = oracle.run(s, T, B, 6, seed=6)
        for i in range(2):
            assert np.array_equal(c.spins(i), ref["spins"][i])


# --------------------------------------------------------------------------- resident sweep
# One persistent launch per temperature/field step: each block takes whole instances
# (largest first) and runs every MCS on them. Same per-site arithmetic and random numbers
# as the per-class sweep, so the spins must agree bit for bit.

def _uneven_batch():
    return nanoparticle_batch(7, seed=11, r_max=7.0) + [core_shell_particle(seed=2, radius=5.0, core_radius=3.5)]


@pytest.mark.parametrize("R", [1, 4])
def test_resident_sweep_equals_per_class_sweep(R):
    samples = _uneven_batch()
    n = len(samples) * R
    T = np.stack([np.linspace(0.3, 2.5, 3) * (1 + 0.05 * i) for i in range(n)])
    B = np.stack([np.array([0.4, -0.2, 0.1]) * (1 + 0.1 * i) for i in range(n)])
    with ctx(samples, replicas=R, seed=13, variant=0, accept_log_mcs=3) as a, \
            ctx(samples, replicas=R, seed=13, variant=1, accept_log_mcs=3) as b:
        a.run(T, B, 7)
        b.run(T, B, 7)
        assert a.stats()["variant"] == 0 and b.stats()["variant"] == 1
        for i in range(n):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        for i in range(n):
            assert_fp32_history_close(a.history()[i], b.history()[i], samples[i // R].n_sites)
        assert np.array_equal(a.accept_log(), b.accept_log())


@pytest.mark.parametrize("R,aniso", [(1, True), (4, True), (2, False)])
def test_resident_sweep_with_spins_in_shared_memory(R, aniso):
    """The resident sweep with each instance's spins in shared memory for the whole step equals
    the per-class sweep bit for bit (spins, accept log) across runs and steps; with and without
    an instance with anisotropy (without, the kernel leaves the anisotropy terms out)."""
    samples = _uneven_batch() if aniso else nanoparticle_batch(8, seed=12, r_max=7.0)
    n = len(samples) * R
    T = np.stack([np.linspace(0.3, 2.5, 3) * (1 + 0.05 * i) for i in range(n)])
    B = np.stack([np.array([0.4, -0.2, 0.1]) * (1 + 0.1 * i) for i in range(n)])
    with ctx(samples, replicas=R, seed=13, variant=0, accept_log_mcs=3) as a, \
            ctx(samples, replicas=R, seed=13, variant=1, resident_smem=1, accept_log_mcs=3) as b:
        a.run(T, B, 7)
        b.run(T[:, :1], B[:, :1], 7)
        b.run(T[:, 1:], B[:, 1:], 7)
        st = b.stats()
        assert vb.sweep_kernel_names(st["sweep_kernels"]) == ["resident32_smem"] and st["block_threads"] == 512
        for i in range(n):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        for i in range(n):
            assert_fp32_history_close(a.history()[i], b.history()[i], samples[i // R].n_sites)
        assert np.array_equal(a.accept_log(), b.accept_log())


def test_resident_shared_memory_groups_policies_and_types():
    """Small instances several to a block, each group with its own region of shared memory,
    with update policies (adaptive width included) and per-type statistics."""
    ps = nanoparticle_batch(9, seed=14, r_max=8.0)
    for p in ps:
        p.type = (np.arange(p.n_sites) % 2).astype(np.int32)
        p.with_policy([oracle.ADAPTIVE, oracle.HINZKE_NOWAK], [0.8, 0.4])
    T = np.linspace(0.4, 2.0, 2 * len(ps))[:, None] * np.array([[1.0, 0.8]])
    B = np.full_like(T, 0.1)
    with ctx(ps, replicas=2, seed=30, variant=1, resident_smem=1, group_threads=128, group_sites=600,
             type_stats=True) as a, ctx(ps, replicas=2, seed=30, variant=0, type_stats=True) as b:
        a.run(T, B, 6)
        b.run(T, B, 6)
        st = a.stats()
        assert vb.sweep_kernel_names(st["sweep_kernels"]) == ["resident32_smem"]
        assert st["group_threads"] == 128 and 0 < st["group_sites"] <= 600
        for i in range(2 * len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        n = max(p.n_sites for p in ps)
        assert np.all(np.abs(a.history() - b.history()) <= 1e-6 * n)
        assert np.all(np.abs(a.type_history() - b.type_history()) <= 1e-6 * n)
        assert np.array_equal(a.accept_history(), b.accept_history())
        assert np.array_equal(a.adaptive_width(), b.adaptive_width())


def test_resident_shared_memory_refuses_instances_that_do_not_fit():
    with pytest.raises(vb.VegasError) as e:
        ctx([sc_periodic(30)], variant=1, resident_smem=1)  # 27,000 sites x 12 bytes
    assert e.value.status == vb.EINVAL and "shared memory" in str(e.value)


def test_resident_split_runs_and_autotune():
    samples = _uneven_batch()
    T = np.linspace(0.5, 2.0, len(samples))[:, None] * np.ones((1, 2))
    with ctx(samples, seed=17, variant=1) as a, ctx(samples, seed=17, variant=-1) as b, \
            ctx(samples, seed=17, variant=1) as c:
        a.run(T, np.zeros_like(T), 12)
        b.run(T, np.zeros_like(T), 12)  # first run times both sweeps, then keeps the faster
        c.run(T[:, :1], np.zeros((len(samples), 1)), 12)
        c.run(T[:, 1:], np.zeros((len(samples), 1)), 12)
        assert b.stats()["variant"] in (0, 1)
        for i in range(len(samples)):
            assert np.array_equal(a.spins(i), b.spins(i))
            assert np.array_equal(a.spins(i), c.spins(i))
        assert np.array_equal(a.history(), c.history())


# --------------------------------------------------------------------------- cooperative sweep
# One launch per step for one sample: all blocks sweep every class together and meet at a
# bounded grid barrier. Same arithmetic and random numbers: spins equal the per-class sweep.

@pytest.mark.parametrize("make,R", [(lambda: sc_periodic(16, k_uni=0.05), 1), (lambda: sc_periodic(12, bimodal_seed=2), 4),
                                    (lambda: core_shell_particle(seed=3, radius=5.0, core_radius=3.5), 2),
                                    (lambda: fcc_sphere(4.5).with_policy([oracle.GAUSSIAN], [0.4]), 2)])
def test_cooperative_sweep_equals_per_class_sweep(make, R):
    """Rows of six links take the uniform-degree form, rows of at most twelve the padded
    fixed rows (with and without a policy table): the per-class sweep's spins bit for bit."""
    s = make()
    T = np.stack([np.array([2.0, 0.9, 0.5]) * (1 + 0.1 * i) for i in range(R)])
    B = np.stack([np.array([0.5, -0.5, 1.0]) for _ in range(R)])
    with ctx([s], replicas=R, seed=21, variant=0, accept_log_mcs=2) as a, \
            ctx([s], replicas=R, seed=21, variant=2, accept_log_mcs=2) as b:
        a.run(T, B, 9)
        b.run(T, B, 9)
        assert b.stats()["variant"] == 2
        for i in range(R):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        assert_fp32_history_close(a.history(), b.history(), s.n_sites)
        assert np.array_equal(a.accept_log(), b.accept_log())
        assert np.array_equal(a.accept_history(), b.accept_history())  # recorded one MCS late, in order


@pytest.mark.parametrize("case", ["sc8", "core_shell_policies"])
def test_fp64_cooperative_sweep_bitwise(case):
    """The FP64 cooperative sweep (one launch per step, all blocks on every colour class with
    grid barriers between them) against the oracle: spins, accept log and accepted counts bit
    for bit, history within 1e-12; on the 8^3 ferromagnet and on a core/shell particle of
    uneven rows with a table of (non-adaptive) update policies, two replicas."""
    if case == "sc8":
        s, R = sc_periodic(8), 1
    else:
        s = core_shell_particle(seed=2, radius=4.0, core_radius=2.5).with_policy(
            [oracle.HINZKE_NOWAK, oracle.GAUSSIAN], [0.5, 0.3])
        R = 2
    T = np.stack([[3.0 - 0.5 * r, 1.0, 0.3] for r in range(R)])
    B = np.stack([[0.0, 0.2 * r, -0.1] for r in range(R)])
    mcs = 8
    with ctx([s], precision=64, replicas=R, seed=21, variant=2, accept_log_mcs=3 * mcs) as c:
        c.run(T, B, mcs)
        assert vb.sweep_kernel_names(c.stats()["sweep_kernels"]) == ["coop64"]
        ref = oracle.run(s, T, B, mcs, seed=21, log_mcs=3 * mcs, n_threads=R)
        assert ref["err"] == 0
        alog = c.accept_log().reshape(3 * mcs, R, -1)
        for r in range(R):
            assert first_divergence(c.spins(r), ref["spins"][r]) is None, r
            assert np.array_equal(alog[:, r], ref["accept_log"][r]), r
            assert np.array_equal(c.accept_history()[r], ref["accepted"][r]), r
            assert_history_close(c.history()[r], ref["history"][r], s.n_sites)


@pytest.mark.parametrize("precision", [32, 64])
def test_cooperative_barrier_timeout_is_reported_not_hung(precision):
    """One block leaves before its first grid barrier (host-requested fault injection): the
    other blocks give up after timeout_ns, the run fails with ETIMEOUT, and the context
    refuses further work. No trap, no hang."""
    s = sc_periodic(12)
    with ctx([s], precision=precision, seed=1, variant=2, timeout_ns=50_000_000, fault_inject=1) as c:
        with pytest.raises(vb.VegasError) as e:
            c.run([[1.0]], [[0.0]], 3)
        assert e.value.status == vb.ETIMEOUT
        assert c.stats()["device_error"] & 8
        with pytest.raises(vb.VegasError) as e2:
            c.run([[1.0]], [[0.0]], 1)
        assert e2.value.status == vb.ESTATE


@pytest.mark.parametrize("precision", [64, 32])
def test_whole_run_is_one_graph_launch(precision):
    """With graphs on, a run of the per-class sweep is one launch of a graph whose conditional
    while node repeats one temperature/field step; spins, history and snapshots equal the
    launch-by-launch path, and later runs with other step counts reuse the graph."""
    s = sc_periodic(6, k_uni=0.1)
    T = np.array([[2.0, 1.5, 1.0, 0.7, 0.5]])
    B = np.array([[0.2, 0.1, 0.0, -0.1, -0.2]])
    with ctx([s], precision=precision, seed=27, variant=0, snapshots=True) as a, \
            ctx([s], precision=precision, seed=27, variant=0, snapshots=True, graphs=False) as b, \
            ctx([s], precision=precision, seed=27, variant=0, snapshots=True, graphs=2) as c:
        g0 = a.stats()["graph_launches"]
        a.run(T, B, 7)
        assert a.stats()["graph_launches"] == g0 + 1
        a.run(T[:, :2], B[:, :2], 7)
        assert a.stats()["graph_launches"] == g0 + 2
        b.run(T, B, 7)
        b.run(T[:, :2], B[:, :2], 7)
        assert b.stats()["graph_launches"] == 0
        c.run(T, B, 7)
        c.run(T[:, :2], B[:, :2], 7)
        assert c.stats()["graph_launches"] == 7  # one per step
        assert np.array_equal(c.spins(0), b.spins(0)) and np.array_equal(c.history(), b.history())
        assert np.array_equal(a.spins(0), b.spins(0))
        assert np.array_equal(a.history(), b.history())
        assert np.array_equal(a.accept_history(), b.accept_history())
        for k in range(7):
            assert np.array_equal(a.snapshot(0, k), b.snapshot(0, k)), k


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_persistent_run_is_one_graph_launch(variant):
    """The run graph of the resident, cooperative and cluster sweeps: one launch per run (a
    persistent launch per step inside the conditional loop), the same chain as without
    graphs."""
    ps = nanoparticle_batch(6, seed=14, r_max=5.5) if variant != 2 else [sc_periodic(10, k_uni=0.1)]
    T = np.linspace(0.4, 2.0, len(ps))[:, None] * np.array([[1.0, 0.8, 0.6, 0.5]])
    B = np.full_like(T, 0.1)
    with ctx(ps, seed=30, variant=variant, snapshots=True) as a, \
            ctx(ps, seed=30, variant=variant, snapshots=True, graphs=False) as b:
        a.run(T, B, 6)
        b.run(T, B, 6)
        assert a.stats()["graph_launches"] == 1 and b.stats()["graph_launches"] == 0
        assert a.stats()["variant"] == variant
        for i in range(len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
            for k in range(4):
                assert np.array_equal(a.snapshot(i, k), b.snapshot(i, k)), (i, k)
        assert np.array_equal(a.history(), b.history())


@pytest.mark.parametrize("timing", [False, True])
def test_per_class_sweep_merges_the_samples_passes(timing):
    """The per-class sweep sends the direct passes of one colour class of every sample of a
    batch out as one launch (each block runs the block it runs in its pass's own launch): far
    fewer launches than passes, and the spins of the resident sweep bit for bit, with one
    graph per run and with direct launches timed by events."""
    ps = nanoparticle_batch(10, seed=15, r_max=6.0)
    T = np.linspace(0.4, 2.0, len(ps))[:, None] * np.array([[1.0, 0.8]])
    B = np.full_like(T, 0.2)
    mcs = 6
    with ctx(ps, seed=31, variant=0, timing=timing, accept_log_mcs=2) as a, \
            ctx(ps, seed=31, variant=1, accept_log_mcs=2) as b:
        a.run(T, B, mcs)
        b.run(T, B, mcs)
        st = a.stats()
        assert st["variant"] == 0
        # two steps of four colour classes, at most three kernels (lower-link modes) per class
        assert st["sweep_launches"] <= 2 * mcs * 4 * 3 < 2 * mcs * 4 * len(ps)
        for i in range(len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        assert np.array_equal(a.accept_log(), b.accept_log())
        assert_fp32_history_close(a.history(), b.history(), max(p.n_sites for p in ps))


def test_autotuner_picks_a_sweep_and_block_shape():
    """The first run times every eligible sweep and block shape (threads per block of the
    resident sweep, blocks per cluster of the cluster sweep) on the real chain; whatever it
    keeps, the chain is the per-class sweep's bit for bit, and the stats name the shape."""
    ps = nanoparticle_batch(12, seed=9, r_max=6.5)
    T = np.linspace(0.4, 2.0, len(ps))[:, None]
    B = np.full_like(T, 0.1)
    with ctx(ps, seed=24, variant=-1) as a, ctx(ps, seed=24, variant=0) as b:
        a.run(T, B, 40)
        b.run(T, B, 40)
        st = a.stats()
        assert st["variant"] in (0, 1, 2, 3)
        if st["variant"] == 1:
            assert st["block_threads"] in (256, 512) and st["cluster_blocks"] == 0
        elif st["variant"] == 3:
            assert st["cluster_blocks"] >= 2 and st["block_threads"] in (256, 512)
        else:
            assert st["block_threads"] == 256 and st["cluster_blocks"] == 0
        for i in range(len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        a.run(T, B, 10)  # the chosen shape keeps serving later runs (step graphs included)
        b.run(T, B, 10)
        assert a.stats()["variant"] == st["variant"] and a.stats()["block_threads"] == st["block_threads"]
        for i in range(len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i


def test_autotuner_three_way():
    s = sc_periodic(10, k_uni=0.1)
    with ctx([s], seed=23, variant=-1) as a, ctx([s], seed=23, variant=0) as b:
        a.run([[1.0, 0.7]], [[0.2, 0.1]], 24)
        b.run([[1.0, 0.7]], [[0.2, 0.1]], 24)
        assert a.stats()["variant"] in (0, 1, 2, 3)
        assert np.array_equal(a.spins(0), b.spins(0))


# --------------------------------------------------------------------------- cluster sweep
# A thread-block cluster per instance, the hardware cluster barrier between colour classes.

@pytest.mark.parametrize("make,R", [(lambda: core_shell_particle(seed=3, radius=7.0, core_radius=5.0), 1),
                                    (lambda: sc_periodic(24, bimodal_seed=2, k_uni=0.1), 4),
                                    (lambda: fcc_sphere(5.5), 2)])
def test_cluster_sweep_equals_per_class_sweep(make, R):
    s = make()
    T = np.stack([np.array([2.0, 0.9, 0.5]) * (1 + 0.1 * i) for i in range(R)])
    B = np.stack([np.array([0.5, -0.5, 1.0]) for _ in range(R)])
    with ctx([s], replicas=R, seed=24, variant=0, accept_log_mcs=2) as a, \
            ctx([s], replicas=R, seed=24, variant=3, accept_log_mcs=2) as b:
        a.run(T, B, 9)
        b.run(T, B, 9)
        assert b.stats()["variant"] == 3
        for i in range(R):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        assert_fp32_history_close(a.history(), b.history(), s.n_sites)
        assert np.array_equal(a.accept_log(), b.accept_log())
        assert np.array_equal(a.accept_history(), b.accept_history())


@pytest.mark.parametrize("split", [0, 200, 10**6])
def test_cluster_sweep_splits_small_instances_to_single_blocks(split):
    """Instances of at most cluster_split sites are swept by one block each (the blocks of a
    cluster leave the cluster loop at the first one: instances are queued largest first),
    larger ones by the whole cluster; either way the chain is the per-class sweep's."""
    ps = nanoparticle_batch(9, seed=12, r_max=6.5)
    T = np.linspace(0.4, 2.0, len(ps))[:, None] * np.array([[1.0, 0.7]])
    B = np.full_like(T, 0.2)
    with ctx(ps, seed=28, variant=3, cluster_split=split) as a, ctx(ps, seed=28, variant=0) as b:
        a.run(T, B, 6)
        b.run(T, B, 6)
        assert a.stats()["variant"] == 3 and a.stats()["split_sites"] == split
        for i in range(len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        Ha, Hb = a.history(), b.history()
        assert np.all(np.abs(Ha - Hb) <= 1e-6 * max(p.n_sites for p in ps))
        assert np.array_equal(a.accept_history(), b.accept_history())


@pytest.mark.parametrize("variant,group,kw", [
    (1, 128, {}), (1, 64, {}), (1, 256, {}),
    (3, 128, dict(cluster_blocks=2, cluster_threads=512, cluster_split=700)),
])
def test_small_instances_several_to_a_block(variant, group, kw):
    """Instances of at most group_sites sites are swept several to a block, group_threads
    threads each meeting at their own named barrier (the resident sweep, and the single-block
    phase of the cluster sweep); the chain stays the per-class sweep's, with the acceptance
    counts and (with per-type statistics) the magnetization of every type."""
    ps = nanoparticle_batch(11, seed=13, r_max=6.0)
    for p in ps:
        p.type = (np.arange(p.n_sites) % 2).astype(np.int32)
    T = np.linspace(0.4, 2.0, len(ps))[:, None] * np.array([[1.0, 0.8]])
    B = np.full_like(T, 0.1)
    with ctx(ps, seed=29, variant=variant, group_threads=group, group_sites=600, type_stats=True, **kw) as a, \
            ctx(ps, seed=29, variant=0, type_stats=True) as b:
        a.run(T, B, 5)
        b.run(T, B, 5)
        st = a.stats()
        grouped = group < (256 if variant == 1 else 512)  # the blocks' threads (256: instances < 4096 sites)
        assert st["variant"] == variant and st["group_threads"] == (group if grouped else 0)
        assert st["group_sites"] == (600 if grouped else 0)
        for i in range(len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        n = max(p.n_sites for p in ps)
        assert np.all(np.abs(a.history() - b.history()) <= 1e-6 * n)
        assert np.all(np.abs(a.type_history() - b.type_history()) <= 1e-6 * n)
        assert np.array_equal(a.accept_history(), b.accept_history())


def test_cluster_sweep_batch_with_policies_and_types():
    ps = nanoparticle_batch(6, seed=6, r_max=9.0)
    for p in ps:
        p.type = (np.arange(p.n_sites) % 2).astype(np.int32)
        p.with_policy([oracle.ADAPTIVE, oracle.HINZKE_NOWAK], [0.8, 0.4])
    T = np.linspace(0.4, 2.0, 12)[:, None]
    B = np.full_like(T, 0.2)
    with ctx(ps, replicas=2, seed=25, variant=0, type_stats=True) as a, \
            ctx(ps, replicas=2, seed=25, variant=3, type_stats=True) as b:
        a.run(T, B, 10)
        b.run(T, B, 10)
        assert np.array_equal(a.accept_history(), b.accept_history())
        assert np.array_equal(a.adaptive_width(), b.adaptive_width())
        for i in range(12):
            assert np.array_equal(a.spins(i), b.spins(i)), i
            n = ps[i // 2].n_sites
            assert np.all(np.abs(a.type_history()[i] - b.type_history()[i]) <= 1e-6 * n)


@pytest.mark.parametrize("cs,threads,split,group", [(2, 512, 0, 0), (4, 512, 700, 0), (2, 256, 700, 128)])
def test_cluster_sweep_with_spin_copies_in_shared_memory(cs, threads, split, group):
    """The cluster sweep with a copy of the instance's spins in every block's shared memory
    (accepted spins written to all copies through distributed shared memory), with and
    without small instances swept alone or in groups, equals the per-class sweep bit for
    bit over two steps and two runs."""
    ps = nanoparticle_batch(7, seed=15, r_max=9.0)
    T = np.linspace(0.4, 2.4, 2 * len(ps))[:, None] * np.array([[1.0, 0.7]])
    B = np.full_like(T, 0.15)
    kw = dict(cluster_blocks=cs, cluster_threads=threads, cluster_split=split, group_threads=group, group_sites=600)
    with ctx(ps, replicas=2, seed=33, variant=3, resident_smem=1, accept_log_mcs=3, **kw) as a, \
            ctx(ps, replicas=2, seed=33, variant=0, accept_log_mcs=3) as b:
        a.run(T[:, :1], B[:, :1], 5)
        a.run(T[:, 1:], B[:, 1:], 5)
        b.run(T, B, 5)
        st = a.stats()
        assert vb.sweep_kernel_names(st["sweep_kernels"]) == ["cluster32_smem"]
        assert st["cluster_blocks"] == cs and st["split_sites"] == split
        for i in range(2 * len(ps)):
            assert np.array_equal(a.spins(i), b.spins(i)), i
        n = max(p.n_sites for p in ps)
        assert np.all(np.abs(a.history() - b.history()) <= 1e-6 * n)
        assert np.array_equal(a.accept_log(), b.accept_log())


def test_cluster_shared_memory_with_policies_and_types():
    ps = nanoparticle_batch(6, seed=16, r_max=9.0)
    for p in ps:
        p.type = (np.arange(p.n_sites) % 2).astype(np.int32)
        p.with_policy([oracle.ADAPTIVE, oracle.HINZKE_NOWAK], [0.8, 0.4])
    T = np.linspace(0.4, 2.0, 12)[:, None]
    B = np.full_like(T, 0.2)
    with ctx(ps, replicas=2, seed=26, variant=0, type_stats=True) as a, \
            ctx(ps, replicas=2, seed=26, variant=3, resident_smem=1, cluster_blocks=2, cluster_threads=512,
                cluster_split=1500, type_stats=True) as b:
        a.run(T, B, 10)
        b.run(T, B, 10)
        assert vb.sweep_kernel_names(b.stats()["sweep_kernels"]) == ["cluster32_smem"]
        assert np.array_equal(a.accept_history(), b.accept_history())
        assert np.array_equal(a.adaptive_width(), b.adaptive_width())
        for i in range(12):
            assert np.array_equal(a.spins(i), b.spins(i)), i
            n = ps[i // 2].n_sites
            assert np.all(np.abs(a.type_history()[i] - b.type_history()[i]) <= 1e-6 * n)


def test_cluster_rejected_for_fp64():
    with pytest.raises(vb.VegasError) as e:
        ctx([sc_periodic(4)], precision=64, variant=3)
    assert e.value.status == vb.EINVAL


def test_resident_rejected_for_fp64():
    with pytest.raises(vb.VegasError) as e:
        ctx([sc_periodic(4)], precision=64, variant=1)
    assert e.value.status == vb.EINVAL


# --------------------------------------------------------------------------- FP32 batching

def test_fp32_replica_batch_equals_plain_runs():
    s = sc_periodic(12, bimodal_seed=3)
    R = 32
    T = (0.1 * 20.0 ** (np.arange(R) / (R - 1.0)))[:, None]
    with ctx([s], precision=32, replicas=R, seed=11) as c:
        c.run(T, np.zeros_like(T), 30)
        H = c.history()
        for p in (0, 7, 31):
            with ctx([s], precision=32, replicas=1, inst_base=p, seed=11) as q:
                q.run(T[p:p + 1], np.zeros((1, 1)), 30)
                assert np.array_equal(c.spins(p), q.spins(0)), p
                assert_fp32_history_close(H[p], q.history()[0], s.n_sites)


def test_fp32_sample_batch_equals_single_sample_runs():
    samples = nanoparticle_batch(6, seed=4, r_max=6.0)
    T = np.linspace(0.3, 2.0, 6)[:, None]
    with ctx(samples, precision=32, seed=2) as c:
        c.run(T, np.full_like(T, 0.1), 25)
        H = c.history()
        for p in (0, 3, 5):
            with ctx([samples[p]], precision=32, inst_base=p, seed=2) as q:
                q.run(T[p:p + 1], np.full((1, 1), 0.1), 25)
                assert np.array_equal(c.spins(p), q.spins(0))
                assert_fp32_history_close(H[p], q.history()[0], samples[p].n_sites)


# --------------------------------------------------------------------------- FP32 precision statement

def _precision_case(samples, T, B, mcs, R=1):
    worst = 0.0
    with ctx(samples, precision=32, replicas=R, seed=21) as c:
        for step in range(T.shape[1]):
            c.run(T[:, step:step + 1], B[:, step:step + 1], mcs)
            H = c.history()
            for i in range(c.n_instances):
                s = samples[i // R]
                S = c.spins(i)
                e_ref = oracle.energy(s, S, B[i, step]) / s.n_sites
                worst = max(worst, abs(H[i, -1, 0] / s.n_sites - e_ref))
                np.testing.assert_allclose(H[i, -1, 1:], S.sum(axis=0), rtol=0, atol=1e-5 * s.n_sites)
                norms = np.linalg.norm(S, axis=1)
                sn = s.param("spin_norm")
                assert np.all(np.abs(norms - sn) < 1e-5 * sn)
    return worst


def test_fp32_history_energy_matches_oracle_energy_of_same_spins():
    cases = [
        ([sc_periodic(16, k_uni=0.05)], np.full((1, 3), 0.5), np.array([[2.0, 0.0, -2.0]]), 20, 1),
        ([core_shell_particle(seed=1, radius=6.0, core_radius=4.5)], np.array([[3.0, 1.0, 0.1]]),
         np.full((1, 3), 0.5), 20, 1),
        (nanoparticle_batch(5, seed=7, r_max=7.0), np.full((5, 2), 0.8), np.zeros((5, 2)), 15, 1),
        ([sc_periodic(10, bimodal_seed=5)], np.tile([[0.2, 1.0]], (8, 1)), np.zeros((8, 2)), 15, 8),
        ([random_graph(300, 0.02, 3)], np.array([[1.5, 0.5]]), np.array([[0.7, -0.4]]), 15, 1),
    ]
    for samples, T, B, mcs, R in cases:
        worst = _precision_case(samples, T, B, mcs, R)
        assert worst < 1e-3, (samples[0].name, worst)
        assert worst < 1e-5, (samples[0].name, worst)  # what FP32 spins with FP64 sums deliver


# --------------------------------------------------------------------------- FP32 statistics

@pytest.mark.parametrize("T,B", [(0.9, 0.0), (1.4, 0.0), (2.5, 0.3)])
def test_fp32_observables_match_oracle(T, B):
    """<E>/N, <|M|>/N, C_v and chi of the FP32 path against the FP64 oracle within 3 standard
    errors (4 chains each side, independent seeds; a point fails only if it fails again with
    fresh seeds), and the energy per site of the two within 1e-3 or their errors."""
    s = sc_periodic(8)
    N, R, mcs = s.n_sites, 4, 4000

    def run(attempt):
        with ctx([s], precision=32, replicas=R, seed=31 + 2 * attempt) as c:
            c.run(np.full((R, 1), T), np.full((R, 1), B), mcs)
            H = c.history()
        Hr = oracle.run(s, np.full((R, 1), T), np.full((R, 1), B), mcs, seed=32 + 2 * attempt, n_threads=R)["history"]
        return [(chain_observables(H, N, T), chain_observables(Hr, N, T))]

    g, o = assert_statistically_equal(run, label=f"8^3 T={T}")[0]
    d_e = abs(g["e"][0] - o["e"][0])
    print(f"T={T} B={B}: |d(E/N)| = {d_e:.2e} (errors {g['e'][1]:.1e}, {o['e'][1]:.1e})")
    assert d_e < 1e-3 or d_e < 3 * np.hypot(g["e"][1], o["e"][1])


def test_fp32_closed_forms():
    """FP32 GPU path against the exact results used to pin the oracle."""
    n = 4000
    # Langevin with a tilted field axis, three fields at once (one instance each)
    axis = np.array([1.0, 2.0, 2.0]) / 3.0
    Bs = np.array([0.5, 2.0, 8.0])
    with ctx([free_spins(n, field_axis=axis)], precision=32, replicas=4, seed=41) as c:
        c.run(np.ones((4, 1)), np.append(Bs, 1.0)[:, None], 400)
        H = c.history()
    for k, B in enumerate(Bs):
        m, se = binned(H[k, :, 1:] @ axis / n)
        L = 1 / np.tanh(B) - 1 / B
        assert abs(m - L) < 4 * se + 2e-5, (B, m, se, L)
    # open chain, antiferromagnetic
    N, R, beta = 64, 16, 2.0
    with ctx([chain_open(N, J=-1.0)], precision=32, replicas=R, seed=42) as c:
        c.run(np.full((R, 1), 1 / beta), np.zeros((R, 1)), 1500)
        H = c.history()
    u = 1 / np.tanh(-beta) + 1 / beta
    U = (N - 1) * u
    means = [binned(h) for h in H[:, :, 0]]
    m = np.mean([a for a, _ in means])
    se = np.sqrt(np.sum([b ** 2 for _, b in means])) / R
    assert abs(m - U) < 4 * se, (m, se, U)
    # frustrated three-spin ring (three colour classes)
    P, T = 2000, 0.7
    with ctx([triangles(P, J=-1.0)], precision=32, seed=43) as c:
        c.run([[T]], [[0.0]], 500)
        H = c.history()
    ref = oracle.run(triangles(P, J=-1.0), [[T]], [[0.0]], 500, seed=44)
    a, sa = binned(H[0, :, 0] / P)
    b, sb = binned(ref["history"][0, :, 0] / P)
    assert abs(a - b) < 4 * np.hypot(sa, sb)


def test_fp32_dimer_detailed_balance():
    P, J, T = 20000, 1.0, 0.5
    with ctx([dimers(P, J=J)], precision=32, seed=45) as c:
        c.run([[T]], [[0.0]], 200)
        S = c.spins(0)
    from scipy import stats

    cth = np.einsum("ij,ij->i", S[0::2], S[1::2])
    K = J / T
    edges = np.linspace(-1, 1, 21)
    obs, _ = np.histogram(np.clip(cth, -1, 1), bins=edges)
    p = (np.exp(K * edges[1:]) - np.exp(K * edges[:-1])) / (np.exp(K) - np.exp(-K))
    chi2 = float(((obs - P * p) ** 2 / (P * p)).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-4, 19), chi2


# --------------------------------------------------------------------------- errors and edge cases

def test_errors_leave_context_usable():
    s = sc_periodic(4)
    with ctx([s], seed=1) as c:
        for T in (0.0, -1.0, np.nan, np.inf):
            with pytest.raises(vb.VegasError) as e:
                c.run([[T]], [[0.0]], 1)
            assert e.value.status == vb.EINVAL
        with pytest.raises(vb.VegasError):
            c.run([[1.0]], [[np.nan]], 1)
        with pytest.raises(vb.VegasError):
            vb.vegas_get_spins(c.ptr, 5, 64)
        with pytest.raises(vb.VegasError):
            c.set_spins(0, np.full((64, 3), np.nan))
        c.run([[1.0]], [[0.0]], 0)
        assert c.history().shape == (1, 0, 4)
        c.run([[1.0]], [[0.0]], 3)
        assert c.history().shape == (1, 3, 4)
        st = c.stats()
        assert st["mcs_done"] == 3 and st["device_error"] == 0 and st["records"] == 3


def test_extreme_temperatures():
    s = sc_periodic(6)
    with ctx([s], precision=32, replicas=2, seed=3) as c:
        up = np.tile([0, 0, 1.0], (s.n_sites, 1))
        c.set_spins(0, up)
        c.set_spins(1, up)
        c.run(np.array([[1e-6], [1e6]]), np.zeros((2, 1)), 20)
        H = c.history()
    assert np.all(H[0, :, 0] / s.n_sites < -2.9999)  # only downhill moves at T -> 0
    assert abs(H[1, -5:, 0].mean() / s.n_sites) < 0.5  # near-random at T -> infinity
