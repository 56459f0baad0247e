"""Per-phase magnetization and per-step final states (Sec. II) on the GPU, against the oracle.

FP64: the magnetization of every site type after every MCS agrees with the oracle's to
1e-12 relative (the GPU sums block partials in another order) and the final state of every
step equals the oracle's bit for bit, for packed samples with different numbers of types.
FP32: the types add up to the history's magnetization, the last record of a step matches the
snapshot's sums, the per-class and resident sweeps agree, and storing sites type by type does
not change a single spin.
"""

import numpy as np
import pytest

import oracle
import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import core_shell_particle, nanoparticle_batch, random_graph, sc_periodic

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


def _samples():
    cs = core_shell_particle(seed=2, radius=4.0, core_radius=2.5)                 # types 0, 1
    rg = random_graph(60, 0.1, 5, all_terms=True)                                  # types 0, 1, 2
    plain = sc_periodic(4)                                                         # no types
    return [cs, rg, plain]


def test_fp64_type_history_and_snapshots_match_oracle():
    samples = _samples()
    R, mcs = 2, 5
    n_inst = len(samples) * R
    T = np.stack([np.array([2.0, 1.0, 0.5]) * (1 + 0.1 * i) for i in range(n_inst)])
    B = np.stack([np.array([0.1, 0.4, -0.3]) for _ in range(n_inst)])
    with ctx(samples, precision=64, replicas=R, seed=21, type_stats=True, snapshots=True) as c:
        c.run(T, B, mcs)
        H, TH = c.history(), c.type_history()
        assert c.stats()["n_types"] == 3 and c.stats()["snapshot_steps"] == 3
        for si, s in enumerate(samples):
            rows = slice(si * R, (si + 1) * R)
            ref = oracle.run(s, T[rows], B[rows], mcs, seed=21, inst_base=si * R, n_types=3, snapshots=True)
            for r in range(R):
                i = si * R + r
                assert np.array_equal(c.spins(i), ref["spins"][r])
                assert np.allclose(TH[i], ref["type_history"][r], rtol=0, atol=1e-12 * s.n_sites)
                assert np.allclose(TH[i].sum(axis=1), H[i, :, 1:], rtol=0, atol=1e-12 * s.n_sites)
                for k in range(3):
                    assert np.array_equal(c.snapshot(i, k), ref["snapshots"][r, k]), (s.name, r, k)


def _typed_particles(n=6):
    ps = nanoparticle_batch(n, seed=4, r_max=4.5)
    for p in ps:
        p.type = (np.arange(p.n_sites) % 3).astype(np.int32)
    return ps


@pytest.mark.parametrize("variant", [0, 1])
def test_fp32_types_add_up_and_match_snapshots(variant):
    ps = _typed_particles()
    T = np.tile([[1.5, 0.6]], (len(ps), 1))
    B = np.full_like(T, 0.3)
    mcs = 7
    with ctx(ps, seed=22, variant=variant, type_stats=True, snapshots=True) as c:
        c.run(T, B, mcs)
        H, TH = c.history(), c.type_history()
        for i, p in enumerate(ps):
            n = p.n_sites
            assert np.all(np.abs(TH[i].sum(axis=1) - H[i, :, 1:]) <= 1e-6 * n)
            for k in range(2):
                S = c.snapshot(i, k)
                for ty in range(3):
                    want = S[p.type == ty].sum(axis=0)
                    assert np.all(np.abs(TH[i, (k + 1) * mcs - 1, ty] - want) <= 1e-5 * n), (i, k, ty)
            assert np.array_equal(c.snapshot(i, 1), c.spins(i))


def test_fp32_resident_and_per_class_type_statistics_agree():
    ps = _typed_particles()
    T = np.linspace(0.4, 2.0, len(ps))[:, None]
    B = np.full_like(T, 0.2)
    with ctx(ps, seed=23, variant=0, type_stats=True) as a, ctx(ps, seed=23, variant=1, type_stats=True) as b:
        a.run(T, B, 9)
        b.run(T, B, 9)
        for i, p in enumerate(ps):
            assert np.array_equal(a.spins(i), b.spins(i))
            assert np.all(np.abs(a.type_history()[i] - b.type_history()[i]) <= 1e-6 * p.n_sites)


@pytest.mark.parametrize("R", [1, 32])
def test_type_major_storage_changes_no_spin(R):
    s = sc_periodic(16, bimodal_seed=7)
    s.type = np.random.default_rng(3).integers(0, 2, size=s.n_sites).astype(np.int32)
    T = np.linspace(0.5, 2.5, R)[:, None]
    with ctx([s], replicas=R, seed=24, variant=0) as a, ctx([s], replicas=R, seed=24, variant=0, type_stats=True) as b:
        a.run(T, np.zeros_like(T), 4)
        b.run(T, np.zeros_like(T), 4)
        assert np.array_equal(a.accept_history(), b.accept_history())
        for i in (0, R - 1):
            assert np.array_equal(a.spins(i), b.spins(i))
        TH, H = b.type_history(), b.history()
        assert np.all(np.abs(TH.sum(axis=2) - H[..., 1:]) <= 1e-6 * s.n_sites)


def test_snapshots_continue_across_runs_and_graphs():
    s = core_shell_particle(seed=5, radius=4.0, core_radius=2.5)
    with ctx([s], seed=25, snapshots=True) as a, ctx([s], seed=25, snapshots=True, graphs=False) as b:
        a.run([[1.0, 0.8]], [[0.1, 0.2]], 6)
        a.run([[0.6]], [[0.3]], 6)
        b.run([[1.0, 0.8, 0.6]], [[0.1, 0.2, 0.3]], 6)
        assert a.stats()["snapshot_steps"] == 3
        for k in range(3):
            assert np.array_equal(a.snapshot(0, k), b.snapshot(0, k))
        assert np.array_equal(a.snapshot(0, 2), a.spins(0))


def test_output_option_errors():
    s = core_shell_particle(seed=5, radius=4.0, core_radius=2.5)
    with ctx([s]) as c:
        c.run([[1.0]], [[0.0]], 2)
        with pytest.raises(vb.VegasError) as e:
            c.type_history()
        assert e.value.status == vb.EINVAL
        with pytest.raises(vb.VegasError):
            c.snapshot(0, 0)
    with ctx([s], snapshots=True) as c:
        c.run([[1.0]], [[0.0]], 2)
        with pytest.raises(vb.VegasError):
            c.snapshot(0, 1)
        c.snapshot(0, 0)
    with pytest.raises(vb.VegasError):
        ctx([s], variant=2, type_stats=True)
    many = core_shell_particle(seed=5, radius=4.0, core_radius=2.5)
    many.type = (np.arange(many.n_sites) % 9).astype(np.int32)
    with pytest.raises(vb.VegasError):
        ctx([many], variant=1, type_stats=True)
