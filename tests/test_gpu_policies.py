"""Update policies on the GPU (Sec. II; Sec. IV.C) through the C-ABI, against the CPU oracle.

FP64: spins, accept/reject bits, accepted counts per MCS and the adaptive widths match the
oracle bit for bit, for every policy and for mixed per-type tables. FP32: the equilibrium
laws each policy must reach (Langevin, uniaxial quadrature, Ising chain for spin flips),
the adaptive control law recomputed from the GPU's own counts, bit identity between the
sweep variants, and the accepted counts against the accept/reject log (which also covers
the replica-batched R = 32 kernel).
"""

import math

import numpy as np
import pytest
from scipy import special

from conftest import binned

import oracle
import paper_1803_07030_gb300 as vg
from lattices import chain_open, core_shell_particle, free_spins, nanoparticle_batch, random_graph, sc_periodic

pytestmark = pytest.mark.gpu

ALL = [oracle.RANDOM, oracle.SPIN_FLIP, oracle.SMALL_STEP, oracle.GAUSSIAN, oracle.HINZKE_NOWAK, oracle.ADAPTIVE]
PARAM = [0.0, 0.0, 0.4, 0.35, 0.6, 0.9]


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


def mixed_sc(L=6, seed=3, policies=ALL, params=PARAM):
    """Periodic +-J sc with anisotropy, random site types over a six-entry policy table."""
    s = sc_periodic(L, k_uni=0.3, bimodal_seed=seed)
    rng = np.random.default_rng(seed)
    s.type = rng.integers(0, 6, size=s.n_sites).astype(np.int32)
    return s.with_policy(policies, params)


# --------------------------------------------------------------------------- FP64 bit identity

@pytest.mark.parametrize("policy,param", list(zip(ALL, PARAM)))
def test_fp64_each_policy_bitwise(policy, param):
    s = sc_periodic(5, k_uni=0.2).with_policy([policy], [param])
    T = np.array([[1.5, 0.6]])
    B = np.array([[0.3, -0.2]])
    mcs = 10  # two adaptive MCS per step
    with ctx([s], precision=64, seed=5, accept_log_mcs=20) as c:
        c.run(T, B, mcs)
        ref = oracle.run(s, T, B, mcs, seed=5, log_mcs=20)
        assert ref["err"] == 0
        assert first_divergence(c.accept_log().reshape(20, -1), ref["accept_log"][0]) is None
        assert first_divergence(c.spins(0), ref["spins"][0]) is None
        assert np.array_equal(c.accept_history()[0], ref["accepted"][0])
        if policy == oracle.ADAPTIVE:
            assert c.adaptive_width()[0] == ref["sigma"][0]
        else:
            assert c.adaptive_width()[0] == 0.0


def test_fp64_mixed_table_replicas_bitwise():
    s = mixed_sc()
    R, base, mcs = 4, 3, 15
    T = np.stack([[2.0 - 0.3 * r, 0.8 + 0.1 * r] for r in range(R)])
    B = np.stack([[0.1 * r, -0.4] for r in range(R)])
    with ctx([s], precision=64, replicas=R, inst_base=base, seed=11) as c:
        c.run(T, B, mcs)
        ref = oracle.run(s, T, B, mcs, seed=11, inst_base=base, n_threads=R)
        acc = c.accept_history()
        sig = c.adaptive_width()
        for r in range(R):
            assert first_divergence(c.spins(r), ref["spins"][r]) is None, r
            assert np.array_equal(acc[r], ref["accepted"][r])
            assert sig[r] == ref["sigma"][r]


def test_fp64_core_shell_and_ragged_samples_bitwise():
    cs = core_shell_particle(seed=2, radius=4.0, core_radius=2.5).with_policy(
        [oracle.HINZKE_NOWAK, oracle.ADAPTIVE], [0.5, 1.2])
    rg = random_graph(70, 0.08, 4, all_terms=True)
    rg.with_policy([oracle.GAUSSIAN, oracle.SPIN_FLIP, oracle.SMALL_STEP], [0.3, 0.0, 1.0])
    plain = sc_periodic(4)
    samples = [cs, rg, plain]
    R, mcs = 2, 12
    n_inst = len(samples) * R
    T = np.linspace(0.5, 2.5, n_inst)[:, None]
    B = np.linspace(-0.5, 0.5, n_inst)[:, None]
    with ctx(samples, precision=64, replicas=R, seed=17) as c:
        c.run(T, B, mcs)
        acc, sig = c.accept_history(), c.adaptive_width()
        for si, s in enumerate(samples):
            rows = slice(si * R, (si + 1) * R)
            ref = oracle.run(s, T[rows], B[rows], mcs, seed=17, inst_base=si * R)
            for r in range(R):
                i = si * R + r
                assert first_divergence(c.spins(i), ref["spins"][r]) is None, (s.name, r)
                assert np.array_equal(acc[i], ref["accepted"][r])
                assert sig[i] == ref["sigma"][r]


def test_fp64_adaptive_width_checkpoint():
    s = free_spins(300).with_policy([oracle.ADAPTIVE], [1.0])
    with ctx([s], precision=64, seed=8) as a:
        a.run([[0.5, 0.5]], [[2.0, 2.0]], 10)
        full = a.spins(0), a.adaptive_width()[0]
    with ctx([s], precision=64, seed=8) as b:
        b.run([[0.5]], [[2.0]], 10)
        S, w = b.spins(0), b.adaptive_width()
    with ctx([s], precision=64, seed=8) as c:  # resume in a fresh context
        c.set_spins(0, S)
        c.set_adaptive_width(w)
        c.run([[0.5]], [[2.0]], 10)  # a fresh context starts its MCS counter at t = 0
        resumed = c.spins(0)
    ref = oracle.run(s, [[0.5]], [[2.0]], 10, seed=8, spins=S[None], sigma=w, t0=0)
    assert np.array_equal(resumed, ref["spins"][0])
    b2 = oracle.run(s, [[0.5]], [[2.0]], 10, seed=8, spins=S[None], sigma=w, t0=10)
    assert np.array_equal(full[0], b2["spins"][0]) and full[1] == b2["sigma"][0]


# --------------------------------------------------------------------------- FP32 physics

@pytest.mark.parametrize("policy,param", [(oracle.SMALL_STEP, 0.5), (oracle.GAUSSIAN, 0.4),
                                          (oracle.HINZKE_NOWAK, 0.3), (oracle.ADAPTIVE, 1.0)])
def test_fp32_policy_langevin_and_uniaxial(policy, param):
    n, mcs = 4000, 500
    s = free_spins(n).with_policy([policy], [param])
    with ctx([s], precision=32, replicas=2, seed=21) as c:
        c.run(np.ones((2, 1)), np.array([[1.5], [0.5]]), mcs)
        H = c.history()
    for k, B in enumerate((1.5, 0.5)):
        m, se = binned(H[k, mcs // 5:, 3] / n)
        L = 1 / math.tanh(B) - 1 / B
        assert abs(m - L) < 4 * se + 2e-5, (B, m, se, L)
    k_, e = 2.0, np.array([0.0, 1.0, 1.0]) / np.sqrt(2.0)
    s = free_spins(n, k_uni=k_, e_uni=e).with_policy([policy], [param])
    with ctx([s], precision=32, seed=22) as c:
        c.run([[1.0]], [[0.0]], mcs)
        H = c.history()
    m, se = binned(-H[0, mcs // 5:, 0] / (k_ * n))
    exact = np.exp(k_) / (np.sqrt(np.pi * k_) * special.erfi(np.sqrt(k_))) - 1.0 / (2.0 * k_)
    assert abs(m - exact) < 4 * se + 2e-5, (m, se, exact)


@pytest.mark.parametrize("J", [1.0, -1.0])
def test_fp32_spin_flip_ising_chain(J):
    N, T = 4000, 1.5
    s = chain_open(N, J=J).with_policy([oracle.SPIN_FLIP], [0.0])
    s.init_spins = np.tile([0.0, 0.0, 1.0], (N, 1))
    with ctx([s], precision=32, seed=23) as c:
        c.run([[T]], [[0.0]], 400)
        H = c.history()
        S = c.spins(0)
    assert np.all(np.abs(np.abs(S[:, 2]) - 1.0) < 1e-6)
    m, se = binned(H[0, :, 0])
    U = -(N - 1) * J * math.tanh(J / T)
    assert abs(m - U) < 4 * se + 1e-5 * N, (m, se, U)


def test_fp32_adaptive_control_law_from_gpu_counts():
    n, mcs = 4000, 100
    s = free_spins(n).with_policy([oracle.ADAPTIVE], [2.0])
    s.init_spins = np.tile([0.0, 0.0, 1.0], (n, 1))
    with ctx([s], precision=32, replicas=2, seed=24) as c:
        c.run(np.ones((2, 1)), np.array([[8.0], [6.0]]), mcs)
        acc = c.accept_history()
        w = c.adaptive_width()
    for r in range(2):
        sg = 2.0
        for m in range(mcs // 5):
            sg = min(max(sg * (0.5 / max(1.0 - acc[r, m] / n, 0.01)), 1e-4), 100.0)
        assert w[r] == sg
        assert abs(acc[r, mcs // 5:].mean() / n - 0.5) < 0.05


def test_fp32_policy_observables_match_oracle():
    # no spin-flip-only type: such sites keep their initial axis, which differs between seeds
    s = mixed_sc(L=6, seed=9, policies=[oracle.RANDOM, oracle.HINZKE_NOWAK, oracle.SMALL_STEP, oracle.GAUSSIAN,
                                        oracle.HINZKE_NOWAK, oracle.ADAPTIVE], params=[0.0, 0.7, 0.4, 0.35, 0.2, 0.9])
    mcs = 1500
    with ctx([s], precision=32, seed=25) as c:
        c.run([[1.2]], [[0.4]], mcs)
        H = c.history()[0]
    ref = oracle.run(s, [[1.2]], [[0.4]], mcs, seed=26)["history"][0]
    n = s.n_sites
    for q in (0, 3):
        a, sa = binned(H[mcs // 5:, q] / n)
        b, sb = binned(ref[mcs // 5:, q] / n)
        assert abs(a - b) < 4 * np.hypot(sa, sb) + 1e-5, (q, a, sa, b, sb)


# --------------------------------------------------------------------------- variants and counts

def test_policy_sweep_variants_agree():
    samples = nanoparticle_batch(5, seed=3, r_max=4.5)
    for p in samples:
        p.type = (np.arange(p.n_sites) % 3).astype(np.int32)
        p.with_policy([oracle.HINZKE_NOWAK, oracle.ADAPTIVE, oracle.GAUSSIAN], [0.4, 0.8, 0.3])
    T = np.linspace(0.4, 2.0, 10)[:, None]
    B = np.full_like(T, 0.2)
    with ctx(samples, replicas=2, seed=31, variant=0, accept_log_mcs=4) as a, \
            ctx(samples, replicas=2, seed=31, variant=1, accept_log_mcs=4) as b:
        a.run(T, B, 12)
        b.run(T, B, 12)
        assert np.array_equal(a.accept_log(), b.accept_log())
        assert np.array_equal(a.accept_history(), b.accept_history())
        assert np.array_equal(a.adaptive_width(), b.adaptive_width())
        for i in range(10):
            assert np.array_equal(a.spins(i), b.spins(i)), i


def test_cooperative_sweep_with_policies_and_no_adaptive():
    s = core_shell_particle(seed=4, radius=5.0, core_radius=3.5).with_policy(
        [oracle.RANDOM, oracle.HINZKE_NOWAK], [0.0, 0.5])
    with ctx([s], replicas=2, seed=32, variant=0) as a, ctx([s], replicas=2, seed=32, variant=2) as b:
        a.run([[1.0], [0.5]], [[0.3], [0.3]], 6)
        b.run([[1.0], [0.5]], [[0.3], [0.3]], 6)
        assert np.array_equal(a.accept_history(), b.accept_history())
        for i in range(2):
            assert np.array_equal(a.spins(i), b.spins(i))
    ad = core_shell_particle(seed=4, radius=5.0, core_radius=3.5).with_policy(
        [oracle.RANDOM, oracle.ADAPTIVE], [0.0, 0.5])
    with pytest.raises(vg.VegasError):
        ctx([ad], variant=2)


def test_random_sites_on_the_policy_path_equal_the_plain_path():
    """A table whose non-random type no site has: the policy kernels' random branch must
    reproduce the plain (staged) kernels bit for bit."""
    plain = sc_periodic(8, bimodal_seed=2)
    tabled = sc_periodic(8, bimodal_seed=2)
    tabled.type = np.zeros(tabled.n_sites, dtype=np.int32)
    tabled.with_policy([oracle.RANDOM, oracle.SPIN_FLIP], [0.0, 0.0])
    for R in (1, 4, 32):
        with ctx([plain], replicas=R, seed=33) as a, ctx([tabled], replicas=R, seed=33) as b:
            T = np.full((R, 1), 1.3)
            a.run(T, np.zeros_like(T), 5)
            b.run(T, np.zeros_like(T), 5)
            assert np.array_equal(a.accept_history(), b.accept_history())
            for i in (0, R - 1):
                assert np.array_equal(a.spins(i), b.spins(i)), (R, i)


@pytest.mark.parametrize("R", [1, 32])
def test_accept_counts_equal_the_accept_log(R):
    s = sc_periodic(16, bimodal_seed=5)
    with ctx([s], replicas=R, seed=34, accept_log_mcs=3) as c:
        T = np.linspace(0.5, 3.0, R)[:, None]
        c.run(T, np.zeros_like(T), 3)
        log = c.accept_log().reshape(3, R, s.n_sites)
        acc = c.accept_history()
    assert np.array_equal(acc.T, log.sum(axis=2).astype(np.uint32))


def test_invalid_policy_tables_rejected_on_device_context():
    s = sc_periodic(4)
    s.type = np.full(s.n_sites, 2, dtype=np.int32)
    s.with_policy([oracle.RANDOM, oracle.GAUSSIAN], [0.0, 0.5])
    with pytest.raises(vg.VegasError) as e:
        ctx([s])
    assert "outside the policy table" in str(e.value)


def test_replica_batched_policy_kernel_equals_direct_kernel():
    """R = 32 on six-link rows: the staged kernel with policies against the direct kernel."""
    s = mixed_sc(L=16, seed=12)
    T = np.linspace(0.3, 2.5, 32)[:, None]
    B = np.full_like(T, 0.1)
    with ctx([s], replicas=32, seed=35, variant=0) as a, \
            ctx([s], replicas=32, seed=35, variant=0, pipeline_depth=1) as b:
        a.run(T, B, 10)
        b.run(T, B, 10)
        assert np.array_equal(a.accept_history(), b.accept_history())
        assert np.array_equal(a.adaptive_width(), b.adaptive_width())
        for i in (0, 13, 31):
            assert np.array_equal(a.spins(i), b.spins(i)), i


# --------------------------------------------------------------------------- qIsing

def _mixed_spin_lattice(L=6, seed=4):
    """Ferrimagnet-like sc lattice: sublattice A spin 1/2, sublattice B spin 1 (both qIsing),
    a few random Heisenberg sites of norm 1; field and crystal field along z."""
    s = sc_periodic(L, J=-1.0, k_uni=0.4)
    idx = np.arange(s.n_sites)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    s.type = ((x + y + z) % 2).astype(np.int32)
    rng = np.random.default_rng(seed)
    s.type[rng.choice(s.n_sites, 10, replace=False)] = 2
    s.spin_norm = np.where(s.type == 0, 0.5, 1.0)
    return s.with_policy([oracle.QISING, oracle.QISING, oracle.RANDOM], [0.0, 0.0, 0.0])


def test_fp64_qising_bitwise():
    s = _mixed_spin_lattice()
    T = np.array([[1.2, 0.5], [2.0, 0.8]])
    B = np.array([[0.3, -0.2], [0.0, 0.5]])
    with ctx([s], precision=64, replicas=2, seed=41, accept_log_mcs=6) as c:
        c.run(T, B, 6)
        ref = oracle.run(s, T, B, 6, seed=41, log_mcs=6, n_threads=2)
        assert first_divergence(c.accept_log().reshape(6, 2, -1), ref["accept_log"].transpose(1, 0, 2)) is None
        for r in range(2):
            assert first_divergence(c.spins(r), ref["spins"][r]) is None, r
        assert np.array_equal(c.accept_history(), ref["accepted"])
        S = c.spins(0)
        q = s.type < 2
        assert np.all(S[q, :2] == 0.0) and np.all(np.isin(S[q, 2], [-1.0, -0.5, 0.0, 0.5, 1.0]))


@pytest.mark.parametrize("sn,B,k", [(1.0, 0.6, 0.8), (1.5, 0.4, -0.3)])
def test_fp32_qising_free_spins_boltzmann(sn, B, k):
    n, T, mcs = 8000, 1.0, 300
    fs = free_spins(n, spin_norm=sn, k_uni=k, e_uni=(0.0, 0.0, 1.0)).with_policy([oracle.QISING], [0.0])
    with ctx([fs], precision=32, seed=42) as c:
        c.run([[T]], [[B]], mcs)
        H = c.history()[0]
        S = c.spins(0)
    m = np.arange(-sn, sn + 0.5, 1.0)
    w = np.exp((B * m + k * m * m) / T)
    w /= w.sum()
    got, se = binned(H[:, 3] / n)
    assert abs(got - (w * m).sum()) < 4 * se + 1e-4, (got, se)
    assert np.all(S[:, :2] == 0.0) and np.all(np.isin(S[:, 2], m))


def test_qising_replica_batched_kernel_equals_direct_kernel():
    s = _mixed_spin_lattice(L=16, seed=5)
    T = np.linspace(0.4, 2.4, 32)[:, None]
    B = np.full_like(T, 0.2)
    with ctx([s], replicas=32, seed=43, variant=0) as a, \
            ctx([s], replicas=32, seed=43, variant=0, pipeline_depth=1) as b:
        a.run(T, B, 6)
        b.run(T, B, 6)
        assert np.array_equal(a.accept_history(), b.accept_history())
        for i in (0, 17, 31):
            assert np.array_equal(a.spins(i), b.spins(i)), i


def test_qising_needs_half_integer_norms():
    s = free_spins(10, spin_norm=0.7).with_policy([oracle.QISING], [0.0])
    with pytest.raises(vg.VegasError) as e:
        ctx([s])
    assert "qIsing" in str(e.value)


SPECIALISED = [(oracle.SPIN_FLIP, 0.0), (oracle.SMALL_STEP, 0.6), (oracle.GAUSSIAN, 0.4), (oracle.HINZKE_NOWAK, 0.5),
               (oracle.ADAPTIVE, 0.8), (oracle.QISING, 0.0)]


@pytest.mark.parametrize("policy,param", SPECIALISED, ids=[str(p) for p, _ in SPECIALISED])
def test_single_policy_kernel_equals_table_kernels(policy, param):
    """A sample whose sites all have one policy runs the R = 32 kernel compiled for that policy
    alone; its spins, accepted counts and adaptive widths equal the table-driven direct
    kernel's bit for bit. Two site types with the same policy but different parameters keep
    the per-site parameter in play."""
    s = sc_periodic(12, k_uni=0.3)
    s.type = (np.arange(s.n_sites) % 3 == 0).astype(np.int32)
    if policy == oracle.QISING:
        s.spin_norm = np.where(s.type == 0, 0.5, 1.0)
    s.with_policy([policy, policy], [param, 1.5 * param if param else 0.0])
    T = np.linspace(0.3, 2.5, 32)[:, None]
    B = np.full_like(T, 0.15)
    with ctx([s], replicas=32, seed=36, variant=0) as a, \
            ctx([s], replicas=32, seed=36, variant=0, pipeline_depth=1) as b:
        a.run(T, B, 10)
        b.run(T, B, 10)
        assert vg.vegas.sweep_kernel_names(a.stats()["sweep_kernels"]) == ["pass32_r32_one_policy"]
        assert vg.vegas.sweep_kernel_names(b.stats()["sweep_kernels"]) == ["pass32_direct"]
        assert np.array_equal(a.accept_history(), b.accept_history())
        assert np.array_equal(a.adaptive_width(), b.adaptive_width())
        for i in (0, 13, 31):
            assert np.array_equal(a.spins(i), b.spins(i)), i


def test_policy_kernel_per_colour_class():
    """Each colour class gets its own kernel: a class whose sites all move at random runs the
    kernel without a table, a class of one other policy the specialised kernel; the spins
    equal the direct kernel's."""
    s = sc_periodic(10)
    colour, _ = vg.vegas_greedy_colour(s.row_ptr, s.col)
    s.type = colour.astype(np.int32)  # type = class: class 0 random, class 1 Gaussian
    s.with_policy([oracle.RANDOM, oracle.GAUSSIAN], [0.0, 0.3])
    T = np.linspace(0.5, 2.0, 32)[:, None]
    B = np.zeros_like(T)
    with ctx([s], replicas=32, seed=37, variant=0) as a, \
            ctx([s], replicas=32, seed=37, variant=0, pipeline_depth=1) as b:
        a.run(T, B, 8)
        b.run(T, B, 8)
        assert sorted(vg.vegas.sweep_kernel_names(a.stats()["sweep_kernels"])) == \
            ["pass32_r32", "pass32_r32_one_policy"]
        for i in (0, 31):
            assert np.array_equal(a.spins(i), b.spins(i)), i
