"""The five workloads on the GPU (through the C-ABI).

Full size, in the launch configuration bench.py times (32 replicas of the 256^3 +-J glass,
FP32, automatic variant and pipeline): the history's energy and magnetization of sampled
replicas against the oracle's energy and sum of the same spins, unit norms, and one replica
bit-identical to a plain single-replica run. The headline's own kernel on a +-J glass with 32
replicas, and reduced-size twins of the other workloads (the hysteresis loop, its reversal
steps as an ensemble, the core/shell particle, a nanoparticle batch, the largest particles
through cluster blocks): <E>/N, <|M|>/N, C_v and chi against the oracle (independent seeds)
within 3 standard errors, a point failing only if it fails again with fresh seeds. The
device error path: a NaN energy change poisons the context, without any GPU fault.
"""

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from conftest import assert_statistically_equal, chain_observables

import oracle
import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import core_shell_particle, nanoparticle_batch, sc_periodic
from lattices.workloads import hysteresis_fields

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


def test_spin_glass_full_size_bench_configuration():
    s = sc_periodic(256, bimodal_seed=1)
    R, mcs = 32, 2
    T = (0.1 * 20.0 ** (np.arange(R) / (R - 1.0)))[:, None]
    N = s.n_sites
    with ctx([s], precision=32, replicas=R, seed=1, timing=True) as c:
        c.run(T, np.zeros_like(T), mcs)
        H = c.history()
        st = c.stats()
        assert st["device_error"] == 0 and st["records"] == mcs
        for i in (0, 15, 31):
            S = c.spins(i)
            norms = np.linalg.norm(S, axis=1)
            assert np.all(np.abs(norms - 1.0) < 1e-5)
            e = oracle.energy(s, S, 0.0)
            assert abs(H[i, -1, 0] - e) / N < 1e-5, (i, H[i, -1, 0] / N, e / N)
            assert np.all(np.abs(H[i, -1, 1:] - S.sum(axis=0)) < 1e-5 * N)
        batched7 = c.spins(7)
    with ctx([s], precision=32, replicas=1, inst_base=7, seed=1) as p:
        p.run(T[7:8], np.zeros((1, 1)), mcs)
        assert np.array_equal(p.spins(0), batched7)


def oracle_threads():
    return max(1, min(32, os.cpu_count() or 1))


def oracle_many(jobs):
    """Several oracle runs at once on host threads (the oracle is C called through ctypes,
    which releases the interpreter lock): jobs = [(sample, T, B, mcs, seed, inst_base)]."""
    def one(j):
        smp, T, B, mcs, seed, base = j
        return oracle.run(smp, T, B, mcs, seed=seed, inst_base=base, n_threads=max(1, oracle_threads() // len(jobs)))
    with ThreadPoolExecutor(max_workers=min(len(jobs), oracle_threads())) as ex:
        return list(ex.map(one, jobs))


def steps_of(H, n_steps, mcs):
    """[chains, n_steps * mcs, 4] history -> [n_steps][chains, mcs, 4]."""
    return [H[:, k * mcs:(k + 1) * mcs] for k in range(n_steps)]


# headline temperatures of the +-J glass: T_k = 0.1 * 20^(k/31); four of them, 8 replicas each
GLASS_K = (10, 17, 24, 31)


def test_headline_kernel_statistics_pm_j_glass_r32():
    """The kernel that sweeps the benchmarked workload (pass32_r32: one warp per site x 32
    replicas) on its own kind of input, a +-J glass with 32 replicas, against the FP64 oracle:
    <E>/N, <|M|>/N, C_v and chi within 3 standard errors at four of the headline's
    temperatures (8 independent chains each side, independent seeds)."""
    s = sc_periodic(16, bimodal_seed=1)
    N, R, mcs = s.n_sites, 32, 2000
    Tq = 0.1 * 20.0 ** (np.array(GLASS_K) / 31.0)
    T = np.repeat(Tq, R // len(Tq))[:, None]
    B = np.zeros_like(T)

    def run(attempt):
        with ctx([s], precision=32, replicas=R, seed=101 + 2 * attempt, variant=0) as c:
            c.run(T, B, mcs)
            st = c.stats()
            # the headline kernel, its step's last class-1 pass with the renormalisation folded in
            assert vb.sweep_kernel_names(st["sweep_kernels"]) == ["pass32_r32", "pass32_r32_renorm"], st["sweep_kernels"]
            H = c.history()
        ref = oracle.run(s, T, B, mcs, seed=102 + 2 * attempt, n_threads=oracle_threads())["history"]
        pts = []
        for q in range(len(Tq)):
            rows = slice(q * (R // len(Tq)), (q + 1) * (R // len(Tq)))
            g, o = chain_observables(H[rows], N, Tq[q]), chain_observables(ref[rows], N, Tq[q])
            print(f"+-J 16^3 T={Tq[q]:.3f}: |d(E/N)| = {abs(g['e'][0] - o['e'][0]):.2e} "
                  f"(errors {g['e'][1]:.1e}, {o['e'][1]:.1e})")
            pts.append((g, o))
        return pts

    assert_statistically_equal(run, label="pass32_r32 +-J glass")


def test_hysteresis_twin_equilibrium_steps():
    """8^3 sc, J = 1, K = 0.05 along z, T = 0.5, the loop's field steps (every 20th), 4 chains:
    all four observables within 3 standard errors at every step where the magnetization
    follows the field (the reversal steps are compared as an ensemble below)."""
    s = sc_periodic(8, k_uni=0.05)
    Bf = hysteresis_fields()[::20]  # 2.0, 1.0, 0.0, -1.0, -2.0, -1.0, 0.0, 1.0, 2.0
    R, mcs = 4, 400
    B = np.tile(Bf, (R, 1))
    T = np.full_like(B, 0.5)
    N = s.n_sites

    def run(attempt):
        with ctx([s], replicas=R, seed=3 + 2 * attempt) as c:
            c.run(T, B, mcs)
            H = c.history()
        ref = oracle.run(s, T, B, mcs, seed=4 + 2 * attempt, n_threads=R)["history"]
        return [(chain_observables(g, N, 0.5), chain_observables(o, N, 0.5))
                for k, (g, o) in enumerate(zip(steps_of(H, len(Bf), mcs), steps_of(ref, len(Bf), mcs)))
                if k not in (3, 7)]

    pts = assert_statistically_equal(run, label="hysteresis 8^3")
    # the loop: the magnetization follows the field at the extremes
    assert pts[0][0]["m"][0] > 0.9 and pts[3][0]["m"][0] > 0.9


def test_hysteresis_reversal_ensemble():
    """The reversal steps of the loop (the field turned against the magnetization, B = -1 and
    later +1) are transients, not equilibrium averages: 32 chains on each side go through the
    same schedule, and the switching time (first MCS of the step with M_z of the new sign)
    must have the same distribution (two-sample Kolmogorov-Smirnov) and the ensemble mean of
    M_z(m)/N the same trajectory (3 errors of the mean at checkpoints). The GPU side runs 32
    replicas, i.e. the 32-replica kernel of the headline on the loop's lattice."""
    from scipy import stats

    s = sc_periodic(8, k_uni=0.05)
    Bf = hysteresis_fields()[::20]
    R, mcs = 32, 200
    B = np.tile(Bf, (R, 1))
    T = np.full_like(B, 0.5)
    N = s.n_sites
    marks = [0, 2, 5, 10, 20, 40, 80, 160, 199]

    def trajectories(H):
        out = []
        for k, sign in ((3, -1.0), (7, 1.0)):
            mz = sign * H[:, k * mcs:(k + 1) * mcs, 3] / N  # > 0 once switched
            tau = np.array([int(np.argmax(r > 0)) if np.any(r > 0) else mcs for r in mz])
            out.append((tau, mz))
        return out

    def run(attempt):
        with ctx([s], replicas=R, seed=21 + 2 * attempt, variant=0) as c:
            c.run(T, B, mcs)
            assert vb.sweep_kernel_names(c.stats()["sweep_kernels"]) == ["pass32_r32", "pass32_r32_renorm"]
            H = c.history()
        ref = oracle.run(s, T, B, mcs, seed=22 + 2 * attempt, n_threads=oracle_threads())["history"]
        return trajectories(H), trajectories(ref)

    def check(g, o):
        bad = []
        for (tg, mg), (to, mo) in zip(g, o):
            if stats.ks_2samp(tg, to).pvalue < 1e-3:
                bad.append(("tau", float(tg.mean()), float(to.mean())))
            for m in marks:
                a, b = mg[:, m], mo[:, m]
                se = np.hypot(a.std(ddof=1), b.std(ddof=1)) / np.sqrt(R)
                if abs(a.mean() - b.mean()) > 3 * se + 1e-6:
                    bad.append(("mz", m, float(a.mean()), float(b.mean()), float(se)))
        return bad

    g, o = run(0)
    bad = check(g, o)
    if bad:  # a point fails only if it fails again with fresh seeds
        print("reversal: first seeds", bad)
        g, o = run(1)
        again = check(g, o)
        assert not again, again
    # both reversals complete within the step on both sides
    for (tg, _), (to, _) in zip(g, o):
        assert np.all(tg < mcs) and np.all(to < mcs)


def test_core_shell_twin():
    """Core/shell particle (radius 5, core 3.5: J_c = 1, J_s = 0.5, J_cs = -0.3, radial
    surface anisotropy 0.5), B = 0.5, two temperatures, 4 chains: 3 standard errors."""
    s = core_shell_particle(seed=5, radius=5.0, core_radius=3.5)
    Tv = [1.5, 0.6]
    R, mcs = 4, 800
    T = np.tile(Tv, (R, 1))
    B = np.full_like(T, 0.5)
    N = s.n_sites

    def run(attempt):
        with ctx([s], replicas=R, seed=6 + 2 * attempt) as c:
            c.run(T, B, mcs)
            H = c.history()
        ref = oracle.run(s, T, B, mcs, seed=7 + 2 * attempt, n_threads=R)["history"]
        return [(chain_observables(g, N, Tv[k]), chain_observables(o, N, Tv[k]))
                for k, (g, o) in enumerate(zip(steps_of(H, 2, mcs), steps_of(ref, 2, mcs)))]

    assert_statistically_equal(run, label="core/shell")


def test_nanoparticle_batch_twin():
    """Six fcc particles (radius 3 .. 5), one temperature each, 4 replicas per particle, in
    one resident launch: 3 standard errors on all four observables per particle."""
    samples = nanoparticle_batch(6, seed=8, r_max=5.0)
    temps = np.array([0.3, 0.8, 1.3, 1.8, 2.3, 2.8])
    R, mcs = 4, 800
    T = np.repeat(temps, R)[:, None]

    def run(attempt):
        with ctx(samples, replicas=R, seed=9 + 2 * attempt, variant=1) as c:
            c.run(T, np.zeros_like(T), mcs)
            assert vb.sweep_kernel_names(c.stats()["sweep_kernels"]) == ["resident32"]
            H = c.history()
        refs = oracle_many([(smp, T[p * R:(p + 1) * R], np.zeros((R, 1)), mcs, 10 + 2 * attempt, p * R)
                            for p, smp in enumerate(samples)])
        return [(chain_observables(H[p * R:(p + 1) * R], smp.n_sites, temps[p]),
                 chain_observables(refs[p]["history"], smp.n_sites, temps[p])) for p, smp in enumerate(samples)]

    assert_statistically_equal(run, label="nanoparticles")


def test_large_particles_through_cluster_blocks():
    """Particles of the batch's largest radii (about 10k and 14k sites) swept by thread-block
    clusters of several blocks (the shapes the automatic choice sizes for them), with small
    particles beside them swept one per block (cluster split), against the oracle: 3 standard
    errors on all four observables for every particle."""
    big = nanoparticle_batch(2, seed=31, r_min=13.5, r_max=15.0)
    small = nanoparticle_batch(4, seed=32, r_min=3.0, r_max=5.0)
    samples = big + small
    temps = np.array([0.9, 2.2, 0.5, 1.4, 2.0, 2.8])
    R, mcs = 2, 400
    T = np.repeat(temps, R)[:, None]

    def run(attempt):
        with ctx(samples, replicas=R, seed=41 + 2 * attempt, variant=3, cluster_blocks=4, cluster_threads=512,
                 cluster_split=2000) as c:
            c.run(T, np.zeros_like(T), mcs)
            st = c.stats()
            assert vb.sweep_kernel_names(st["sweep_kernels"]) == ["cluster32"] and st["cluster_blocks"] == 4
            assert st["split_sites"] == 2000
            H = c.history()
        refs = oracle_many([(smp, T[p * R:(p + 1) * R], np.zeros((R, 1)), mcs, 42 + 2 * attempt, p * R)
                            for p, smp in enumerate(samples)])
        return [(chain_observables(H[p * R:(p + 1) * R], smp.n_sites, temps[p]),
                 chain_observables(refs[p]["history"], smp.n_sites, temps[p])) for p, smp in enumerate(samples)]

    assert all(smp.n_sites > 9000 for smp in big)
    assert_statistically_equal(run, label="large particles, clusters")


def test_nan_energy_change_poisons_the_context():
    """Spins near the FP32 limit make the local field +inf in x and -inf in y; the energy
    change is then NaN, the kernel flags it (no trap), and the context refuses further work."""
    s = sc_periodic(4)
    colour, _ = vg.vegas_greedy_colour(s.row_ptr, s.col)
    big = np.where(colour[:, None] == 0, [[3e38, 3e38, 0.0]], [[3e38, -3e38, 0.0]])
    with ctx([s], seed=1) as c:
        c.set_spins(0, big)
        with pytest.raises(vb.VegasError) as e:
            c.run([[1.0]], [[0.0]], 1)
        assert e.value.status == vb.EDEVICE and "NaN" in str(e.value)
        assert c.stats()["device_error"] & 1
        with pytest.raises(vb.VegasError) as e2:
            c.run([[1.0]], [[0.0]], 1)
        assert e2.value.status == vb.ESTATE
