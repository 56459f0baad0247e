"""The five workloads on the GPU (through the C-ABI).

Full size, in the launch configuration bench.py times (32 replicas of the 256^3 +-J glass,
FP32, automatic variant and pipeline): the history's energy and magnetization of sampled
replicas against the oracle's energy and sum of the same spins, unit norms, and one replica
bit-identical to a plain single-replica run. Reduced-size twins of the other workloads:
observables against the oracle (independent seeds) within 4 standard errors. The device
error path: a NaN energy change poisons the context, without any GPU fault.
"""

import numpy as np
import pytest

from conftest import binned

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


def _compare(gpu_hist, ora_hist, N, keys=("e", "m")):
    out = {}
    for name, h in (("gpu", gpu_hist), ("ora", ora_hist)):
        e = h[..., 0] / N
        m = np.linalg.norm(h[..., 1:], axis=-1) / N
        stats = {}
        for k, x in (("e", e), ("m", m)):
            means = [binned(xi) for xi in np.atleast_2d(x)]
            stats[k] = (np.mean([a for a, _ in means]), np.sqrt(np.sum([b ** 2 for _, b in means])) / len(means))
        out[name] = stats
    for k in keys:
        (a, sa), (b, sb) = out["gpu"][k], out["ora"][k]
        assert abs(a - b) < 4 * np.hypot(sa, sb) + 1e-9, (k, a, sa, b, sb)


def test_hysteresis_twin():
    """8^3 sc, J = 1, K = 0.05 along z, T = 0.5, field steps of the loop (reduced)."""
    s = sc_periodic(8, k_uni=0.05)
    B = hysteresis_fields()[::20][None, :]  # 2.0, 1.0, 0.0, -1.0, -2.0, ... back to 2.0
    T = np.full_like(B, 0.5)
    mcs = 300
    with ctx([s], seed=3) as c:
        c.run(T, B, mcs)
        H = c.history()[0].reshape(B.shape[1], mcs, 4)
    ref = oracle.run(s, T, B, mcs, seed=4)["history"][0].reshape(B.shape[1], mcs, 4)
    for k in range(B.shape[1]):
        if k in (3, 7):  # the steps where the field reverses the magnetization: a switching
            continue     # transient of random length, not an equilibrium average
        _compare(H[k][None], ref[k][None], s.n_sites)
    # the loop: magnetization follows the field at the extremes
    assert H[0, -50:, 3].mean() > 0.9 * s.n_sites and H[4, -50:, 3].mean() < -0.9 * s.n_sites


def test_core_shell_twin():
    s = core_shell_particle(seed=5, radius=5.0, core_radius=3.5)
    T = np.array([[1.5, 0.6]])
    B = np.full_like(T, 0.5)
    mcs = 600
    with ctx([s], seed=6) as c:
        c.run(T, B, mcs)
        H = c.history()[0].reshape(2, mcs, 4)
    ref = oracle.run(s, T, B, mcs, seed=7)["history"][0].reshape(2, mcs, 4)
    for k in range(2):
        _compare(H[k][None], ref[k][None], s.n_sites)


def test_nanoparticle_batch_twin():
    samples = nanoparticle_batch(6, seed=8, r_max=5.0)
    temps = np.array([0.3, 0.8, 1.3, 1.8, 2.3, 2.8])
    mcs = 800
    with ctx(samples, seed=9, variant=1) as c:
        c.run(temps[:, None], np.zeros((6, 1)), mcs)
        H = c.history()
    for p, smp in enumerate(samples):
        ref = oracle.run(smp, [[temps[p]]], [[0.0]], mcs, seed=10, inst_base=p)["history"][0]
        _compare(H[p][None], ref[None], smp.n_sites, keys=("e",))


def test_spin_glass_twin_replicas():
    s = sc_periodic(6, bimodal_seed=4)
    R, mcs = 4, 800
    T = np.array([0.9, 1.2, 1.6, 2.0])[:, None]
    with ctx([s], replicas=R, seed=11) as c:
        c.run(T, np.zeros_like(T), mcs)
        H = c.history()
    ref = oracle.run(s, T, np.zeros_like(T), mcs, seed=12, n_threads=R)["history"]
    for r in range(R):
        _compare(H[r][None], ref[r][None], s.n_sites, keys=("e",))


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
