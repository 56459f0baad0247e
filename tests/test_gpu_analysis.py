"""History analysis on the GPU (thermal averages, cumulants, autocorrelation times,
reweighting) against the numpy oracle, on histories from the GPU sweep and on synthetic
series. Both sides are FP64; they sum in different orders, so values agree to ~1e-10
relative (v1, v2 to 1e-10 of <E>, the scale of the terms that cancel in the oracle's form)."""

import numpy as np
import pytest

from oracle import analysis
import paper_1803_07030_gb300 as vg
from lattices import sc_periodic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _compare(gpu_row, ref, Escale):
    for k, name in enumerate(vg.AVG_FIELDS):
        a, b = gpu_row[k], ref[name]
        if name in ("v1", "v2"):
            assert abs(a - b) <= 1e-10 * Escale + 1e-12, (name, a, b)
        elif name in ("tau_e", "tau_m"):
            assert abs(a - b) <= 1e-8 * abs(b), (name, a, b)
        else:
            assert abs(a - b) <= 1e-9 * abs(b) + 1e-300, (name, a, b)


def test_thermal_averages_of_gpu_histories():
    s = sc_periodic(8)
    R, mcs = 32, 1000
    T = np.linspace(0.6, 2.4, R)[:, None]
    with vg.Context([s], replicas=R, seed=3, stream=None) as c:
        c.run(T, np.zeros_like(T), mcs)
        H = c.history()
    out = vg.thermal_averages(H, 200, 20, T[:, 0], s.n_sites)
    for r in range(R):
        ref = analysis.thermal_averages(H[r], 200, 20, T[r, 0], s.n_sites)
        _compare(out[r], ref, abs(H[r, 200:, 0].mean()))
    # the ferromagnet orders below T_c ~ 1.44: |M| per site grows as T falls
    assert out[0, 2] > 0.8 and out[-1, 2] < 0.3
    assert np.array_equal(out, vg.thermal_averages(H, 200, 20, T[:, 0], s.n_sites))  # deterministic


def test_thermal_averages_of_long_synthetic_series():
    rng = np.random.default_rng(7)
    ns, ln = 12, 50000
    phi = 0.9
    x = np.zeros((ns, ln))
    xi = rng.normal(size=(ns, ln)) * np.sqrt(1 - phi * phi)
    for i in range(1, ln):
        x[:, i] = phi * x[:, i - 1] + xi[:, i]
    H = np.stack([-5000.0 + 30.0 * x, 100.0 * rng.normal(size=(ns, ln)), 100.0 * x,
                  200.0 + 50.0 * rng.normal(size=(ns, ln))], axis=2)
    Tv = np.linspace(1.0, 2.0, ns)
    out = vg.thermal_averages(H, 5000, 40, Tv, 4096.0)
    for s in range(ns):
        _compare(out[s], analysis.thermal_averages(H[s], 5000, 40, Tv[s], 4096.0), 5000.0)


def _langevin_samples(rng, n_conf, N, beta, B):
    a = beta * B
    u = rng.random((n_conf, N))
    c = np.log(np.exp(-a) + u * (np.exp(a) - np.exp(-a))) / a
    Mz = c.sum(axis=1)
    return -B * Mz, Mz


@pytest.mark.parametrize("K", [1, 4])
def test_reweighting_matches_oracle(K):
    rng = np.random.default_rng(8)
    N, B = 10, 1.0
    betas = np.array([0.5, 0.8, 1.1, 1.4])[:K]
    runs = [_langevin_samples(rng, 50000, N, b, B) for b in betas]
    E = np.stack([r[0] for r in runs])
    O = np.stack([np.column_stack([r[0], r[1], r[1] ** 2]) for r in runs])
    targets = np.array([0.45, 0.65, 0.95, 1.25, 1.5])
    out, g, it = vg.reweight(E, O, betas, targets, tol=1e-12)
    ref, gref, itref = analysis.reweight(E, O, betas, targets, tol=1e-12)
    assert abs(it - itref) <= 1
    assert np.allclose(g, gref, rtol=0, atol=1e-9)
    assert np.allclose(out, ref, rtol=1e-9, atol=1e-12)
