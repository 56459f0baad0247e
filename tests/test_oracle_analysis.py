"""Pins of the oracle's history analysis (oracle/analysis.py) to facts outside itself (no GPU).

  thermal averages  iid Gaussian energies and an isotropic Gaussian 3D magnetization: the
                    means, c = sigma^2 / (N T^2), chi, Binder u4 = 4/9, tau = 1/2; the binned
                    and jackknife errors against the spread over independent repetitions
  autocorrelation   an AR(1) series: tau_int = (1 + phi) / (2 (1 - phi))
  cumulants         independent Ising spins in a field (binomial law, exact sums): v1, v2
                    from samples against the exact values, and the exact v_j against a
                    finite-difference d ln<|M|^j> / d beta
  reweighting       exact Boltzmann samples of free classical spins in a field: single
                    histogram <E>(beta) near beta0 and multiple histogram interpolation against
                    the Langevin law; the free energies g_k against the exact ln Z_k - ln Z_0
"""

import math

import numpy as np
from scipy import special

from oracle import analysis


def _gauss_series(rng, n, mu, sigma, sm):
    E = rng.normal(mu, sigma, n)
    M = rng.normal(0.0, sm, (n, 3))
    return np.column_stack([E, M])


def test_thermal_averages_of_gaussian_series():
    rng = np.random.default_rng(1)
    N, T, mu, sigma, sm = 1000.0, 2.0, -3000.0, 40.0, 25.0
    reps = [analysis.thermal_averages(_gauss_series(rng, 20000, mu, sigma, sm), 1000, 20, T, N) for _ in range(20)]
    r = reps[0]
    assert abs(r["e"] - mu / N) < 4 * r["e_err"]
    assert abs(r["e_err"] - sigma / math.sqrt(19000 // 20 * 20) / N) < 0.4 * r["e_err"]
    assert abs(r["c"] - sigma ** 2 / (N * T * T)) < 4 * r["c_err"]
    # |M| of an isotropic 3D Gaussian: Maxwell law, <|M|> = 2 sm sqrt(2/pi), var = sm^2 (3 - 8/pi)
    assert abs(r["m"] - 2 * sm * math.sqrt(2 / math.pi) / N) < 4 * r["m_err"]
    assert abs(r["chi"] - sm ** 2 * (3 - 8 / math.pi) / (N * T)) < 4 * r["chi_err"]
    assert abs(r["u4"] - 4.0 / 9.0) < 4 * r["u4_err"]
    assert abs(r["tau_e"] - 0.5) < 0.2 and abs(r["tau_m"] - 0.5) < 0.2
    assert r["n"] == 19000 and r["bins"] == 20
    # error bars against the spread of independent repetitions
    for k in ("e", "c", "chi", "u4"):
        spread = np.std([x[k] for x in reps], ddof=1)
        mean_err = np.mean([x[k + "_err"] for x in reps])
        assert 0.6 < mean_err / spread < 1.6, (k, mean_err, spread)


def test_tau_of_ar1_series():
    rng = np.random.default_rng(2)
    for phi in (0.5, 0.8):
        n = 400000
        x = np.empty(n)
        x[0] = rng.normal()
        xi = rng.normal(size=n) * math.sqrt(1 - phi * phi)
        for i in range(1, n):
            x[i] = phi * x[i - 1] + xi[i]
        exact = (1 + phi) / (2 * (1 - phi))
        assert abs(analysis.tau_int(x) - exact) < 0.08 * exact, (phi, analysis.tau_int(x), exact)


def _ising_paramagnet_exact(N, beta, h, j):
    """<E>, <|M|^j>, <|M|^j E> for N independent Ising spins, E = -h M (binomial sums)."""
    k = np.arange(N + 1)
    M = 2.0 * k - N
    logw = special.gammaln(N + 1) - special.gammaln(k + 1) - special.gammaln(N - k + 1) + beta * h * M
    w = np.exp(logw - logw.max())
    w /= w.sum()
    E = -h * M
    Aj = np.abs(M) ** j
    return (w * E).sum(), (w * Aj).sum(), (w * Aj * E).sum()


def test_cumulants_v1_v2_of_independent_ising_spins():
    N, beta, h = 64, 0.4, 0.05
    rng = np.random.default_rng(3)
    n = 400000
    p = math.exp(beta * h) / (math.exp(beta * h) + math.exp(-beta * h))
    k = rng.binomial(N, p, n)
    M = 2.0 * k - N
    series = np.column_stack([-h * M, np.zeros(n), np.zeros(n), M])
    r = analysis.thermal_averages(series, 0, 20, 1.0 / beta, N)
    for j, key in ((1, "v1"), (2, "v2")):
        e, a, ae = _ising_paramagnet_exact(N, beta, h, j)
        exact = e - ae / a
        # the definition is the logarithmic derivative d ln<|M|^j> / d beta
        d = 1e-5
        fd = (math.log(_ising_paramagnet_exact(N, beta + d, h, j)[1]) -
              math.log(_ising_paramagnet_exact(N, beta - d, h, j)[1])) / (2 * d)
        assert abs(fd - exact) < 1e-6 * max(1.0, abs(exact))
        assert abs(r[key] - exact) < 0.03 * abs(exact), (key, r[key], exact)


def _langevin_samples(rng, n_conf, N, beta, B):
    """Exact Boltzmann samples of N free unit spins in a field B along z: returns E, Mz per
    configuration (cos theta by the inverse of its CDF, proportional to exp(beta B c))."""
    a = beta * B
    u = rng.random((n_conf, N))
    c = np.log(np.exp(-a) + u * (np.exp(a) - np.exp(-a))) / a
    Mz = c.sum(axis=1)
    return -B * Mz, Mz


def _langevin(x):
    return 1.0 / np.tanh(x) - 1.0 / x


def test_single_histogram_reweighting_of_free_spins():
    rng = np.random.default_rng(4)
    N, B, beta0 = 20, 1.0, 1.0
    E, Mz = _langevin_samples(rng, 200000, N, beta0, B)
    out, g, it = analysis.reweight(E[None, :], np.column_stack([E, Mz])[None], [beta0], [0.9, 1.0, 1.1])
    assert g.shape == (1,) and g[0] == 0.0
    for b, (e, m) in zip((0.9, 1.0, 1.1), out):
        assert abs(m - N * _langevin(b * B)) < 0.02, (b, m, N * _langevin(b * B))
        assert abs(e + N * B * _langevin(b * B)) < 0.02


def test_multiple_histogram_interpolation_and_free_energies():
    rng = np.random.default_rng(5)
    N, B = 10, 1.0
    betas = np.array([0.5, 0.8, 1.1, 1.4])
    runs = [_langevin_samples(rng, 100000, N, b, B) for b in betas]
    E = np.stack([r[0] for r in runs])
    O = np.stack([np.column_stack([r[0], r[1]]) for r in runs])
    mid = [0.65, 0.95, 1.25]
    out, g, it = analysis.reweight(E, O, betas, mid)
    assert it < 10000
    for b, (e, m) in zip(mid, out):
        assert abs(m - N * _langevin(b * B)) < 0.015, (b, m)
    # ln Z of N free spins: N ln(4 pi sinh(beta B) / (beta B))
    lnz = N * np.log(np.sinh(betas * B) / (betas * B))
    assert np.allclose(g, lnz - lnz[0], atol=0.02), (g, lnz - lnz[0])


def test_single_run_is_the_single_histogram_formula():
    rng = np.random.default_rng(6)
    E = rng.normal(-10.0, 2.0, 5000)
    O = rng.normal(size=(5000, 2))
    out, g, _ = analysis.reweight(E[None], O[None], [1.0], [1.3])
    w = np.exp(-0.3 * (E - E.min()))
    assert np.allclose(out[0], (w[:, None] * O).sum(axis=0) / w.sum(), rtol=1e-12, atol=1e-14)
