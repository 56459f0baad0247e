"""The statistics of the parity tests on series with known laws (CPU).

chain_observables follows the thermal averages of Sec. IV.A with binned and jackknife
errors; here its values and errors are checked on independent Gaussian records, where the
mean, the variance and the standard errors are known exactly, and the match criterion is
checked to accept equal laws and reject a shifted one."""

import numpy as np

from conftest import assert_statistically_equal, chain_observables, failing_observables


def gaussian_history(rng, chains, records, N, mu, sigma, mz):
    H = np.zeros((chains, records, 4))
    H[:, :, 0] = N * rng.normal(mu, sigma, size=(chains, records))
    H[:, :, 3] = N * rng.normal(mz, sigma, size=(chains, records))
    return H


def test_values_and_errors_of_independent_records():
    rng = np.random.default_rng(5)
    chains, records, N, T, mu, sigma = 4, 20000, 100, 2.0, -1.5, 0.2
    H = gaussian_history(rng, chains, records, N, mu, sigma, 0.8)
    o = chain_observables(H, N, T)
    used = chains * (records - records // 5)
    assert abs(o["e"][0] - mu) < 4 * sigma / np.sqrt(used)
    assert 0.6 < o["e"][1] / (sigma / np.sqrt(used)) < 1.6
    assert abs(o["m"][0] - 0.8) < 4 * sigma / np.sqrt(used)
    # C_v = N var(e) / T^2, chi = N var(|m|) / T (|m| = m here: m stays far from 0)
    assert abs(o["cv"][0] - N * sigma ** 2 / T ** 2) < 5 * o["cv"][1]
    assert abs(o["chi"][0] - N * sigma ** 2 / T) < 5 * o["chi"][1]
    # var(s^2) = 2 sigma^4 for a Gaussian: error of the variance over `used` records
    se_var = np.sqrt(2.0 / used) * sigma ** 2
    assert 0.5 < o["cv"][1] / (N * se_var / T ** 2) < 2.0


def test_between_chain_spread_counts_when_chains_disagree():
    """Chains that sit at different values (still relaxing) have a small within-chain error
    but a large spread; the error of the average must reflect the spread."""
    rng = np.random.default_rng(6)
    H = np.concatenate([gaussian_history(rng, 1, 4000, 10, mu, 0.01, 0.5) for mu in (-1.0, -0.8, -1.2, -0.9)])
    o = chain_observables(H, 10, 1.0)
    assert o["e"][1] > 0.05


def test_match_criterion_accepts_equal_laws_and_rejects_a_shift():
    rng = np.random.default_rng(7)
    N, T = 50, 1.5

    def pair(shift):
        a = chain_observables(gaussian_history(rng, 4, 5000, N, -1.0, 0.1, 0.6), N, T)
        b = chain_observables(gaussian_history(rng, 4, 5000, N, -1.0 + shift, 0.1, 0.6), N, T)
        return a, b

    fails = sum(bool(failing_observables(*pair(0.0))) for _ in range(40))
    assert fails <= 3  # 4 observables x 0.27% x 40 ~ 0.4 expected
    assert failing_observables(*pair(0.01)) == ["e"]
    calls = []

    def run(attempt):
        calls.append(attempt)
        return [pair(0.0)]

    assert_statistically_equal(run)
    assert calls[0] == 0 and len(calls) <= 2
