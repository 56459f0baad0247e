"""Pins of the oracle's Ising model (spin-flip policy, Sec. II) to facts outside itself (no GPU).

  4x4 lattice        exact <E> and <|M|> by enumerating all 2^16 states; the energy histogram
                     against the exact Boltzmann law (chi^2)
  paramagnet         J = 0: <M>/N = tanh(beta h)
  2D, L = 64         Onsager's energy per site above and below T_c and Yang's spontaneous
                     magnetization below it
  3D                 the same physics as the Heisenberg oracle's spin-flip policy on z-aligned
                     spins (an independently pinned function)
  continuation       a run split in two equals the whole run bit for bit
"""

import itertools
import math

import numpy as np
from scipy import special, stats

from conftest import binned

import oracle
from lattices import sc_periodic

from test_oracle_pins import pooled


def _exact_4x4(J, h, T):
    L = 4
    states = np.array(list(itertools.product((-1, 1), repeat=L * L)), dtype=np.int64).reshape(-1, L, L)
    bonds = (states * np.roll(states, -1, axis=2)).sum(axis=(1, 2)) + (states * np.roll(states, -1, axis=1)).sum(axis=(1, 2))
    M = states.sum(axis=(1, 2))
    E = -J * bonds - h * M
    w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    return E, M, w


def test_four_by_four_exact_averages():
    J, h, T = 1.0, 0.1, 2.5
    E, M, w = _exact_4x4(J, h, T)
    R = 16
    r = oracle.ising_run(2, 4, J, np.full((R, 1), T), np.full((R, 1), h), 20000, seed=3)
    e, se = pooled(r["history"][:, :, 0])
    m, sm = pooled(np.abs(r["history"][:, :, 1]))
    assert abs(e - (w * E).sum()) < 4 * se, (e, se, (w * E).sum())
    assert abs(m - (w * np.abs(M)).sum()) < 4 * sm, (m, sm, (w * np.abs(M)).sum())


def test_four_by_four_energy_histogram():
    J, h, T = 1.0, -0.2, 3.0
    E, M, w = _exact_4x4(J, h, T)
    levels = np.unique(np.round(E, 9))
    p = np.array([w[np.isclose(E, v)].sum() for v in levels])
    R = 64
    r = oracle.ising_run(2, 4, J, np.full((R, 1), T), np.full((R, 1), h), 3000, seed=4)
    samples = r["history"][:, 500::25, 0].ravel()  # thinned: nearly independent draws
    obs = np.array([np.isclose(samples, v).sum() for v in levels])
    assert obs.sum() == samples.size
    keep = samples.size * p > 5
    exp_ = samples.size * p[keep]
    chi2 = float((((obs[keep] - exp_) ** 2) / exp_).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-4, keep.sum() - 1), chi2


def test_paramagnet_tanh_law():
    L, T, h = 32, 1.5, 0.4
    r = oracle.ising_run(2, L, 0.0, [[T]], [[h]], 2000, seed=5)
    m, se = binned(r["history"][0, :, 1] / L ** 2)
    assert abs(m - math.tanh(h / T)) < 4 * se + 1e-4, (m, se)
    assert np.allclose(r["history"][0, :, 0], -h * r["history"][0, :, 1])


def _onsager_energy(T, J=1.0):
    K = J / T
    kappa = 2.0 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    K1 = special.ellipk(kappa * kappa)
    return -J / math.tanh(2 * K) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * K) ** 2 - 1.0) * K1)


def test_onsager_energy_and_spontaneous_magnetization():
    L, R = 64, 4
    for T in (1.8, 3.0):
        start = np.ones((R, L * L), dtype=np.int8) if T < 2.269 else None
        r = oracle.ising_run(2, L, 1.0, np.full((R, 1), T), np.zeros((R, 1)), 3000, seed=6, spins=start)
        e, se = pooled(r["history"][:, :, 0] / L ** 2)
        assert abs(e - _onsager_energy(T)) < 4 * se + 2e-3, (T, e, se, _onsager_energy(T))
        if T < 2.269:
            m, sm = pooled(np.abs(r["history"][:, :, 1]) / L ** 2)
            exact = (1.0 - math.sinh(2.0 / T) ** -4) ** 0.125
            assert abs(m - exact) < 4 * sm + 2e-3, (m, sm, exact)


def test_three_dimensional_ising_equals_heisenberg_spin_flip():
    L, T, R, mcs = 6, 4.0, 8, 4000
    r = oracle.ising_run(3, L, 1.0, np.full((R, 1), T), np.zeros((R, 1)), mcs, seed=7)
    s = sc_periodic(L).with_policy([oracle.SPIN_FLIP], [0.0])
    rng = np.random.default_rng(8)
    S0 = np.zeros((R, L ** 3, 3))
    S0[:, :, 2] = rng.choice([-1.0, 1.0], size=(R, L ** 3))
    q = oracle.run(s, np.full((R, 1), T), np.zeros((R, 1)), mcs, seed=9, spins=S0, n_threads=R)
    a, sa = pooled(r["history"][:, :, 0] / L ** 3)
    b, sb = pooled(q["history"][:, :, 0] / L ** 3)
    assert abs(a - b) < 4 * math.hypot(sa, sb), (a, sa, b, sb)
    a, sa = pooled(np.abs(r["history"][:, :, 1]) / L ** 3)
    b, sb = pooled(np.abs(q["history"][:, :, 3]) / L ** 3)
    assert abs(a - b) < 4 * math.hypot(sa, sb), (a, sa, b, sb)


def test_ising_continuation_bitwise():
    T = np.array([[2.6, 2.2], [1.9, 1.5]])
    h = np.array([[0.1, -0.1], [0.0, 0.3]])
    full = oracle.ising_run(2, 8, 1.0, T, h, 7, seed=10, inst_base=4)
    a = oracle.ising_run(2, 8, 1.0, T[:, :1], h[:, :1], 7, seed=10, inst_base=4)
    b = oracle.ising_run(2, 8, 1.0, T[:, 1:], h[:, 1:], 7, seed=10, inst_base=4, spins=a["spins"], t0=7)
    assert np.array_equal(full["spins"], b["spins"])
    assert np.array_equal(full["history"], np.concatenate([a["history"], b["history"]], axis=1))
