"""Pins of the oracle's update policies (Sec. II; Sec. IV.C) to facts outside itself (no GPU).

  logarithm        the oracle's own atanh-series ln against libm, within 4 ulp
  small step       trials are unit vectors inside the cap; cos(angle) uniform on
                   [cos theta, 1] and the azimuth uniform in a frame built here (KS)
  Gaussian         for a tiny width the three offsets are independent standard normals
                   (KS, moments); for a huge width the trial is uniform on the sphere (iid
                   normals); for a finite width the angle to S follows the projected normal
                   density (quadrature, chi^2)
  spin flip        the trial is -S; a free spin flipped in a field has <S_z> = tanh(beta B);
                   flips on z-aligned spins of an open chain give the Ising chain's
                   U = -(N-1) J tanh(beta J)
  Hinzke-Nowak     a third of the trials are flips, a third uniform, a third in the cap
  equilibrium      every policy reaches the same Boltzmann law: Langevin law, uniaxial and
                   cubic quadratures, dimer bond-angle histogram (chi^2)
  adaptive         the acceptance rate settles at 1/2; the width follows the control law
                   from the recorded acceptance counts and stays frozen after the first
                   fifth of the step; the frozen part samples the Langevin law; in the
                   ordered phase its energy decorrelates several times faster than under
                   uniform trials (the efficiency the paper reports for it, Sec. IV.C)
  table            an all-random table gives the caller bit-identical chains; per-type
                   policies apply per site type
"""

import math

import numpy as np
import pytest
from scipy import integrate, special, stats

from conftest import binned

import oracle
from lattices import chain_open, core_shell_particle, dimers, free_spins, sc_periodic
from oracle.analysis import tau_int

from test_oracle_pins import langevin, sphere_grid


def _one_site(policy, param):
    return free_spins(1).with_policy([policy], [param])


def _trials(policy, param, S, count, sigma=0.0, seed=11):
    s = _one_site(policy, param)
    out = np.zeros((count, 3))
    for t in range(count):
        out[t], err = oracle.trial(s, np.asarray(S, dtype=np.float64)[None, :], 0, seed, t, 3, sigma)
        assert err == 0
    return out


def _frame(u):
    """An orthonormal pair perpendicular to u, by Gram-Schmidt on a fixed vector."""
    a = np.array([0.3, -0.7, 0.64])
    e1 = a - (a @ u) * u
    e1 /= np.linalg.norm(e1)
    return e1, np.cross(u, e1)


# --------------------------------------------------------------------------- logarithm

def test_log_series_matches_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([10.0 ** rng.uniform(-300, 300, 4000), rng.uniform(0.0, 1.0, 4000) + 1e-300,
                         1.0 + rng.uniform(-1e-3, 1e-3, 1000), [1.0, 2.0, 0.5, 1.4142135623730951, 0.7071067811865476]])
    for x in xs:
        got, want = oracle.log(x), math.log(x)
        assert abs(got - want) <= 4 * np.spacing(abs(want)) + 1e-300, (x, got, want)
    assert oracle.log(1.0) == 0.0


# --------------------------------------------------------------------------- trial generators

@pytest.mark.parametrize("theta", [0.2, 1.0, np.pi])
def test_small_step_uniform_in_cap(theta):
    S = np.array([0.8, -1.1, 1.9])  # not unit: the policy uses the direction only
    u = S / np.linalg.norm(S)
    v = _trials(oracle.SMALL_STEP, theta, S, 6000)
    assert np.all(np.abs(np.linalg.norm(v, axis=1) - 1.0) < 1e-14)
    c = v @ u
    ct = math.cos(theta)
    assert np.all(c >= ct - 1e-12)
    assert stats.kstest(c, stats.uniform(loc=ct, scale=1.0 - ct).cdf).pvalue > 1e-3
    e1, e2 = _frame(u)
    phi = np.arctan2(v @ e2, v @ e1)
    assert stats.kstest(phi, stats.uniform(loc=-np.pi, scale=2 * np.pi).cdf).pvalue > 1e-3


def test_gaussian_offsets_are_standard_normals():
    sigma = 1e-5
    g = []
    for S, (i, j, k) in (([0.0, 0.0, 2.0], (0, 1, 2)), ([1.0, 0.0, 0.0], (1, 2, 0))):
        v = _trials(oracle.GAUSSIAN, sigma, S, 5000, seed=12)
        g.append(v[:, i] / v[:, k] / sigma)
        g.append(v[:, j] / v[:, k] / sigma)
    # offsets 0, 1 (first pair, S = z) and 1, 2 (S = x): the second pair's first normal
    for x in g:
        assert abs(x.mean()) < 5 / np.sqrt(len(x))
        assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / len(x))
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(g[0], g[1])[0, 1]) < 5 / np.sqrt(len(g[0]))


def test_gaussian_wide_is_uniform():
    """sigma -> infinity: the trial is the direction of three iid normals, uniform on the sphere."""
    v = _trials(oracle.GAUSSIAN, 1e8, [1.0, 0.0, 0.0], 6000, seed=15)
    for q in range(3):
        assert stats.kstest(v[:, q], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    c = np.corrcoef(v.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 5 / np.sqrt(len(v)))
    phi = np.arctan2(v[:, 1], v[:, 0])
    assert stats.kstest(phi, stats.uniform(loc=-np.pi, scale=2 * np.pi).cdf).pvalue > 1e-3


def test_gaussian_projected_normal_angle():
    sigma = 0.7
    S = np.array([0.0, 0.6, 0.8])
    v = _trials(oracle.GAUSSIAN, sigma, S, 8000, seed=13)
    c = v @ S
    # direction of S + sigma g: density of c = cos(angle) proportional to
    # int_0^inf r^2 exp(-(r^2 - 2 r c + 1) / (2 sigma^2)) dr
    def dens(x):
        return integrate.quad(lambda r: r * r * np.exp(-(r * r - 2 * r * x + 1) / (2 * sigma ** 2)), 0, np.inf)[0]

    edges = np.linspace(-1, 1, 21)
    p = np.array([integrate.quad(dens, a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    p /= p.sum()
    obs, _ = np.histogram(c, bins=edges)
    n = len(c)
    keep = n * p > 5
    chi2 = float(((obs[keep] - n * p[keep]) ** 2 / (n * p[keep])).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-4, keep.sum() - 1), chi2


def test_spin_flip_trial_is_minus_s():
    S = np.array([0.36, -0.48, 0.8])  # unit norm, the default spin norm
    v = _trials(oracle.SPIN_FLIP, 0.0, S, 5)
    assert np.array_equal(v, np.tile(-S / 1.0, (5, 1)))


def test_hinzke_nowak_mixture():
    theta = 0.4
    S = np.array([0.0, 0.0, 1.0])
    n = 9000
    v = _trials(oracle.HINZKE_NOWAK, theta, S, n, seed=14)
    flip = np.all(v == -S, axis=1)
    incap = (v @ S >= math.cos(theta)) & ~flip
    p_flip, p_cap = 1 / 3, 1 / 3 + (1 / 3) * (1 - math.cos(theta)) / 2
    for k, p in ((flip.sum(), p_flip), (incap.sum(), p_cap)):
        assert abs(k - n * p) < 5 * math.sqrt(n * p * (1 - p)), (k, n * p)
    rest = v[~flip & ~incap] @ S  # the uniform third outside the cap: cos uniform on [-1, cos theta)
    assert stats.kstest(rest, stats.uniform(loc=-1, scale=1 + math.cos(theta)).cdf).pvalue > 1e-3


# --------------------------------------------------------------------------- chains

def test_flip_free_spin_in_field():
    n, B, T = 3000, 0.7, 1.0
    s = free_spins(n).with_policy([oracle.SPIN_FLIP], [0.0])
    up = np.tile([0.0, 0.0, 1.0], (1, n, 1))
    r = oracle.run(s, [[T]], [[B]], 300, seed=15, spins=up)
    m, se = binned(r["history"][0, :, 3] / n)
    assert abs(m - math.tanh(B / T)) < 4 * se + 1e-4, (m, se)
    assert np.allclose(np.abs(r["spins"][0][:, 2]), 1.0, atol=1e-15)


@pytest.mark.parametrize("J", [1.0, -1.0])
def test_flip_ising_chain(J):
    N, T = 2000, 1.5
    s = chain_open(N, J=J).with_policy([oracle.SPIN_FLIP], [0.0])
    up = np.tile([0.0, 0.0, 1.0], (1, N, 1))
    r = oracle.run(s, [[T]], [[0.0]], 400, seed=16, spins=up)
    m, se = binned(r["history"][0, :, 0])
    U = -(N - 1) * J * math.tanh(J / T)
    assert abs(m - U) < 4 * se + 1e-6, (m, se, U)


POLICIES = [(oracle.SMALL_STEP, 0.5), (oracle.GAUSSIAN, 0.4), (oracle.HINZKE_NOWAK, 0.3), (oracle.ADAPTIVE, 1.0)]


@pytest.mark.parametrize("policy,param", POLICIES)
def test_policy_langevin_law(policy, param):
    n, B, T = 3000, 1.5, 1.0
    s = free_spins(n).with_policy([policy], [param])
    mcs = 500
    r = oracle.run(s, [[T]], [[B]], mcs, seed=17)
    assert r["err"] == 0
    m, se = binned(r["history"][0, mcs // 5:, 3] / n)
    assert abs(m - langevin(B / T)) < 4 * se + 1e-4, (m, se, langevin(B / T))


@pytest.mark.parametrize("policy,param", POLICIES)
def test_policy_uniaxial(policy, param):
    n, T, k = 3000, 1.0, 2.0
    e = np.array([0.0, 1.0, 1.0]) / np.sqrt(2.0)
    s = free_spins(n, k_uni=k, e_uni=e).with_policy([policy], [param])
    mcs = 500
    r = oracle.run(s, [[T]], [[0.0]], mcs, seed=18)
    m, se = binned(-r["history"][0, mcs // 5:, 0] / (k * n))
    a = k / T
    exact = np.exp(a) / (np.sqrt(np.pi * a) * special.erfi(np.sqrt(a))) - 1.0 / (2.0 * a)
    assert abs(m - exact) < 4 * se + 1e-5, (m, se, exact)


@pytest.mark.parametrize("policy,param", [(oracle.HINZKE_NOWAK, 0.5), (oracle.GAUSSIAN, 0.5)])
def test_policy_cubic(policy, param):
    n, T, kc = 3000, 0.8, -2.5
    s = free_spins(n, k_cub=kc).with_policy([policy], [param])
    r = oracle.run(s, [[T]], [[0.0]], 500, seed=19)
    m, se = binned(r["history"][0, 100:, 0] / n)
    v, w = sphere_grid(64, 96)
    x2, y2, z2 = (v ** 2).T
    cub = x2 * y2 + y2 * z2 + x2 * z2
    bw = w * np.exp(kc * cub / T)
    exact = -kc * np.sum(bw * cub) / np.sum(bw)
    assert abs(m - exact) < 4 * se + 1e-5, (m, se, exact)


@pytest.mark.parametrize("policy,param", [(oracle.SMALL_STEP, 0.6), (oracle.GAUSSIAN, 0.5),
                                          (oracle.HINZKE_NOWAK, 0.3)])
def test_policy_detailed_balance_dimer(policy, param):
    P, J, T = 20000, 1.0, 0.5
    s = dimers(P, J=J).with_policy([policy], [param])
    r = oracle.run(s, [[T]], [[0.0]], 300, seed=20)
    S = r["spins"][0]
    c = np.einsum("ij,ij->i", S[0::2], S[1::2])
    K = J / T
    edges = np.linspace(-1, 1, 21)
    obs, _ = np.histogram(c, bins=edges)
    p = (np.exp(K * edges[1:]) - np.exp(K * edges[:-1])) / (np.exp(K) - np.exp(-K))
    chi2 = float(((obs - P * p) ** 2 / (P * p)).sum())
    assert chi2 < stats.chi2.ppf(1 - 1e-4, 19), chi2


def test_adaptive_acceptance_and_control_law():
    n, B, T = 4000, 8.0, 1.0  # beta B = 8: uniform trials are accepted about 1 time in 8
    s = free_spins(n).with_policy([oracle.ADAPTIVE], [2.0])
    mcs = 200
    up = np.tile([0.0, 0.0, 1.0], (1, n, 1))  # start in equilibrium-like order
    r = oracle.run(s, [[T]], [[B]], mcs, seed=21, spins=up)
    acc = r["accepted"][0]
    rate = acc / n
    assert rate[0] < 0.3  # the starting width is far from the target
    assert abs(rate[mcs // 5:].mean() - 0.5) < 0.05, rate[mcs // 5:].mean()
    # the width: every factor 0.5 / max(1 - R, 0.01) of the first fifth, clamped, then frozen
    sg = 2.0
    for m in range(mcs // 5):
        sg = min(max(sg * (0.5 / max(1.0 - acc[m] / n, 0.01)), 1e-4), 100.0)
    assert r["sigma"][0] == sg
    m, se = binned(r["history"][0, mcs // 5:, 3] / n)
    assert abs(m - langevin(B / T)) < 4 * se + 1e-4, (m, se)
    # random policy at the same temperature: acceptance far below 1/2
    r0 = oracle.run(free_spins(n), [[T]], [[B]], 20, seed=21, spins=up)
    assert r0["accepted"][0].mean() / n < 0.25


def test_adaptive_policy_shortens_the_energy_autocorrelation():
    """6^3 ferromagnet at T = 0.3 (ordered; T_c is about 1.44), four replicas started aligned:
    uniform trials are accepted about 5% of the time and the energy's integrated
    autocorrelation time is tens of MCS; the adaptive width holds the acceptance near 1/2 and
    the time falls by more than half (Sec. IV.C: the adaptive policy is the efficient one)."""
    R, mcs, cut = 4, 4000, 800
    up = np.tile([0.0, 0.0, 1.0], (R, 216, 1))
    out = {}
    for name, pol, par in (("random", oracle.RANDOM, 0.0), ("adaptive", oracle.ADAPTIVE, 0.5)):
        s = sc_periodic(6).with_policy([pol], [par])
        r = oracle.run(s, np.full((R, 1), 0.3), np.zeros((R, 1)), mcs, seed=31, spins=up, n_threads=R)
        taus = [tau_int(e) for e in r["history"][:, cut:, 0]]
        out[name] = (float(np.mean(taus)), r["accepted"][:, cut:].mean() / s.n_sites)
    (tau_r, acc_r), (tau_a, acc_a) = out["random"], out["adaptive"]
    assert acc_r < 0.1 and abs(acc_a - 0.5) < 0.05, out
    assert tau_a < 0.5 * tau_r, out


def test_adaptive_width_frozen_then_continued():
    """Two calls: the second starts from the first's width and adapts again (a new step)."""
    n = 500
    s = free_spins(n).with_policy([oracle.ADAPTIVE], [1.0])
    a = oracle.run(s, [[0.5, 0.5]], [[2.0, 2.0]], 10, seed=22)
    b1 = oracle.run(s, [[0.5]], [[2.0]], 10, seed=22)
    b2 = oracle.run(s, [[0.5]], [[2.0]], 10, seed=22, spins=b1["spins"], t0=10, sigma=b1["sigma"])
    assert np.array_equal(a["spins"], b2["spins"])
    assert a["sigma"][0] == b2["sigma"][0]
    assert np.array_equal(a["accepted"][0], np.concatenate([b1["accepted"][0], b2["accepted"][0]]))


def test_all_random_table_is_the_default_chain():
    s = core_shell_particle(seed=2, radius=4.0, core_radius=2.5)
    a = oracle.run(s, [[0.9]], [[0.3]], 20, seed=23)
    s.with_policy([oracle.RANDOM, oracle.RANDOM], [0.0, 0.0])
    b = oracle.run(s, [[0.9]], [[0.3]], 20, seed=23)
    assert np.array_equal(a["spins"], b["spins"]) and np.array_equal(a["accepted"], b["accepted"])


def test_per_type_policies_apply_per_type():
    """Core random, shell spin flip: every shell spin stays on its initial axis."""
    s = core_shell_particle(seed=2, radius=4.0, core_radius=2.5)
    s.with_policy([oracle.RANDOM, oracle.SPIN_FLIP], [0.0, 0.0])
    S0 = oracle.init_spins(s, 24, 0)
    r = oracle.run(s, [[0.9]], [[0.3]], 50, seed=24)
    S = r["spins"][0]
    shell = s.type == 1
    cosang = np.einsum("ij,ij->i", S, S0) / (np.linalg.norm(S, axis=1) * np.linalg.norm(S0, axis=1))
    assert np.all(np.abs(np.abs(cosang[shell]) - 1.0) < 1e-12)
    assert np.mean(np.abs(cosang[~shell]) < 0.99) > 0.5  # the core moved
    assert np.any(cosang[shell] < 0) and np.any(cosang[shell] > 0)


# --------------------------------------------------------------------------- qIsing (mixed spin Ising)

def _qising_free(n, s, B=0.0, k=0.0):
    fs = free_spins(n, spin_norm=s, k_uni=k, e_uni=(0.0, 0.0, 1.0))
    return fs.with_policy([oracle.QISING], [0.0])


def _brillouin_like(s, beta, B, k):
    m = np.arange(-s, s + 0.5, 1.0)
    w = np.exp(beta * (B * m + k * m * m))
    w /= w.sum()
    return m, w


def test_qising_values_stay_discrete_and_start_uniform():
    s = 1.5
    fs = _qising_free(6000, s)
    S0 = oracle.init_spins(fs, 31, 0)
    assert np.all(S0[:, :2] == 0.0)
    vals, counts = np.unique(S0[:, 2], return_counts=True)
    assert np.array_equal(vals, [-1.5, -0.5, 0.5, 1.5])
    assert stats.chisquare(counts).pvalue > 1e-3
    r = oracle.run(fs, [[1.0, 0.7]], [[0.3, -0.2]], 20, seed=31)
    S = r["spins"][0]
    assert np.all(S[:, :2] == 0.0) and set(np.unique(S[:, 2])) == {-1.5, -0.5, 0.5, 1.5}


@pytest.mark.parametrize("s,B,k", [(1.0, 0.6, 0.8), (1.5, 0.4, -0.3), (0.5, 1.0, 0.0)])
def test_qising_free_spins_boltzmann(s, B, k):
    n, T = 4000, 1.0
    fs = _qising_free(n, s, B, k)
    mcs = 300
    r = oracle.run(fs, [[T]], [[B]], mcs, seed=32)
    m, w = _brillouin_like(s, 1.0 / T, B, k)
    mean_m = (w * m).sum()
    got, se = binned(r["history"][0, :, 3] / n)
    assert abs(got - mean_m) < 4 * se + 1e-4, (got, se, mean_m)
    e_exact = -(B * mean_m + k * (w * m * m).sum())
    ge, see = binned(r["history"][0, :, 0] / n)
    assert abs(ge - e_exact) < 4 * see + 1e-4, (ge, see, e_exact)
    # detailed balance: the distribution of m over the final states
    obs = np.array([(r["spins"][0][:, 2] == v).sum() for v in m])
    assert stats.chisquare(obs, n * w).pvalue > 1e-4


def test_qising_half_spin_chain_is_the_ising_chain():
    N, T, J = 2000, 0.6, 1.0
    ch = chain_open(N, J=J)
    ch.spin_norm = np.full(N, 0.5)
    ch.with_policy([oracle.QISING], [0.0])
    r = oracle.run(ch, [[T]], [[0.0]], 400, seed=33)
    m, se = binned(r["history"][0, :, 0])
    U = -(N - 1) * (J / 4) * math.tanh(J / (4 * T))
    assert abs(m - U) < 4 * se + 1e-6, (m, se, U)
