"""The FP32 attempt's random trial and acceptance against their exact laws (Sec. III.B, Eq. 4).

The FP32 path draws the uniform-on-the-sphere trial from two 23-bit uniforms through the
SFU's sine/cosine and reciprocal square root, and decides with the SFU exponential against
a 32-bit uniform. Their error bounds (stated with the kernels) make the bias of the
stationary law far smaller than any statistical test can see; these tests check that no
larger mistake hides there:

- free spins at B = 0: every energy change is 0, so every trial is accepted and the spins
  are the trials; their z and azimuth are uniform (Kolmogorov-Smirnov on 10^6 trials), the
  moments <S_a> = 0 and <S_a S_b> = delta_ab / 3 hold, and |S| = 1 to FP32 rounding;
- the end-of-step renormalisation rounds like the FP64 formula s S/|S|;
- spin-1/2 free spins (the qIsing policy) in a field: the trial is always the other value,
  so the stationary law is set by the acceptance probability exp(-beta dE) alone,
  <S_z> = tanh(beta B / 2) / 2, checked to about 1e-4.
"""

import numpy as np
import pytest

from conftest import binned

import oracle
import paper_1803_07030_gb300 as vg
from lattices import free_spins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    vg.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_random_trials_are_uniform_on_the_sphere():
    from scipy import stats

    n, R, rounds = 31250, 4, 8  # 10^6 trials
    with vg.Context([free_spins(n)], precision=32, replicas=R, seed=77, stream=None) as c:
        S = []
        for _ in range(rounds):
            c.run(np.ones((R, 1)), np.zeros((R, 1)), 1)  # B = 0: every trial accepted
            S.extend(c.spins(i) for i in range(R))
        acc = c.accept_history()
    assert np.all(acc == n)  # every attempt accepted: the spins are the trials
    S = np.concatenate(S)
    assert S.shape == (n * R * rounds, 3)
    r = np.linalg.norm(S, axis=1)
    assert np.max(np.abs(r - 1.0)) < 1e-6  # FP32 rounding (the renormalisation leaves ~1 ulp)
    z = S[:, 2] / r
    phi = np.arctan2(S[:, 1], S[:, 0])
    assert stats.kstest(z, "uniform", args=(-1.0, 2.0)).pvalue > 1e-4
    assert stats.kstest(phi, "uniform", args=(-np.pi, 2.0 * np.pi)).pvalue > 1e-4
    m = S.shape[0]
    mean = S.mean(axis=0)
    assert np.all(np.abs(mean) < 4.0 * np.sqrt(1.0 / 3.0 / m))
    cov = S.T @ S / m
    # var(S_a^2) = 1/5 - 1/9 = 4/45, var(S_a S_b) = 1/15 for a uniform unit vector
    assert np.all(np.abs(np.diag(cov) - 1.0 / 3.0) < 4.0 * np.sqrt(4.0 / 45.0 / m))
    off = cov[~np.eye(3, dtype=bool)]
    assert np.all(np.abs(off) < 4.0 * np.sqrt(1.0 / 15.0 / m))


@pytest.mark.parametrize("beta_B", [1.0, 3.0])
def test_acceptance_probability_sets_the_two_state_law(beta_B):
    n, mcs, T = 100000, 1200, 1.0
    fs = free_spins(n, spin_norm=0.5).with_policy([oracle.QISING], [0.0])
    with vg.Context([fs], precision=32, seed=78, stream=None) as c:
        c.run([[T]], [[beta_B * T]], mcs)
        H = c.history()[0]
    got, se = binned(H[:, 3] / n)
    exact = 0.5 * np.tanh(beta_B / 2.0)
    assert abs(got - exact) < 4.0 * se + 2e-6, (got, se, exact)
    assert se < 2e-4


@pytest.mark.parametrize("norm", [1.0, 2.0])
def test_fp32_renormalisation_rounds_like_the_fp64_formula(norm):
    """The end-of-step renormalisation of FP32 spins (S <- s S/|S|, |S|^2 - 1 from FP32 products
    and sums with their exact errors, the FP64 formula off the series' range) against
    the FP64 formula evaluated on the host and rounded to FP32, for spins whose norm is off by
    up to 1e-7 (what Metropolis steps leave) and 1e-5 (the series' range), 2^-11, 0.5 and 2
    (the direct formula), with spin norms s = 1 and 2. A ferromagnet held at T = 1e-6 rejects every
    move, so only the renormalisation changes the spins (the accept log confirms it)."""
    from lattices import sc_periodic

    s = sc_periodic(8)
    n = s.n_sites
    s.spin_norm = np.full(n, norm)
    rng = np.random.default_rng(5)
    # |S| / s - 1 up to these: spins longer than s, so that no unit trial lowers the energy
    cases = [1e-7, 1e-5, 2.0 ** -11, 0.5, 2.0]
    R = 8  # the five cases, then unperturbed spins
    starts = []
    for k in range(R):
        d = np.tile([0.0, 0.0, 1.0], (n, 1)) + rng.normal(0.0, 1e-4, size=(n, 3))
        d *= norm / np.linalg.norm(d, axis=1)[:, None]
        if k < len(cases):
            d *= 1.0 + cases[k] * rng.uniform(0.0, 1.0, size=(n, 1))
        starts.append(d)
    with vg.Context([s], precision=32, replicas=R, seed=79, accept_log_mcs=1, stream=None) as c:
        for k in range(R):
            c.set_spins(k, starts[k])
        got0 = [c.spins(k) for k in range(R)]  # the FP32 values the kernels hold
        c.run(np.full((R, 1), 1e-6), np.full((R, 1), 0.5), 1)
        assert not c.accept_log().any()
        got = [c.spins(k) for k in range(R)]
    for k in range(R):
        v = got0[k].astype(np.float32).astype(np.float64)
        f = norm / np.sqrt((v * v).sum(axis=1))
        want = (v * f[:, None]).astype(np.float32)
        exact = np.mean(got[k].astype(np.float32) == want)
        ulps = np.abs(got[k].astype(np.float32).view(np.int32) - want.view(np.int32))
        assert exact > 0.9999 and ulps.max() <= 1, (k, exact, ulps.max())
