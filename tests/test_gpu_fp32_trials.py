"""The FP32 attempt's random trial and acceptance against their exact laws (Sec. III.B, Eq. 4).

The FP32 path draws the uniform-on-the-sphere trial from two 23-bit uniforms through the
SFU's sine/cosine and reciprocal square root, and decides with the SFU exponential against
a 32-bit uniform. Their error bounds (stated with the kernels) make the bias of the
stationary law far smaller than any statistical test can see; these tests check that no
larger mistake hides there:

- free spins at B = 0: every energy change is 0, so every trial is accepted and the spins
  are the trials; their z and azimuth are uniform (Kolmogorov-Smirnov on 10^6 trials), the
  moments <S_a> = 0 and <S_a S_b> = delta_ab / 3 hold, and |S| = 1 to FP32 rounding;
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
