"""Pins of the oracle's per-phase and per-step outputs (Sec. II) to facts outside itself (no GPU).

  per-type M      the types' magnetizations add up to the total of the history; each equals
                  numpy's sum over that type's sites of the step's final state; sites of an
                  untracked type are left out; two decoupled phases with field axes z and x
                  each follow the Langevin law along their own axis
  snapshots       the last step's snapshot is the final state; the snapshot of step k is the
                  final state of a run of the first k + 1 steps
"""

import numpy as np

from conftest import binned

import oracle
from lattices import core_shell_particle, free_spins

from test_oracle_pins import langevin


def _core_shell():
    return core_shell_particle(seed=3, radius=4.5, core_radius=3.0)


def test_type_magnetizations_add_up_and_match_the_final_states():
    s = _core_shell()
    T = np.array([[1.5, 0.7, 0.3]])
    B = np.array([[0.2, 0.5, -0.4]])
    mcs = 6
    r = oracle.run(s, T, B, mcs, seed=4, n_types=2, snapshots=True)
    th, h, snaps = r["type_history"][0], r["history"][0], r["snapshots"][0]
    n = s.n_sites
    assert th.shape == (3 * mcs, 2, 3)
    assert np.allclose(th.sum(axis=1), h[:, 1:], rtol=0, atol=1e-12 * n)
    for k in range(3):
        S = snaps[k]
        for ty in range(2):
            want = S[s.type == ty].sum(axis=0)
            # the record precedes the step's renormalisation by one rounding per spin
            assert np.allclose(th[(k + 1) * mcs - 1, ty], want, rtol=0, atol=1e-12 * n)


def test_untracked_types_are_left_out():
    s = _core_shell()
    r = oracle.run(s, [[0.9]], [[0.1]], 3, seed=5, n_types=1, snapshots=True)
    S = r["snapshots"][0, 0]
    assert np.allclose(r["type_history"][0, -1, 0], S[s.type == 0].sum(axis=0), atol=1e-12 * s.n_sites)
    assert not np.allclose(r["type_history"][0, -1, 0], r["history"][0, -1, 1:], atol=1e-6)


def test_two_phases_follow_their_own_field_axes():
    n, B, T = 4000, 1.2, 1.0
    axis = np.zeros((n, 3))
    typ = (np.arange(n) % 2).astype(np.int32)
    axis[typ == 0, 2] = 1.0
    axis[typ == 1, 0] = 1.0
    s = free_spins(n)
    s.field_axis = axis
    s.type = typ
    mcs = 300
    r = oracle.run(s, [[T]], [[B]], mcs, seed=6, n_types=2)
    th = r["type_history"][0, mcs // 5:] / (n / 2)
    for ty, along, across in ((0, 2, 0), (1, 0, 2)):
        m, se = binned(th[:, ty, along])
        assert abs(m - langevin(B / T)) < 4 * se + 1e-4, (ty, m, se)
        c, sc = binned(th[:, ty, across])
        assert abs(c) < 4 * sc + 1e-4, (ty, c, sc)


def test_snapshots_are_the_final_states_per_step():
    s = _core_shell()
    T = np.array([[2.0, 1.0, 0.5, 0.25]])
    B = np.array([[0.0, 0.3, 0.6, 0.9]])
    mcs = 5
    full = oracle.run(s, T, B, mcs, seed=7, snapshots=True)
    assert np.array_equal(full["snapshots"][0, -1], full["spins"][0])
    for k in range(3):
        part = oracle.run(s, T[:, :k + 1], B[:, :k + 1], mcs, seed=7)
        assert np.array_equal(full["snapshots"][0, k], part["spins"][0]), k
