"""The seeded synthetic inputs: the shapes of the five workloads and the properties of the
generated samples that the sweeps rely on (symmetric links, proper colourings).

These run on the CPU only; they check the generators, which hold none of the method's
arithmetic.
"""

import numpy as np
import pytest

import oracle
from lattices import core_shell_particle, fcc_sphere, nanoparticle_batch, sc_periodic, workload


def _sources(s):
    return np.repeat(np.arange(s.n_sites), np.diff(s.row_ptr))


def _assert_symmetric(s):
    src = _sources(s)
    fwd = {(int(i), int(j)): float(J) for i, j, J in zip(src, s.col, s.J)}
    for (i, j), J in fwd.items():
        assert fwd.get((j, i)) == J, (i, j)


@pytest.mark.parametrize("make", [
    lambda: fcc_sphere(4.3),
    lambda: fcc_sphere(3.0, a=4.0 ** (1.0 / 3.0), centre=(0.3, 0.1, 0.7)),
    lambda: core_shell_particle(seed=3, radius=6.0, core_radius=4.0),
    lambda: nanoparticle_batch(4, seed=5, r_max=7.0)[2],
])
def test_fcc_samples_carry_a_proper_four_colouring(make):
    """The sublattice colouring of an fcc sample: 4 classes, no link inside a class, and the
    greedy colouring of the same graph needs more."""
    s = make()
    c = np.asarray(s.colour)
    assert c.dtype == np.int32 and c.shape == (s.n_sites,)
    assert set(np.unique(c).tolist()) <= {0, 1, 2, 3} and len(np.unique(c)) == 4
    assert np.all(c[_sources(s)] != c[s.col])
    greedy, n_greedy = oracle.greedy_colour(s)
    assert n_greedy > 4
    _assert_symmetric(s)


def test_sc_lattices_are_two_coloured_and_symmetric():
    s = sc_periodic((6, 4, 8), bimodal_seed=2)
    _assert_symmetric(s)
    assert set(np.unique(s.J).tolist()) == {-1.0, 1.0}
    _, nc = oracle.greedy_colour(s)
    assert nc == 2


@pytest.mark.parametrize("name,n_inst,n_sites,steps,mcs,precision", [
    ("sc8_fp64", 1, 512, 30, 1000, 64),          # 8^3 ferromagnet, 30 temperatures
    ("sc64_hyst", 1, 262144, 161, 500, 32),      # 64^3 hysteresis, B 2 -> -2 -> 2 in 0.05 steps
    ("coreshell_fc", 1, None, 60, 2000, 32),     # fcc core/shell particle, 60 field-cooled steps
    ("np256", 256, None, 1, 5000, 32),           # 256 fcc particles, one step of 5000 MCS
])
def test_workload_shapes(name, n_inst, n_sites, steps, mcs, precision):
    w = workload(name)
    assert w.n_inst == n_inst and w.T.shape == (n_inst, steps) and w.mcs == mcs and w.precision == precision
    if n_sites is not None:
        assert w.n_sites_total == n_sites
    if name == "coreshell_fc":
        assert 25000 < w.n_sites_total < 33000  # about 29k sites (radius 12, a = 1)
    if name == "np256":
        sizes = [s.n_sites for s in w.samples]
        assert min(sizes) > 50 and max(sizes) < 16000 and 0.9e6 < sum(sizes) < 1.4e6
    if name == "sc64_hyst":
        B = w.B[0]
        assert B[0] == pytest.approx(2.0) and B[80] == pytest.approx(-2.0) and B[-1] == pytest.approx(2.0)
        assert np.allclose(np.abs(np.diff(B)), 0.05)


def test_core_shell_recipe():
    """Types by distance from the centre, exchange by the endpoint types, radial uniaxial
    anisotropy on the surface sites (fewer than 12 links) only."""
    s = core_shell_particle(seed=4, radius=6.0, core_radius=4.0)
    centre_dist = np.linalg.norm(s.positions - s.positions.mean(axis=0), axis=1)
    t = np.asarray(s.type)
    assert set(np.unique(t).tolist()) == {0, 1}
    assert centre_dist[t == 0].max() < centre_dist[t == 1].max()
    src = _sources(s)
    pair = {(0, 0): 1.0, (1, 1): 0.5, (0, 1): -0.3, (1, 0): -0.3}
    assert all(J == pair[(int(t[i]), int(t[j]))] for i, j, J in zip(src, s.col, s.J))
    _assert_symmetric(s)
    deg = np.diff(s.row_ptr)
    surf = deg < 12
    assert surf.any() and (~surf).any() and deg.max() == 12
    assert np.all(np.asarray(s.k_uni)[surf] == 0.5) and np.all(np.asarray(s.k_uni)[~surf] == 0.0)
    e = np.asarray(s.e_uni)[surf]
    assert np.allclose(np.linalg.norm(e, axis=1), 1.0)
    r = s.positions[surf] - s.positions.mean(axis=0)
    assert np.mean(np.sum(e * r, axis=1) / np.linalg.norm(r, axis=1)) > 0.95  # about radial


def test_nanoparticle_batch_recipe():
    """One site per unit volume (cube side 4^(1/3)): a radius-r particle holds about
    (4/3) pi r^3 sites; radii between 3 and 15; temperatures 0.05 + (p mod 64) 2.95/63."""
    w = workload("np256", mcs=1)
    sizes = np.array([s.n_sites for s in w.samples])
    radii = np.array([float(s.name.split("_r")[1]) for s in w.samples])
    assert radii.min() >= 3.0 and radii.max() <= 15.0
    ratio = sizes / (4.0 / 3.0 * np.pi * radii ** 3)
    assert np.all(np.abs(ratio - 1.0) < 0.25) and abs(np.median(ratio) - 1.0) < 0.05
    p = np.arange(256)
    assert np.allclose(w.T[:, 0], 0.05 + (p % 64) * 2.95 / 63.0) and np.all(w.B == 0.0)


def test_spin_glass_bonds_are_bimodal_and_shared():
    """The +-J glass: J = +-1 per undirected bond, about half each, one realisation for every
    replica (the workload has one sample)."""
    w = workload("sg256x32", scale=1 / 16)
    assert len(w.samples) == 1 and w.replicas == 32
    J = np.asarray(w.samples[0].J)
    assert set(np.unique(J).tolist()) == {-1.0, 1.0} and abs(np.mean(J)) < 0.05
    _assert_symmetric(w.samples[0])
    k = np.arange(32)
    assert np.allclose(w.T[:, 0], 0.1 * 20.0 ** (k / 31.0)) and np.all(w.B == 0.0)  # 0.1 -> 2.0, geometric
